// Device helpers shared by the GRNND kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace grnnd {

constexpr uint64_t kEmpty = ~0ull;
constexpr int kMaxR = 64;  // pool capacity handled by the 64-bit prune masks

// Counter-based hash of the design notes (reading C9): five chained SplitMix64
// steps, each the published gamma increment followed by the 30/27/31 finaliser.
__host__ __device__ __forceinline__ uint64_t splitmix_step(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t counter_hash(uint64_t seed, uint64_t t1, uint64_t t2,
                                                          uint64_t v, uint64_t x) {
  uint64_t h = splitmix_step(seed);
  h = splitmix_step(h ^ t1);
  h = splitmix_step(h ^ t2);
  h = splitmix_step(h ^ v);
  return splitmix_step(h ^ x);
}

// The same hash in two parts: the first three steps depend only on (seed, t1, t2), so a
// kernel computes them once, and hash_tail(hash_head(seed, t1, t2), v, x) equals
// counter_hash(seed, t1, t2, v, x) bit for bit.
__host__ __device__ __forceinline__ uint64_t hash_head(uint64_t seed, uint64_t t1, uint64_t t2) {
  return splitmix_step(splitmix_step(splitmix_step(seed) ^ t1) ^ t2);
}
__host__ __device__ __forceinline__ uint64_t hash_tail(uint64_t head, uint64_t v, uint64_t x) {
  return splitmix_step(splitmix_step(head ^ v) ^ x);
}

// ---- pool keys: (ordered float bits << 32) | (id << 1) | old -------------------------
__device__ __forceinline__ uint32_t ordered_bits(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}
__device__ __forceinline__ uint64_t make_key(float dist, uint32_t id, uint32_t old) {
  return ((uint64_t)ordered_bits(dist) << 32) | ((uint64_t)id << 1) | (uint64_t)old;
}
__device__ __forceinline__ uint32_t key_id(uint64_t k) { return (uint32_t)(k >> 1) & 0x7fffffffu; }
__device__ __forceinline__ float key_dist(uint64_t k) { return from_ordered((uint32_t)(k >> 32)); }
__device__ __forceinline__ uint32_t key_old(uint64_t k) { return (uint32_t)k & 1u; }

// ---- canonical FP32 distance -------------------------------------------------------------
// Four partial sums, s_j over the dimensions k = j (mod 4) in ascending k, each step one
// rounded op: L2SQ t = a - b, s_j = fma(t, t, s_j); IP s_j = fma(a, b, s_j).  The result
// is (s_0 + s_1) + (s_2 + s_3) (IP: 1 - that).  Every kernel that records a distance uses
// exactly this evaluation, so a pair gets the same bits wherever it is computed.
template <int METRIC>
__device__ __forceinline__ float dist_step(float acc, float a, float b) {
  if (METRIC == 0) {
    float t = __fsub_rn(a, b);
    return __fmaf_rn(t, t, acc);
  }
  return __fmaf_rn(a, b, acc);
}
template <int METRIC>
__device__ __forceinline__ void dist_step4(float4& acc, float4 a, float4 b) {
  acc.x = dist_step<METRIC>(acc.x, a.x, b.x);
  acc.y = dist_step<METRIC>(acc.y, a.y, b.y);
  acc.z = dist_step<METRIC>(acc.z, a.z, b.z);
  acc.w = dist_step<METRIC>(acc.w, a.w, b.w);
}
template <int METRIC>
__device__ __forceinline__ float dist_finish4(float4 acc) {
  const float s = __fadd_rn(__fadd_rn(acc.x, acc.y), __fadd_rn(acc.z, acc.w));
  return METRIC == 0 ? s : __fsub_rn(1.0f, s);
}
// Single-accumulator finish for the query-side kernels (their order is free).
template <int METRIC>
__device__ __forceinline__ float dist_finish(float acc) {
  return METRIC == 0 ? acc : __fsub_rn(1.0f, acc);
}
// Keeps the first `keep` (0..3) components of v and zeroes the others.
__device__ __forceinline__ float4 mask4(float4 v, int keep) {
  if (keep < 4) v.w = 0.0f;
  if (keep < 3) v.z = 0.0f;
  if (keep < 2) v.y = 0.0f;
  if (keep < 1) v.x = 0.0f;
  return v;
}

// Canonical distance of two rows in global memory (16-byte aligned rows, d dims).
template <int METRIC>
__device__ __forceinline__ float row_dist(const float* __restrict__ a, const float* __restrict__ b,
                                          int d) {
  float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  int k = 0;
  for (; k + 4 <= d; k += 4)
    dist_step4<METRIC>(acc, __ldg(reinterpret_cast<const float4*>(a + k)),
                       __ldg(reinterpret_cast<const float4*>(b + k)));
  if (k < d) {
    const int r = d - k;
    float4 x = make_float4(0.0f, 0.0f, 0.0f, 0.0f), y = x;
    x.x = __ldg(a + k);
    y.x = __ldg(b + k);
    if (r > 1) { x.y = __ldg(a + k + 1); y.y = __ldg(b + k + 1); }
    if (r > 2) { x.z = __ldg(a + k + 2); y.z = __ldg(b + k + 2); }
    dist_step4<METRIC>(acc, x, y);
  }
  return dist_finish4<METRIC>(acc);
}

// ---- warp bitonic sort of 32*E uint64 values, element index e = j*32 + lane ----------
template <int E>
__device__ __forceinline__ void warp_sort_u64(uint64_t (&x)[E]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
    for (int s = k >> 1; s > 0; s >>= 1) {
      if (s >= 32) {
        const int js = s >> 5;
#pragma unroll
        for (int j = 0; j < E; ++j) {
          if ((j & js) == 0) {
            const int j2 = j | js;
            const bool up = (((j << 5) | lane) & k) == 0;
            uint64_t a = x[j], b = x[j2];
            bool sw = up ? (a > b) : (a < b);
            x[j] = sw ? b : a;
            x[j2] = sw ? a : b;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const int e = (j << 5) | lane;
          const bool up = (e & k) == 0;
          const bool lower = (e & s) == 0;
          uint64_t o = __shfl_xor_sync(0xffffffffu, x[j], s);
          uint64_t mn = x[j] < o ? x[j] : o;
          uint64_t mx = x[j] < o ? o : x[j];
          x[j] = (lower == up) ? mn : mx;
        }
      }
    }
  }
}

// ---- bounded mbarrier wait (every wait has an iteration limit) ----------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(a),
      "r"(bytes)
      : "memory");
}
// Returns true when the phase with the given parity completed, false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// Bulk copy global -> shared (no tensor map); completion counted on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gmem_src, uint32_t bytes,
                                         uint64_t* bar) {
  uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
      "l"(gmem_src), "r"(bytes), "r"(b)
      : "memory");
}

// Status word written by kernels whose bounded waits gave up.
constexpr int kErrTimeout = 1;
constexpr int kErrBounds = 2;

// Bounds checks of the checked build (-DGRNND_CHECKS=1, the stand-in for a memory checker): an
// index outside its buffer records kErrBounds in the step's status word (so the rest of the
// step does nothing) and the access is skipped.  In the normal build they compile to nothing.
#ifdef GRNND_CHECKS
__device__ __forceinline__ bool in_bounds(bool ok, int32_t* err) {
  if (!ok) atomicCAS(err, 0, kErrBounds);
  return ok;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(bool, int32_t*) { return true; }
#endif

}  // namespace grnnd
