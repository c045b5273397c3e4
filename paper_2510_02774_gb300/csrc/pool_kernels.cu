// GRNND pool kernels for sm_103a.
//
//   rnd_init      Alg 3, INITIAL_NEIGHBORS
//   prep          list of the vertices whose pool holds a new entry (the others cannot fire)
//   rnd_join      Alg 4's pair loop with the rule of Eq 2: gather + dist_tile + rng_prune
//   rev_merge     bucket the redirects by target, then per target keep the R smallest
//                 distinct keys of (kept pool, redirects): the end state of WARP_INSERT
//                 (Alg 6) over fixed-capacity pools (Sec 3.5)
//   reverse       reverse-edge sampling (Sec 3.6) feeding the same merge
//   quantize      BF16 copy of the points + per-row norm and residual for the BF16 form
#include <cuda.h>  // CUtensorMap and the types of cuTensorMapEncodeTiled (fetched at run time)
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cstdio>

#include "common.cuh"
#include "internal.h"
#include "kernels.cuh"
#include <atomic>
#include <type_traits>
#include <mutex>

namespace grnnd {

namespace {

constexpr uint32_t kWaitLimit = 1u << 18;  // mbarrier try_wait rounds before a wait gives up (about 1 s: a try that does not complete returns after about 3.8 us)

// Per-kernel launch set-up kept out of stream captures: the dynamic shared-memory opt-in
// (once) and the resident blocks per SM (cached per shared-memory size).  Shared by host
// threads, so guarded by a mutex.
struct KernelSetup {
  bool attr = false;
  size_t smem[2] = {0, 0};
  int per_sm[2] = {0, 0};
};
std::mutex g_setup_mu;

template <typename K>
cudaError_t setup_kernel(KernelSetup& ks, K kern, int threads, size_t smem_max, size_t smem, int* per_sm) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!ks.attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    if (e != cudaSuccess) return e;
    ks.attr = true;
  }
  for (int i = 0; i < 2; ++i)
    if (ks.per_sm[i] > 0 && ks.smem[i] == smem) {
      *per_sm = ks.per_sm[i];
      return cudaSuccess;
    }
  int v = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, threads, smem);
  if (e != cudaSuccess) return e;
  if (v < 1) v = 1;
  const int slot = ks.per_sm[0] == 0 ? 0 : 1;
  ks.smem[slot] = smem;
  ks.per_sm[slot] = v;
  *per_sm = v;
  return cudaSuccess;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ uint64_t bits_below(int i) { return i == 0 ? 0ull : (~0ull >> (64 - i)); }

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

}  // namespace

int sm_count() {
  static std::atomic<int> cached{0};  // read by the worker threads of the serving loop too
  int v = cached.load(std::memory_order_relaxed);
  if (v == 0) {
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    v = c > 0 ? c : 152;
    cached.store(v, std::memory_order_relaxed);
  }
  return v;
}

// 16-byte asynchronous copy global -> shared (the L1-bypassing form): nbytes (0..16) are read
// from g, the rest of the 16 bytes are written as zeros; both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* sm, const void* g, int nbytes) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(sm);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(g), "r"(nbytes) : "memory");
}
// waits for every cp_async16 this thread issued (a hardware wait: the copies always complete)
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// =====================================================================================
// rnd_init: one warp per vertex.
//   Sampling follows the sequential definition exactly: candidate j = 0, 1, 2, ... is
//   accepted iff its id differs from every earlier accepted id, until S are accepted.
//   32 candidates are tested per step; a lane is rejected if its id matches an accepted
//   id or an earlier lane of the same step.
// =====================================================================================
// E: pool entries per lane (32 E >= R); IW: warps per CTA (E = 2, pools of up to 64 entries:
// 4 warps; E = 8, up to 256 entries: 2 warps, so that the staged rows stay within the static
// shared memory); IC: FP32 dimensions per staged chunk (4 IC bytes of each row per round
// trip); SR: staged rows per warp (S + 1 at most: the drawn rows and v's own).  A BF16 source
// is staged in the same bytes as bfloat16 values, 2 IC dimensions per chunk.  Samples of up to
// 32 entries stage 33 rows of 128-byte chunks; larger ones 32 E + 1 rows of 64-byte chunks (a
// bigger buffer would cost resident warps).
// Xb (may be null): a BF16 copy of the rows (ldb elements per row); when qflags say that every
// value is exact in BF16, the drawn rows are read from it -- the same values in half the bytes.
template <int METRIC, int E, int IW, int IC, int SR>
__global__ void __launch_bounds__(IW * 32) rnd_init_kernel(const float* __restrict__ X, int64_t n,
                                                           int d, int ld, int S, int R, uint64_t seed,
                                                           uint64_t* __restrict__ keys,
                                                           int32_t* __restrict__ deg,
                                                           const int2* __restrict__ vseg,
                                                           const __nv_bfloat16* __restrict__ Xb, int ldb,
                                                           const unsigned* __restrict__ qflags,
                                                           uint64_t magic) {
  constexpr int RSF = IC + 4;       // staged row stride in floats (16-byte granules)
  constexpr int RSB = 2 * RSF;      // ... in bfloat16 values
  constexpr int GF = IC / 4;        // FP32 granules (4 dimensions) per staged row chunk
  constexpr int GB = IC / 4;        // BF16 granules (8 dimensions) per staged row chunk
  __shared__ int32_t acc_ids[IW][32 * E];
  // the chunk of each drawn row (rows 0..S-1) and of v itself (row S), 16-byte granules
  __shared__ __align__(16) float stage[IW][SR][RSF];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* acc = acc_ids[warp];
  float(*rows)[RSF] = stage[warp];
  uint16_t* rows_b = reinterpret_cast<uint16_t*>(&stage[warp][0][0]);
  const uint64_t head = hash_head(seed, 0, 0);
  const unsigned below = lanemask_lt();
  const bool use_b = Xb != nullptr && (qflags[0] & 2u) == 0u;  // every value exact in BF16
  const uint16_t* Xbs = reinterpret_cast<const uint16_t*>(Xb);
  for (int64_t v = (int64_t)blockIdx.x * IW + warp; v < n; v += (int64_t)gridDim.x * IW) {
    // the vertex's build: ids [lo, lo + nb); draws use the local id v - lo
    const int64_t lo = vseg ? vseg[v].x : 0;
    const uint64_t nm1 = (uint64_t)((vseg ? (int64_t)vseg[v].y : n) - 1);
    const uint64_t vl = (uint64_t)(v - lo);
    // h mod nm1 without a division: q = high 64 bits of h * floor((2^64 - 1) / nm1) is
    // h / nm1 rounded down, or one less, so one correction gives the exact remainder
    const uint64_t mg = vseg ? (~0ull / nm1) : magic;
    int cnt = 0;
    // S <= nb - 1, so the draws cover enough distinct ids long before the bound.
    for (uint64_t base = 0; cnt < S && base < (1ull << 32); base += 32) {
      const uint64_t hv = hash_tail(head, vl, base + lane);
      uint64_t r = hv - __umul64hi(hv, mg) * nm1;
      if (r >= nm1) r -= nm1;
      const int32_t u = (int32_t)(lo + (int64_t)(r + (r >= vl ? 1u : 0u)));
      bool dup = false;
      for (int j = 0; j < cnt; ++j) dup |= (acc[j] == u);
      const unsigned same = __match_any_sync(0xffffffffu, u);
      dup |= (same & below) != 0u;
      const unsigned ok = __ballot_sync(0xffffffffu, !dup);
      const int pos = cnt + __popc(ok & below);
      if (!dup && pos < S) acc[pos] = u;
      cnt = min(S, cnt + __popc(ok));
      __syncwarp();
    }
    // canonical distances, lane e for entries e, e + 32, ...: the rows are staged a chunk of
    // dimensions at a time with coalesced 16-byte loads; each lane then advances its four
    // partial sums over the chunk in ascending dimension order, exactly as row_dist does
    float4 ps[E];
#pragma unroll
    for (int j = 0; j < E; ++j) ps[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const int CH = use_b ? 2 * IC : IC;  // dimensions per chunk
    for (int c0 = 0; c0 < d; c0 += CH) {
      const int clen = min(CH, d - c0);
      // every 16-byte granule of the chunk is copied asynchronously (all of them in flight at
      // once, no registers held); the bytes past d are filled with zeros by the copy itself
      if (use_b) {
        // row t / GB, granule t % GB of 8 BF16 values
        for (int t = lane; t < (S + 1) * GB; t += 32) {
          const int r = t / GB, q = t % GB;  // (GB is a power of two)
          const int64_t src = r < S ? (int64_t)acc[r] : v;
          const int nbytes = 2 * max(0, min(8, clen - 8 * q));
          cp_async16(rows_b + r * RSB + 8 * q, Xbs + src * ldb + c0 + (nbytes ? 8 * q : 0), nbytes);
        }
      } else {
        // row t / GF, granule t % GF of 4 FP32 values (past d: zero, as row_dist's tail)
        for (int t = lane; t < (S + 1) * GF; t += 32) {
          const int r = t / GF, q = t % GF;  // (GF is a power of two)
          const int64_t src = r < S ? (int64_t)acc[r] : v;
          const int nbytes = 4 * max(0, min(4, clen - 4 * q));
          cp_async16(&rows[r][4 * q], X + src * ld + c0 + (nbytes ? 4 * q : 0), nbytes);
        }
      }
      cp_async_wait_all();
      __syncwarp();
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int e = j * 32 + lane;
        if (e >= S) continue;
        if (use_b) {
          for (int q = 0; 8 * q < clen; ++q) {  // eight BF16 values, widened exactly
            const uint4 a = *reinterpret_cast<const uint4*>(rows_b + S * RSB + 8 * q);
            const uint4 b = *reinterpret_cast<const uint4*>(rows_b + e * RSB + 8 * q);
            float4 a0 = make_float4(__uint_as_float(a.x << 16), __uint_as_float(a.x & 0xffff0000u),
                                    __uint_as_float(a.y << 16), __uint_as_float(a.y & 0xffff0000u));
            float4 a1 = make_float4(__uint_as_float(a.z << 16), __uint_as_float(a.z & 0xffff0000u),
                                    __uint_as_float(a.w << 16), __uint_as_float(a.w & 0xffff0000u));
            float4 b0 = make_float4(__uint_as_float(b.x << 16), __uint_as_float(b.x & 0xffff0000u),
                                    __uint_as_float(b.y << 16), __uint_as_float(b.y & 0xffff0000u));
            float4 b1 = make_float4(__uint_as_float(b.z << 16), __uint_as_float(b.z & 0xffff0000u),
                                    __uint_as_float(b.w << 16), __uint_as_float(b.w & 0xffff0000u));
            const int rem = clen - 8 * q;  // past d: zero, as row_dist's tail
            if (rem < 8) {
              a0 = mask4(a0, rem);
              b0 = mask4(b0, rem);
              a1 = mask4(a1, rem - 4);
              b1 = mask4(b1, rem - 4);
            }
            dist_step4<METRIC>(ps[j], a0, b0);
            if (rem > 4) dist_step4<METRIC>(ps[j], a1, b1);
          }
        } else {
          const int gr = (clen + 3) >> 2;  // granules of the chunk
          for (int q = 0; q < gr; ++q)
            dist_step4<METRIC>(ps[j], *reinterpret_cast<const float4*>(&rows[S][4 * q]),
                               *reinterpret_cast<const float4*>(&rows[e][4 * q]));
        }
      }
      __syncwarp();
    }
    uint64_t kk[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int e = j * 32 + lane;
      kk[j] = e < S ? make_key(dist_finish4<METRIC>(ps[j]), (uint32_t)acc[e], 0u) : kEmpty;
    }
    // sort the registers that hold entries (the others hold only empty keys, which are last)
    if (S <= 32) {
      uint64_t k1[1] = {kk[0]};
      warp_sort_u64<1>(k1);
      kk[0] = k1[0];
    } else if (E == 2 || S <= 64) {
      uint64_t k2[2] = {kk[0], kk[1]};
      warp_sort_u64<2>(k2);
      kk[0] = k2[0];
      kk[1] = k2[1];
    } else {
      warp_sort_u64<E>(kk);
    }
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int e = j * 32 + lane;
      if (e < R) keys[v * R + e] = kk[j];
    }
    if (lane == 0) deg[v] = S;
    __syncwarp();
  }
}

cudaError_t launch_pool_init(const float* X, int64_t n, int d, int ld, int metric, int S, int R,
                             uint64_t seed, uint64_t* keys, int32_t* deg, cudaStream_t st,
                             const int2* vseg, const void* Xb16, int ldb, const unsigned* qflags) {
  const __nv_bfloat16* Xb = (Xb16 && qflags) ? static_cast<const __nv_bfloat16*>(Xb16) : nullptr;
  const uint64_t magic = ~0ull / (uint64_t)(n - 1);  // the draws' modulus of a single build (n >= 2)
  ProfScope ps("rnd_init", st);
  if (R <= kTeamMaxM && S <= 32) {
    constexpr int IW = 4;
    const int64_t blocks = std::min<int64_t>(ceil_div(n, IW), (int64_t)sm_count() * 16);
    if (metric == 0)
      rnd_init_kernel<0, 2, IW, 32, 33><<<(unsigned)blocks, IW * 32, 0, st>>>(X, n, d, ld, S, R, seed, keys, deg, vseg, Xb, ldb, qflags, magic);
    else
      rnd_init_kernel<1, 2, IW, 32, 33><<<(unsigned)blocks, IW * 32, 0, st>>>(X, n, d, ld, S, R, seed, keys, deg, vseg, Xb, ldb, qflags, magic);
  } else if (R <= kTeamMaxM) {
    constexpr int IW = 4;
    const int64_t blocks = std::min<int64_t>(ceil_div(n, IW), (int64_t)sm_count() * 16);
    if (metric == 0)
      rnd_init_kernel<0, 2, IW, 16, 65><<<(unsigned)blocks, IW * 32, 0, st>>>(X, n, d, ld, S, R, seed, keys, deg, vseg, Xb, ldb, qflags, magic);
    else
      rnd_init_kernel<1, 2, IW, 16, 65><<<(unsigned)blocks, IW * 32, 0, st>>>(X, n, d, ld, S, R, seed, keys, deg, vseg, Xb, ldb, qflags, magic);
  } else {  // pools of up to 256 entries
    constexpr int IW = 2;
    const int64_t blocks = std::min<int64_t>(ceil_div(n, IW), (int64_t)sm_count() * 32);
    if (metric == 0)
      rnd_init_kernel<0, 8, IW, 16, 257><<<(unsigned)blocks, IW * 32, 0, st>>>(X, n, d, ld, S, R, seed, keys, deg, vseg, Xb, ldb, qflags, magic);
    else
      rnd_init_kernel<1, 8, IW, 16, 257><<<(unsigned)blocks, IW * 32, 0, st>>>(X, n, d, ld, S, R, seed, keys, deg, vseg, Xb, ldb, qflags, magic);
  }
  return cudaGetLastError();
}

__global__ void localize_ids_kernel(int64_t n, int R, int32_t* __restrict__ ids, const int2* __restrict__ vseg) {
  const int64_t total = n * R;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = ids[i];
    if (u >= 0) ids[i] = u - vseg[i / R].x;
  }
}

cudaError_t launch_localize_ids(int64_t n, int R, int32_t* ids, const int2* vseg, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>(ceil_div(n * R, 256), (int64_t)sm_count() * 8);
  localize_ids_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, R, ids, vseg);
  return cudaGetLastError();
}

// =====================================================================================
// quantize: BF16 rows (dp = d rounded up to 16 elements, zero padded) followed by a 32-byte
// tail (norm^2 of the BF16 row, ||x - bf16(x)|| rounded up, then zeros), so that a row's bulk
// copy brings its terms along; ldb = dp + 16 elements is the row stride.  The same terms go to
// aux, and the dataset flags: qflags[0] bit 0 = some value is not an integer, bit 1 = some
// value is not exact in BF16; qflags[1] = max |x| (bits).
// =====================================================================================
__global__ void quantize_kernel(const float* __restrict__ X, int64_t n, int d, int ld,
                                __nv_bfloat16* __restrict__ Xb, int ldb, float2* __restrict__ aux,
                                unsigned* __restrict__ qflags) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int dp = ldb - kRowTail16;  // padded dimensions of a row
  unsigned fl = 0, mx = 0;
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; r < n;
       r += (int64_t)gridDim.x * (blockDim.x >> 5)) {
    float nrm = 0.0f, res = 0.0f;
    for (int k = lane; k < dp; k += 32) {
      const float x = k < d ? X[r * ld + k] : 0.0f;
      const __nv_bfloat16 b = __float2bfloat16_rn(x);
      Xb[r * ldb + k] = b;
      const float xf = __bfloat162float(b);
      nrm = __fmaf_rn(xf, xf, nrm);
      // |x - xf|, its square and the running sum rounded upward: res stays an upper bound
      // of the squared residual norm
      const float e = x >= xf ? __fsub_ru(x, xf) : __fsub_ru(xf, x);
      res = __fmaf_ru(e, e, res);
      fl |= (x != rintf(x)) ? 1u : 0u;
      fl |= (xf != x) ? 2u : 0u;
      mx = max(mx, __float_as_uint(fabsf(x)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
      res = __fadd_ru(res, __shfl_xor_sync(0xffffffffu, res, o));
    }
    if (lane == 0) {
      const float2 t = make_float2(nrm, __fsqrt_ru(res));
      aux[r] = t;
      *reinterpret_cast<float4*>(Xb + r * ldb + dp) = make_float4(t.x, t.y, 0.0f, 0.0f);
      *reinterpret_cast<float4*>(Xb + r * ldb + dp + 8) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fl |= __shfl_xor_sync(0xffffffffu, fl, o);
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) {
    if (fl) atomicOr(&qflags[0], fl);
    atomicMax(&qflags[1], mx);
  }
}

// =====================================================================================
// quantize, FP8 form: e4m3 rows (dp = d rounded up to 32 bytes, zero padded, then the same
// 32-byte tail as the BF16 rows; ldb = dp + 32) with one power-of-two scale per row,
// x_hat = 2^e q.  e = E - 8 for max |x| = f 2^E, f in [0.5, 1),
// so every |x| 2^-e < 256 stays inside e4m3's finite range (448) and the scaling itself is
// exact.  aux = (norm^2 of x_hat, ||x - x_hat|| rounded up); the low byte of the residual's
// bits carries e + 127 (the residual is first rounded up to a multiple of 256 units in its
// last place, so the stored value is still an upper bound).  qflags as for BF16, with
// bit 1 = some value is not exact in the quantized row.
// =====================================================================================
__global__ void quantize_fp8_kernel(const float* __restrict__ X, int64_t n, int d, int ld,
                                    uint8_t* __restrict__ Xq, int ldb, float2* __restrict__ aux,
                                    unsigned* __restrict__ qflags) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned fl = 0, mx = 0;
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; r < n;
       r += (int64_t)gridDim.x * (blockDim.x >> 5)) {
    float amax = 0.0f;
    for (int k = lane; k < d; k += 32) amax = fmaxf(amax, fabsf(X[r * ld + k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    int E = 0;
    if (amax > 0.0f) frexpf(amax, &E);
    const int e = amax > 0.0f ? min(127, max(-126, E - 8)) : 0;
    const float inv = ldexpf(1.0f, -e), sc = ldexpf(1.0f, e);
    const int dp = ldb - kRowTail8;  // padded dimensions of a row
    float nrm = 0.0f, res = 0.0f;
    for (int k = lane; k < dp; k += 32) {
      const float x = k < d ? X[r * ld + k] : 0.0f;
      const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(x * inv, __NV_SATFINITE, __NV_E4M3);
      Xq[r * ldb + k] = (uint8_t)q;
      const float xf = __half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3))) * sc;
      nrm = __fmaf_rn(xf, xf, nrm);
      // |x - xf|, its square and the running sum rounded upward: res stays an upper bound
      // of the squared residual norm
      const float e = x >= xf ? __fsub_ru(x, xf) : __fsub_ru(xf, x);
      res = __fmaf_ru(e, e, res);
      fl |= (x != rintf(x)) ? 1u : 0u;
      fl |= (xf != x) ? 2u : 0u;
      mx = max(mx, __float_as_uint(fabsf(x)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
      res = __fadd_ru(res, __shfl_xor_sync(0xffffffffu, res, o));
    }
    if (lane == 0) {
      uint32_t rb = __float_as_uint(__fsqrt_ru(res));
      rb = ((rb + 255u) & ~255u) | (uint32_t)(e + 127);
      aux[r] = make_float2(nrm, __uint_as_float(rb));
      *reinterpret_cast<float4*>(Xq + r * ldb + dp) = make_float4(nrm, __uint_as_float(rb), 0.0f, 0.0f);
      *reinterpret_cast<float4*>(Xq + r * ldb + dp + 16) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fl |= __shfl_xor_sync(0xffffffffu, fl, o);
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) {
    if (fl) atomicOr(&qflags[0], fl);
    atomicMax(&qflags[1], mx);
  }
}

cudaError_t launch_quantize(const float* X, int64_t n, int d, int ld, void* Xbv, int ldb,
                            float2* aux, unsigned* qflags, int precision, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(qflags, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::min<int64_t>(ceil_div(n, 8), (int64_t)sm_count() * 16);
  ProfScope ps("quantize", st);
  if (precision == 2)
    quantize_fp8_kernel<<<(unsigned)blocks, 256, 0, st>>>(X, n, d, ld, static_cast<uint8_t*>(Xbv), ldb, aux,
                                                          qflags);
  else
    quantize_kernel<<<(unsigned)blocks, 256, 0, st>>>(X, n, d, ld, static_cast<__nv_bfloat16*>(Xbv), ldb, aux,
                                                      qflags);
  return cudaGetLastError();
}

// =====================================================================================
// prep: active flag of the vertices whose pool holds a new entry, and for each of them a work
// record in the list of its pool-size class.  Records go to one of five
// regions by pool size (entries <= 8, <= 16, <= 32, <= 64, more; pools of up to 64 entries
// all to the fourth region when the warp kernels cannot take the rows), so that a warp can
// take several small pools at once.  A record of a region holding up to cap entries:
//   word 0: v | (first id of v's build) << 32    word 1: m
// (the joins read the m pool keys from v's own row).
// Also counts the entries of every pool (each one is proposed once, explicitly or in place).
// With `hint` (the flags the last merge of the same pools wrote) no pool key is read for
// the active test.
// =====================================================================================
struct RecSet {
  uint64_t* rec[kNumClasses];
  int w[kNumClasses];
  int cap[kNumClasses];
};

constexpr int kPrepWarps = 8;  // warps per prep block (256 threads)
__global__ void __launch_bounds__(kPrepWarps * 32) prep_kernel(const uint64_t* __restrict__ keys, const int32_t* __restrict__ deg,
                            int64_t n, int R, uint8_t* __restrict__ active,
                            int32_t* __restrict__ list_n, int warp_ok, int3 gmax, RecSet rs,
                            const int2* __restrict__ vseg,
                            const uint8_t* __restrict__ hint, int64_t* __restrict__ stats,
                            int32_t* __restrict__ zero_count, int64_t* __restrict__ zero_new) {
  // (zero_count, zero_new: the round's redirect counts and new-entry counter, cleared here
  // instead of by separate memsets)
  if (zero_new && blockIdx.x == 0 && threadIdx.x == 0) *zero_new = 0;
  // record places: a warp counts its active vertices per class (ballots), the block adds
  // its warps' counts up and takes one range per class from list_n (one atomic per block and
  // class, not per warp: the class counters are few addresses that every block hits)
  __shared__ int s_cnt[kPrepWarps][kNumClasses];  // per warp; then its first place in the block's range
  __shared__ int s_base[kNumClasses];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long props = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < n; b0 += stride) {  // uniform over the block
    const int64_t v = b0 + threadIdx.x;
    bool act = false;
    int m = 0;
    if (v < n) {
      if (zero_count) zero_count[v] = 0;
      m = deg[v];
      props += m;
      if (hint)  // the last merge of these pools recorded which rows hold a new entry
        act = hint[v] != 0;
      else
        for (int j = 0; j < m && !act; ++j) act = !(keys[v * R + j] & 1ull);
      active[v] = act ? 1 : 0;
    }
    const int cls = m > kTeamMaxM ? 4 : !warp_ok ? 3 : (m <= gmax.x ? 0 : (m <= gmax.y ? 1 : (m <= gmax.z ? 2 : 3)));
    unsigned bc[kNumClasses];
#pragma unroll
    for (int c = 0; c < kNumClasses; ++c) {
      bc[c] = __ballot_sync(0xffffffffu, act && cls == c);
      if (lane == 0) s_cnt[warp][c] = __popc(bc[c]);
    }
    __syncthreads();
    if (threadIdx.x < kNumClasses) {
      const int c = threadIdx.x;
      int tot = 0;
      for (int w = 0; w < kPrepWarps; ++w) {
        const int x = s_cnt[w][c];
        s_cnt[w][c] = tot;
        tot += x;
      }
      s_base[c] = tot ? atomicAdd(&list_n[c], tot) : 0;
    }
    __syncthreads();
    // each active vertex writes its record: v and its build's first id, and m (the join reads
    // the pool keys from the vertex's own row, which nothing else writes before its join)
    if (act) {
      unsigned mb = bc[0];
      int o = s_base[0] + s_cnt[warp][0];
      uint64_t* rg = rs.rec[0];
      int W = rs.w[0];
#pragma unroll
      for (int q = 1; q < kNumClasses; ++q)
        if (cls == q) {
          mb = bc[q];
          o = s_base[q] + s_cnt[warp][q];
          rg = rs.rec[q];
          W = rs.w[q];
        }
      uint64_t* r = rg + (int64_t)(o + __popc(mb & lanemask_lt())) * W;
      r[0] = (uint64_t)v | ((uint64_t)(vseg ? vseg[v].x : 0) << 32);
      r[1] = (uint64_t)m;
    }
  }
  if (stats) {  // (every thread of the block gets here: the loop above is uniform over it)
    __shared__ long long s_props[kPrepWarps];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) props += __shfl_xor_sync(0xffffffffu, props, o);
    if (lane == 0) s_props[warp] = props;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long t = 0;
      for (int w = 0; w < kPrepWarps; ++w) t += s_props[w];
      if (t) atomicAdd(reinterpret_cast<unsigned long long*>(&stats[4]), (unsigned long long)t);
    }
  }
}

// =====================================================================================
// rnd_join, batched.  A CTA walks a contiguous range of the active list.  It takes the
// vertices in batches (at most BV vertices, BR pool entries, BP pairs or BT mma tiles)
// and runs every phase for the whole batch at once, so that each latency (global loads,
// the gather round trip, barriers, the slot reservation) is paid once per batch:
//
//  0. set-up, one warp per vertex: pool keys, visit order pi = rank of
//     (h(seed,t1,t2,v,id), id) (or ascending / descending key), rows laid out new-first
//     so that the pairs with a new side -- the only ones that can fire (design reading
//     C10) -- are local rows i < k, j > i: k(m-1) - k(k-1)/2 pairs per vertex;
//  1. gather: one bulk copy (TMA engine) per row and dimension chunk into a shared row
//     arena, all completing on one mbarrier; the next batch's rows are in flight while
//     the current batch computes (two stages);
//  2. dist_tile, FP32 form: one thread per pair, the canonical four-accumulator FP32
//     distance over dimension chunks (partial sums in registers); BF16 form: Gram tiles
//     on the tensor cores (mma.sync m16n8k16, FP32 accumulate), D = (|x_i|^2 - g) +
//     (|x_j|^2 - g), with a per-pair error bound; a decision inside the bound is re-taken
//     with canonical FP32 distances read from the FP32 rows;
//  3. rng_prune: fire bits F[b] = {a < b : d(a,b) < max(d(v,a), d(v,b))} in pi order,
//     then one thread per vertex replays the sequential pair scan of Alg 4 on the bits:
//     in column b, the live firing a's are taken in order; each one that is farther than
//     b becomes bottom (absorbed by b) until one that is closer makes b bottom;
//  4. emit: survivors in key order into the output pool (old); each bottom entry is one
//     redirect (absorber, d(close, far), new) in a compact list.
// =====================================================================================
namespace {

constexpr int JT = 256;                        // threads per join CTA
constexpr int JW = JT / 32;                    // warps per join CTA
constexpr int BV = 16;                         // vertices per batch at most
constexpr int BR = 208;                        // pool entries (rows) per batch at most
constexpr int BRA = BR + 16;                   // allocated rows: partial mma tiles read past the end
constexpr int BP = 2048;                       // pairs per batch at most
constexpr int SPW = 12;                        // FP32 tile: row segments per warp
constexpr int BSEG = 288;                      // row segments per batch at most
constexpr int BT = 64;                         // mma output tiles per batch at most
constexpr int TPW = BT / JW;                   // mma tiles per warp
constexpr int RECW_MAX = 2;                    // work-record words
constexpr int RED_CHUNK = kRedChunk;           // redirect slots reserved per CTA at a time

// A row segment is up to 32 consecutive pairs (i, j0..j0+31) of one new row i: one warp
// takes a segment, one lane a partner j.
template <int PREC>
__host__ __device__ constexpr int seg_budget() { return PREC == 0 ? JW * SPW : BSEG; }

template <int PREC>
struct Prec;
template <>
struct Prec<0> {
  using T = float;
  static constexpr int DC = 32;     // dimensions per staged chunk
  static constexpr int RS = DC + 4; // 144-byte rows: 16-byte loads of 8 rows hit distinct banks
  static constexpr int VEC = 4;     // copy granule in elements (16 bytes)
};
template <>
struct Prec<1> {
  using T = __nv_bfloat16;
  static constexpr int DC = 64;
  static constexpr int RS = DC + 8; // 144-byte rows: ldmatrix rows hit distinct banks
  static constexpr int VEC = 16;    // whole k16 steps (32 bytes)
};

struct __align__(16) Batch {
  // indexed by batch row (rowbase of the vertex + local row)
  int32_t rid[BRA];         // point id of the row
  int32_t roff[BR];         // batch pair index of the first pair of a new row
  float rnrm[BR];           // BF16 form: norm^2 of the quantized row
  float rdq[BR];            // BF16 form: quantization residual norm
  uint8_t rpos[BR];         // pi position of the row
  uint8_t rvb[BR];          // vertex (in the batch) of the row
  // indexed by rowbase of the vertex + pi position
  uint64_t pkey[BR];
  int32_t pid[BR];
  uint8_t prow[BR];         // local row of the pi position
  uint8_t pslot[BR];        // storage slot of the pi position
  uint16_t seg[BSEG];       // (batch row of the new row << 8) | first partner
  // per vertex
  int64_t v[BV];
  int32_t m[BV], k[BV], np[BV];
  int32_t rowbase[BV + 1], pairbase[BV + 1], tilebase[BV + 1], segbase[BV + 1];
  uint16_t tiles[BT];       // (vb << 8) | (I << 4) | J
  int nb, nent, ncopy, npairs, ntiles, nseg, nchunks;
};

template <int PREC>
struct __align__(16) JoinSmem {
  typename Prec<PREC>::T rows[2][BRA][Prec<PREC>::RS];
  Batch bt[2];
  float pd[BP];             // pair distances in batch pair order
  uint64_t fire[BR];        // fire bits by rowbase + pi position
  uint64_t closer[BR];      // fire bits whose lower pi position is also the closer entry
  uint64_t colkill[BR];     // entries made bottom in column b (absorbed by b)
  uint8_t colf[BR];         // absorber of b when b itself became bottom, else 0xFF
  uint64_t fcol[BV];        // columns with a fire bit, per vertex
  uint64_t alive[BV];
  uint64_t smask[BV];       // survivors by storage slot
  int32_t deadrank[BV];     // rank of a vertex's first redirect within the batch
  // batch formation
  uint64_t window[BV * RECW_MAX];  // work records of the next candidates (bulk prefetch)
  int64_t cv[BV];
  int32_t cm[BV], ck[BV], cnp[BV], cnt_[BV], cns[BV];
  unsigned long long red_next, red_end;  // this CTA's reserved redirect slots
  unsigned long long red_b0, red_b1;     // the batch's redirects: avail at red_b0, the rest at red_b1
  int32_t red_avail;
  uint64_t bar[2];
  uint64_t wbar;
};

// two CTAs per SM: 233472 bytes of shared memory minus 1 KB reserved per CTA
static_assert(sizeof(JoinSmem<0>) <= 115 * 1024 && sizeof(JoinSmem<1>) <= 115 * 1024,
              "join shared memory must allow two CTAs per SM");

__device__ __forceinline__ int tiles_of(int m, int k) {
  int nt = 0;
  const int KI = (k + 15) >> 4, NJ = (m + 7) >> 3;
  for (int I = 0; I < KI; ++I)
    for (int J = 0; J < NJ; ++J) nt += (J * 8 + 7 > I * 16) ? 1 : 0;
  return nt;
}

// ---- batch formation and per-vertex set-up (all threads) --------------------------------
// Candidates are the next BV list entries of the CTA's range; warp w loads candidates w
// and w + JW and keeps their keys in registers for the set-up.  Returns the number of
// list entries consumed (0 when the range is exhausted).
template <int PREC>
__device__ __forceinline__ void join_prefetch(JoinSmem<PREC>& s, int64_t pos, int64_t end, const JoinArgs& a) {
  const int64_t cnt = min((int64_t)BV, end - pos);
  if (cnt <= 0) return;
  const uint32_t bytes = (uint32_t)(cnt * a.rec_w[3] * 8);
  mbar_expect_tx(&s.wbar, bytes);
  bulk_g2s(s.window, a.rec[3] + pos * a.rec_w[3], bytes, &s.wbar);
}

template <int PREC>
__device__ int join_form_batch(JoinSmem<PREC>& s, Batch& B, int64_t pos, int64_t end,
                               uint32_t& wph, const JoinArgs& a) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int R = a.R, W = a.rec_w[3];
  if (pos >= end) return 0;
  const bool ok = mbar_wait(&s.wbar, wph, kWaitLimit);
  wph ^= 1u;
  if (__syncthreads_or(!ok)) {  // the records never arrived: report and stop the CTA
    if (tid == 0) atomicExch(a.err, kErrTimeout);
    if (!ok) mbar_wait(&s.wbar, wph ^ 1u, kWaitLimit);
    return -1;
  }
  uint64_t kx[2][2];
  float2 ax[2][2];
  int64_t vx[2];
  uint32_t lox[2];  // first id of the vertex's build (visit orders use local ids)
  int mx[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c = warp + h * JW;
    const int64_t p = pos + c;
    vx[h] = -1;
    mx[h] = 0;
    kx[h][0] = kx[h][1] = kEmpty;
    if (p < end) {
      const uint64_t* r = s.window + c * W;
      const int64_t v = (int64_t)(r[0] & 0xffffffffull);
      const int m = (int)r[1];
      vx[h] = v;
      lox[h] = (uint32_t)(r[0] >> 32);
      mx[h] = m;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int e = j * 32 + lane;
        if (e < m && in_bounds((uint64_t)v < (uint64_t)a.n, a.err)) kx[h][j] = a.keys_in[v * a.R + e];
        if (PREC == 1 && e < m) ax[h][j] = a.P.aux[key_id(kx[h][j])];
      }
      const int k = __popc(__ballot_sync(0xffffffffu, lane < m && !key_old(kx[h][0]))) +
                    __popc(__ballot_sync(0xffffffffu, lane + 32 < m && !key_old(kx[h][1])));
      if (lane == 0) {
        s.cv[c] = v;
        s.cm[c] = m;
        s.ck[c] = k;
        s.cnp[c] = k * (m - 1) - k * (k - 1) / 2;
        s.cnt_[c] = (PREC == 1) ? tiles_of(m, k) : 0;
        s.cns[c] = min(k, m - 1) + min(k, max(0, m - 33));
      }
    } else if (lane == 0) {
      s.cv[c] = -1;
    }
  }
  __syncthreads();
  if (warp == 0) {  // take the longest prefix of candidates that fits every budget
    const bool have = lane < BV && s.cv[lane] >= 0;
    int m = have ? s.cm[lane] : 0, np = have ? s.cnp[lane] : 0, nt = have ? s.cnt_[lane] : 0;
    int ns = have ? s.cns[lane] : 0;
    int cp = (have && np > 0) ? m : 0;
    int im = m, inp = np, inti = nt, icp = cp, ins = ns;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int a1 = __shfl_up_sync(0xffffffffu, im, o), a2 = __shfl_up_sync(0xffffffffu, inp, o);
      const int a3 = __shfl_up_sync(0xffffffffu, inti, o), a4 = __shfl_up_sync(0xffffffffu, icp, o);
      const int a5 = __shfl_up_sync(0xffffffffu, ins, o);
      if (lane >= o) {
        im += a1;
        inp += a2;
        inti += a3;
        icp += a4;
        ins += a5;
      }
    }
    const bool fits = have && (lane == 0 || (im <= BR && inp <= BP && inti <= BT && ins <= seg_budget<PREC>()));
    const int nb = __popc(__ballot_sync(0xffffffffu, fits));  // the fitting lanes form a prefix
    if (lane < nb) {
      B.v[lane] = s.cv[lane];
      B.m[lane] = m;
      B.k[lane] = s.ck[lane];
      B.np[lane] = np;
      B.rowbase[lane + 1] = im;
      B.pairbase[lane + 1] = inp;
      B.tilebase[lane + 1] = inti;
      B.segbase[lane + 1] = ins;
    }
    if (lane == 0) {
      B.rowbase[0] = B.pairbase[0] = B.tilebase[0] = B.segbase[0] = 0;
      B.nb = nb;
    }
    if (nb > 0 && lane == nb - 1) {
      B.nent = im;
      B.ncopy = icp;
      B.npairs = inp;
      B.ntiles = inti;
      B.nseg = ins;
      B.nchunks = inp > 0 ? (a.P.d + Prec<PREC>::DC - 1) / Prec<PREC>::DC : 0;
    }
    if (nb == 0 && lane == 0) {
      B.nent = B.ncopy = B.npairs = B.ntiles = B.nseg = B.nchunks = 0;
    }
  }
  __syncthreads();
  const int nb = B.nb;
  const uint64_t head = hash_head(a.seed, (uint64_t)a.t1, (uint64_t)a.t2);  // visit-order hash, uniform part
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int vb = warp + h * JW;
    if (vb >= nb) continue;
    const int64_t v = vx[h];
    const int m = mx[h], k = B.k[vb], rb = B.rowbase[vb];
    uint64_t hk[2];
    uint32_t id[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int e = j * 32 + lane;
      id[j] = key_id(kx[h][j]);
      hk[j] = (a.order == 0)   ? hash_tail(head, (uint64_t)(v - lox[h]),
                                              (uint64_t)(id[j] - lox[h]))
              : (a.order == 1) ? (uint64_t)e
                               : (uint64_t)(m - 1 - e);
    }
    int p[2] = {0, 0};
    for (int f = 0; f < m; ++f) {
      const uint64_t hf = __shfl_sync(0xffffffffu, (f < 32) ? hk[0] : hk[1], f & 31);
      const uint32_t idf = __shfl_sync(0xffffffffu, (f < 32) ? id[0] : id[1], f & 31);
#pragma unroll
      for (int j = 0; j < 2; ++j) p[j] += (hf < hk[j]) || (hf == hk[j] && idf < id[j]);
    }
    // new entries by pi position
    uint32_t nlo = 0, nhi = 0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int e = j * 32 + lane;
      if (e < m && !key_old(kx[h][j])) {
        if (p[j] < 32) nlo |= 1u << p[j];
        else nhi |= 1u << (p[j] - 32);
      }
    }
    nlo = __reduce_or_sync(0xffffffffu, nlo);
    nhi = __reduce_or_sync(0xffffffffu, nhi);
    const uint64_t newm = ((uint64_t)nhi << 32) | nlo;
    const uint64_t valid = (m >= 64) ? ~0ull : ((1ull << m) - 1ull);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int e = j * 32 + lane;
      if (e >= m) continue;
      const int pp = p[j];
      const uint64_t lo = bits_below(pp);
      const int row = ((newm >> pp) & 1ull) ? __popcll(newm & lo) : k + __popcll(~newm & valid & lo);
      B.rid[rb + row] = (int32_t)id[j];
      B.rpos[rb + row] = (uint8_t)pp;
      B.rvb[rb + row] = (uint8_t)vb;
      if (row < k) B.roff[rb + row] = B.pairbase[vb] + row * (m - 1) - row * (row - 1) / 2;
      B.pkey[rb + pp] = kx[h][j];
      B.pid[rb + pp] = (int32_t)id[j];
      B.prow[rb + pp] = (uint8_t)row;
      B.pslot[rb + pp] = (uint8_t)e;
      if (PREC == 1) {
        B.rnrm[rb + row] = ax[h][j].x;
        B.rdq[rb + row] = ax[h][j].y;
      }
    }
    {  // row segments of the new rows i = lane, lane + 32: one if it has a pair, two past 32
      int cnt[2], ex[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int i = j * 32 + lane, len = m - 1 - i;
        cnt[j] = i < k ? (len >= 1) + (len > 32) : 0;
      }
      int inc0 = cnt[0], inc1 = cnt[1];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y0 = __shfl_up_sync(0xffffffffu, inc0, o), y1 = __shfl_up_sync(0xffffffffu, inc1, o);
        if (lane >= o) {
          inc0 += y0;
          inc1 += y1;
        }
      }
      ex[0] = inc0 - cnt[0];
      ex[1] = __shfl_sync(0xffffffffu, inc0, 31) + inc1 - cnt[1];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int i = j * 32 + lane;
        const int sb = B.segbase[vb] + ex[j];
        if (cnt[j] > 0) B.seg[sb] = (uint16_t)(((rb + i) << 8) | (i + 1));
        if (cnt[j] > 1) B.seg[sb + 1] = (uint16_t)(((rb + i) << 8) | (i + 33));
      }
    }
    if (PREC == 1) {  // this vertex's mma tiles, lane (I, J) = (lane / 8, lane % 8)
      const int KI = (k + 15) >> 4, NJ = (m + 7) >> 3;
      const int I = lane >> 3, J = lane & 7;
      const bool ok = I < KI && J < NJ && J * 8 + 7 > I * 16;
      const unsigned bm = __ballot_sync(0xffffffffu, ok);
      if (ok) B.tiles[B.tilebase[vb] + __popc(bm & lanemask_lt())] = (uint16_t)((vb << 8) | (I << 4) | J);
    }
  }
  __syncthreads();
  if (tid == 0) join_prefetch<PREC>(s, pos + nb, end, a);  // the next batch's candidates
  return nb;
}

// ---- bulk copies of one dimension chunk of a batch's rows (all threads) ------------------
template <int PREC>
__device__ __forceinline__ void join_issue(JoinSmem<PREC>& s, const Batch& B, int chunk, int buf,
                                           const JoinArgs& a) {
  using C = Prec<PREC>;
  const int c0 = chunk * C::DC;
  const int clen = min(C::DC, a.P.d - c0);
  const int cpy = (clen + C::VEC - 1) / C::VEC * C::VEC;
  const uint32_t bytes = (uint32_t)(cpy * sizeof(typename C::T));
  if (threadIdx.x == 0) mbar_expect_tx(&s.bar[buf], (uint32_t)B.ncopy * bytes);
  for (int r = threadIdx.x; r < B.nent; r += JT) {
    if (B.np[B.rvb[r]] == 0) continue;
    const typename C::T* src =
        (PREC == 0) ? reinterpret_cast<const typename C::T*>(a.P.X + (int64_t)B.rid[r] * a.P.ld + c0)
                    : reinterpret_cast<const typename C::T*>(a.P.Xb) + (int64_t)B.rid[r] * a.P.ldb + c0;
    bulk_g2s(&s.rows[buf][r][0], src, bytes, &s.bar[buf]);
  }
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldmatrix_x2(uint32_t (&r)[2], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(a));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_e4m3(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// One k-step of a quantized tile: m16n8k16 over BF16 rows, m16n8k32 over e4m3 rows.  Both
// read 32 bytes of each row per step with the same fragment-to-byte layout, so ldmatrix
// addresses are the same in bytes for the two forms.
template <int PREC>
__device__ __forceinline__ void mma_q(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  if constexpr (PREC == 2)
    mma_e4m3(c, a, b);
  else
    mma_bf16(c, a, b);
}
// FP8 form: the power-of-two scale of a quantized row, from the low byte of its residual.
__device__ __forceinline__ float q_scale(float rdq) { return __uint_as_float((__float_as_uint(rdq) & 0xffu) << 23); }

// Bound on |D_tile(i,j) - D_fp32(i,j)| for the BF16 form (Higham-style: u = 2^-23 covers a
// truncating accumulator; gamma_K = K u / (1 - K u)).  L2SQ:
//   arithmetic  (gamma_d + 2u) (sqrt(n_i) + sqrt(n_j))^2
//   quantization (e_i + e_j) (2 sqrt(D + arith) + e_i + e_j)
//   FP32 reference rounding (d + 3) u (D + the two above)
// IP: (gamma_d + 2u) sqrt(n_i n_j) + 2u |D| + e_i sqrt(n_j) + e_j sqrt(n_i) + e_i e_j, plus the
// same reference term.  n = squared norm of the BF16 row, e = ||x - bf16(x)||.
template <int METRIC>
__device__ __forceinline__ float bf16_bound(float D, float ni, float nj, float ei, float ej, int d) {
  const float u = 1.1920929e-07f;  // 2^-23
  const float g = (float)d * u / (1.0f - (float)d * u);
  const float si = sqrtf(fmaxf(ni, 0.0f)), sj = sqrtf(fmaxf(nj, 0.0f));
  float ar, qz, base;
  if (METRIC == 0) {
    ar = (g + 2.0f * u) * (si + sj) * (si + sj);
    const float e = ei + ej;
    qz = e * (2.0f * sqrtf(fmaxf(D, 0.0f) + ar) + e);
    base = fmaxf(D, 0.0f);
  } else {
    ar = (g + 2.0f * u) * si * sj + 2.0f * u * fabsf(D);
    qz = ei * sj + ej * si + ei * ej;
    base = fabsf(D) + si * sj;
  }
  const float tot = ar + qz;
  return (tot + ((float)d + 3.0f) * u * (base + tot)) * 1.0001f;
}

template <int METRIC, int PREC>
__global__ void __launch_bounds__(JT) rnd_join_kernel(JoinArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  JoinSmem<PREC>& s = *reinterpret_cast<JoinSmem<PREC>*>(smem_raw);
  using C = Prec<PREC>;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the pools of the last size class: records [0, cnt) of that class
  const int64_t cnt = a.list_n[3];
  const int64_t per = (cnt + gridDim.x - 1) / gridDim.x;
  int64_t pos = (int64_t)blockIdx.x * per;
  const int64_t end = min(cnt, pos + per);
  if (pos >= end || *(volatile int32_t*)a.err) return;  // nothing to do, or the round has failed
  if (tid == 0) {
    mbar_init(&s.bar[0], 1);
    mbar_init(&s.bar[1], 1);
    mbar_init(&s.wbar, 1);
    fence_mbar_init();
    s.red_next = s.red_end = 0;
  }
  for (int t = tid; t < BR; t += JT) {
    s.fire[t] = 0;
    s.closer[t] = 0;
  }
  if (tid < BV) s.fcol[tid] = 0;
  __syncthreads();
  bool exact = false;
  if (PREC == 1) {
    const unsigned fl = a.P.qflags[0];
    const float mxa = __uint_as_float(a.P.qflags[1]);
    exact = (fl == 0u) && ((double)a.P.d * (double)mxa * (double)mxa < 16777216.0);
  }
  const int R = a.R;
  uint32_t ph[2] = {0u, 0u};
  long long st_vert = 0, st_rows = 0, st_pairs = 0, st_fired = 0, st_check = 0;

  uint32_t wph = 0;
  if (tid == 0) join_prefetch<PREC>(s, pos, end, a);
  {
    const int nb0 = join_form_batch<PREC>(s, s.bt[0], pos, end, wph, a);
    if (nb0 < 0) return;
    pos += nb0;
  }
  if (s.bt[0].nchunks > 0) join_issue<PREC>(s, s.bt[0], 0, 0, a);
  int bcur = 0, ccur = 0, sbuf = 0;

  float4 facc[PREC == 0 ? SPW : 1];
  float cacc[PREC == 1 ? TPW : 1][4];

  for (;;) {
    Batch& B = s.bt[bcur];
    // ---- next stage: the next chunk of this batch, or the next batch ----------------------
    int bnext = bcur, cnext = ccur + 1;
    bool have_next = true;
    if (cnext >= B.nchunks) {
      if (pos < end) {
        bnext = bcur ^ 1;
        cnext = 0;
        const int nbn = join_form_batch<PREC>(s, s.bt[bnext], pos, end, wph, a);
        if (nbn < 0) {  // let the current stage's copies land before leaving
          if (B.nchunks > 0) mbar_wait(&s.bar[sbuf], ph[sbuf], kWaitLimit);
          return;
        }
        pos += nbn;
      } else {
        have_next = false;
      }
    }
    if (have_next && s.bt[bnext].nchunks > 0) join_issue<PREC>(s, s.bt[bnext], cnext, sbuf ^ 1, a);

    // ---- current stage: one dimension chunk of every tile of the batch ------------------
    if (B.nchunks > 0) {
      const bool ok = mbar_wait(&s.bar[sbuf], ph[sbuf], kWaitLimit);
      ph[sbuf] ^= 1u;
      if (__syncthreads_or(!ok)) {
        // a bounded wait gave up: report, let in-flight copies land, and stop.
        if (tid == 0) atomicExch(a.err, kErrTimeout);
        if (!ok) mbar_wait(&s.bar[sbuf], ph[sbuf] ^ 1u, kWaitLimit);
        if (have_next && s.bt[bnext].nchunks > 0) mbar_wait(&s.bar[sbuf ^ 1], ph[sbuf ^ 1], kWaitLimit);
        return;
      }
      const int c0 = ccur * C::DC;
      const int clen = min(C::DC, a.P.d - c0);
      const bool last = (ccur + 1 == B.nchunks);
      if (PREC == 0) {
        const float* rows = reinterpret_cast<const float*>(&s.rows[sbuf][0][0]);
        const int full4 = clen & ~3, rem = clen & 3;
#pragma unroll
        for (int t = 0; t < SPW; ++t) {
          const int sidx = warp + t * JW;
          if (sidx < B.nseg) {
            const int code = B.seg[sidx];
            const int row = code >> 8, j = (code & 255) + lane;
            const int vb = B.rvb[row], rb = B.rowbase[vb];
            if (j < B.m[vb]) {
              const float* ra = rows + row * C::RS;
              const float* rbp = rows + (rb + j) * C::RS;
              if (ccur == 0) facc[t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
              float4 acc = facc[t];
              for (int u = 0; u < full4; u += 4)
                dist_step4<METRIC>(acc, *reinterpret_cast<const float4*>(ra + u),
                                   *reinterpret_cast<const float4*>(rbp + u));
              if (rem)
                dist_step4<METRIC>(acc, mask4(*reinterpret_cast<const float4*>(ra + full4), rem),
                                   mask4(*reinterpret_cast<const float4*>(rbp + full4), rem));
              facc[t] = acc;
              if (last) s.pd[B.roff[row] + (j - (row - rb) - 1)] = dist_finish4<METRIC>(acc);
            }
          }
        }
      } else {
        const __nv_bfloat16* rows = reinterpret_cast<const __nv_bfloat16*>(&s.rows[sbuf][0][0]);
        const int ksteps = (clen + 15) >> 4;
#pragma unroll
        for (int t = 0; t < TPW; ++t) {
          const int ti = warp + t * JW;
          if (ti < B.ntiles) {
            const int code = B.tiles[ti];
            const int vb = code >> 8, I = (code >> 4) & 15, J = code & 15;
            const int rb = B.rowbase[vb];
            if (ccur == 0) cacc[t][0] = cacc[t][1] = cacc[t][2] = cacc[t][3] = 0.0f;
            const int ra = min(rb + I * 16 + (lane & 15), BRA - 1);
            const int rbb = min(rb + J * 8 + (lane & 7), BRA - 1);
            const __nv_bfloat16* pa = rows + ra * C::RS + ((lane >> 4) << 3);
            const __nv_bfloat16* pb = rows + rbb * C::RS + (((lane >> 3) & 1) << 3);
            for (int ks = 0; ks < ksteps; ++ks) {
              uint32_t fa[4], fb[2];
              ldmatrix_x4(fa, pa + ks * 16);
              ldmatrix_x2(fb, pb + ks * 16);
              mma_bf16(cacc[t], fa, fb);
            }
            if (last) {
              const int g = lane >> 2, tg = lane & 3;
              const int m = B.m[vb], k = B.k[vb];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int i = I * 16 + g + ((e >> 1) << 3);
                const int j = J * 8 + 2 * tg + (e & 1);
                if (i < k && j > i && j < m) {
                  const float gij = cacc[t][e];
                  float Dt;
                  if (METRIC == 0)
                    Dt = __fadd_rn(__fsub_rn(B.rnrm[rb + i], gij), __fsub_rn(B.rnrm[rb + j], gij));
                  else
                    Dt = __fsub_rn(1.0f, gij);
                  s.pd[B.roff[rb + i] + (j - i - 1)] = Dt;
                }
              }
            }
          }
        }
      }
    }
    __syncthreads();

    // ---- last chunk done: prune and emit the whole batch --------------------------------
    if (ccur + 1 >= B.nchunks) {
      const int nb = B.nb;
      // fire bits, one warp per row segment
      for (int sidx = warp; sidx < B.nseg; sidx += JW) {
        const int code = B.seg[sidx];
        const int row = code >> 8, j = (code & 255) + lane;
        const int vb = B.rvb[row], rb = B.rowbase[vb];
        const int i = row - rb;
        if (j < B.m[vb]) {
          const int q = B.roff[row] + (j - i - 1);
          const int pa = B.rpos[rb + i], pb = B.rpos[rb + j];
          const int lo = min(pa, pb), hi = max(pa, pb);
          const float dab = s.pd[q];
          const float dva = key_dist(B.pkey[rb + pa]), dvb = key_dist(B.pkey[rb + pb]);
          const float mx = fmaxf(dva, dvb);
          bool fire = dab < mx;
          if (PREC == 1 && !exact) {
            const float tol =
                bf16_bound<METRIC>(dab, B.rnrm[rb + i], B.rnrm[rb + j], B.rdq[rb + i], B.rdq[rb + j], a.P.d);
            if (fabsf(dab - mx) <= tol) {  // re-decide with the canonical FP32 d(a,b)
              const float* xa = a.P.X + (int64_t)B.pid[rb + pa] * a.P.ld;
              const float* xb = a.P.X + (int64_t)B.pid[rb + pb] * a.P.ld;
              const float d_ab = row_dist<METRIC>(xa, xb, a.P.d);
              fire = d_ab < mx;
              s.pd[q] = d_ab;
              ++st_check;
            }
          }
          if (fire) {
            atomicOr(reinterpret_cast<unsigned long long*>(&s.fire[rb + hi]), 1ull << lo);
            atomicOr(reinterpret_cast<unsigned long long*>(&s.fcol[vb]), 1ull << hi);
            if ((B.pkey[rb + lo] >> 1) < (B.pkey[rb + hi] >> 1))
              atomicOr(reinterpret_cast<unsigned long long*>(&s.closer[rb + hi]), 1ull << lo);
          }
        }
      }
      __syncthreads();
      if (warp == 0) {  // one chain per vertex, in parallel
        int ndead = 0;
        if (lane < nb) {
          const int m = B.m[lane], rb = B.rowbase[lane];
          uint64_t alive = (m >= 64) ? ~0ull : ((1ull << m) - 1ull);
          uint64_t cols = s.fcol[lane];
          // only columns with a fire bit can change anything; in column b the live firing
          // partners are taken in pi order: farther ones are absorbed by b until the first
          // closer one, which makes b the far side
          while (cols) {
            const int b = __ffsll((long long)cols) - 1;
            cols &= cols - 1;
            const uint64_t cand = s.fire[rb + b] & alive;
            uint64_t kill = cand;
            uint8_t f = 0xFF;
            const uint64_t x = cand & s.closer[rb + b];
            if (x) {
              f = (uint8_t)(__ffsll((long long)x) - 1);
              kill = cand & bits_below(f);
              alive &= ~(1ull << b);
            }
            alive &= ~kill;
            s.colkill[rb + b] = kill;
            s.colf[rb + b] = f;
          }
          s.alive[lane] = alive;
          s.smask[lane] = 0;
          ndead = m - __popcll(alive);
          if (B.np[lane] > 0) {
            st_vert += 1;
            st_rows += m;
            st_pairs += B.np[lane];
          }
          st_fired += ndead;
        }
        if (a.emit_redirects) {  // one reservation per batch
          int incl = ndead;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
          }
          const int total = __shfl_sync(0xffffffffu, incl, 31);
          // fill the current chunk to its end, then continue in a fresh one (a batch has at
          // most BV * 63 <= RED_CHUNK redirects), so only each CTA's last chunk has a tail
          const unsigned long long base = s.red_next, end = s.red_end;
          unsigned long long b1 = base, next = base + (unsigned long long)total;
          int avail = total;
          if (next > end) {
            avail = (int)(end - base);
            unsigned long long nbase = 0;
            if (lane == 0) nbase = atomicAdd(a.red_n, (unsigned long long)RED_CHUNK);
            b1 = __shfl_sync(0xffffffffu, nbase, 0);
            next = b1 + (unsigned long long)(total - avail);
            if (lane == 0) s.red_end = b1 + RED_CHUNK;
          }
          if (lane == 0) {
            s.red_next = next;
            s.red_b0 = base;
            s.red_b1 = b1;
            s.red_avail = avail;
          }
          if (lane < nb) s.deadrank[lane] = incl - ndead;
        }
      }
      __syncthreads();
      // emit, one thread per pool entry of the batch (indexed by rowbase + pi position)
      const int t = tid;
      int ev = -1, ep = 0;
      uint64_t ealive = 0;
      if (t < B.nent) {
        ev = B.rvb[t];  // entries and rows share the batch index range
        ep = t - B.rowbase[ev];
        ealive = s.alive[ev];
        if ((ealive >> ep) & 1ull)
          atomicOr(reinterpret_cast<unsigned long long*>(&s.smask[ev]), 1ull << B.pslot[t]);
      }
      __syncthreads();
      if (ev >= 0) {
        const int rb = B.rowbase[ev];
        const int64_t v = B.v[ev];
        if ((ealive >> ep) & 1ull) {
          const int slot = B.pslot[t];
          a.keys_out[v * R + __popcll(s.smask[ev] & bits_below(slot))] = B.pkey[t] | 1ull;
        } else if (a.emit_redirects) {
          const int m = B.m[ev];
          const uint64_t valid = (m >= 64) ? ~0ull : ((1ull << m) - 1ull);
          const uint64_t cols = s.fcol[ev];
          int cpos = ((cols >> ep) & 1ull) ? s.colf[t] : 0xFF;
          if (cpos == 0xFF) {  // absorbed by a later column b: the one whose kill mask holds it
            uint64_t later = cols & ~bits_below(ep + 1);
            while (later) {
              const int b = __ffsll((long long)later) - 1;
              later &= later - 1;
              if ((s.colkill[rb + b] >> ep) & 1ull) {
                cpos = b;
                break;
              }
            }
          }
          const int ri = B.prow[rb + cpos], rj = B.prow[t];
          const int i = min(ri, rj), j = max(ri, rj);
          const float dd = s.pd[B.roff[rb + i] + (j - i - 1)];
          const int32_t tgt = B.pid[rb + cpos];
          const int g = s.deadrank[ev] + __popcll(~ealive & valid & bits_below(ep));
          const unsigned long long slot =
              g < s.red_avail ? s.red_b0 + (unsigned long long)g : s.red_b1 + (unsigned long long)(g - s.red_avail);
          if (in_bounds(slot < (unsigned long long)a.red_cap && (uint64_t)tgt < (uint64_t)a.n, a.err)) {
            a.red_tgt[slot] = tgt;
            a.red_key[slot] = make_key(dd, (uint32_t)B.pid[t], 0u);
            atomicAdd(&a.count[tgt], 1);
          }
        }
      }
      for (int u = tid; u < nb * R; u += JT) {
        const int vb = u / R, jj = u - vb * R;
        if (jj >= __popcll(s.alive[vb])) a.keys_out[B.v[vb] * R + jj] = kEmpty;
      }
      if (tid < nb) a.deg_out[B.v[tid]] = __popcll(s.alive[tid]);
      for (int q = tid; q < B.nent; q += JT) {
        s.fire[q] = 0;
        s.closer[q] = 0;
      }
      if (tid < nb) s.fcol[tid] = 0;
      __syncthreads();
    }
    if (!have_next) break;
    bcur = bnext;
    ccur = cnext;
    sbuf ^= 1;
  }
  __syncthreads();
  if (a.emit_redirects)
    for (unsigned long long i = s.red_next + tid; i < s.red_end; i += JT) a.red_tgt[i] = -1;
  if (a.stats && warp == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      st_vert += __shfl_xor_sync(0xffffffffu, st_vert, o);
      st_rows += __shfl_xor_sync(0xffffffffu, st_rows, o);
      st_pairs += __shfl_xor_sync(0xffffffffu, st_pairs, o);
      st_fired += __shfl_xor_sync(0xffffffffu, st_fired, o);
    }
    if (lane == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[0]), (unsigned long long)st_vert);
      atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[1]), (unsigned long long)st_rows);
      atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[2]), (unsigned long long)st_pairs);
      atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[3]), (unsigned long long)st_fired);
    }
  }
  if (a.stats && PREC == 1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) st_check += __shfl_xor_sync(0xffffffffu, st_check, o);
    if (lane == 0 && st_check) atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[7]), (unsigned long long)st_check);
  }
}

template <int METRIC, int PREC>
cudaError_t launch_join_t(const JoinArgs& a, cudaStream_t st, const char* name, bool setup_only = false) {
  const size_t smem = sizeof(JoinSmem<PREC>);
  static KernelSetup ks;
  auto kern = rnd_join_kernel<METRIC, PREC>;
  int per_sm = 0;
  cudaError_t e = setup_kernel(ks, kern, JT, smem, smem, &per_sm);
  if (e != cudaSuccess || setup_only) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t blocks = std::min<int64_t>(std::min<int64_t>(std::max<int64_t>(a.n, 1), (int64_t)sm_count() * per_sm),
                                            kMaxJoinGrid);
  ProfScope ps(name, st);
  kern<<<(unsigned)blocks, JT, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

// =====================================================================================
// rnd_join for pools of at most 32 entries: a warp takes one vertex of 17..32 entries,
// two of 9..16 or four of at most 8 at a time (lane groups of VW = 32, 16 or 8 lanes),
// end to end, with no block-wide barrier.
//   order    bitonic sort of (h(seed,t1,t2,v,id), id) (or the key order) within each
//            lane group -> pi
//   gather   one bulk copy per row (lane s: the row of storage slot s; rows hold the new
//            entries first, then the old ones, each part in slot order), completing on the
//            warp's own mbarrier, in chunks of 128 dimensions; the first chunk's copies are
//            issued before the visit order is sorted
//   tile     BF16 / FP8: mma.sync m16n8k16 / m16n8k32 tiles (six for one vertex, the four
//            diagonal ones for lane groups), partial dot products kept between chunks,
//            fire decisions taken from the accumulators; FP32 (d <= 128): each group's
//            lanes take its pairs one by one with the canonical four-accumulator distance;
//            a pair that fires sets its bit in the later position's mask (shared atomic)
//   prune    the outcome of the group's sequential mask chain as a fixed point, one column
//            (pi position) per lane: each lane learns whether its entry survives and, if
//            not, its absorber
//   emit     survivors in key order in place; redirects into per-warp slot chunks
// =====================================================================================
namespace {

constexpr int WW = 4;      // warps per CTA
constexpr int WM = 32;     // pool entries a warp holds at a time
constexpr int WRED = 256;  // redirect slots a warp reserves at a time
constexpr int WDC = 128;   // dimensions per gathered chunk
constexpr int WRQ = 128;   // re-decisions a warp queues per item (more are taken in place)

template <int PREC>
struct WPrec;
template <>
struct WPrec<0> {
  using T = float;
  static constexpr int RS = WDC + 4;
  static constexpr int VEC = 4;
  static constexpr int RSB = RS * 4;    // bytes per staged row
  static constexpr int GB = 4 * RSB;    // bytes per four rows (rows are contiguous: no gather4)
};
template <>
struct WPrec<1> {
  using T = __nv_bfloat16;
  static constexpr int RS = WDC + 8;
  static constexpr int VEC = 16;
  static constexpr int RSB = RS * 2;                 // 272 bytes: one gather4 box row
  static constexpr int GB = (4 * RSB + 127) & ~127;  // four rows of one gather4, 128-byte aligned
};
template <>
struct WPrec<2> {
  using T = uint8_t;                  // e4m3 bytes
  static constexpr int RS = WDC + 16; // 144-byte rows, as for BF16 in bytes per 64 columns
  static constexpr int VEC = 32;      // whole k32 steps (32 bytes)
  static constexpr int RSB = RS;
  static constexpr int GB = (4 * RSB + 127) & ~127;
};

// The staged rows of a warp: row r (group base + local row) at (r / 4) * GS + (r % 4) * RSB
// bytes.  With one bulk copy per row GS = 4 * RSB: rows are contiguous, and the 8 rows of an
// ldmatrix phase (RSB / 16 odd) hit distinct banks.  With gather4 copies (TMA) GS = GB, so
// that every four rows, the destination of one copy, start on a 128-byte boundary; rows r and
// r + 4 then share banks (a 2-way conflict in every ldmatrix phase).
template <int PREC, bool TMA>
struct WLayout {
  static constexpr int GS = TMA ? WPrec<PREC>::GB : 4 * WPrec<PREC>::RSB;
};
template <int PREC, bool TMA>
struct __align__(128) WarpSlot {
  unsigned char rowb[(WM / 4) * WLayout<PREC, TMA>::GS];
  int32_t rid[WM];              // by row: the point id whose row is staged there
  float pd[WM * (WM - 1) / 2];  // group g's pairs from g * VW (VW - 1) / 2
  int32_t pid[WM];              // by position: group base + local pi position
  uint32_t fire[WM];            // by position; bits: earlier local positions that fired with it
  float2 rnd[WM];               // by row: (squared norm of the BF16 row, recorded dist to v)
  float rdq[WM];                // by row: norm of the quantization residual
  int32_t roff[WM];             // by row: local index of the first pair of new row i
  uint8_t rpos[WM], prow[WM];   // local position of a row / local row of a position
  uint8_t src[WM];              // by position (group base + position): local storage slot
  uint8_t kil[WM];              // by position: the column that absorbed it (chain rounds)
  uint16_t rq[WRQ];             // pairs (row i << 5 | row j) whose decision is re-taken in FP32
  int32_t nrq;                  // queued re-decisions of the item
  int32_t gk[4], gm[4];         // per group: new entries, entries
  uint64_t bar;
  unsigned long long red_next, red_end;
};

template <int PREC, bool TMA>
__device__ __forceinline__ typename WPrec<PREC>::T* wrow(WarpSlot<PREC, TMA>& s, int r) {
  return reinterpret_cast<typename WPrec<PREC>::T*>(s.rowb + (r >> 2) * WLayout<PREC, TMA>::GS +
                                                    (r & 3) * WPrec<PREC>::RSB);
}

// TMA gather of four rows (y0..y3) of a 2-D tensor, columns x .. x + box - 1, into four
// consecutive box rows at dst (128-byte aligned); completion counted on `bar` (4 x box bytes,
// out-of-range elements read as zero).  x times the element size is a multiple of 16 bytes.
__device__ __forceinline__ void tma_gather4(void* dst, const TmaMap* map, int x, int y0, int y1, int y2, int y3,
                                            uint64_t* bar) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(d),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(b)
      : "memory");
}

__device__ __forceinline__ uint32_t lanes_below32(int p) { return p == 0 ? 0u : (0xffffffffu >> (32 - p)); }
__device__ __forceinline__ uint32_t low_bits32(int w) { return w >= 32 ? 0xffffffffu : ((1u << w) - 1u); }

// One work item: the vertices of lane group lane / VW; class 2 items first (one vertex of
// 17..32 entries), then class 1 (two of 9..16), then class 0 (four of at most 8).
struct WItem {
  int cls;
  int m;
  uint32_t lo;  // first id of the vertex's build
  int64_t v;
  uint64_t key;
};

// The work record of item w for this lane's group: the vertex word and m (m = 0: the group
// has no vertex).  cnt: records per class 0..2.  Class 2 items come first (one vertex of
// 17..32 entries per warp), then class 1 (two of 9..16), then class 0 (four of at most 8).
struct WRec {
  ulonglong2 r;
  int cls;
};
__device__ __forceinline__ void warp_rec_load(const JoinArgs& a, int64_t w, int64_t n2, int64_t n1, const int cnt[3],
                                              int lane, WRec& x) {
  int cls;
  int64_t it;
  if (w < n2) {
    cls = 2;
    it = w;
  } else if (w < n2 + n1) {
    cls = 1;
    it = w - n2;
  } else {
    cls = 0;
    it = w - n2 - n1;
  }
  const int lw = 3 + cls;  // log2 of the group width
  const int64_t rr = it * (32 >> lw) + (lane >> lw);
  x.cls = cls;
  x.r = make_ulonglong2(0ull, 0ull);
  if (rr < (int64_t)(cls == 2 ? cnt[2] : cls == 1 ? cnt[1] : cnt[0])) x.r = *reinterpret_cast<const ulonglong2*>(a.rec[cls] + rr * a.rec_w[cls]);
}
// The item of a loaded record: this lane's pool key (storage slot lane % group width).
__device__ __forceinline__ void warp_item_of(const JoinArgs& a, const WRec& r, int lane, WItem& x) {
  x.cls = r.cls;
  x.m = (int)r.r.y;
  x.v = x.m > 0 ? (int64_t)(r.r.x & 0xffffffffull) : -1;
  x.lo = (uint32_t)(r.r.x >> 32);
  x.key = kEmpty;
  const int gl = lane & ((8 << r.cls) - 1);
  if (gl < x.m && in_bounds((uint64_t)x.v < (uint64_t)a.n, a.err)) x.key = a.keys_in[x.v * a.R + gl];
}

// TMA: quantized rows staged by gather4 copies through a.rows_map (else one bulk copy per row)
template <int METRIC, int PREC, bool TMA>
__global__ void __launch_bounds__(WW * 32, 4) rnd_join_warp_kernel(const __grid_constant__ JoinArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using C = WPrec<PREC>;
  using T = typename C::T;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // the warp slots start on a 128-byte boundary (the launch adds 128 bytes for this)
  unsigned char* const sbase = smem_raw + ((128u - ((uint32_t)__cvta_generic_to_shared(smem_raw) & 127u)) & 127u);
  WarpSlot<PREC, TMA>& s = reinterpret_cast<WarpSlot<PREC, TMA>*>(sbase)[wid];
  static_assert(!TMA || PREC >= 1, "gather4 copies are for quantized rows");
  const int cnt[3] = {a.list_n[0], a.list_n[1], a.list_n[2]};
  const int64_t n2 = cnt[2], n1 = (cnt[1] + 1) / 2, n0 = (cnt[0] + 3) / 4;
  const int64_t items = n2 + n1 + n0;
  const int64_t gw = (int64_t)blockIdx.x * WW + wid, GW = (int64_t)gridDim.x * WW;
  // The counters (a.stats) of the CTA's warps are added up in shared memory; the last warp
  // to leave adds them to the global counters: one atomic per CTA and counter, not per warp
  // (the counters are a few addresses that every CTA hits when the launch ends).
  __shared__ unsigned long long s_st[5];
  __shared__ int s_left;
  if (threadIdx.x < 5) s_st[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) s_left = WW;
  __syncthreads();
  auto leave = [&](long long c0, long long c1, long long c2, long long c3, long long c4) {  // lane 0
    if (!a.stats) return;
    if (c0) atomicAdd(&s_st[0], (unsigned long long)c0);
    if (c1) atomicAdd(&s_st[1], (unsigned long long)c1);
    if (c2) atomicAdd(&s_st[2], (unsigned long long)c2);
    if (c3) atomicAdd(&s_st[3], (unsigned long long)c3);
    if (c4) atomicAdd(&s_st[4], (unsigned long long)c4);
    __threadfence_block();
    if (atomicSub(&s_left, 1) == 1) {  // the CTA's last warp
      __threadfence_block();
      unsigned long long* g = reinterpret_cast<unsigned long long*>(a.stats);
      const int slot[5] = {0, 1, 2, 3, 7};
#pragma unroll
      for (int q = 0; q < 5; ++q)
        if (s_st[q]) atomicAdd(&g[slot[q]], s_st[q]);
    }
  };
  if (gw >= items || *(volatile int32_t*)a.err) {  // nothing to do, or the round has failed
    if (lane == 0) leave(0, 0, 0, 0, 0);
    return;
  }
  const int R = a.R, d = a.P.d;
  const int nchd = (d + WDC - 1) / WDC;
  const uint64_t head = hash_head(a.seed, (uint64_t)a.t1, (uint64_t)a.t2);  // visit-order hash, uniform part
  if (lane == 0) {
    mbar_init(&s.bar, 1);
    fence_mbar_init();
    s.red_next = s.red_end = 0;
  }
  __syncwarp();
  bool exact = false;
  if (PREC >= 1) {
    const unsigned fl = a.P.qflags[0];
    const float mxa = __uint_as_float(a.P.qflags[1]);
    exact = (fl == 0u) && ((double)d * (double)mxa * (double)mxa < 16777216.0);
  }
  uint32_t phb = 0u;  // mbarrier phase
  bool inflight = false;
  int st_vert = 0, st_rows = 0, st_pairs = 0, st_fired = 0, st_check = 0;  // per lane; summed at the end

  // Items below S go to the warps in turn (warp gw takes gw, gw + GW, ...); the last ones,
  // S, S + 1, ..., come from a device work queue in the order warps ask, which evens out the
  // end of the launch without an atomic per item.  Loads are pipelined so that no item waits
  // for memory: when item w starts, the pool keys of the next item w1 (whose record arrived
  // during item w - 1) and the record of the item after, w2, are requested; a queue ticket is
  // asked one item before it is needed.
  const int64_t S = items > 5 * GW ? items - 4 * GW : (items < GW ? items : GW);
  WItem nx;
  WRec nrec;
  warp_rec_load(a, gw, n2, n1, cnt, lane, nrec);
  warp_item_of(a, nrec, lane, nx);
  unsigned int tq = 0;
  int64_t wnext = gw + GW;
  if (wnext >= S) {
    if (lane == 0) tq = atomicAdd(a.work_q, 1u);
    wnext = S + (int64_t)__shfl_sync(0xffffffffu, tq, 0);
  }
  if (wnext < items) {
    warp_rec_load(a, wnext, n2, n1, cnt, lane, nrec);
    if (lane == 0 && wnext + GW >= S) tq = atomicAdd(a.work_q, 1u);
  }
  for (int64_t w = gw; w < items;) {
    const WItem cur = nx;
    int64_t w2 = items;
    if (wnext < items) {
      warp_item_of(a, nrec, lane, nx);
      w2 = wnext + GW < S ? wnext + GW : S + (int64_t)__shfl_sync(0xffffffffu, tq, 0);
      if (w2 < items) {
        warp_rec_load(a, w2, n2, n1, cnt, lane, nrec);
        if (lane == 0 && w2 + GW >= S) tq = atomicAdd(a.work_q, 1u);
      }
    }
    // the item's work, compiled once per lane-group width (VW = 32, 16 or 8 lanes per pool),
    // for quantized rows per mode (EX: the tiles are exact, no decision is re-taken), and for
    // rows of one chunk (ONE: d <= WDC) apart from longer rows
    bool quit = false;  // a bounded wait gave up: the warp stops
    auto item = [&](auto vw_tag, auto ex_tag, auto one_tag) {
      constexpr int VW = decltype(vw_tag)::value, lw = VW == 32 ? 5 : (VW == 16 ? 4 : 3), G = 32 / VW;
      constexpr bool EX = decltype(ex_tag)::value, ONE = decltype(one_tag)::value;
      const int g = lane >> lw, gl = lane & (VW - 1), gb = g << lw;
      const uint32_t gmask = low_bits32(VW);
      const int m = cur.m;
      const int64_t v = cur.v;
      const uint64_t keyl = cur.key;
      // ---- rows, and the first chunk's gather in flight while the visit order is sorted ----
      // Rows hold the new entries first, then the old ones, each part in storage-slot order
      // (lane gb + s holds slot s here): the pairs are enumerated over rows (new row i, any
      // later row j), so the order inside each part does not matter.
      const uint32_t validm = low_bits32(m);
      const bool valid_s = gl < m;
      const uint32_t news = (__ballot_sync(0xffffffffu, valid_s && !key_old(keyl)) >> gb) & gmask;
      const int k = __popc(news);
      const int np = k * (m - 1) - k * (k - 1) / 2;
      const uint32_t below_s = lanes_below32(gl);
      const int row_s = ((news >> gl) & 1u) ? __popc(news & below_s) : k + __popc(~news & validm & below_s);
      const uint32_t id_s = key_id(keyl);
      const bool need = valid_s && np > 0 &&  // rows of groups with pairs only
                        in_bounds((uint64_t)id_s < (uint64_t)a.n, a.err);
      const uint32_t needm = __ballot_sync(0xffffffffu, need);
      const int nch = needm ? nchd : 0;
      if (TMA && valid_s) s.rid[gb + row_s] = (int32_t)id_s;
      auto issue = [&](int c) {  // the copies of chunk c, completing on the warp's mbarrier
        const int c0 = c * WDC;
        if constexpr (TMA) {
          // one gather4 per four rows of a group with pairs, issued by the lane of the first of
          // them (rows gb + gl .. gb + gl + 3 = lane .. lane + 3); a group's last copy repeats
          // its first row in the places past m.  Each copies whole boxes: the chunk's columns
          // and, after the last chunk, the first 16 bytes of the row's tail.
          const bool iss = need && (gl & 3) == 0;
          const uint32_t im = __ballot_sync(0xffffffffu, iss);
          if (lane == 0) mbar_expect_tx(&s.bar, (uint32_t)__popc(im) * 4u * (uint32_t)C::RSB);
          inflight = true;
          __syncwarp();
          if (iss) {
            int4 q = *reinterpret_cast<const int4*>(&s.rid[lane]);
            if (gl + 1 >= m) q.y = q.x;
            if (gl + 2 >= m) q.z = q.x;
            if (gl + 3 >= m) q.w = q.x;
            tma_gather4(wrow(s, lane), &a.rows_map, c0, q.x, q.y, q.z, q.w, &s.bar);
          }
          return;
        }
        const int cpy = (min(WDC, d - c0) + C::VEC - 1) / C::VEC * C::VEC;
        // a quantized row's last chunk brings the row's terms (norm^2, residual) along
        const uint32_t bytes = (uint32_t)(cpy * sizeof(T)) + ((PREC >= 1 && (ONE || c + 1 == nchd)) ? (uint32_t)kTailCopy : 0u);
        if (lane == 0) mbar_expect_tx(&s.bar, (uint32_t)__popc(needm) * bytes);
        inflight = true;
        __syncwarp();
        if (need) {
          const T* src = (PREC == 0) ? reinterpret_cast<const T*>(a.P.X + (int64_t)id_s * a.P.ld + c0)
                                     : reinterpret_cast<const T*>(a.P.Xb) + (int64_t)id_s * a.P.ldb + c0;
          bulk_g2s(wrow(s, gb + row_s), src, bytes, &s.bar);
        }
      };
      if (nch > 0) issue(0);

      // ---- visit order: the position of each entry is its rank in (h, id) order in its group --
      // Ranks count, per entry, the group's entries with a smaller key: over the high 32 bits
      // of h alone when those are distinct in every group (two of 32 hashes share them with
      // probability about 1e-7), else over the full (h, id).  (The serial orders put their
      // index in the high bits.)
      const uint32_t idl = key_id(keyl);
      uint64_t h = ~0ull;
      if (valid_s)
        h = (a.order == 0)   ? hash_tail(head, (uint64_t)(v - cur.lo), (uint64_t)(idl - cur.lo))
            : (a.order == 1) ? (uint64_t)gl << 32
                             : (uint64_t)(m - 1 - gl) << 32;
      int pi_s = gl;  // this storage slot's position (slots past m keep positions m .. VW - 1)
      {
        const uint32_t k32 = (uint32_t)(h >> 32);
        const uint64_t mv = valid_s ? (((uint64_t)g << 32) | k32) : (~0ull << 32) | (uint64_t)lane;
        const bool tie = __any_sync(0xffffffffu, __popc(__match_any_sync(0xffffffffu, mv)) > 1);
        int r = 0;
        if (!tie) {
  #pragma unroll 8
          for (int j = 0; j < VW; ++j) {
            const uint32_t kj = __shfl_sync(0xffffffffu, k32, gb + j);
            r += (j < m && kj < k32) ? 1 : 0;
          }
        } else {
          for (int j = 0; j < VW; ++j) {
            const uint64_t hj = __shfl_sync(0xffffffffu, h, gb + j);
            const uint32_t ij = __shfl_sync(0xffffffffu, idl, gb + j);
            r += (j < m && (hj < h || (hj == h && ij < idl))) ? 1 : 0;
          }
        }
        if (valid_s) {
          pi_s = r;
          s.src[gb + r] = (uint8_t)gl;
        }
      }
      __syncwarp();
      // lane gb + p takes local pi position p: its source lane hs (storage slot hs - gb)
      const int hs = gb + (gl < m ? (int)s.src[lane] : gl);
      const int slot = hs - gb;
      const uint64_t key = __shfl_sync(0xffffffffu, keyl, (int)hs);
      const bool valid_p = gl < m;
      const uint32_t below = lanes_below32(gl);
      const int row = __shfl_sync(0xffffffffu, row_s, (int)hs);  // the row of this position's entry
      const int32_t id = (int32_t)key_id(key);
      const int P = gb + gl;
      if (valid_p) {
        s.pid[P] = id;
        s.prow[P] = (uint8_t)row;
        s.rpos[gb + row] = (uint8_t)gl;
        if (row < k) s.roff[gb + row] = row * (m - 1) - row * (row - 1) / 2;
        // (BF16 / FP8: the quantized row's norm^2 and residual arrive with its last chunk)
        s.rnd[gb + row] = make_float2(0.0f, key_dist(key));
      }
      if (lane == 0) s.nrq = 0;
      if (gl == 0) {
        s.gk[g] = k;
        s.gm[g] = m;
      }
      s.fire[lane] = 0u;  // fire bits are set by the pairs that fire (shared atomics)
      __syncwarp();
      // "closer to v" is storage-slot order (rows hold their keys in ascending order): the
      // closer mask of a position is the prefix OR, over the slots before its own, of the
      // slots' position bits
      uint32_t closer_p;
      {
        const uint32_t bit = valid_s ? (1u << pi_s) : 0u;  // this lane as storage slot
        uint32_t x = bit;
  #pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
          if (dd >= VW) break;
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, dd, VW);
          if (gl >= dd) x |= y;
        }
        closer_p = __shfl_sync(0xffffffffu, x ^ bit, (int)hs);
      }

      // ---- gather + tile ---------------------------------------------------------------
      const int pdb = g * ((VW * (VW - 1)) >> 1);
      bool ok = true;
      for (int c = 0; c < nch; ++c) {
        const int c0 = c * WDC;
        const int clen = min(WDC, d - c0);
        if (!ONE && c > 0) issue(c);  // (chunk 0 is in flight since before the visit order)
        ok = mbar_wait(&s.bar, phb, kWaitLimit);
        if (!__all_sync(0xffffffffu, ok)) break;
        phb ^= 1u;
        inflight = false;
        if (PREC >= 1 && (ONE || c + 1 == nch)) {  // each row's terms, from its tail
          if (need) {
            const int cpy = (clen + C::VEC - 1) / C::VEC * C::VEC;
            const float2 t = *reinterpret_cast<const float2*>(wrow(s, gb + row_s) + cpy);
            s.rnd[gb + row_s].x = t.x;
            s.rdq[gb + row_s] = t.y;
          }
          __syncwarp();
        }
        if (PREC >= 1) {
          // tiles one at a time; partial dot products wait in pd between chunks (d > 128),
          // and the last chunk takes the fire decisions straight from the accumulators
          constexpr int KB = 16 / (int)sizeof(T);  // elements per 16 bytes
          const int ksteps = (clen + 2 * KB - 1) / (2 * KB);
          const int KI = (k + 15) >> 4, NJ = (m + 7) >> 3;  // used when one vertex fills the warp
          const bool first_c = ONE || c == 0, last_c = ONE || c + 1 == nch;
          const int g8 = lane >> 2, tg = lane & 3;
          const int npg = (VW * (VW - 1)) >> 1;  // pairs per lane group
          for (int t = 0; t < 6; ++t) {
            // tiles (I, J): (0,0..3), (1,2), (1,3); lane groups use the diagonal ones only
            const int I = t < 4 ? 0 : 1, J = t < 4 ? t : t - 2;
            const bool use = (VW == 32) ? (I < KI && J < NJ) : (t != 2 && t != 3);
            if (!use) continue;
            // this lane's elements: rows i0, i0 + 8 of the warp's row space, columns j0, j0 + 1
            const int i0 = I * 16 + g8, j0 = J * 8 + 2 * tg;
            int q[4];
            bool ve[4];
  #pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int i = i0 + ((e >> 1) << 3), j = j0 + (e & 1);
              const int ge = i >> lw;  // the lane group both rows must belong to
              const int eb = ge << lw, li = i - eb, lj = j - eb;
              const int ke = (VW == 32) ? k : s.gk[ge], me = (VW == 32) ? m : s.gm[ge];
              ve[e] = ((j >> lw) == ge) && li < ke && lj > li && lj < me;
              q[e] = ve[e] ? ge * npg + s.roff[i] + (lj - li - 1) : 0;
            }
            float acc[4];
  #pragma unroll
            for (int e = 0; e < 4; ++e) acc[e] = (!first_c && ve[e]) ? s.pd[q[e]] : 0.0f;
            const int ra = I * 16 + (lane & 15);
            const int rb = J * 8 + (lane & 7);
            const T* pa = wrow(s, ra) + (lane >> 4) * KB;
            const T* pb = wrow(s, rb) + ((lane >> 3) & 1) * KB;
            for (int ks = 0; ks < ksteps; ++ks) {
              uint32_t fa[4], fb[2];
              ldmatrix_x4(fa, pa + ks * 2 * KB);
              ldmatrix_x2(fb, pb + ks * 2 * KB);
              mma_q<PREC>(acc, fa, fb);
            }
            if (!last_c) {
  #pragma unroll
              for (int e = 0; e < 4; ++e)
                if (ve[e]) s.pd[q[e]] = acc[e];
              continue;
            }
            const float2 rI[2] = {s.rnd[i0], s.rnd[i0 + 8]};
            const float2 rJ[2] = {s.rnd[j0], s.rnd[j0 + 1]};
            const int pI[2] = {s.rpos[i0], s.rpos[i0 + 8]};
            const int pJ[2] = {s.rpos[j0], s.rpos[j0 + 1]};
            float scI[2] = {1.0f, 1.0f}, scJ[2] = {1.0f, 1.0f};
            if (PREC == 2) {  // the rows' power-of-two scales (exact products)
              scI[0] = q_scale(s.rdq[i0]);
              scI[1] = q_scale(s.rdq[i0 + 8]);
              scJ[0] = q_scale(s.rdq[j0]);
              scJ[1] = q_scale(s.rdq[j0 + 1]);
            }
  #pragma unroll
            for (int e = 0; e < 4; ++e) {
              if (!ve[e]) continue;
              const int i = i0 + ((e >> 1) << 3), j = j0 + (e & 1);
              const int ge = i >> lw, eb = ge << lw;
              const float gij = (PREC == 2) ? acc[e] * scI[e >> 1] * scJ[e & 1] : acc[e];
              const float2 ri = rI[e >> 1], rj = rJ[e & 1];
              float dab = (METRIC == 0) ? __fadd_rn(__fsub_rn(ri.x, gij), __fsub_rn(rj.x, gij))
                                        : __fsub_rn(1.0f, gij);
              const float mx = fmaxf(ri.y, rj.y);
              bool fire = dab < mx;
              const int pa2 = pI[e >> 1], pb2 = pJ[e & 1];
              if constexpr (!EX) {
                const float eqi = s.rdq[i], eqj = s.rdq[j];
                const float tol = bf16_bound<METRIC>(dab, ri.x, rj.x, eqi, eqj, d);
                if (fabsf(dab - mx) <= tol) {  // re-decide with the canonical FP32 d(a,b)
                  ++st_check;
                  const int slot = atomicAdd(&s.nrq, 1);
                  if (slot < WRQ) {
                    s.rq[slot] = (uint16_t)((i << 5) | j);  // taken below, all together
                    continue;
                  }
                  const float* xa = a.P.X + (int64_t)s.pid[eb + pa2] * a.P.ld;
                  const float* xb = a.P.X + (int64_t)s.pid[eb + pb2] * a.P.ld;
                  dab = row_dist<METRIC>(xa, xb, d);
                  fire = dab < mx;
                }
              }
              s.pd[q[e]] = dab;
              if (fire) atomicOr(&s.fire[eb + max(pa2, pb2)], 1u << min(pa2, pb2));
            }
          }
        } else {
          const int full4 = clen & ~3, rem = clen & 3;
          for (int q = gl; q < np; q += VW) {
            int i = 0;  // the new local row owning pair q
  #pragma unroll
            for (int w2 = 16; w2 > 0; w2 >>= 1)
              if (i + w2 < k && s.roff[gb + i + w2] <= q) i += w2;
            const int j = i + 1 + (q - s.roff[gb + i]);
            const float* ra = reinterpret_cast<const float*>(wrow(s, gb + i));
            const float* rb = reinterpret_cast<const float*>(wrow(s, gb + j));
            float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            for (int u = 0; u < full4; u += 4)
              dist_step4<METRIC>(acc, *reinterpret_cast<const float4*>(ra + u),
                                 *reinterpret_cast<const float4*>(rb + u));
            if (rem)
              dist_step4<METRIC>(acc, mask4(*reinterpret_cast<const float4*>(ra + full4), rem),
                                 mask4(*reinterpret_cast<const float4*>(rb + full4), rem));
            const float dab = dist_finish4<METRIC>(acc);
            s.pd[pdb + q] = dab;
            const int pa = s.rpos[gb + i], pb = s.rpos[gb + j];
            if (dab < fmaxf(s.rnd[gb + i].y, s.rnd[gb + j].y)) atomicOr(&s.fire[gb + max(pa, pb)], 1u << min(pa, pb));
          }
        }
        __syncwarp();
      }
      if (!__all_sync(0xffffffffu, ok)) {  // a bounded wait gave up: report and stop the warp
        if (lane == 0) atomicExch(a.err, kErrTimeout);
        if (inflight) mbar_wait(&s.bar, phb, kWaitLimit);  // let this warp's copies land
        if (a.emit_redirects)
          for (unsigned long long i = s.red_next + lane; i < s.red_end; i += 32) a.red_tgt[i] = -1;
        if (lane == 0) leave(0, 0, 0, 0, 0);
        quit = true;
        return;
      }
      // queued re-decisions, one per lane: the FP32 rows of every pair load at once
      if (PREC >= 1 && !EX && nch > 0) {
        const int nq = min(s.nrq, WRQ);
        for (int t = lane; t < nq; t += 32) {
          const int i = s.rq[t] >> 5, j = s.rq[t] & 31;
          const int ge = i >> lw, eb = ge << lw, li = i - eb, lj = j - eb;
          const int pa2 = s.rpos[i], pb2 = s.rpos[j];
          const float* xa = a.P.X + (int64_t)s.pid[eb + pa2] * a.P.ld;
          const float* xb = a.P.X + (int64_t)s.pid[eb + pb2] * a.P.ld;
          const float dab = row_dist<METRIC>(xa, xb, d);
          s.pd[ge * ((VW * (VW - 1)) >> 1) + s.roff[i] + (lj - li - 1)] = dab;
          if (dab < fmaxf(s.rnd[i].y, s.rnd[j].y)) atomicOr(&s.fire[eb + max(pa2, pb2)], 1u << min(pa2, pb2));
        }
        __syncwarp();
      }
      __syncwarp();

      // ---- prune: the chain's outcome, one column (pi position) per lane of the group -------
      // Column b of the sequential pair scan kills K_b: its live firing partners before the
      // first closer one f, then b itself (absorbed by f); all of them when none is closer.
      // Its live partners are the valid positions that no column c < b killed, so the scan's
      // outcome is the fixed point of K_b = rule(fire[b] & valid & ~OR_{c<b} K_c).  Rounds
      // that apply the rule to every column at once, from K = 0, reach it: after round r the
      // columns 0..r hold their final value, so it takes at most m rounds; the first round
      // whose K has the prefix it was computed from (in every group of the warp) is the fixed
      // point and ends the loop.
      uint32_t alive = validm;
      int mykill = -1;
      {
        const uint32_t fb = s.fire[P];
        uint32_t K = 0u, before = 0u, inc = 0u;  // before: the OR of K over the earlier columns
        int f = -1;
        for (int r = 0;; ++r) {
          const uint32_t cand = fb & validm & ~before;
          const uint32_t x = cand & closer_p;
          const uint32_t low = x & (0u - x);  // first closer partner (0: none)
          f = x ? __ffs(x) - 1 : -1;
          K = x ? ((cand & (low - 1u)) | (1u << gl)) : cand;
          inc = K;  // inclusive prefix OR over the group's columns
  #pragma unroll
          for (int dd = 1; dd < 32; dd <<= 1) {
            if (dd >= VW) break;
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, dd, VW);
            if (gl >= dd) inc |= y;
          }
          uint32_t bn = __shfl_up_sync(0xffffffffu, inc, 1, VW);
          if (gl == 0) bn = 0u;
          // the new K has the prefix this round used: it is the fixed point
          if (!__any_sync(0xffffffffu, bn != before) || r >= WM) break;
          before = bn;
        }
        alive = validm & ~__shfl_sync(0xffffffffu, inc, gb + VW - 1);
        for (uint32_t ab = K & ~(1u << gl); ab; ab &= ab - 1) s.kil[gb + __ffs(ab) - 1] = (uint8_t)gl;
        __syncwarp();
        if (valid_p && !((alive >> gl) & 1u)) mykill = f >= 0 ? f : (int)s.kil[P];
      }
      __syncwarp();
      // ---- emit ----------------------------------------------------------------------------
      const bool surv = valid_p && ((alive >> gl) & 1u);
      const uint32_t smask = (__reduce_or_sync(0xffffffffu, surv ? (1u << hs) : 0u) >> gb) & gmask;
      const int nkeep = __popc(alive & validm);
      if (m > 0 && in_bounds((uint64_t)v < (uint64_t)a.n, a.err)) {
        if (surv) a.keys_out[v * R + __popc(smask & lanes_below32(slot))] = key | 1ull;
        // in place, the slots past m are empty already (pool rows end in empty slots)
        const int pend = a.keys_out == a.keys_in ? m : R;
        for (int t = nkeep + gl; t < pend; t += VW) a.keys_out[v * R + t] = kEmpty;
        if (gl == 0) a.deg_out[v] = nkeep;
      }
      const int ndead = m - nkeep;
      // redirects of all groups: one reservation per warp, groups in order
      int pre = 0, tot = 0;
  #pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int nd = __shfl_sync(0xffffffffu, ndead, (q << lw) & 31);
        if (q < G) {
          if (q < g) pre += nd;
          tot += nd;
        }
      }
      if (a.emit_redirects && tot > 0) {
        // fill the warp's chunk to its end, then continue in a fresh one (tot < WRED)
        const unsigned long long base = s.red_next, end = s.red_end;
        unsigned long long b1 = base, next = base + (unsigned long long)tot;
        int avail = tot;
        if (next > end) {
          avail = (int)(end - base);
          unsigned long long nb2 = 0;
          if (lane == 0) nb2 = atomicAdd(a.red_n, (unsigned long long)WRED);
          b1 = __shfl_sync(0xffffffffu, nb2, 0);
          next = b1 + (unsigned long long)(tot - avail);
          if (lane == 0) s.red_end = b1 + WRED;
        }
        __syncwarp();
        if (lane == 0) s.red_next = next;
        if (valid_p && !surv) {
          const int ri = s.prow[gb + mykill], rj = row;
          const int i = min(ri, rj), j = max(ri, rj);
          const float dd = s.pd[pdb + s.roff[gb + i] + (j - i - 1)];
          const int32_t tgt = s.pid[gb + mykill];
          const int rk = pre + __popc(~alive & validm & below);
          const unsigned long long sl = rk < avail ? base + (unsigned long long)rk : b1 + (unsigned long long)(rk - avail);
          if (in_bounds(sl < (unsigned long long)a.red_cap && (uint64_t)(uint32_t)tgt < (uint64_t)a.n, a.err)) {
            a.red_tgt[sl] = tgt;
            a.red_key[sl] = make_key(dd, (uint32_t)id, 0u);
            atomicAdd(&a.count[tgt], 1);
          }
        }
      }
      if (gl == 0 && m > 0) {
        if (np > 0) {
          st_vert += 1;
          st_rows += m;
          st_pairs += np;
        }
        st_fired += ndead;
      }
      __syncwarp();
    };
    auto by_width = [&](auto ex_tag, auto one_tag) {
      if (cur.cls == 2)
        item(std::integral_constant<int, 32>{}, ex_tag, one_tag);
      else if (cur.cls == 1)
        item(std::integral_constant<int, 16>{}, ex_tag, one_tag);
      else
        item(std::integral_constant<int, 8>{}, ex_tag, one_tag);
    };
    auto by_chunks = [&](auto ex_tag) {
      if constexpr (PREC == 1) {  // (the one-chunk variant for the BF16 form only: compile time)
        if (nchd == 1)
          by_width(ex_tag, std::true_type{});
        else
          by_width(ex_tag, std::false_type{});
      } else {
        by_width(ex_tag, std::false_type{});
      }
    };
    if constexpr (PREC >= 1) {
      if (exact)
        by_chunks(std::true_type{});
      else
        by_chunks(std::false_type{});
    } else {
      by_chunks(std::false_type{});
    }
    if (quit) return;
    w = wnext;
    wnext = w2;
  }
  if (a.emit_redirects)
    for (unsigned long long i = s.red_next + lane; i < s.red_end; i += 32) a.red_tgt[i] = -1;
  if (a.stats) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      st_vert += __shfl_xor_sync(0xffffffffu, st_vert, o);
      st_rows += __shfl_xor_sync(0xffffffffu, st_rows, o);
      st_pairs += __shfl_xor_sync(0xffffffffu, st_pairs, o);
      st_fired += __shfl_xor_sync(0xffffffffu, st_fired, o);
      st_check += __shfl_xor_sync(0xffffffffu, st_check, o);
    }
    if (lane == 0) leave(st_vert, st_rows, st_pairs, st_fired, PREC >= 1 ? st_check : 0);
  }
}

template <int METRIC, int PREC, bool TMA>
cudaError_t launch_join_warp_v(const JoinArgs& a, cudaStream_t st, const char* name, bool setup_only) {
  const size_t smem = sizeof(WarpSlot<PREC, TMA>) * WW + 128;  // + alignment of the slots
  static KernelSetup ks;
  auto kern = rnd_join_warp_kernel<METRIC, PREC, TMA>;
  int per_sm = 0;
  cudaError_t e = setup_kernel(ks, kern, WW * 32, smem, smem, &per_sm);
  if (e != cudaSuccess || setup_only) return e;
  if (a.warp_ctas > 0) per_sm = std::min(per_sm, a.warp_ctas);
  if (per_sm < 1) per_sm = 1;
  const int64_t blocks = std::min<int64_t>((int64_t)sm_count() * per_sm, kMaxJoinGrid);
  ProfScope ps(name, st);
  kern<<<(unsigned)blocks, WW * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <int METRIC, int PREC>
cudaError_t launch_join_warp_t(const JoinArgs& a, cudaStream_t st, const char* name, bool setup_only = false) {
  if constexpr (PREC >= 1)
    if (a.rows_tma) return launch_join_warp_v<METRIC, PREC, true>(a, st, name, setup_only);
  return launch_join_warp_v<METRIC, PREC, false>(a, st, name, setup_only);
}

}  // namespace


// =====================================================================================
// rnd_join for pools of 33..64 entries: a team of two warps (one 64-thread CTA) per
// vertex; thread t owns pool entry t (storage slot t).
//   order   rank of (h, id) among the m entries (16-byte keys in shared memory);
//   gather  one bulk copy per row and 128-column chunk (two stages when d > 128); rows hold
//           the new entries first, then the old ones, each part in slot order, so the first
//           chunk's copies are issued before the visit order is ranked;
//   tile    BF16 / FP8: mma.sync tiles over new rows x all rows, shared between the two
//           warps and taken one at a time; partial dot products wait in shared memory
//           between chunks, and the last chunk decides the fire bits straight from the
//           accumulators (a pair that fires sets its bit in the later position's mask by
//           a shared atomic).  FP32 (d <= 128): one thread per pair, canonical distance;
//   chain   the sequential outcome of the pair scan over the fire bits as a fixed point,
//           one column (pi position) per thread; for each entry made bottom, the entry
//           that absorbed it;
//   emit    survivors rewritten in place as old; redirects into reserved slots.
// =====================================================================================
namespace {

constexpr int TM = 64;     // pool entries per team
constexpr int TRED = 512;  // redirect slots a team reserves at a time
constexpr int TDC = 128;   // columns per gathered chunk
constexpr int TRQ = 64;    // re-decisions a team queues per vertex (more are taken in place)

template <int PREC>
struct TPrec;
template <>
struct TPrec<0> {
  using T = float;
  static constexpr int RS = TDC + 4;  // row stride (elements): 528 B, conflict-free float4 reads
  static constexpr int VEC = 4;
};
template <>
struct TPrec<1> {
  using T = __nv_bfloat16;
  static constexpr int RS = TDC + 8;  // 272 B: the 8 rows of an ldmatrix phase hit distinct banks
  static constexpr int VEC = 16;
};
template <>
struct TPrec<2> {
  using T = uint8_t;                  // e4m3 bytes
  static constexpr int RS = TDC + 16; // 144 B: the 8 rows of an ldmatrix phase hit distinct banks
  static constexpr int VEC = 32;
};

struct __align__(16) TeamKey {
  uint64_t h;
  uint32_t id;
  uint32_t pad;
};

struct __align__(16) TeamSmem {
  union {
    struct {
      TeamKey hk[TM];               // order key by storage slot (visit order), until the tiles
      uint32_t hk32[TM];            // its high 32 hash bits (~0 past m)
    };
    float pd[TM * (TM - 1) / 2];    // per pair: its distance (partial dot product between chunks)
  };
  uint64_t fire[TM], closer[TM];  // by pi position; bit a < b: pair (a, b) fired / a is closer
  float2 rnd[TM];                 // by row: (squared norm of the BF16 row, recorded dist to v)
  float rdq[TM];                  // by row: norm of the quantization residual
  int32_t pid[TM];                // by pi position
  uint16_t roff[TM + 1];          // first pair index of new row i
  uint8_t rpos[TM], prow[TM], killer[TM];
  uint16_t rq[TRQ];               // pairs (row i << 6 | row j) whose decision is re-taken in FP32
  int32_t nrq;
  uint64_t alive, wtot;
  uint64_t kor[2][2];             // chain rounds: per warp, the OR of its columns' kill sets
  uint32_t sm32[2];
  uint64_t bar[2];
  unsigned long long red_next, red_end, red_b0, red_b1;
  int32_t red_avail;
  int64_t next_p;                 // the team's next record (device work queue)
};
constexpr size_t kTeamRowsOff = (sizeof(TeamSmem) + 127) & ~(size_t)127;  // staged rows follow
// BF16 rows of up to 128 dimensions: eight team CTAs fit one SM (233,472 bytes of shared
// memory, 1,024 reserved per CTA), as many as the 128-register threads allow
static_assert(8 * (kTeamRowsOff + (size_t)TM * (TDC + 8) * 2 + 1024) <= 233472,
              "team shared memory must allow eight CTAs per SM");

constexpr int kTeamTiles = 20;  // (I, J) with I < 4, J < 8 and J >= 2I (some j > i in the tile)

__device__ __forceinline__ void team_tile(int t, int& I, int& J) {
  if (t < 8) { I = 0; J = t; }
  else if (t < 14) { I = 1; J = t - 6; }
  else if (t < 18) { I = 2; J = t - 10; }
  else { I = 3; J = t - 12; }
}

template <int METRIC, int PREC>
__global__ void __launch_bounds__(TM, 8) rnd_join_team_kernel(JoinArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using C = TPrec<PREC>;
  using T = typename C::T;
  TeamSmem& s = *reinterpret_cast<TeamSmem*>(smem_raw);
  T* const rowbase = reinterpret_cast<T*>(smem_raw + kTeamRowsOff);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t cnt = a.list_n[3];  // records of the last size class
  int64_t p = blockIdx.x;
  if (p >= cnt || *(volatile int32_t*)a.err) return;  // nothing to do, or the round has failed
  const int R = a.R, W = a.rec_w[3], d = a.P.d;
  const int nchd = (d + TDC - 1) / TDC;  // chunks per row
  const uint64_t head = hash_head(a.seed, (uint64_t)a.t1, (uint64_t)a.t2);  // visit-order hash, uniform part
  const int nst = nchd > 1 ? 2 : 1;      // stages
  if (tid == 0) {
    mbar_init(&s.bar[0], 1);
    mbar_init(&s.bar[1], 1);
    fence_mbar_init();
    s.red_next = s.red_end = 0;
  }
  __syncthreads();
  bool exact = false;
  if (PREC >= 1) {
    const unsigned fl = a.P.qflags[0];
    const float mxa = __uint_as_float(a.P.qflags[1]);
    exact = (fl == 0u) && ((double)d * (double)mxa * (double)mxa < 16777216.0);
  }
  uint32_t phb = 0u, infl = 0u;  // mbarrier phase bit and copies-in-flight bit per stage
  int stage = 0;
  long long st_vert = 0, st_rows = 0, st_pairs = 0, st_fired = 0, st_check = 0;

  const uint64_t* r0 = a.rec[3] + p * W;
  int64_t nv = (int64_t)(r0[0] & 0xffffffffull);
  uint32_t nlo = (uint32_t)(r0[0] >> 32);
  int nm = (int)r0[1];
  uint64_t nkey = (tid < nm && in_bounds((uint64_t)nv < (uint64_t)a.n, a.err)) ? a.keys_in[nv * R + tid] : kEmpty;
  // The first record of each team is its block index; the later ones come from a device work
  // queue (records gridDim.x, gridDim.x + 1, ... in the order teams ask).  Loads are pipelined
  // so that no record waits for memory: when record p starts, the pool keys of the next record
  // (whose words arrived during the record before) are requested, the ticket asked then is
  // published, and the words of the record it names are requested.
  if (tid == 0) s.next_p = (int64_t)gridDim.x + (int64_t)atomicAdd(a.work_q + 1, 1u);
  __syncthreads();
  int64_t pnext = s.next_p;
  __syncthreads();  // (thread 0 writes the next ticket there when the first record starts)
  uint64_t qr0 = 0;  // the words of record pnext
  int qm = 0;
  unsigned int tq = 0;  // thread 0: the ticket of the record after pnext
  if (pnext < cnt) {
    const uint64_t* rn = a.rec[3] + pnext * W;
    qr0 = rn[0];
    qm = (int)rn[1];
    if (tid == 0) tq = atomicAdd(a.work_q + 1, 1u);
  }

  while (p < cnt) {
    // the record's work, compiled per mode for quantized rows (EX: exact tiles, no decision
    // is re-taken) and, for BF16 rows, per length (ONE: one chunk of columns)
    int64_t p2 = cnt;
    bool quit = false;  // a bounded wait gave up: the team stops
    auto record = [&](auto ex_tag, auto one_tag) {
      constexpr bool EX = decltype(ex_tag)::value, ONE = decltype(one_tag)::value;
      const int64_t v = nv;
      const uint32_t lo = nlo;  // first id of the vertex's build
      const int m = nm;
      const uint64_t keyl = tid < m ? nkey : kEmpty;
      if (pnext < cnt) {
        nv = (int64_t)(qr0 & 0xffffffffull);
        nlo = (uint32_t)(qr0 >> 32);
        nm = qm;
        nkey = (tid < nm && in_bounds((uint64_t)nv < (uint64_t)a.n, a.err)) ? a.keys_in[nv * R + tid] : kEmpty;
        if (tid == 0) s.next_p = (int64_t)gridDim.x + (int64_t)tq;
      }
      // ---- visit order: rank of (h, id) among the m entries --------------------------------
      const uint32_t idl = key_id(keyl);
      const bool has = tid < m;
      uint64_t h = ~0ull;
      if (has)  // (the serial orders put their index in the high bits)
        h = (a.order == 0)   ? hash_tail(head, (uint64_t)(v - lo),
                                            (uint64_t)(idl - lo))
            : (a.order == 1) ? (uint64_t)tid << 32
                             : (uint64_t)(m - 1 - tid) << 32;
      {
        TeamKey hk;
        hk.h = h;
        hk.id = has ? idl : 0xffffffffu;
        hk.pad = 0u;
        s.hk[tid] = hk;
        s.hk32[tid] = has ? (uint32_t)(h >> 32) : 0xffffffffu;
      }
      {
        const unsigned nw = __ballot_sync(0xffffffffu, has && !key_old(keyl));  // new entries by slot
        if (lane == 0) s.sm32[warp] = nw;
      }
      if (tid == 0) s.nrq = 0;
      __syncthreads();
      p2 = pnext < cnt ? s.next_p : cnt;  // the record after pnext
      if (p2 < cnt) {
        const uint64_t* rn = a.rec[3] + p2 * W;
        qr0 = rn[0];
        qm = (int)rn[1];
        if (tid == 0) tq = atomicAdd(a.work_q + 1, 1u);
      }
      // rows: the new entries first, then the old ones, each part in storage-slot order (the
      // pairs are enumerated over rows: new row i, any later row j, so the order inside each
      // part does not matter); the first chunk's copies are in flight while the visit order
      // is ranked
      const uint64_t news = (uint64_t)s.sm32[0] | ((uint64_t)s.sm32[1] << 32);
      const int k = __popcll(news);
      const int np = k * (m - 1) - k * (k - 1) / 2;
      const uint64_t valid = (m >= 64) ? ~0ull : ((1ull << m) - 1ull);
      int row = 0;
      if (has) {
        const uint64_t bt = bits_below(tid);
        row = ((news >> tid) & 1ull) ? __popcll(news & bt) : k + __popcll(~news & valid & bt);
      }
      const int nch = np > 0 ? nchd : 0;
      auto issue = [&](int c, int st) {
        const int c0 = c * TDC;
        const int clen = min(TDC, d - c0);
        const int cpy = (clen + C::VEC - 1) / C::VEC * C::VEC;
        // a quantized row's last chunk brings the row's terms (norm^2, residual) along
        const uint32_t bytes = (uint32_t)(cpy * sizeof(T)) + ((PREC >= 1 && (ONE || c + 1 == nchd)) ? (uint32_t)kTailCopy : 0u);
        if (tid == 0) mbar_expect_tx(&s.bar[st], (uint32_t)m * bytes);
        infl |= 1u << st;
        __syncthreads();
        // (checked build: a row id out of range is not copied; the stage's wait then gives up)
        if (has && in_bounds((uint64_t)idl < (uint64_t)a.n, a.err)) {
          const T* src = (PREC == 0) ? reinterpret_cast<const T*>(a.P.X + (int64_t)idl * a.P.ld + c0)
                                     : reinterpret_cast<const T*>(a.P.Xb) + (int64_t)idl * a.P.ldb + c0;
          bulk_g2s(rowbase + ((size_t)st * TM + row) * C::RS, src, bytes, &s.bar[st]);
        }
      };
      if (nch > 0) issue(0, stage);
      // position = rank of the entry's key among the m entries: over the high 32 hash bits
      // (entries past m hold ~0 there and never count), then checked: equal high bits leave
      // two entries with one rank, and the ranks are taken again over the full (h, id)
      int pi = 0;
      if (has) {
        const uint32_t k32 = (uint32_t)(h >> 32);
        for (int f = 0; f < m; f += 4) {
          const uint4 o = *reinterpret_cast<const uint4*>(&s.hk32[f]);
          pi += (o.x < k32 ? 1 : 0) + (o.y < k32 ? 1 : 0) + (o.z < k32 ? 1 : 0) + (o.w < k32 ? 1 : 0);
        }
        s.prow[pi] = (uint8_t)tid;  // this rank's claim
      }
      // "closer to v" is storage-slot order (rows hold their keys in ascending order): the
      // closer mask of a position is the OR of the position bits of the slots before its own
      uint64_t pbit = has ? (1ull << pi) : 0ull;
      uint64_t pre = pbit;
  #pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, pre, dd);
        if (lane >= dd) pre |= y;
      }
      if (warp == 0 && lane == 31) s.wtot = pre;
      __syncthreads();
      if (__syncthreads_or(has && s.prow[pi] != (uint8_t)tid)) {  // a tie in the high bits
        pi = 0;
        if (has)
          for (int f = 0; f < m; ++f) {
            const TeamKey o = s.hk[f];
            pi += (o.h < h) || (o.h == h && o.id < idl);
          }
        pbit = has ? (1ull << pi) : 0ull;
        pre = pbit;
  #pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
          const uint64_t y = __shfl_up_sync(0xffffffffu, pre, dd);
          if (lane >= dd) pre |= y;
        }
        if (warp == 0 && lane == 31) s.wtot = pre;
        __syncthreads();
      }
      if (warp == 1) pre |= s.wtot;
      if (has) {
        s.pid[pi] = (int32_t)idl;
        s.prow[pi] = (uint8_t)row;
        s.rpos[row] = (uint8_t)pi;
        s.closer[pi] = pre ^ pbit;
        // (BF16 / FP8: the quantized row's norm^2 and residual arrive with its last chunk)
        s.rnd[row] = make_float2(0.0f, key_dist(keyl));
      }
      if (tid <= k) s.roff[tid] = tid * (m - 1) - tid * (tid - 1) / 2;
      s.fire[tid] = 0ull;  // fire bits are set by the pairs that fire (shared atomics)
      __syncthreads();

      // ---- gather + tile (chunk 0 is in flight since before the visit order) --------------
      bool fail = false;
      for (int c = 0; c < nch; ++c) {
        const int st = stage;
        if (!ONE && nst > 1 && c + 1 < nch) issue(c + 1, st ^ 1);
        const bool ok = mbar_wait(&s.bar[st], (phb >> st) & 1u, kWaitLimit);
        if (__syncthreads_or(!ok)) {  // uniform over the team
          fail = true;
          break;
        }
        phb ^= 1u << st;
        infl &= ~(1u << st);
        const int clen = min(TDC, d - c * TDC);
        const T* rows = rowbase + (size_t)st * TM * C::RS;
        if (PREC >= 1 && (ONE || c + 1 == nch)) {  // each row's terms, from its tail
          if (has) {
            const int cpy = (clen + C::VEC - 1) / C::VEC * C::VEC;
            const float2 t = *reinterpret_cast<const float2*>(rows + (size_t)row * C::RS + cpy);
            s.rnd[row].x = t.x;
            s.rdq[row] = t.y;
          }
          __syncthreads();
        }
        if (PREC >= 1) {
          constexpr int KB = 16 / (int)sizeof(T);  // elements per 16 bytes
          const int ksteps = (clen + 2 * KB - 1) / (2 * KB);
          const int KI = (k + 15) >> 4, NJ = (m + 7) >> 3;
          const bool first_c = ONE || c == 0, last_c = ONE || c + 1 == nch;
          const int g = lane >> 2, tg = lane & 3;
          for (int t = warp; t < kTeamTiles; t += 2) {
            int I, J;
            team_tile(t, I, J);
            if (I >= KI || J >= NJ) continue;
            // this lane's four elements: rows i0, i0 + 8 and columns j0, j0 + 1
            const int i0 = I * 16 + g, j0 = J * 8 + 2 * tg;
            int q[4];
            bool ve[4];
  #pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int i = i0 + ((e >> 1) << 3), j = j0 + (e & 1);
              ve[e] = (i < k) && (j > i) && (j < m);
              q[e] = ve[e] ? s.roff[i] + (j - i - 1) : 0;
            }
            float acc[4];
  #pragma unroll
            for (int e = 0; e < 4; ++e) acc[e] = (!first_c && ve[e]) ? s.pd[q[e]] : 0.0f;
            const int ra = min(I * 16 + (lane & 15), TM - 1);
            const int rb = J * 8 + (lane & 7);
            const T* pa = rows + ra * C::RS + (lane >> 4) * KB;
            const T* pb = rows + rb * C::RS + ((lane >> 3) & 1) * KB;
            for (int ks = 0; ks < ksteps; ++ks) {
              uint32_t fa[4], fb[2];
              ldmatrix_x4(fa, pa + ks * 2 * KB);
              ldmatrix_x2(fb, pb + ks * 2 * KB);
              mma_q<PREC>(acc, fa, fb);
            }
            if (!last_c) {
  #pragma unroll
              for (int e = 0; e < 4; ++e)
                if (ve[e]) s.pd[q[e]] = acc[e];
              continue;
            }
            // last chunk: distance and fire decision of each element
            const float2 rI[2] = {s.rnd[min(i0, TM - 1)], s.rnd[min(i0 + 8, TM - 1)]};
            const float2 rJ[2] = {s.rnd[j0], s.rnd[j0 + 1]};
            float scI[2] = {1.0f, 1.0f}, scJ[2] = {1.0f, 1.0f};
            if (PREC == 2) {  // the rows' power-of-two scales (exact products)
              scI[0] = q_scale(s.rdq[min(i0, TM - 1)]);
              scI[1] = q_scale(s.rdq[min(i0 + 8, TM - 1)]);
              scJ[0] = q_scale(s.rdq[j0]);
              scJ[1] = q_scale(s.rdq[j0 + 1]);
            }
  #pragma unroll
            for (int e = 0; e < 4; ++e) {
              if (!ve[e]) continue;
              const int i = i0 + ((e >> 1) << 3), j = j0 + (e & 1);
              const float2 ri = rI[e >> 1], rj = rJ[e & 1];
              const float gij = (PREC == 2) ? acc[e] * scI[e >> 1] * scJ[e & 1] : acc[e];
              float dab = (METRIC == 0) ? __fadd_rn(__fsub_rn(ri.x, gij), __fsub_rn(rj.x, gij))
                                        : __fsub_rn(1.0f, gij);
              const float mx = fmaxf(ri.y, rj.y);
              bool fire = dab < mx;
              if constexpr (!EX) {
                const float eqi = s.rdq[i], eqj = s.rdq[j];
                const float tol = bf16_bound<METRIC>(dab, ri.x, rj.x, eqi, eqj, d);
                if (fabsf(dab - mx) <= tol) {  // re-decide with the canonical FP32 d(a,b)
                  ++st_check;
                  const int slot = atomicAdd(&s.nrq, 1);
                  if (slot < TRQ) {
                    s.rq[slot] = (uint16_t)((i << 6) | j);  // taken below, all together
                    continue;
                  }
                  const float* xa = a.P.X + (int64_t)s.pid[s.rpos[i]] * a.P.ld;
                  const float* xb = a.P.X + (int64_t)s.pid[s.rpos[j]] * a.P.ld;
                  dab = row_dist<METRIC>(xa, xb, d);
                  fire = dab < mx;
                }
              }
              s.pd[q[e]] = dab;
              const int pa2 = s.rpos[i], pb2 = s.rpos[j];
              if (fire)
                atomicOr(reinterpret_cast<unsigned long long*>(&s.fire[max(pa2, pb2)]), 1ull << min(pa2, pb2));
            }
          }
        } else {
          const float* rf = reinterpret_cast<const float*>(rows);
          const int full4 = clen & ~3, rem = clen & 3;
          for (int q = tid; q < np; q += TM) {
            int i = 0;  // the new row owning pair q
  #pragma unroll
            for (int w = 32; w > 0; w >>= 1)
              if (i + w < k && s.roff[i + w] <= q) i += w;
            const int j = i + 1 + (q - s.roff[i]);
            const float* ra = rf + i * C::RS;
            const float* rb = rf + j * C::RS;
            float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            for (int u = 0; u < full4; u += 4)
              dist_step4<METRIC>(acc, *reinterpret_cast<const float4*>(ra + u),
                                 *reinterpret_cast<const float4*>(rb + u));
            if (rem)
              dist_step4<METRIC>(acc, mask4(*reinterpret_cast<const float4*>(ra + full4), rem),
                                 mask4(*reinterpret_cast<const float4*>(rb + full4), rem));
            const float dab = dist_finish4<METRIC>(acc);
            s.pd[q] = dab;
            const int pa = s.rpos[i], pb = s.rpos[j];
            if (dab < fmaxf(s.rnd[i].y, s.rnd[j].y))
              atomicOr(reinterpret_cast<unsigned long long*>(&s.fire[max(pa, pb)]), 1ull << min(pa, pb));
          }
        }
        __syncthreads();
        if (nst > 1) stage ^= 1;
      }
      if (fail) {  // a bounded wait gave up: report, let the copies in flight land, stop
        if (tid == 0) atomicExch(a.err, kErrTimeout);
        for (int t = 0; t < 2; ++t)
          if ((infl >> t) & 1u) mbar_wait(&s.bar[t], (phb >> t) & 1u, kWaitLimit);
        if (a.emit_redirects)
          for (unsigned long long i = s.red_next + tid; i < s.red_end; i += TM) a.red_tgt[i] = -1;
        quit = true;
        return;
      }

      // queued re-decisions, one per thread: the FP32 rows of every pair load at once
      if (PREC >= 1 && !EX && nch > 0 && s.nrq > 0) {
        const int nq = min(s.nrq, TRQ);
        for (int t = tid; t < nq; t += TM) {
          const int i = s.rq[t] >> 6, j = s.rq[t] & 63;
          const int pa2 = s.rpos[i], pb2 = s.rpos[j];
          const float* xa = a.P.X + (int64_t)s.pid[pa2] * a.P.ld;
          const float* xb = a.P.X + (int64_t)s.pid[pb2] * a.P.ld;
          const float dab = row_dist<METRIC>(xa, xb, d);
          s.pd[s.roff[i] + (j - i - 1)] = dab;
          if (dab < fmaxf(s.rnd[i].y, s.rnd[j].y))
            atomicOr(reinterpret_cast<unsigned long long*>(&s.fire[max(pa2, pb2)]), 1ull << min(pa2, pb2));
        }
        __syncthreads();
      }
      // ---- prune: the chain's outcome, one column (pi position) per thread ------------------
      // Column b of the sequential pair scan kills K_b: its live firing partners before the
      // first closer one f, then b itself (absorbed by f); all of them when none is closer.
      // Its live partners are the valid positions that no column c < b killed, so the scan's
      // outcome is the fixed point of K_b = rule(fire[b] & valid & ~OR_{c<b} K_c).  Rounds
      // that apply the rule to every column at once, from K = 0, reach it: after round r the
      // columns 0..r hold their final value, so it takes at most m rounds; the first round
      // whose K has the prefix it was computed from is the fixed point and ends the loop.
      {
        const uint64_t fb = s.fire[tid], cb = s.closer[tid];
        // the OR of K over the earlier columns: bw of this warp's, t0 of warp 0's (for warp 1)
        uint64_t K = 0ull, bw = 0ull, t0 = 0ull;
        int f = -1, r = 0;
        for (;; ++r) {
          const uint64_t cand = fb & valid & ~(bw | (warp == 1 ? t0 : 0ull));
          const uint64_t x = cand & cb;
          f = x ? __ffsll((long long)x) - 1 : -1;
          K = x ? ((cand & bits_below(f)) | (1ull << tid)) : cand;
          uint64_t inc = K;  // inclusive prefix OR over the warp's columns
  #pragma unroll
          for (int dd = 1; dd < 32; dd <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, inc, dd);
            if (lane >= dd) inc |= y;
          }
          uint64_t bwn = __shfl_up_sync(0xffffffffu, inc, 1);
          if (lane == 0) bwn = 0ull;
          if (lane == 31) s.kor[r & 1][warp] = inc;
          // the new K has the prefix this round used: it is the fixed point
          const bool moved = __syncthreads_or(bwn != bw || (warp == 0 && lane == 31 && inc != t0)) != 0;
          if (!moved || r >= TM) break;
          bw = bwn;
          t0 = s.kor[r & 1][0];
        }
        // absorbers: b for the partners it kills, f for b itself
        for (uint64_t ab = K & ~(1ull << tid); ab; ab &= ab - 1) s.killer[__ffsll((long long)ab) - 1] = (uint8_t)tid;
        if (f >= 0) s.killer[tid] = (uint8_t)f;
        if (tid == 0) s.alive = valid & ~(s.kor[r & 1][0] | s.kor[r & 1][1]);
      }
      __syncthreads();
      // ---- emit ------------------------------------------------------------------------------
      const uint64_t alive = s.alive;
      const bool surv = has && ((alive >> pi) & 1ull);
      const unsigned sb = __ballot_sync(0xffffffffu, surv);
      if (lane == 0) s.sm32[warp] = sb;
      const int nkeep = __popcll(alive & valid);
      const int ndead = m - nkeep;
      if (a.emit_redirects && tid == 0 && ndead > 0) {
        // fill the team's chunk to its end, then continue in a fresh one (ndead < TRED)
        const unsigned long long base = s.red_next;
        unsigned long long b1 = base, next = base + (unsigned long long)ndead;
        int avail = ndead;
        if (next > s.red_end) {
          avail = (int)(s.red_end - base);
          b1 = atomicAdd(a.red_n, (unsigned long long)TRED);
          next = b1 + (unsigned long long)(ndead - avail);
          s.red_end = b1 + TRED;
        }
        s.red_next = next;
        s.red_b0 = base;
        s.red_b1 = b1;
        s.red_avail = avail;
      }
      __syncthreads();
      const uint64_t smask = (uint64_t)s.sm32[0] | ((uint64_t)s.sm32[1] << 32);  // survivors by slot
      const bool vok = in_bounds((uint64_t)v < (uint64_t)a.n, a.err);
      if (surv && vok) a.keys_out[v * R + __popcll(smask & bits_below(tid))] = keyl | 1ull;
      // in place, the slots past m are empty already (pool rows end in empty slots)
      const int pend = a.keys_out == a.keys_in ? m : R;
      for (int t = nkeep + tid; vok && t < pend; t += TM) a.keys_out[v * R + t] = kEmpty;
      if (tid == 0 && vok) a.deg_out[v] = nkeep;
      if (a.emit_redirects && has && !surv) {
        const int kp = s.killer[pi];
        const int ri = s.prow[kp], rj = row;
        const int i = min(ri, rj), j = max(ri, rj);
        const float dd = s.pd[s.roff[i] + (j - i - 1)];
        const int32_t tgt = s.pid[kp];
        const int g = __popcll(~alive & valid & bits_below(pi));
        const unsigned long long sl =
            g < s.red_avail ? s.red_b0 + (unsigned long long)g : s.red_b1 + (unsigned long long)(g - s.red_avail);
        if (in_bounds(sl < (unsigned long long)a.red_cap && (uint64_t)(uint32_t)tgt < (uint64_t)a.n, a.err)) {
          a.red_tgt[sl] = tgt;
          a.red_key[sl] = make_key(dd, idl, 0u);
          atomicAdd(&a.count[tgt], 1);
        }
      }
      if (tid == 0) {
        if (np > 0) {
          st_vert += 1;
          st_rows += m;
          st_pairs += np;
        }
        st_fired += ndead;
      }
      __syncthreads();
    };
    auto by_chunks = [&](auto ex_tag) {
      if constexpr (PREC == 1) {  // (the one-chunk variant for the BF16 form only: compile time)
        if (nchd == 1)
          record(ex_tag, std::true_type{});
        else
          record(ex_tag, std::false_type{});
      } else {
        record(ex_tag, std::false_type{});
      }
    };
    if constexpr (PREC >= 1) {
      if (exact)
        by_chunks(std::true_type{});
      else
        by_chunks(std::false_type{});
    } else {
      by_chunks(std::false_type{});
    }
    if (quit) return;
    p = pnext;
    pnext = p2;
  }
  if (a.emit_redirects)
    for (unsigned long long i = s.red_next + tid; i < s.red_end; i += TM) a.red_tgt[i] = -1;
  if (a.stats) {
    if (tid == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[0]), (unsigned long long)st_vert);
      atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[1]), (unsigned long long)st_rows);
      atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[2]), (unsigned long long)st_pairs);
      atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[3]), (unsigned long long)st_fired);
    }
    if (PREC >= 1) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) st_check += __shfl_xor_sync(0xffffffffu, st_check, o);
      if (lane == 0 && st_check)
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[7]), (unsigned long long)st_check);
    }
  }
}

template <int METRIC, int PREC>
cudaError_t launch_join_team_t(const JoinArgs& a, cudaStream_t st, const char* name, bool setup_only = false) {
  using C = TPrec<PREC>;
  const int nchd = (a.P.d + TDC - 1) / TDC;
  const size_t smem = kTeamRowsOff + (size_t)(nchd > 1 ? 2 : 1) * TM * C::RS * sizeof(typename C::T);
  const size_t smem_max = kTeamRowsOff + (size_t)2 * TM * C::RS * sizeof(typename C::T);
  static KernelSetup ks;
  auto kern = rnd_join_team_kernel<METRIC, PREC>;
  int per_sm = 0;
  cudaError_t e = setup_kernel(ks, kern, TM, smem_max, smem, &per_sm);
  if (e != cudaSuccess || setup_only) return e;
  if (a.team_ctas > 0) per_sm = std::min(per_sm, a.team_ctas);
  if (per_sm < 1) per_sm = 1;
  const int64_t blocks = std::min<int64_t>((int64_t)sm_count() * per_sm, kMaxJoinGrid);
  ProfScope ps(name, st);
  kern<<<(unsigned)blocks, TM, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

// =====================================================================================
// rev_merge: exclusive scan of the per-target counts, scatter of the redirect keys into
// per-target buckets, and a per-target select of the R smallest distinct ids among the
// target's base pool (kept survivors, or its untouched pool) and its bucket.
// =====================================================================================
namespace {

constexpr int SCAN_T = 256;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_IPT;

__device__ __forceinline__ int64_t warp_sum64(int64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__global__ void __launch_bounds__(SCAN_T) scan_reduce_kernel(const int32_t* __restrict__ cnt,
                                                             int64_t n,
                                                             int64_t* __restrict__ bsum) {
  __shared__ int64_t red[SCAN_T / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t s = 0;
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T) {
    const int64_t idx = base + i;
    if (idx < n) s += cnt[idx];
  }
  s = warp_sum64(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    int64_t t = threadIdx.x < SCAN_T / 32 ? red[threadIdx.x] : 0;
    t = warp_sum64(t);
    if (threadIdx.x == 0) bsum[blockIdx.x] = t;
  }
}

// Each block first adds up the sums of the blocks before it (a few thousand int64 at most,
// from L2), then scans its own tile; the last block also writes the total to off[n].
__global__ void __launch_bounds__(SCAN_T) scan_apply_kernel(const int32_t* __restrict__ cnt,
                                                            int64_t n,
                                                            const int64_t* __restrict__ bsum,
                                                            int64_t* __restrict__ off) {
  __shared__ int64_t wsum[SCAN_T / 32];
  __shared__ int64_t bpre_s;
  {
    int64_t x = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += SCAN_T) x += bsum[b];
    x = warp_sum64(x);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t t = 0;
      for (int w = 0; w < SCAN_T / 32; ++w) t += wsum[w];
      bpre_s = t;
    }
    __syncthreads();
  }
  const int64_t bpre = bpre_s;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
  int32_t v[SCAN_IPT];
  int64_t tsum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_IPT; ++i) {
    v[i] = (base + i < n) ? cnt[base + i] : 0;
    tsum += v[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  __syncthreads();  // (wsum is reused)
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  int64_t wpre = 0;
  for (int w = 0; w < warp; ++w) wpre += wsum[w];
  int64_t run = bpre + wpre + inc - tsum;
#pragma unroll
  for (int i = 0; i < SCAN_IPT; ++i) {
    if (base + i < n) off[base + i] = run;
    run += v[i];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_T - 1) off[n] = run;  // the total
}

__global__ void scatter_kernel(const int32_t* __restrict__ tgt, const uint64_t* __restrict__ pk,
                               const unsigned long long* __restrict__ nred,
                               const int64_t* __restrict__ off, int32_t* __restrict__ count,
                               uint64_t* __restrict__ bucket, int32_t* __restrict__ err, int64_t n,
                               int64_t red_cap, int64_t bucket_cap) {
  if (*err) return;  // a join wait gave up: the slots are incomplete, merge nothing
  const int64_t nslots = (int64_t)*nred;
  if (!in_bounds(nslots <= red_cap, err)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nslots;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = tgt[i];
    if (t < 0) continue;  // unused tail of a reserved chunk
    if (!in_bounds(t < n, err)) continue;
    const int pos = atomicSub(&count[t], 1) - 1;
    if (!in_bounds(pos >= 0 && off[t] + pos < bucket_cap, err)) continue;
    bucket[off[t] + pos] = pk[i];
  }
}

// ---- per-target select -----------------------------------------------------------------
// Inserts key b into a sorted, duplicate-free list (x0 holds elements 0..31 by lane, x1
// elements 32..63) that keeps the R smallest keys: a copy of an id already listed keeps
// the smaller key and the old bit of either copy.
__device__ __forceinline__ void list_insert(uint64_t& x0, uint64_t& x1, uint64_t b, int R) {
  const int lane = threadIdx.x & 31;
  const uint32_t idb = key_id(b);
  const unsigned d0 = __ballot_sync(0xffffffffu, x0 != kEmpty && key_id(x0) == idb);
  const unsigned d1 = __ballot_sync(0xffffffffu, x1 != kEmpty && key_id(x1) == idb);
  if (d0 | d1) {
    const int e = d0 ? __ffs(d0) - 1 : 32 + __ffs(d1) - 1;
    const uint64_t xe = __shfl_sync(0xffffffffu, e < 32 ? x0 : x1, e & 31);
    if ((b >> 1) >= (xe >> 1)) {  // the listed copy is not farther: keep it
      if (b & 1ull) {
        if (lane == e) x0 |= 1ull;
        if (lane + 32 == e) x1 |= 1ull;
      }
      return;
    }
    b |= xe & 1ull;  // the nearer copy replaces the listed one: remove element e first
    const uint64_t x1first = __shfl_sync(0xffffffffu, x1, 0);
    uint64_t n0 = __shfl_down_sync(0xffffffffu, x0, 1);
    uint64_t n1 = __shfl_down_sync(0xffffffffu, x1, 1);
    if (lane == 31) {
      n0 = x1first;
      n1 = kEmpty;
    }
    if (lane >= e) x0 = n0;
    if (lane + 32 >= e) x1 = n1;
  }
  const int pos = __popc(__ballot_sync(0xffffffffu, x0 < b)) + __popc(__ballot_sync(0xffffffffu, x1 < b));
  if (pos >= R) return;
  const uint64_t x0last = __shfl_sync(0xffffffffu, x0, 31);
  uint64_t u0 = __shfl_up_sync(0xffffffffu, x0, 1);
  uint64_t u1 = __shfl_up_sync(0xffffffffu, x1, 1);
  if (lane == 0) u1 = x0last;
  x0 = lane > pos ? u0 : (lane == pos ? b : x0);
  x1 = lane + 32 > pos ? u1 : (lane + 32 == pos ? b : x1);
  if (lane >= R) x0 = kEmpty;
  if (lane + 32 >= R) x1 = kEmpty;
}

// list_insert when every copy of an id carries one key up to the old bit (a build's canonical
// distances) and b is new: a copy already listed sits where b would go, and stays as it is.
// Keys compare through (key | 1), which orders them as (dist, id) whatever the old bits.
__device__ __forceinline__ void list_insert_exact(uint64_t& x0, uint64_t& x1, uint64_t b, int R) {
  const int lane = threadIdx.x & 31;
  const uint64_t bk = b | 1ull;
  const int pos = __popc(__ballot_sync(0xffffffffu, (x0 | 1ull) < bk)) + __popc(__ballot_sync(0xffffffffu, (x1 | 1ull) < bk));
  if (pos >= R) return;
  const uint64_t at = __shfl_sync(0xffffffffu, pos < 32 ? x0 : x1, pos & 31);
  if ((at | 1ull) == bk) return;  // listed already (an empty slot never matches a finite key)
  const uint64_t x0last = __shfl_sync(0xffffffffu, x0, 31);
  uint64_t u0 = __shfl_up_sync(0xffffffffu, x0, 1);
  uint64_t u1 = __shfl_up_sync(0xffffffffu, x1, 1);
  if (lane == 0) u1 = x0last;
  x0 = lane > pos ? u0 : (lane == pos ? b : x0);
  x1 = lane + 32 > pos ? u1 : (lane + 32 == pos ? b : x1);
  if (lane >= R) x0 = kEmpty;
  if (lane + 32 >= R) x1 = kEmpty;
}

// Per-warp scratch of merge_chunk.
struct __align__(16) MergeScratch {
  uint64_t row[64];   // the row as it came in (by index), then its kept entries, compacted
  uint64_t prop[32];  // the kept proposals, compacted
  uint64_t out[96];   // the merged row by rank
  uint32_t hid[128];  // hash of the row's ids (open addressing) ...
  uint8_t hix[128];   // ... and their row indices
  uint8_t rrm[64];    // row entry replaced by a nearer proposal
  uint8_t rold[64];   // row entry kept, with the old bit of a proposal
  uint32_t oid[128];  // hash of the ids the target's row held as old before its first chunk
};

__device__ __forceinline__ uint32_t id_slot(uint32_t id) { return (id * 0x9E3779B1u) >> 25; }

// Merges up to 32 proposals (key b per lane, kEmpty for none) into the sorted, duplicate-free
// row (x0: elements 0..31 by lane, x1: 32..63) that keeps the R smallest keys, under the
// merge rule (one copy per id: the smaller key, old if any copy is old):
//   proposals sorted; one copy per id among them (__match_any_sync); ids already in the row
//   found through a small hash of the row's ids, the nearer copy kept; then every kept
//   element's rank = its index in its own sorted list + the number of smaller keys in the
//   other list (binary search), which places it in the merged row.
__device__ __forceinline__ void merge_chunk(uint64_t& x0, uint64_t& x1, uint64_t b, int R, MergeScratch& ms) {
  const int lane = threadIdx.x & 31;
  const uint32_t below = lane == 0 ? 0u : (0xffffffffu >> (32 - lane));
  {
    uint64_t t[1] = {b};
    warp_sort_u64<1>(t);
    b = t[0];
  }
  const bool hb = b != kEmpty;
  const uint32_t idb = key_id(b);
  const unsigned same = __match_any_sync(0xffffffffu, hb ? idb : 0xffffffffu);
  const unsigned olds = __ballot_sync(0xffffffffu, hb && (b & 1ull));
  bool keep = hb && lane == __ffs(same) - 1;  // sorted: the first copy is the nearest
  if (keep && (olds & same)) b |= 1ull;
  ms.row[lane] = x0;
  ms.row[lane + 32] = x1;
  ms.rrm[lane] = ms.rrm[lane + 32] = 0;
  ms.rold[lane] = ms.rold[lane + 32] = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) ms.hid[lane + 32 * q] = 0xffffffffu;
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // the row's ids are distinct: each insert finds a free slot
    const uint64_t xk = h ? x1 : x0;
    if (xk != kEmpty) {
      const uint32_t id = key_id(xk);
      uint32_t sl = id_slot(id);
      for (int probe = 0; probe < 128; ++probe) {
        if (atomicCAS(&ms.hid[sl], 0xffffffffu, id) == 0xffffffffu) {
          ms.hix[sl] = (uint8_t)(lane + 32 * h);
          break;
        }
        sl = (sl + 1) & 127u;
      }
    }
  }
  __syncwarp();
  if (keep) {  // the id is listed already: the nearer copy stays, old if either is old
    uint32_t sl = id_slot(idb);
    for (int probe = 0; probe < 128; ++probe) {
      const uint32_t h = ms.hid[sl];
      if (h == idb) {
        const int e = ms.hix[sl];
        const uint64_t re = ms.row[e];
        if ((b >> 1) < (re >> 1)) {
          ms.rrm[e] = 1;
          b |= re & 1ull;
        } else {
          keep = false;
          if (b & 1ull) ms.rold[e] = 1;
        }
        break;
      }
      if (h == 0xffffffffu) break;
      sl = (sl + 1) & 127u;
    }
  }
  __syncwarp();
  const bool k0 = x0 != kEmpty && !ms.rrm[lane], k1 = x1 != kEmpty && !ms.rrm[lane + 32];
  if (ms.rold[lane]) x0 |= 1ull;
  if (ms.rold[lane + 32]) x1 |= 1ull;
  const unsigned kb = __ballot_sync(0xffffffffu, keep);
  const unsigned r0 = __ballot_sync(0xffffffffu, k0), r1 = __ballot_sync(0xffffffffu, k1);
  const int nb = __popc(kb), nr = __popc(r0) + __popc(r1);
  const int ib = __popc(kb & below), i0 = __popc(r0 & below), i1 = __popc(r0) + __popc(r1 & below);
  __syncwarp();
  if (keep) ms.prop[ib] = b;
  if (k0) ms.row[i0] = x0;
  if (k1) ms.row[i1] = x1;
  __syncwarp();
  // rank = own index + number of smaller keys in the other list
  if (keep) {
    int lo = 0, hi = nr;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((ms.row[mid] >> 1) < (b >> 1)) lo = mid + 1; else hi = mid;
    }
    ms.out[ib + lo] = b;
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const bool kk = h ? k1 : k0;
    if (kk) {
      const uint64_t xk = h ? x1 : x0;
      int lo = 0, hi = nb;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((ms.prop[mid] >> 1) < (xk >> 1)) lo = mid + 1; else hi = mid;
      }
      ms.out[(h ? i1 : i0) + lo] = xk;
    }
  }
  __syncwarp();
  const int tot = min(nb + nr, R);
  x0 = lane < tot ? ms.out[lane] : kEmpty;
  x1 = lane + 32 < tot ? ms.out[lane + 32] : kEmpty;
  __syncwarp();
}

// merge_chunk when every copy of an id proposed to the target carries the same distance (the
// pools' distances all come from the library's canonical FP32 arithmetic or exact tiles, as
// in a whole build) and the proposals are new: copies of one id then have equal keys up to the
// old bit, so duplicates are found by comparing keys, with no id hash and no sort:
//   gap    each proposal's lower bound lo in the row (the number of row entries with a smaller
//          key; a fixed six-step search), which is also where a row copy of it would sit (the
//          row's copy, old or not, is the one kept); proposals with lo >= R fall past the
//          truncation and take no further part (every kept proposal before them is smaller);
//   rank   the proposals ordered by gap: six ballots over the bits of lo give each proposal the
//          set of proposals in lower gaps and the set in its own gap; within a gap (mostly a
//          single proposal) duplicates keep their lowest lane, and keys are compared directly;
//   place  a kept proposal's merged position is its rank among the kept proposals plus lo; the
//          row entries fill the other positions in order, so position p that no proposal
//          took holds row entry p - (positions below p that proposals took): two ballots
//          (warp OR reductions) of the taken positions replace a search per row entry.
// Keys compare through (key | 1): (x | 1) < (y | 1) iff x >> 1 < y >> 1 (order and equality
// of (dist, id), whatever the old bits).
__device__ __forceinline__ void merge_chunk_exact(uint64_t& x0, uint64_t& x1, uint64_t b, int R, MergeScratch& ms) {
  const int lane = threadIdx.x & 31;
  const uint32_t below = lane == 0 ? 0u : (0xffffffffu >> (32 - lane));
  const uint64_t bk = b | 1ull;
  ms.row[lane] = x0;
  ms.row[lane + 32] = x1;
  const int nr = __popc(__ballot_sync(0xffffffffu, x0 != kEmpty)) + __popc(__ballot_sync(0xffffffffu, x1 != kEmpty));
  __syncwarp();
  // gap: row entries with a smaller key (empty slots, all ones, never are)
  int lo = 0;
#pragma unroll
  for (int st = 32; st > 0; st >>= 1)
    if ((ms.row[lo + st - 1] | 1ull) < bk) lo += st;
  if (lo == 63 && (ms.row[63] | 1ull) < bk) lo = 64;
  const bool cand = b != kEmpty && lo < R && (ms.row[lo] | 1ull) != bk;  // not listed already
  // rank: the proposals in lower gaps (lt) and in this one (eq), among the candidates
  unsigned eq = __ballot_sync(0xffffffffu, cand), lt = 0u;
#pragma unroll
  for (int bit = 5; bit >= 0; --bit) {
    const bool one = (lo >> bit) & 1;
    const unsigned B = __ballot_sync(0xffffffffu, one);
    lt |= one ? (eq & ~B) : 0u;
    eq &= one ? B : ~B;
  }
  ms.prop[lane] = bk;
  __syncwarp();
  const unsigned others = eq & ~(1u << lane);
  bool keep = cand;
  if (cand)
    for (unsigned g = others & below; g; g &= g - 1)
      if (ms.prop[__ffs(g) - 1] == bk) {  // a lower lane holds the same key
        keep = false;
        break;
      }
  const unsigned kb = __ballot_sync(0xffffffffu, keep);
  int w = 0;  // kept proposals of the same gap with a smaller key
  if (keep)
    for (unsigned g = others & kb; g; g &= g - 1) w += ms.prop[__ffs(g) - 1] < bk ? 1 : 0;
  // place
  const int pos = __popc(lt & kb) + w + lo;
  if (keep && pos < 64) ms.out[pos] = b;
  const unsigned t0 = __reduce_or_sync(0xffffffffu, (keep && pos < 32) ? 1u << pos : 0u);
  const unsigned t1 = __reduce_or_sync(0xffffffffu, (keep && pos >= 32 && pos < 64) ? 1u << (pos - 32) : 0u);
  __syncwarp();
  const int tot = min(__popc(kb) + nr, R);
  const int f0 = lane - __popc(t0 & below);                        // row entries before position lane
  const int f1 = 32 - __popc(t0) + lane - __popc(t1 & below);      // ... before position lane + 32
  x0 = lane < tot ? (((t0 >> lane) & 1u) ? ms.out[lane] : ms.row[f0]) : kEmpty;
  x1 = lane + 32 < tot ? (((t1 >> lane) & 1u) ? ms.out[lane + 32] : ms.row[f1]) : kEmpty;
  __syncwarp();
}

__global__ void __launch_bounds__(256, 5) select_kernel(SelectArgs a) {
  __shared__ MergeScratch scratch[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  MergeScratch& ms = scratch[warp];
  const int R = a.R;
  long long n_new = 0, n_in = 0;
  // in place (keys_out == keys_in): every row already holds the target's base pool
  const bool in_place = a.keys_out == a.keys_in;
  // the new-entry and proposal counts of the block's warps are added up in shared memory and
  // the last warp to leave adds them to the global counters (one atomic per block, not per
  // warp: the counters are two addresses that every block hits)
  __shared__ unsigned long long s_cnt[2];
  __shared__ int s_left;
  if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) s_left = blockDim.x >> 5;
  __syncthreads();
  auto leave = [&](long long nn, long long ni) {  // lane 0
    if (nn) atomicAdd(&s_cnt[0], (unsigned long long)nn);
    if (ni) atomicAdd(&s_cnt[1], (unsigned long long)ni);
    __threadfence_block();
    if (atomicSub(&s_left, 1) == 1) {  // the block's last warp
      __threadfence_block();
      if (s_cnt[0]) atomicAdd(reinterpret_cast<unsigned long long*>(a.round_new), s_cnt[0]);
      if (a.stats && s_cnt[1]) atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[6]), s_cnt[1]);
    }
  };
  if (*a.err) {
    if (lane == 0) leave(0, 0);
    return;
  }
  bool old_pass = a.old_pass != 0;
  if (!old_pass && a.qflags) {
    const float mxa = __uint_as_float(a.qflags[1]);
    old_pass = !(a.qflags[0] == 0u && (double)a.d * (double)mxa * (double)mxa < 16777216.0);
  }
  // a warp scans 32 consecutive targets at once (one per lane) and merges, one after the
  // other, only those that received proposals or still need their base pool copied
  for (int64_t u0 = ((int64_t)blockIdx.x * 8 + warp) * 32; u0 < a.n; u0 += (int64_t)gridDim.x * 8 * 32) {
    const int64_t ul = u0 + lane;
    int64_t b0l = 0;
    int cl = 0;  // a target's proposal count (its bucket count is an int32_t)
    bool keptl = true;
    if (ul < a.n) {
      if (a.bucket) {
        b0l = a.off[ul];
        cl = (int)(a.off[ul + 1] - b0l);
      }
      keptl = in_place || (a.active && a.active[ul]);
    }
    // a target with nothing proposed whose pool is in place is final already (and holds no
    // new entry: the join rewrote every row it pruned as old)
    unsigned work = __ballot_sync(0xffffffffu, ul < a.n && (cl != 0 || !keptl));
    const unsigned keptm = __ballot_sync(0xffffffffu, keptl);
    const bool merged_l = (work >> lane) & 1u;
    // the base pool sizes of the targets to merge, in one load
    const int nal = merged_l ? (keptl ? a.deg_out[ul] : a.deg_in[ul]) : 0;
    bool mynew = false;
    while (work) {
      const int tl = __ffs(work) - 1;
      work &= work - 1;
      const int64_t u = u0 + tl;
      const int64_t b0 = __shfl_sync(0xffffffffu, b0l, tl);
      const int c = __shfl_sync(0xffffffffu, cl, tl);
      const bool kept = (keptm >> tl) & 1u;
      if (!in_bounds(b0 >= 0 && c >= 0 && b0 + c <= a.n * R, a.err)) continue;
      const uint64_t* base = kept ? a.keys_out + u * R : a.keys_in + u * R;
      const int na = __shfl_sync(0xffffffffu, nal, tl);
      n_in += c;
      uint64_t out0, out1;
      if (c == 0) {
        out0 = lane < na ? base[lane] : kEmpty;
        out1 = lane + 32 < na ? base[32 + lane] : kEmpty;
      } else if (c <= 4) {  // a few proposals: insert them one by one into the sorted row
        out0 = lane < na ? base[lane] : kEmpty;
        out1 = lane + 32 < na ? base[32 + lane] : kEmpty;
        uint64_t bl = lane < c ? a.bucket[b0 + lane] : kEmpty;
        // Proposals are new; an id is old in the result iff the row held it as old.  An insert
        // can push that row entry out before a nearer copy of the same id arrives (copies can
        // differ in distance when the tiles are not exact), so proposals take the row's old
        // bit first.
        for (int t = 0; old_pass && t < (int)c; ++t) {
          const uint32_t idt = key_id(__shfl_sync(0xffffffffu, bl, t));
          const bool held = (out0 != kEmpty && (out0 & 1ull) && key_id(out0) == idt) ||
                            (out1 != kEmpty && (out1 & 1ull) && key_id(out1) == idt);
          if (__any_sync(0xffffffffu, held) && lane == t) bl |= 1ull;
        }
        if (old_pass || !a.keys_canonical)
          for (int t = 0; t < (int)c; ++t) list_insert(out0, out1, __shfl_sync(0xffffffffu, bl, t), R);
        else
          for (int t = 0; t < (int)c; ++t) list_insert_exact(out0, out1, __shfl_sync(0xffffffffu, bl, t), R);
      } else {  // chunks of 32 proposals merged into the row
        out0 = lane < na ? base[lane] : kEmpty;
        out1 = lane + 32 < na ? base[32 + lane] : kEmpty;
        // over several chunks, an earlier chunk can push an old row entry out before a later
        // one brings a nearer copy of its id: the ids the row holds as old are hashed first,
        // and each later proposal takes the old bit of its id
        const bool multi = old_pass && c > 32;
        if (multi) {
#pragma unroll
          for (int q = 0; q < 4; ++q) ms.oid[lane + 32 * q] = 0xffffffffu;
          __syncwarp();
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint64_t xk = h ? out1 : out0;
            if (xk != kEmpty && (xk & 1ull)) {  // the row's ids are distinct: a free slot is found
              const uint32_t id = key_id(xk);
              uint32_t sl = id_slot(id);
              for (int probe = 0; probe < 128; ++probe) {
                if (atomicCAS(&ms.oid[sl], 0xffffffffu, id) == 0xffffffffu) break;
                sl = (sl + 1) & 127u;
              }
            }
          }
          __syncwarp();
        }
        for (int64_t done = 0; done < c; done += 32) {
          uint64_t bl = done + lane < c ? a.bucket[b0 + done + lane] : kEmpty;
          if (multi && done > 0 && bl != kEmpty && !(bl & 1ull)) {
            const uint32_t idb = key_id(bl);
            uint32_t sl = id_slot(idb);
            for (int probe = 0; probe < 128; ++probe) {
              const uint32_t hv = ms.oid[sl];
              if (hv == idb) {
                bl |= 1ull;
                break;
              }
              if (hv == 0xffffffffu) break;
              sl = (sl + 1) & 127u;
            }
          }
          if (old_pass || !a.keys_canonical)
            merge_chunk(out0, out1, bl, R, ms);
          else
            merge_chunk_exact(out0, out1, bl, R, ms);
        }
      }
      if (lane >= R) out0 = kEmpty;
      if (lane + 32 >= R) out1 = kEmpty;
      const unsigned v0 = __ballot_sync(0xffffffffu, out0 != kEmpty);
      const unsigned v1 = __ballot_sync(0xffffffffu, out1 != kEmpty);
      const unsigned w0 = __ballot_sync(0xffffffffu, out0 != kEmpty && !(out0 & 1ull));
      const unsigned w1 = __ballot_sync(0xffffffffu, out1 != kEmpty && !(out1 & 1ull));
      if (lane < R) a.keys_out[u * R + lane] = out0;
      if (lane + 32 < R) a.keys_out[u * R + 32 + lane] = out1;
      if (lane == 0) a.deg_out[u] = __popc(v0) + __popc(v1);
      n_new += __popc(w0) + __popc(w1);
      if (lane == tl) mynew = (w0 | w1) != 0u;
    }
    if (a.next_active && ul < a.n && (merged_l || a.next_active_all)) a.next_active[ul] = mynew ? 1 : 0;
  }
  if (lane == 0) leave(n_new, n_in);
}

cudaError_t merge_tail(const Workspace& ws, const SelectArgs& sa, cudaStream_t st, bool new_cleared = false) {
  const int64_t n = ws.n;
  if (sa.bucket) {
    const int64_t nb = ceil_div(n, SCAN_TILE);
    {
      ProfScope ps("scan", st);
      scan_reduce_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(ws.count, n, ws.bsum);
      scan_apply_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(ws.count, n, ws.bsum, ws.off);
    }
    {
      ProfScope ps("scatter", st);
      scatter_kernel<<<(unsigned)(sm_count() * 8), 256, 0, st>>>(ws.red_tgt, ws.red_key, ws.red_n, ws.off,
                                                                 ws.count, ws.bucket, ws.err, n, ws.red_cap,
                                                                 n * ws.R);
    }
  }
  if (!new_cleared) cudaMemsetAsync(ws.round_new, 0, sizeof(int64_t), st);
  if (sa.R > kTeamMaxM) return launch_select_wide(sa, st);  // rows of more than 64 entries
  const int64_t blocks = std::min<int64_t>(ceil_div(n, 256), (int64_t)sm_count() * 16);
  ProfScope ps("select", st);
  select_kernel<<<(unsigned)blocks, 256, 0, st>>>(sa);
  return cudaGetLastError();
}

cudaError_t run_prep(const uint64_t* keys_in, const int32_t* deg_in, const Workspace& ws,
                     const PointsSet& P, const uint8_t* hint, int64_t* stats, cudaStream_t st,
                     bool clear_round = false) {
  const int64_t blocks = std::min<int64_t>(ceil_div(ws.n, kPrepWarps * 32), (int64_t)sm_count() * 8);
  ProfScope ps("prep", st);
  // the warp kernels take FP32 rows of up to 128 dimensions (BF16 rows of any length)
  const int warp_ok = (P.precision == 0 && P.d > 128) ? 0 : 1;
  RecSet rs;
  for (int c = 0; c < kNumClasses; ++c) {
    rs.rec[c] = ws.rec[c];
    rs.w[c] = ws.rec_w[c];
    rs.cap[c] = ws.rec_cap[c];
  }
  const int3 gmax = make_int3(P.group_max[0], P.group_max[1], P.group_max[2]);
  prep_kernel<<<(unsigned)blocks, kPrepWarps * 32, 0, st>>>(keys_in, deg_in, ws.n, ws.R, ws.active, ws.list_n, warp_ok,
                                                gmax, rs, P.vseg, hint, stats, clear_round ? ws.count : nullptr,
                                                clear_round ? ws.round_new : nullptr);
  return cudaGetLastError();
}

namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}
}  // namespace

// The quantized rows (n rows of ldb elements: bfloat16 for BF16, bytes for FP8) as a 2-D
// tensor map whose box is one staged row of the warp join (its 128-column chunk and the 16
// bytes after it) and one row high, for gather4 copies.  False (the join then copies row by
// row) when the rows do not meet the copy's rules: base 16-byte aligned, row pitch a multiple
// of 16 bytes, at most 2^31 - 1 rows.
bool encode_rows_map(TmaMap* m, const void* Xb, int64_t n, int ldb, int precision) {
  static_assert(sizeof(TmaMap) == sizeof(CUtensorMap) && alignof(TmaMap) >= 64, "tensor map layout");
  if (!Xb || n <= 0 || n > INT32_MAX || ldb <= 0) return false;
  const bool bf = precision == GRNND_BF16;
  if (!bf && precision != GRNND_FP8) return false;
  const int esz = bf ? 2 : 1;
  const cuuint32_t box = bf ? (cuuint32_t)WPrec<1>::RS : (cuuint32_t)WPrec<2>::RS;
  if ((reinterpret_cast<uintptr_t>(Xb) & 15u) || ((int64_t)ldb * esz) % 16 != 0) return false;
  const EncodeTiledFn f = encode_tiled();
  if (!f) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)ldb, (cuuint64_t)n};
  const cuuint64_t pitch[1] = {(cuuint64_t)ldb * (cuuint64_t)esz};
  const cuuint32_t boxd[2] = {box, 1u};
  const cuuint32_t es[2] = {1u, 1u};
  const CUresult r = f(reinterpret_cast<CUtensorMap*>(m), bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                       2u, const_cast<void*>(Xb), dims, pitch, boxd, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

JoinArgs make_join_args(const PointsSet& P, int64_t n, int R, const uint64_t* keys_in,
                        const int32_t* deg_in, uint64_t seed, int t1, int t2, int order,
                        const Workspace& ws, uint64_t* keys_out, int32_t* deg_out, int emit,
                        int64_t* stats) {
  JoinArgs a;
  // gather4 copies: fewer copy instructions, but 2-way bank conflicts in the tiles; measured
  // faster for BF16 rows of one 128-column chunk, slower for longer rows and for FP8
  const bool gather4 = P.row_copies == 2 || (P.row_copies == 0 && P.precision == GRNND_BF16 && P.d <= 128);
  a.rows_tma = (gather4 && P.Xb && (P.precision == GRNND_BF16 || P.precision == GRNND_FP8) &&
                encode_rows_map(&a.rows_map, P.Xb, n, P.ldb, P.precision))
                   ? 1
                   : 0;
  a.P.X = P.X;
  a.P.ld = P.ld;
  a.P.Xb = P.Xb;
  a.P.ldb = P.ldb;
  a.P.aux = P.aux;
  a.P.qflags = P.qflags;
  a.P.d = P.d;
  a.n = n;
  a.R = R;
  a.keys_in = keys_in;
  a.deg_in = deg_in;
  a.list_n = ws.list_n;
  for (int c = 0; c < kNumClasses; ++c) {
    a.rec[c] = ws.rec[c];
    a.rec_w[c] = ws.rec_w[c];
    a.rec_cap[c] = ws.rec_cap[c];
  }
  a.seed = seed;
  a.t1 = t1;
  a.t2 = t2;
  a.order = order;
  a.keys_out = keys_out;
  a.deg_out = deg_out;
  a.emit_redirects = emit;
  a.red_tgt = ws.red_tgt;
  a.red_key = ws.red_key;
  a.red_n = ws.red_n;
  a.red_cap = ws.red_cap;
  a.count = ws.count;
  a.stats = stats;
  a.err = ws.err;
  a.work_q = ws.work_q;
  a.warp_ctas = P.warp_ctas;
  a.team_ctas = P.team_ctas;
  return a;
}

template <int METRIC>
cudaError_t launch_warp_p(int prec, const JoinArgs& a, cudaStream_t st, const char* name, bool so) {
  if (prec == 2) return launch_join_warp_t<METRIC, 2>(a, st, name, so);
  if (prec == 1) return launch_join_warp_t<METRIC, 1>(a, st, name, so);
  return launch_join_warp_t<METRIC, 0>(a, st, name, so);
}
template <int METRIC>
cudaError_t launch_team_p(int prec, const JoinArgs& a, cudaStream_t st, const char* name, bool so) {
  if (prec == 2) return launch_join_team_t<METRIC, 2>(a, st, name, so);
  if (prec == 1) return launch_join_team_t<METRIC, 1>(a, st, name, so);
  return launch_join_team_t<METRIC, 0>(a, st, name, so);
}

cudaError_t dispatch_join(const PointsSet& P, const JoinArgs& a, cudaStream_t st, const char* name,
                          bool setup_only = false) {
  if (P.precision >= 1 && (!P.Xb || !P.aux || !P.qflags) && !setup_only) return cudaErrorInvalidValue;
  cudaError_t e;
  // pools of up to 32 entries: one warp per vertex; 33..64 entries: a two-warp team per
  // vertex (batched CTAs with dimension chunks for FP32 rows longer than 128)
  const char* wname = (name[0] == 'r') ? "rnd_join_warp" : "final_prune_warp";
  const bool so = setup_only;
  e = P.metric == 0 ? launch_warp_p<0>(P.precision, a, st, wname, so) : launch_warp_p<1>(P.precision, a, st, wname, so);
  if (e != cudaSuccess) return e;
  if (P.precision >= 1 || P.d <= 128) {  // pools of 33..64 entries: a two-warp team per vertex
    const char* tname = (name[0] == 'r') ? "rnd_join_team" : "final_prune_team";
    e = P.metric == 0 ? launch_team_p<0>(P.precision, a, st, tname, so)
                      : launch_team_p<1>(P.precision, a, st, tname, so);
  } else {  // FP32 rows of more than 128 dimensions: batched CTAs with dimension chunks
    e = P.metric == 0 ? launch_join_t<0, 0>(a, st, name, so) : launch_join_t<1, 0>(a, st, name, so);
  }
  if (e != cudaSuccess || so || a.R <= kTeamMaxM) return e;
  // pools of 65..R entries: the wide join, one CTA per vertex
  return launch_join_wide(a, P.metric, st, (name[0] == 'r') ? "rnd_join_wide" : "final_prune_wide");
}

}  // namespace

cudaError_t prepare_join_kernels(const PointsSet& P) {
  JoinArgs a{};
  a.P.d = P.d;
  return dispatch_join(P, a, nullptr, "rnd_join", true);
}

cudaError_t launch_round(const PointsSet& P, int64_t n, int R, const uint64_t* keys_in,
                         const int32_t* deg_in, uint64_t seed, int t1, int t2, int order,
                         const Workspace& ws, uint64_t* keys_out, int32_t* deg_out, int64_t* stats,
                         cudaStream_t st, bool use_hint, bool keys_canonical) {
  cudaError_t e;
  // list_n, red_n, the work queues and this step's status word with one memset where they are
  // adjacent (the workspace carve puts the status word 256 bytes after list_n); the redirect
  // counts and the new-entry counter are cleared by prep
  const bool adjacent = reinterpret_cast<char*>(ws.err) == reinterpret_cast<char*>(ws.list_n) + 256;
  if (adjacent) {
    if ((e = cudaMemsetAsync(ws.list_n, 0, 256 + 4, st)) != cudaSuccess) return e;
  } else {
    if ((e = cudaMemsetAsync(ws.list_n, 0, 48, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws.err, 0, 4, st)) != cudaSuccess) return e;
  }
  if ((e = run_prep(keys_in, deg_in, ws, P, use_hint ? ws.next_active : nullptr, stats, st, true)) != cudaSuccess)
    return e;
  const JoinArgs a = make_join_args(P, n, R, keys_in, deg_in, seed, t1, t2, order, ws, keys_out,
                                    deg_out, 1, stats);
  if ((e = dispatch_join(P, a, st, "rnd_join")) != cudaSuccess) return e;
  SelectArgs sa;
  sa.n = n;
  sa.R = R;
  sa.bucket = ws.bucket;
  sa.off = ws.off;
  sa.active = ws.active;
  sa.keys_in = keys_in;
  sa.deg_in = deg_in;
  sa.keys_out = keys_out;
  sa.deg_out = deg_out;
  sa.round_new = ws.round_new;
  sa.err = ws.err;
  sa.stats = stats;
  sa.next_active = keys_out == keys_in ? ws.next_active : nullptr;
  sa.next_active_all = 1;
  sa.old_pass = 0;
  sa.qflags = P.precision >= 1 ? P.qflags : nullptr;
  sa.d = P.d;
  sa.keys_canonical = keys_canonical ? 1 : 0;
  return merge_tail(ws, sa, st, true);
}

cudaError_t launch_final(const PointsSet& P, int64_t n, int R, const uint64_t* keys_in,
                         const int32_t* deg_in, uint64_t seed, int t1, int order,
                         const Workspace& ws, uint64_t* keys_out, int32_t* deg_out, cudaStream_t st,
                         bool use_hint) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws.list_n, 0, 48, st)) != cudaSuccess) return e;  // list_n, red_n, work queues
  if ((e = cudaMemsetAsync(ws.err, 0, 4, st)) != cudaSuccess) return e;  // this step's status
  if ((e = run_prep(keys_in, deg_in, ws, P, use_hint ? ws.next_active : nullptr, nullptr, st)) != cudaSuccess)
    return e;
  const JoinArgs a = make_join_args(P, n, R, keys_in, deg_in, seed, t1, 0, order, ws, keys_out,
                                    deg_out, 0, nullptr);
  if ((e = dispatch_join(P, a, st, "final_prune")) != cudaSuccess) return e;
  SelectArgs sa;
  sa.n = n;
  sa.R = R;
  sa.bucket = nullptr;
  sa.off = nullptr;
  sa.active = ws.active;
  sa.keys_in = keys_in;
  sa.deg_in = deg_in;
  sa.keys_out = keys_out;
  sa.deg_out = deg_out;
  sa.round_new = ws.round_new;
  sa.err = ws.err;
  sa.stats = nullptr;
  sa.next_active = nullptr;
  sa.next_active_all = 0;
  sa.old_pass = 0;  // no proposals
  sa.qflags = nullptr;
  sa.d = P.d;
  sa.keys_canonical = 0;
  return merge_tail(ws, sa, st);
}

// =====================================================================================
// Reverse-edge sampling (Sec 3.6): each vertex proposes itself to the first
// floor(rho * deg) entries of its row (the closest ones); every pool is then merged
// with the proposals it received.
// =====================================================================================
// Reverse sampling (Sec 3.6): row v proposes its first floor(rho * deg) entries u (its nearest)
// to u, as (d(v, u), v).  A block takes kRevRows rows at a time (each warp kRevRows / 8 of
// them): the rows' proposal counts are known before any is written, so the block adds them
// up and reserves its slots with one atomic (the slot counter is one address that every
// block hits).
constexpr int kRevWarps = 8, kRevRows = 32;
__global__ void __launch_bounds__(kRevWarps * 32) reverse_propose_kernel(
    int64_t n, int R, float rho, const uint64_t* __restrict__ keys, const int32_t* __restrict__ deg,
    int32_t* __restrict__ tgt, uint64_t* __restrict__ pk, unsigned long long* __restrict__ red_n,
    int32_t* __restrict__ count, int64_t red_cap, int32_t* __restrict__ err) {
  __shared__ int s_r[kRevRows];      // proposals of each row of the block's chunk
  __shared__ int s_pre[kRevRows];    // their first slot, from the chunk's base
  __shared__ unsigned long long s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t r0 = (int64_t)blockIdx.x * kRevRows; r0 < n; r0 += (int64_t)gridDim.x * kRevRows) {  // block-uniform
    if (threadIdx.x < kRevRows) {
      const int64_t v = r0 + threadIdx.x;
      s_r[threadIdx.x] = v < n ? (int)floor((double)rho * (double)deg[v]) : 0;
    }
    __syncthreads();
    if (warp == 0) {  // exclusive prefix over the chunk's rows, one per lane
      const int x = s_r[lane];
      int inc = x;
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, dd);
        if (lane >= dd) inc += y;
      }
      s_pre[lane] = inc - x;
      unsigned long long b = 0;
      if (lane == 31 && inc > 0) b = atomicAdd(red_n, (unsigned long long)inc);
      if (lane == 31) s_base = b;
    }
    __syncthreads();
    for (int q = warp; q < kRevRows; q += kRevWarps) {
      const int64_t v = r0 + q;
      const int r = s_r[q];
      const unsigned long long sb = s_base + (unsigned long long)s_pre[q];
      for (int j = lane; j < r; j += 32) {
        const uint64_t k = keys[v * R + j];
        const int32_t t = (int32_t)key_id(k);
        const unsigned long long slot = sb + (unsigned long long)j;
        if (in_bounds(slot < (unsigned long long)red_cap && (uint64_t)(uint32_t)t < (uint64_t)n, err)) {
          tgt[slot] = t;
          pk[slot] = (k & 0xFFFFFFFF00000000ull) | ((uint64_t)v << 1);
          atomicAdd(&count[t], 1);
        }
      }
    }
    __syncthreads();  // (s_r, s_pre and s_base are rewritten for the next chunk)
  }
}

cudaError_t launch_reverse(int64_t n, int R, float rho, const uint64_t* keys_in,
                           const int32_t* deg_in, const Workspace& ws, uint64_t* keys_out,
                           int32_t* deg_out, int64_t* stats, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws.count, 0, (size_t)n * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(ws.list_n, 0, 48, st)) != cudaSuccess) return e;  // list_n, red_n, work queues
  if ((e = cudaMemsetAsync(ws.err, 0, 4, st)) != cudaSuccess) return e;  // this step's status
  {
    const int64_t blocks = std::min<int64_t>(ceil_div(n, kRevRows), (int64_t)sm_count() * 16);
    ProfScope ps("reverse_propose", st);
    reverse_propose_kernel<<<(unsigned)blocks, kRevWarps * 32, 0, st>>>(n, R, rho, keys_in, deg_in, ws.red_tgt,
                                                            ws.red_key, ws.red_n, ws.count, ws.red_cap,
                                                            ws.err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  SelectArgs sa;
  sa.n = n;
  sa.R = R;
  sa.bucket = ws.bucket;
  sa.off = ws.off;
  sa.active = nullptr;
  sa.keys_in = keys_in;
  sa.deg_in = deg_in;
  sa.keys_out = keys_out;
  sa.deg_out = deg_out;
  sa.round_new = ws.round_new;
  sa.err = ws.err;
  sa.stats = stats;
  sa.next_active = keys_out == keys_in ? ws.next_active : nullptr;  // rows not merged keep their flag
  sa.next_active_all = 0;
  sa.old_pass = 1;  // the points (and so the exactness of the recorded distances) are not known here
  sa.keys_canonical = 0;
  sa.qflags = nullptr;
  sa.d = 0;
  return merge_tail(ws, sa, st);
}

// =====================================================================================
// Export of pool keys to (ids, dists) rows.
// =====================================================================================
__global__ void keys_to_graph_kernel(int64_t total, int R, const uint64_t* __restrict__ keys,
                                     int32_t* __restrict__ ids, float* __restrict__ dists) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    const bool e = (k == kEmpty);
    if (ids) ids[i] = e ? -1 : (int32_t)key_id(k);
    if (dists) dists[i] = e ? __int_as_float(0x7f800000) : key_dist(k);
  }
}

cudaError_t launch_keys_to_graph(int64_t n, int R, const uint64_t* keys, int32_t* ids,
                                 float* dists, int32_t* deg, cudaStream_t st) {
  (void)deg;
  const int64_t total = n * R;
  const int64_t blocks = std::min<int64_t>(ceil_div(total, 256), (int64_t)sm_count() * 32);
  ProfScope ps("export", st);
  keys_to_graph_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(total, R, keys, ids,
                                                                             dists);
  return cudaGetLastError();
}

// ---- workspace layout ------------------------------------------------------------------
namespace {
inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
}

namespace {
// work records of a size class: two words (v and its build's first id, m) per active vertex
// (classes 0..3 hold pools of up to min(R, 8 << c) entries; class 4, only when R > 64, up to R)
inline int rec_cap_of(int R, int c) { return c < 4 ? std::min(R, 8 << c) : (R > kTeamMaxM ? R : 0); }
inline int rec_words(int cap) { return cap > 0 ? 2 : 0; }  // v | build's first id, m
inline size_t rec_region_bytes(int64_t n, int R, int c) {
  const int cap = rec_cap_of(R, c);
  return cap > 0 ? al256((size_t)n * rec_words(cap) * 8) : 0;
}
inline size_t rec_bytes(int64_t n, int R) {
  size_t b = 0;
  for (int c = 0; c < kNumClasses; ++c) b += rec_region_bytes(n, R, c);
  return b;
}
// Redirect slots: a vertex loses at most m - 1 <= R - 1 entries (the one with the smallest
// (dist, id) is never the farther side of a fired pair), and the units of each of the two
// join kernels of a round fill their chunks completely before reserving the next, so each
// kernel leaves at most (its units x its chunk) <= kMaxJoinGrid x RED_CHUNK slots unused.
static_assert(WW * WRED <= RED_CHUNK && TRED <= RED_CHUNK, "per-CTA redirect reservation above the slack");
static_assert(BV * 63 <= RED_CHUNK && WM <= WRED && TM <= TRED, "a batch or vertex must fit one fresh chunk");
// (a third join kernel, the wide one, runs when R > 64)
inline size_t red_slots(int64_t n, int R) {
  return (size_t)n * R + (R > kTeamMaxM ? 3 : 2) * (size_t)kMaxJoinGrid * RED_CHUNK;
}
}  // namespace

size_t workspace_bytes(int64_t n, int R) {
  const size_t slots = red_slots(n, R);
  const size_t nb = (size_t)ceil_div(n, SCAN_TILE) + 1;
  return al256(slots * 4) + al256(slots * 8) + al256((size_t)n * R * 8) + al256((size_t)n * 4) +
         al256(((size_t)n + 1) * 8) + al256(nb * 8) + 2 * al256((size_t)n) + rec_bytes(n, R) + al256(48) +
         al256(4) + al256(8);
}

bool carve_workspace(void* base, size_t bytes, int64_t n, int R, Workspace* ws) {
  if (!base || bytes < workspace_bytes(n, R)) return false;
  if (((uintptr_t)base & 255u) != 0) return false;
  const size_t slots = red_slots(n, R);
  const size_t nb = (size_t)ceil_div(n, SCAN_TILE) + 1;
  char* p = static_cast<char*>(base);
  ws->n = n;
  ws->R = R;
  ws->red_tgt = reinterpret_cast<int32_t*>(p);
  ws->red_cap = (int64_t)slots;
  p += al256(slots * 4);
  ws->red_key = reinterpret_cast<uint64_t*>(p);
  p += al256(slots * 8);
  ws->bucket = reinterpret_cast<uint64_t*>(p);
  p += al256((size_t)n * R * 8);
  ws->count = reinterpret_cast<int32_t*>(p);
  p += al256((size_t)n * 4);
  ws->off = reinterpret_cast<int64_t*>(p);
  p += al256(((size_t)n + 1) * 8);
  ws->bsum = reinterpret_cast<int64_t*>(p);
  p += al256(nb * 8);
  ws->active = reinterpret_cast<uint8_t*>(p);
  p += al256((size_t)n);
  ws->next_active = reinterpret_cast<uint8_t*>(p);
  p += al256((size_t)n);
  for (int c = 0; c < kNumClasses; ++c) {
    ws->rec_cap[c] = rec_cap_of(R, c);
    ws->rec_w[c] = rec_words(ws->rec_cap[c]);
    ws->rec[c] = ws->rec_cap[c] > 0 ? reinterpret_cast<uint64_t*>(p) : nullptr;
    p += rec_region_bytes(n, R, c);
  }
  ws->list_n = reinterpret_cast<int32_t*>(p);  // [5] records per class, then the redirect count
  ws->red_n = reinterpret_cast<unsigned long long*>(p + 24);
  ws->work_q = reinterpret_cast<unsigned int*>(p + 32);  // [3] work queues of the warp and team joins, one spare
  p += al256(48);
  ws->err = reinterpret_cast<int32_t*>(p);
  p += al256(4);
  ws->round_new = reinterpret_cast<int64_t*>(p);
  return true;
}

}  // namespace grnnd
