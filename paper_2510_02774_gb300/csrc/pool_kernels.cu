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
#include <cuda_bf16.h>

#include <cstdio>

#include "common.cuh"
#include "internal.h"

namespace grnnd {

namespace {

constexpr uint32_t kWaitLimit = 1u << 24;

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ uint64_t bits_below(int i) { return i == 0 ? 0ull : (~0ull >> (64 - i)); }

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

}  // namespace

int sm_count() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    cached = c > 0 ? c : 152;
  }
  return cached;
}

// =====================================================================================
// rnd_init: one warp per vertex.
//   Sampling follows the sequential definition exactly: candidate j = 0, 1, 2, ... is
//   accepted iff its id differs from every earlier accepted id, until S are accepted.
//   32 candidates are tested per step; a lane is rejected if its id matches an accepted
//   id or an earlier lane of the same step.
// =====================================================================================
template <int METRIC>
__global__ void __launch_bounds__(256) rnd_init_kernel(const float* __restrict__ X, int64_t n,
                                                        int d, int ld, int S, int R, uint64_t seed,
                                                        uint64_t* __restrict__ keys,
                                                        int32_t* __restrict__ deg) {
  __shared__ int32_t acc_ids[8][kMaxR];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* acc = acc_ids[warp];
  const uint64_t nm1 = (uint64_t)(n - 1);
  const unsigned below = lanemask_lt();
  for (int64_t v = (int64_t)blockIdx.x * 8 + warp; v < n; v += (int64_t)gridDim.x * 8) {
    int cnt = 0;
    // S <= n - 1, so the draws cover enough distinct ids long before the bound.
    for (uint64_t base = 0; cnt < S && base < (1ull << 32); base += 32) {
      const uint64_t r = counter_hash(seed, 0, 0, (uint64_t)v, base + lane) % nm1;
      const int32_t u = (int32_t)(r + (r >= (uint64_t)v ? 1u : 0u));
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
    const float* xv = X + v * (int64_t)ld;
    uint64_t kk[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int e = j * 32 + lane;
      kk[j] = kEmpty;
      if (e < S) {
        const int32_t u = acc[e];
        kk[j] = make_key(row_dist<METRIC>(xv, X + (int64_t)u * ld, d), (uint32_t)u, 0u);
      }
    }
    warp_sort_u64<2>(kk);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int e = j * 32 + lane;
      if (e < R) keys[v * R + e] = kk[j];
    }
    if (lane == 0) deg[v] = S;
    __syncwarp();
  }
}

cudaError_t launch_pool_init(const float* X, int64_t n, int d, int ld, int metric, int S, int R,
                             uint64_t seed, uint64_t* keys, int32_t* deg, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>(ceil_div(n, 8), (int64_t)sm_count() * 16);
  ProfScope ps("rnd_init", st);
  if (metric == 0)
    rnd_init_kernel<0><<<(unsigned)blocks, 256, 0, st>>>(X, n, d, ld, S, R, seed, keys, deg);
  else
    rnd_init_kernel<1><<<(unsigned)blocks, 256, 0, st>>>(X, n, d, ld, S, R, seed, keys, deg);
  return cudaGetLastError();
}

// =====================================================================================
// quantize: BF16 rows (ldb = d rounded up to 16, zero padded), aux = (norm^2 of the BF16
// row, ||x - bf16(x)|| rounded up), and dataset flags: qflags[0] bit 0 = some value is
// not an integer, bit 1 = some value is not exact in BF16; qflags[1] = max |x| (bits).
// =====================================================================================
__global__ void quantize_kernel(const float* __restrict__ X, int64_t n, int d, int ld,
                                __nv_bfloat16* __restrict__ Xb, int ldb, float2* __restrict__ aux,
                                unsigned* __restrict__ qflags) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned fl = 0, mx = 0;
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; r < n;
       r += (int64_t)gridDim.x * (blockDim.x >> 5)) {
    float nrm = 0.0f;
    double res = 0.0;
    for (int k = lane; k < ldb; k += 32) {
      const float x = k < d ? X[r * ld + k] : 0.0f;
      const __nv_bfloat16 b = __float2bfloat16_rn(x);
      Xb[r * ldb + k] = b;
      const float xf = __bfloat162float(b);
      nrm = __fmaf_rn(xf, xf, nrm);
      const double e = (double)x - (double)xf;
      res += e * e;
      fl |= (x != rintf(x)) ? 1u : 0u;
      fl |= (xf != x) ? 2u : 0u;
      mx = max(mx, __float_as_uint(fabsf(x)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
      res += __shfl_xor_sync(0xffffffffu, res, o);
    }
    if (lane == 0) aux[r] = make_float2(nrm, __double2float_ru(sqrt(res) * (1.0 + 1e-12)));
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
                            float2* aux, unsigned* qflags, cudaStream_t st) {
  __nv_bfloat16* Xb = static_cast<__nv_bfloat16*>(Xbv);
  cudaError_t e = cudaMemsetAsync(qflags, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::min<int64_t>(ceil_div(n, 8), (int64_t)sm_count() * 16);
  ProfScope ps("quantize", st);
  quantize_kernel<<<(unsigned)blocks, 256, 0, st>>>(X, n, d, ld, Xb, ldb, aux, qflags);
  return cudaGetLastError();
}

// =====================================================================================
// prep: active flag and list of the vertices whose pool holds a new entry; counts the
// entries of every pool (each one is proposed once, explicitly or in place).
// =====================================================================================
__global__ void prep_kernel(const uint64_t* __restrict__ keys, const int32_t* __restrict__ deg,
                            int64_t n, int R, uint8_t* __restrict__ active,
                            int32_t* __restrict__ list, int32_t* __restrict__ list_n,
                            int64_t* __restrict__ stats) {
  const int lane = threadIdx.x & 31;
  long long props = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t v = base + lane;
    bool act = false;
    if (v < n) {
      const int m = deg[v];
      props += m;
      for (int j = 0; j < m && !act; ++j) act = !(keys[v * R + j] & 1ull);
      active[v] = act ? 1 : 0;
    }
    const unsigned b = __ballot_sync(0xffffffffu, act);
    int off = 0;
    if (lane == 0 && b) off = atomicAdd(list_n, __popc(b));
    off = __shfl_sync(0xffffffffu, off, 0);
    if (act) list[off + __popc(b & lanemask_lt())] = (int32_t)v;
  }
  if (stats) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) props += __shfl_xor_sync(0xffffffffu, props, o);
    if (lane == 0 && props) atomicAdd(reinterpret_cast<unsigned long long*>(&stats[4]), (unsigned long long)props);
  }
}

// =====================================================================================
// rnd_join.  One CTA works through the active list, one vertex at a time, with a
// two-stage pipeline: while a vertex is computed, the rows of the next one are already
// on their way into the other shared-memory stage (one bulk copy per row by the TMA
// engine, completion on an mbarrier).  Per vertex v with m pool entries, k of them new:
//
//  1. visit order pi = rank of (h(seed,t1,t2,v,id), id) (or ascending / descending key);
//  2. rows staged new-first, so the pairs with a new side -- the only ones that can fire
//     (design reading C10) -- are rows i < k, j > i: a dense list of k(m-1) - k(k-1)/2;
//  3. dist_tile, FP32 form: one thread per pair, the canonical four-accumulator FP32
//     distance over dimension chunks of DC; BF16 form: Gram tiles on the tensor cores
//     (mma.sync m16n8k16, FP32 accumulate), D = (|x_i|^2 - g) + (|x_j|^2 - g), with a
//     per-pair error bound; a decision inside the bound is re-taken with canonical FP32
//     distances read from the FP32 rows;
//  4. rng_prune: fire bits F[b] = {a < b : d(a,b) < max(d(v,a), d(v,b))} in pi order; the
//     sequential pair scan of Alg 4 is resolved column by column with 64-bit masks: in
//     column b the live firing a's below the first a that makes b the far side become
//     bottom, and b becomes bottom if such an a exists;
//  5. survivors are written in key order into the output pool (old); each bottom entry
//     becomes one redirect (its absorber, distance d(close, far), new) in a compact list.
// =====================================================================================
namespace {

constexpr int JT = 256;                        // threads per join CTA
constexpr int JW = JT / 32;                    // warps per join CTA
constexpr int MAXP = kMaxR * (kMaxR - 1) / 2;  // 2016 pairs at most
constexpr int PPT = (MAXP + JT - 1) / JT;      // pairs per thread in the FP32 tile
constexpr int MAXTILE = 32;                    // 16 x 8 output tiles of a 64-row vertex
constexpr int TPW = MAXTILE / JW;              // tiles per warp in the BF16 tile

template <int PREC>
struct Prec;
template <>
struct Prec<0> {
  using T = float;
  static constexpr int DC = 128;        // dimensions per staged chunk
  static constexpr int RS = DC + 4;     // row stride: rows fall on different banks
  static constexpr int VEC = 4;         // elements per 16 bytes
};
template <>
struct Prec<1> {
  using T = __nv_bfloat16;
  static constexpr int DC = 128;
  static constexpr int RS = DC + 8;     // 272-byte rows: ldmatrix rows hit distinct banks
  static constexpr int VEC = 16;        // copy granule: whole k16 steps (32 bytes)
};

struct __align__(16) Meta {
  uint64_t pkey[kMaxR];      // key by pi position
  uint64_t skey[kMaxR];      // key by storage slot
  uint64_t hk[kMaxR];        // order key by storage slot
  uint64_t bfar[kMaxR];      // bits a < b with key(a) < key(b)
  int32_t pid[kMaxR];        // id by pi position
  int32_t rowoff[kMaxR + 1]; // first pair index of new row i
  float rnrm[kMaxR];         // BF16 form: norm^2 of the quantized row, by row
  float rdq[kMaxR];          // BF16 form: quantization residual norm, by row
  int16_t pos_of_slot[kMaxR];
  int16_t row_of_pos[kMaxR];
  int16_t pos_of_row[kMaxR];
  uint8_t tiles[MAXTILE];    // BF16 form: (I << 4) | J of the output tiles with a pair
  uint64_t newm;
  int64_t v;
  float vnrm, vdq;
  int m, k, npairs, nchunks, ntiles;
};

template <int PREC>
struct __align__(16) JoinSmem {
  typename Prec<PREC>::T rows[2][kMaxR][Prec<PREC>::RS];
  Meta meta[2];
  float pd[MAXP];           // pair distances in pair-list order
  uint64_t fire[kMaxR];
  int32_t killer[kMaxR];
  uint64_t bar[2];
  uint64_t alive;
  uint64_t mask2;
  unsigned long long red_base;
};

struct PointsDev {
  const float* X;
  int ld;
  const __nv_bfloat16* Xb;
  int ldb;
  const float2* aux;
  const unsigned* qflags;
  int d;
};

struct JoinArgs {
  PointsDev P;
  int64_t n;
  int R;
  const uint64_t* keys_in;
  const int32_t* deg_in;
  const int32_t* list;
  const int32_t* list_n;
  uint64_t seed;
  int t1, t2, order;
  uint64_t* keys_out;  // survivors (in place for the round, final graph for the last pass)
  int32_t* deg_out;
  int emit_redirects;
  int32_t* red_tgt;
  uint64_t* red_key;
  unsigned long long* red_n;
  int32_t* count;
  int64_t* stats;
  int32_t* err;
};

// ---- per-vertex set-up (all threads) --------------------------------------------------------
template <int PREC>
__device__ void join_setup(Meta& M, int64_t v, const JoinArgs& a) {
  const int tid = threadIdx.x;
  const int R = a.R;
  const int m = a.deg_in[v];
  const uint64_t kk = (tid < m) ? a.keys_in[v * R + tid] : kEmpty;
  if (tid < m) {
    const uint32_t id = key_id(kk);
    M.skey[tid] = kk;
    M.hk[tid] = (a.order == 0)   ? counter_hash(a.seed, (uint64_t)a.t1, (uint64_t)a.t2,
                                                (uint64_t)v, (uint64_t)id)
                : (a.order == 1) ? (uint64_t)tid
                                 : (uint64_t)(m - 1 - tid);
  }
  __syncthreads();
  if (tid < m) {
    const uint64_t h = M.hk[tid];
    const uint32_t id = key_id(kk);
    int p = 0;
    for (int j = 0; j < m; ++j) {
      const uint64_t hj = M.hk[j];
      p += (hj < h) || (hj == h && key_id(M.skey[j]) < id);
    }
    M.pos_of_slot[tid] = (int16_t)p;
    M.pkey[p] = kk;
    M.pid[p] = (int32_t)id;
  }
  __syncthreads();
  if (tid < 64) {
    const bool nw = tid < m && !key_old(M.pkey[tid]);
    const unsigned b = __ballot_sync(0xffffffffu, nw);
    if ((tid & 31) == 0) reinterpret_cast<uint32_t*>(&M.newm)[tid >> 5] = b;
  }
  __syncthreads();
  const uint64_t newm = M.newm;
  const int k = __popcll(newm);
  const uint64_t valid = (m >= 64) ? ~0ull : ((1ull << m) - 1ull);
  const int npairs = k * (m - 1) - k * (k - 1) / 2;
  if (tid < m) {
    const uint64_t lo = bits_below(tid);
    const int row = ((newm >> tid) & 1ull) ? __popcll(newm & lo) : k + __popcll(~newm & valid & lo);
    M.row_of_pos[tid] = (int16_t)row;
    M.pos_of_row[row] = (int16_t)tid;
    const uint64_t kb = M.pkey[tid] >> 1;
    uint64_t bf = 0;
    for (int q = 0; q < tid; ++q) bf |= ((M.pkey[q] >> 1) < kb ? 1ull : 0ull) << q;
    M.bfar[tid] = bf;
    if (PREC == 1) {
      const float2 x = a.P.aux[M.pid[tid]];
      M.rnrm[row] = x.x;
      M.rdq[row] = x.y;
    }
  }
  if (tid <= k) M.rowoff[tid] = tid * (m - 1) - tid * (tid - 1) / 2;
  if (tid == 0) {
    M.v = v;
    M.m = m;
    M.k = k;
    M.npairs = npairs;
    M.nchunks = npairs > 0 ? (a.P.d + Prec<PREC>::DC - 1) / Prec<PREC>::DC : 0;
    if (PREC == 1) {
      const float2 x = a.P.aux[v];
      M.vnrm = x.x;
      M.vdq = x.y;
      int nt = 0;
      const int KI = (k + 15) >> 4, NJ = (m + 7) >> 3;
      for (int I = 0; I < KI; ++I)
        for (int J = 0; J < NJ; ++J)
          if (J * 8 + 7 > I * 16) M.tiles[nt++] = (uint8_t)((I << 4) | J);
      M.ntiles = nt;
    }
  }
  __syncthreads();
}

// ---- bulk copies of one chunk of a vertex's rows (thread 0) ----------------------------------
template <int PREC>
__device__ __forceinline__ void join_issue(JoinSmem<PREC>& s, const Meta& M, int chunk, int buf,
                                           const JoinArgs& a) {
  using C = Prec<PREC>;
  const int c0 = chunk * C::DC;
  const int clen = min(C::DC, a.P.d - c0);
  const int cpy = (clen + C::VEC - 1) / C::VEC * C::VEC;
  const uint32_t bytes = (uint32_t)(cpy * sizeof(typename C::T));
  mbar_expect_tx(&s.bar[buf], (uint32_t)M.m * bytes);
  for (int p = 0; p < M.m; ++p) {
    const typename C::T* src =
        (PREC == 0) ? reinterpret_cast<const typename C::T*>(a.P.X + (int64_t)M.pid[p] * a.P.ld + c0)
                    : reinterpret_cast<const typename C::T*>(a.P.Xb + (int64_t)M.pid[p] * a.P.ldb + c0);
    bulk_g2s(&s.rows[buf][M.row_of_pos[p]][0], src, bytes, &s.bar[buf]);
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
  const int list_n = *a.list_n;
  int64_t idx = blockIdx.x;
  if (idx >= list_n) return;
  if (tid == 0) {
    mbar_init(&s.bar[0], 1);
    mbar_init(&s.bar[1], 1);
    fence_mbar_init();
  }
  if (tid < 64) {
    s.fire[tid] = 0;
    s.killer[tid] = -1;
  }
  __syncthreads();
  bool exact = false;
  if (PREC == 1) {
    const unsigned fl = a.P.qflags[0];
    const float mx = __uint_as_float(a.P.qflags[1]);
    exact = (fl == 0u) && ((double)a.P.d * (double)mx * (double)mx < 16777216.0);
  }
  const int R = a.R;
  uint32_t ph[2] = {0u, 0u};
  long long st_vert = 0, st_rows = 0, st_pairs = 0, st_fired = 0, st_check = 0;

  join_setup<PREC>(s.meta[0], a.list[idx], a);
  if (tid == 0 && s.meta[0].nchunks > 0) join_issue<PREC>(s, s.meta[0], 0, 0, a);
  int mcur = 0, ccur = 0, bcur = 0;

  float4 facc[PREC == 0 ? PPT : 1];
  float cacc[PREC == 1 ? TPW : 1][4];

  for (;;) {
    Meta& M = s.meta[mcur];
    // ---- next stage: the next chunk of this vertex, or the next vertex ----------------
    int mnext = mcur, cnext = ccur + 1;
    bool have_next = true;
    if (cnext >= M.nchunks) {
      const int64_t nidx = idx + gridDim.x;
      if (nidx < list_n) {
        mnext = mcur ^ 1;
        cnext = 0;
        join_setup<PREC>(s.meta[mnext], a.list[nidx], a);
      } else {
        have_next = false;
      }
    }
    if (have_next && tid == 0 && s.meta[mnext].nchunks > 0)
      join_issue<PREC>(s, s.meta[mnext], cnext, bcur ^ 1, a);

    // ---- current stage: accumulate one chunk of the tile --------------------------------
    if (M.nchunks > 0) {
      const bool ok = mbar_wait(&s.bar[bcur], ph[bcur], kWaitLimit);
      ph[bcur] ^= 1u;
      if (__syncthreads_or(!ok)) {
        // a bounded wait gave up: report, let in-flight copies land, and stop.
        if (tid == 0) atomicExch(a.err, kErrTimeout);
        if (!ok) mbar_wait(&s.bar[bcur], ph[bcur] ^ 1u, kWaitLimit);
        if (have_next && s.meta[mnext].nchunks > 0) mbar_wait(&s.bar[bcur ^ 1], ph[bcur ^ 1], kWaitLimit);
        return;
      }
      const int c0 = ccur * C::DC;
      const int clen = min(C::DC, a.P.d - c0);
      const bool last = (ccur + 1 == M.nchunks);
      if (PREC == 0) {
        const float* rows = reinterpret_cast<const float*>(&s.rows[bcur][0][0]);
        const int full4 = clen & ~3, rem = clen & 3;
        int i = 0;
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
          const int q = tid + r * JT;
          if (q < M.npairs) {
            while (M.rowoff[i + 1] <= q) ++i;
            const int j = i + 1 + (q - M.rowoff[i]);
            const float* ra = rows + i * C::RS;
            const float* rb = rows + j * C::RS;
            if (ccur == 0) facc[r] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float4 acc = facc[r];
            for (int t = 0; t < full4; t += 4)
              dist_step4<METRIC>(acc, *reinterpret_cast<const float4*>(ra + t),
                                 *reinterpret_cast<const float4*>(rb + t));
            if (rem)
              dist_step4<METRIC>(acc, mask4(*reinterpret_cast<const float4*>(ra + full4), rem),
                                 mask4(*reinterpret_cast<const float4*>(rb + full4), rem));
            facc[r] = acc;
            if (last) s.pd[q] = dist_finish4<METRIC>(acc);
          }
        }
      } else {
        const __nv_bfloat16* rows = reinterpret_cast<const __nv_bfloat16*>(&s.rows[bcur][0][0]);
        const int ksteps = (clen + 15) >> 4;
#pragma unroll
        for (int t = 0; t < TPW; ++t) {
          const int ti = warp + t * JW;
          if (ti < M.ntiles) {
            const int I = M.tiles[ti] >> 4, J = M.tiles[ti] & 15;
            if (ccur == 0) cacc[t][0] = cacc[t][1] = cacc[t][2] = cacc[t][3] = 0.0f;
            const __nv_bfloat16* pa = rows + (I * 16 + (lane & 15)) * C::RS + ((lane >> 4) << 3);
            const __nv_bfloat16* pb = rows + (J * 8 + (lane & 7)) * C::RS + (((lane >> 3) & 1) << 3);
            for (int ks = 0; ks < ksteps; ++ks) {
              uint32_t fa[4], fb[2];
              ldmatrix_x4(fa, pa + ks * 16);
              ldmatrix_x2(fb, pb + ks * 16);
              mma_bf16(cacc[t], fa, fb);
            }
            if (last) {
              const int g = lane >> 2, tg = lane & 3;
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int i = I * 16 + g + ((e >> 1) << 3);
                const int j = J * 8 + 2 * tg + (e & 1);
                if (i < M.k && j > i && j < M.m) {
                  const float gij = cacc[t][e];
                  float Dt;
                  if (METRIC == 0)
                    Dt = __fadd_rn(__fsub_rn(M.rnrm[i], gij), __fsub_rn(M.rnrm[j], gij));
                  else
                    Dt = __fsub_rn(1.0f, gij);
                  s.pd[M.rowoff[i] + (j - i - 1)] = Dt;
                }
              }
            }
          }
        }
      }
    }
    __syncthreads();

    // ---- last chunk done: prune and emit ---------------------------------------------
    if (ccur + 1 >= M.nchunks) {
      const int m = M.m;
      const int64_t v = M.v;
      const uint64_t valid = (m >= 64) ? ~0ull : ((1ull << m) - 1ull);
      {
        int i = 0;
        for (int q = tid; q < M.npairs; q += JT) {
          while (M.rowoff[i + 1] <= q) ++i;
          const int j = i + 1 + (q - M.rowoff[i]);
          const int pa = M.pos_of_row[i], pb = M.pos_of_row[j];
          const int lo = min(pa, pb), hi = max(pa, pb);
          const float dab = s.pd[q];
          const float dva = key_dist(M.pkey[pa]), dvb = key_dist(M.pkey[pb]);
          const float mx = fmaxf(dva, dvb);
          bool fire = dab < mx;
          if (PREC == 1 && !exact) {
            const float tol = bf16_bound<METRIC>(dab, M.rnrm[i], M.rnrm[j], M.rdq[i], M.rdq[j], a.P.d) +
                              fmaxf(bf16_bound<METRIC>(dva, M.vnrm, M.rnrm[i], M.vdq, M.rdq[i], a.P.d),
                                    bf16_bound<METRIC>(dvb, M.vnrm, M.rnrm[j], M.vdq, M.rdq[j], a.P.d));
            if (fabsf(dab - mx) <= tol) {  // re-decide with canonical FP32 distances
              const float* xv = a.P.X + v * a.P.ld;
              const float* xa = a.P.X + (int64_t)M.pid[pa] * a.P.ld;
              const float* xb = a.P.X + (int64_t)M.pid[pb] * a.P.ld;
              const float d_ab = row_dist<METRIC>(xa, xb, a.P.d);
              const float d_va = row_dist<METRIC>(xv, xa, a.P.d);
              const float d_vb = row_dist<METRIC>(xv, xb, a.P.d);
              fire = d_ab < fmaxf(d_va, d_vb);
              s.pd[q] = d_ab;
              ++st_check;
            }
          }
          if (fire) atomicOr(reinterpret_cast<unsigned long long*>(&s.fire[hi]), 1ull << lo);
        }
      }
      __syncthreads();
      if (tid == 0) {
        uint64_t alive = valid;
        for (int b = 1; b < m; ++b) {
          const uint64_t cand = s.fire[b] & alive;
          if (!cand) continue;
          const uint64_t x = cand & M.bfar[b];
          uint64_t kill = cand;
          if (x) {
            const int f = __ffsll((long long)x) - 1;
            kill = cand & bits_below(f);
            alive &= ~(1ull << b);
            s.killer[b] = f;
          }
          alive &= ~kill;
          while (kill) {
            const int q = __ffsll((long long)kill) - 1;
            s.killer[q] = b;
            kill &= kill - 1;
          }
        }
        s.alive = alive;
        const int ndead = m - __popcll(alive);
        if (a.emit_redirects && ndead > 0) s.red_base = atomicAdd(a.red_n, (unsigned long long)ndead);
        if (M.npairs > 0) {
          st_vert += 1;
          st_rows += m;
          st_pairs += M.npairs;
        }
        st_fired += ndead;
      }
      __syncthreads();
      const uint64_t alive = s.alive;
      // survivors, in key order, into the output pool
      if (tid < 64) {
        const bool al = tid < m && ((alive >> M.pos_of_slot[tid]) & 1ull);
        const unsigned b = __ballot_sync(0xffffffffu, al);
        if ((tid & 31) == 0) reinterpret_cast<uint32_t*>(&s.mask2)[tid >> 5] = b;
      }
      if (a.emit_redirects && tid < m && !((alive >> tid) & 1ull)) {
        const int cpos = s.killer[tid];
        const int ri = M.row_of_pos[cpos], rj = M.row_of_pos[tid];
        const int i = min(ri, rj), j = max(ri, rj);
        const float dd = s.pd[M.rowoff[i] + (j - i - 1)];
        const int32_t tgt = M.pid[cpos];
        const unsigned long long slot = s.red_base + (unsigned long long)__popcll(~alive & valid & bits_below(tid));
        a.red_tgt[slot] = tgt;
        a.red_key[slot] = make_key(dd, (uint32_t)M.pid[tid], 0u);
        atomicAdd(&a.count[tgt], 1);
      }
      __syncthreads();
      const uint64_t sm = s.mask2;
      const int cnt = __popcll(sm);
      if (tid < m && ((sm >> tid) & 1ull))
        a.keys_out[v * R + __popcll(sm & bits_below(tid))] = M.skey[tid] | 1ull;
      if (tid >= cnt && tid < R) a.keys_out[v * R + tid] = kEmpty;
      if (tid == 0) a.deg_out[v] = cnt;
      if (tid < 64) {
        s.fire[tid] = 0;
        s.killer[tid] = -1;
      }
      __syncthreads();
      idx += gridDim.x;
    }
    if (!have_next) break;
    mcur = mnext;
    ccur = cnext;
    bcur ^= 1;
  }
  if (tid == 0 && a.stats) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[0]), (unsigned long long)st_vert);
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[1]), (unsigned long long)st_rows);
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[2]), (unsigned long long)st_pairs);
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[3]), (unsigned long long)st_fired);
  }
  if (a.stats && PREC == 1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) st_check += __shfl_xor_sync(0xffffffffu, st_check, o);
    if (lane == 0 && st_check) atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[7]), (unsigned long long)st_check);
  }
}

template <int METRIC, int PREC>
cudaError_t launch_join_t(const JoinArgs& a, cudaStream_t st, const char* name) {
  const size_t smem = sizeof(JoinSmem<PREC>);
  static bool attr_set = false;
  auto kern = rnd_join_kernel<METRIC, PREC>;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, JT, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t blocks = std::min<int64_t>(std::max<int64_t>(a.n, 1), (int64_t)sm_count() * per_sm);
  ProfScope ps(name, st);
  kern<<<(unsigned)blocks, JT, smem, st>>>(a);
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

// Single block: exclusive scan of nb block sums in place, total to off[n].
__global__ void __launch_bounds__(1024) scan_blocks_kernel(int64_t* __restrict__ bsum, int64_t nb,
                                                           int64_t* __restrict__ off_total) {
  __shared__ int64_t wsum[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < nb; base += 1024) {
    const int64_t idx = base + threadIdx.x;
    const int64_t x = idx < nb ? bsum[idx] : 0;
    int64_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      int64_t w = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    const int64_t wpre = warp > 0 ? wsum[warp - 1] : 0;
    const int64_t c = carry;
    if (idx < nb) bsum[idx] = c + wpre + inc - x;
    __syncthreads();
    if (threadIdx.x == 1023) carry = c + wpre + inc;
    __syncthreads();
  }
  if (threadIdx.x == 0) *off_total = carry;
}

__global__ void __launch_bounds__(SCAN_T) scan_apply_kernel(const int32_t* __restrict__ cnt,
                                                            int64_t n,
                                                            const int64_t* __restrict__ bpre,
                                                            int64_t* __restrict__ off) {
  __shared__ int64_t wsum[SCAN_T / 32];
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
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  int64_t wpre = 0;
  for (int w = 0; w < warp; ++w) wpre += wsum[w];
  int64_t run = bpre[blockIdx.x] + wpre + inc - tsum;
#pragma unroll
  for (int i = 0; i < SCAN_IPT; ++i) {
    if (base + i < n) off[base + i] = run;
    run += v[i];
  }
}

__global__ void scatter_kernel(const int32_t* __restrict__ tgt, const uint64_t* __restrict__ pk,
                               const unsigned long long* __restrict__ nred,
                               const int64_t* __restrict__ off, int32_t* __restrict__ count,
                               uint64_t* __restrict__ bucket) {
  const int64_t nslots = (int64_t)*nred;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nslots;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = tgt[i];
    const int pos = atomicSub(&count[t], 1) - 1;
    bucket[off[t] + pos] = pk[i];
  }
}

// ---- per-target select -----------------------------------------------------------------
// idkey = (id << 33) | (ordered dist << 1) | old: sorting by it makes copies of one id
// adjacent, smallest distance first.
__device__ __forceinline__ uint64_t to_idkey(uint64_t k) {
  if (k == kEmpty) return kEmpty;
  return ((uint64_t)key_id(k) << 33) | ((k >> 32) << 1) | (k & 1ull);
}
__device__ __forceinline__ uint64_t from_idkey(uint64_t q) {
  if (q == kEmpty) return kEmpty;
  return (((q >> 1) & 0xFFFFFFFFull) << 32) | ((q >> 33) << 1) | (q & 1ull);
}

// Sort 32*E keys, keep one copy per id (smallest distance, old if any copy is old), and
// sort the survivors by key; duplicates and padding end as kEmpty at the back.
template <int E>
__device__ __forceinline__ void select_pass(uint64_t (&x)[E], uint64_t* buf) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < E; ++j) x[j] = to_idkey(x[j]);
  warp_sort_u64<E>(x);
#pragma unroll
  for (int j = 0; j < E; ++j) buf[j * 32 + lane] = x[j];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int e = j * 32 + lane;
    const uint64_t q = x[j];
    if (q == kEmpty) continue;
    const uint64_t id = q >> 33;
    if (e > 0 && (buf[e - 1] >> 33) == id && buf[e - 1] != kEmpty) {
      x[j] = kEmpty;  // a later copy of the same id
      continue;
    }
    uint64_t old = q & 1ull;
    for (int f = e + 1; f < 32 * E && buf[f] != kEmpty && (buf[f] >> 33) == id; ++f) old |= buf[f] & 1ull;
    x[j] = from_idkey(q | old);
  }
  __syncwarp();
  warp_sort_u64<E>(x);
}

struct SelectArgs {
  int64_t n;
  int R;
  const uint64_t* bucket;  // null: no bucket (every target keeps its base pool)
  const int64_t* off;
  const uint8_t* active;   // null: the base pool of every target is keys_in
  const uint64_t* keys_in;
  const int32_t* deg_in;
  uint64_t* keys_out;      // holds the kept survivors of active targets on entry
  int32_t* deg_out;
  int64_t* round_new;
  int64_t* stats;
};

__global__ void __launch_bounds__(256) select_kernel(SelectArgs a) {
  __shared__ uint64_t bufs[8][128];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t* buf = bufs[warp];
  const int R = a.R;
  long long n_new = 0, n_in = 0;
  for (int64_t u = (int64_t)blockIdx.x * 8 + warp; u < a.n; u += (int64_t)gridDim.x * 8) {
    const bool kept = a.active && a.active[u];
    const uint64_t* base = kept ? a.keys_out + u * R : a.keys_in + u * R;
    const int na = kept ? a.deg_out[u] : a.deg_in[u];
    int64_t b0 = 0, c = 0;
    if (a.bucket) {
      b0 = a.off[u];
      c = a.off[u + 1] - b0;
    }
    n_in += c;
    uint64_t out0, out1;
    if (c == 0) {
      if (kept) continue;  // the kept survivors are already in place (all old)
      out0 = lane < na ? base[lane] : kEmpty;
      out1 = lane + 32 < na ? base[32 + lane] : kEmpty;
    } else {
      uint64_t x[4];
      x[0] = lane < na ? base[lane] : kEmpty;
      x[1] = lane + 32 < na ? base[32 + lane] : kEmpty;
      for (int64_t done = 0; done < c; done += 64) {
#pragma unroll
        for (int j = 2; j < 4; ++j) {
          const int64_t e = done + (j - 2) * 32 + lane;
          x[j] = e < c ? a.bucket[b0 + e] : kEmpty;
        }
        select_pass<4>(x, buf);
        if (lane + 32 >= R) x[1] = kEmpty;
        if (lane >= R) x[0] = kEmpty;
      }
      out0 = x[0];
      out1 = x[1];
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
  }
  if (lane == 0) {
    if (n_new) atomicAdd(reinterpret_cast<unsigned long long*>(a.round_new), (unsigned long long)n_new);
    if (a.stats && n_in) atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[6]), (unsigned long long)n_in);
  }
}

cudaError_t merge_tail(const Workspace& ws, const SelectArgs& sa, cudaStream_t st) {
  const int64_t n = ws.n;
  if (sa.bucket) {
    const int64_t nb = ceil_div(n, SCAN_TILE);
    {
      ProfScope ps("scan", st);
      scan_reduce_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(ws.count, n, ws.bsum);
      scan_blocks_kernel<<<1, 1024, 0, st>>>(ws.bsum, nb, ws.off + n);
      scan_apply_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(ws.count, n, ws.bsum, ws.off);
    }
    {
      ProfScope ps("scatter", st);
      scatter_kernel<<<(unsigned)(sm_count() * 8), 256, 0, st>>>(ws.red_tgt, ws.red_key, ws.red_n, ws.off,
                                                                 ws.count, ws.bucket);
    }
  }
  cudaMemsetAsync(ws.round_new, 0, sizeof(int64_t), st);
  const int64_t blocks = std::min<int64_t>(ceil_div(n, 8), (int64_t)sm_count() * 16);
  ProfScope ps("select", st);
  select_kernel<<<(unsigned)blocks, 256, 0, st>>>(sa);
  return cudaGetLastError();
}

cudaError_t run_prep(const uint64_t* keys_in, const int32_t* deg_in, const Workspace& ws,
                     int64_t* stats, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>(ceil_div(ws.n, 256), (int64_t)sm_count() * 8);
  ProfScope ps("prep", st);
  prep_kernel<<<(unsigned)blocks, 256, 0, st>>>(keys_in, deg_in, ws.n, ws.R, ws.active, ws.list,
                                                ws.list_n, stats);
  return cudaGetLastError();
}

JoinArgs make_join_args(const PointsSet& P, int64_t n, int R, const uint64_t* keys_in,
                        const int32_t* deg_in, uint64_t seed, int t1, int t2, int order,
                        const Workspace& ws, uint64_t* keys_out, int32_t* deg_out, int emit,
                        int64_t* stats) {
  JoinArgs a;
  a.P.X = P.X;
  a.P.ld = P.ld;
  a.P.Xb = static_cast<const __nv_bfloat16*>(P.Xb);
  a.P.ldb = P.ldb;
  a.P.aux = P.aux;
  a.P.qflags = P.qflags;
  a.P.d = P.d;
  a.n = n;
  a.R = R;
  a.keys_in = keys_in;
  a.deg_in = deg_in;
  a.list = ws.list;
  a.list_n = ws.list_n;
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
  a.count = ws.count;
  a.stats = stats;
  a.err = ws.err;
  return a;
}

cudaError_t dispatch_join(const PointsSet& P, const JoinArgs& a, cudaStream_t st, const char* name) {
  if (P.precision == 1 && (!P.Xb || !P.aux || !P.qflags)) return cudaErrorInvalidValue;
  if (P.metric == 0)
    return P.precision == 1 ? launch_join_t<0, 1>(a, st, name) : launch_join_t<0, 0>(a, st, name);
  return P.precision == 1 ? launch_join_t<1, 1>(a, st, name) : launch_join_t<1, 0>(a, st, name);
}

}  // namespace

cudaError_t launch_round(const PointsSet& P, int64_t n, int R, const uint64_t* keys_in,
                         const int32_t* deg_in, uint64_t seed, int t1, int t2, int order,
                         const Workspace& ws, uint64_t* keys_out, int32_t* deg_out, int64_t* stats,
                         cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws.count, 0, (size_t)n * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(ws.list_n, 0, 16, st)) != cudaSuccess) return e;  // list_n and red_n
  if ((e = run_prep(keys_in, deg_in, ws, stats, st)) != cudaSuccess) return e;
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
  sa.stats = stats;
  return merge_tail(ws, sa, st);
}

cudaError_t launch_final(const PointsSet& P, int64_t n, int R, const uint64_t* keys_in,
                         const int32_t* deg_in, uint64_t seed, int t1, int order,
                         const Workspace& ws, uint64_t* keys_out, int32_t* deg_out, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws.list_n, 0, 16, st)) != cudaSuccess) return e;
  if ((e = run_prep(keys_in, deg_in, ws, nullptr, st)) != cudaSuccess) return e;
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
  sa.stats = nullptr;
  return merge_tail(ws, sa, st);
}

// =====================================================================================
// Reverse-edge sampling (Sec 3.6): each vertex proposes itself to the first
// floor(rho * deg) entries of its row (the closest ones); every pool is then merged
// with the proposals it received.
// =====================================================================================
__global__ void reverse_propose_kernel(int64_t n, int R, float rho,
                                       const uint64_t* __restrict__ keys,
                                       const int32_t* __restrict__ deg,
                                       int32_t* __restrict__ tgt, uint64_t* __restrict__ pk,
                                       unsigned long long* __restrict__ red_n,
                                       int32_t* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  const int64_t total = n * R;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
    const int64_t i = base + lane;
    bool emit = false;
    int32_t t = -1;
    uint64_t key = 0;
    if (i < total) {
      const int64_t v = i / R;
      const int j = (int)(i - v * R);
      const int r = (int)floor((double)rho * (double)deg[v]);
      if (j < r) {
        const uint64_t k = keys[i];
        t = (int32_t)key_id(k);
        key = (k & 0xFFFFFFFF00000000ull) | ((uint64_t)v << 1);
        emit = true;
      }
    }
    const unsigned b = __ballot_sync(0xffffffffu, emit);
    unsigned long long off = 0;
    if (lane == 0 && b) off = atomicAdd(red_n, (unsigned long long)__popc(b));
    off = __shfl_sync(0xffffffffu, off, 0);
    if (emit) {
      const unsigned long long slot = off + __popc(b & lanemask_lt());
      tgt[slot] = t;
      pk[slot] = key;
      atomicAdd(&count[t], 1);
    }
  }
}

cudaError_t launch_reverse(int64_t n, int R, float rho, const uint64_t* keys_in,
                           const int32_t* deg_in, const Workspace& ws, uint64_t* keys_out,
                           int32_t* deg_out, int64_t* stats, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws.count, 0, (size_t)n * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(ws.list_n, 0, 16, st)) != cudaSuccess) return e;
  {
    const int64_t blocks = std::min<int64_t>(ceil_div(n * R, 256), (int64_t)sm_count() * 32);
    ProfScope ps("reverse_propose", st);
    reverse_propose_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, R, rho, keys_in, deg_in, ws.red_tgt,
                                                            ws.red_key, ws.red_n, ws.count);
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
  sa.stats = stats;
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

size_t workspace_bytes(int64_t n, int R) {
  const size_t slots = (size_t)n * R;
  const size_t nb = (size_t)ceil_div(n, SCAN_TILE) + 1;
  return al256(slots * 4) + al256(slots * 8) + al256(slots * 8) + al256((size_t)n * 4) +
         al256(((size_t)n + 1) * 8) + al256(nb * 8) + al256((size_t)n * 4) + al256((size_t)n) +
         al256(16) + al256(4) + al256(8);
}

bool carve_workspace(void* base, size_t bytes, int64_t n, int R, Workspace* ws) {
  if (!base || bytes < workspace_bytes(n, R)) return false;
  if (((uintptr_t)base & 255u) != 0) return false;
  const size_t slots = (size_t)n * R;
  const size_t nb = (size_t)ceil_div(n, SCAN_TILE) + 1;
  char* p = static_cast<char*>(base);
  ws->n = n;
  ws->R = R;
  ws->red_tgt = reinterpret_cast<int32_t*>(p);
  p += al256(slots * 4);
  ws->red_key = reinterpret_cast<uint64_t*>(p);
  p += al256(slots * 8);
  ws->bucket = reinterpret_cast<uint64_t*>(p);
  p += al256(slots * 8);
  ws->count = reinterpret_cast<int32_t*>(p);
  p += al256((size_t)n * 4);
  ws->off = reinterpret_cast<int64_t*>(p);
  p += al256(((size_t)n + 1) * 8);
  ws->bsum = reinterpret_cast<int64_t*>(p);
  p += al256(nb * 8);
  ws->list = reinterpret_cast<int32_t*>(p);
  p += al256((size_t)n * 4);
  ws->active = reinterpret_cast<uint8_t*>(p);
  p += al256((size_t)n);
  ws->list_n = reinterpret_cast<int32_t*>(p);  // [0] list length, then the redirect count
  ws->red_n = reinterpret_cast<unsigned long long*>(p + 8);
  p += al256(16);
  ws->err = reinterpret_cast<int32_t*>(p);
  p += al256(4);
  ws->round_new = reinterpret_cast<int64_t*>(p);
  return true;
}

}  // namespace grnnd
