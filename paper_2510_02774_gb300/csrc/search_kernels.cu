// GRNND query-side kernels for sm_103a: search entry, candidate-list search (Sec 4.2),
// exact k-NN ground truth for Recall@k (Sec 2.1), canonical pair distances, and the
// finite-input check of the build.
#include <cfloat>

#include "common.cuh"
#include "internal.h"

namespace grnnd {

namespace {
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

// ---- canonical pair distances -----------------------------------------------------------
template <int METRIC>
__global__ void pair_dist_kernel(const float* __restrict__ X, int d, int ld,
                                 const int32_t* __restrict__ pairs, int64_t np,
                                 float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = pairs[2 * i], b = pairs[2 * i + 1];
    out[i] = row_dist<METRIC>(X + a * ld, X + b * ld, d);
  }
}

cudaError_t launch_pair_dist(const float* X, int d, int ld, int metric, const int32_t* pairs,
                             int64_t np, float* out, cudaStream_t st) {
  if (np == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(np, 128), (int64_t)sm_count() * 16);
  if (metric == 0)
    pair_dist_kernel<0><<<blocks, 128, 0, st>>>(X, d, ld, pairs, np, out);
  else
    pair_dist_kernel<1><<<blocks, 128, 0, st>>>(X, d, ld, pairs, np, out);
  return cudaGetLastError();
}

// ---- finite check ---------------------------------------------------------------------------
// Scans the n x ld floats as 16-byte granules (rows are 16-byte aligned and ld % 4 == 0; the
// padding columns hold zeros, which are finite).
__global__ void check_finite_kernel(const float4* __restrict__ X4, int64_t total4, int32_t* __restrict__ flag) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 x = __ldg(X4 + i);
    bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(x.w));
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}
cudaError_t launch_check_finite(const float* X, int64_t n, int d, int ld, int32_t* flag,
                                cudaStream_t st) {
  (void)d;
  const int64_t total4 = n * (int64_t)ld / 4;
  const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(total4, 256), (int64_t)sm_count() * 8);
  ProfScope ps("check_finite", st);
  check_finite_kernel<<<std::max(blocks, 1u), 256, 0, st>>>(reinterpret_cast<const float4*>(X), total4, flag);
  return cudaGetLastError();
}

// ---- search entry: nearest point to the mean, in FP64 -------------------------------------
// Column sums per block of rows, then per dimension over blocks; every point's distance
// to the mean with unfused FP64 operations in ascending dimension order; argmin by
// (dist, id).
namespace {
constexpr int kEntryBlocks = 512;
}

__global__ void colsum_kernel(const float* __restrict__ X, int64_t n, int d, int ld, int64_t rpb,
                              double* __restrict__ partial) {
  const int64_t r0 = (int64_t)blockIdx.x * rpb;
  const int64_t r1 = std::min<int64_t>(n, r0 + rpb);
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double s = 0.0;
    for (int64_t r = r0; r < r1; ++r) s = __dadd_rn(s, (double)X[r * ld + k]);
    partial[(int64_t)blockIdx.x * d + k] = s;
  }
}

__global__ void mean_kernel(const double* __restrict__ partial, int nb, int d, int64_t n,
                            double* __restrict__ mu) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < d; k += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s = __dadd_rn(s, partial[(int64_t)b * d + k]);
    mu[k] = __ddiv_rn(s, (double)n);
  }
}

__device__ __forceinline__ bool dl_less(double da, int32_t ia, double db, int32_t ib) {
  return da < db || (da == db && ia < ib);
}

// FP32 pre-filter of the nearest point.  For every point, a warp computes the FP32 distance
// d32 to the FP32-rounded mean and a rigorous bound B on |d32 - d64|, where d64 is the FP64
// value that nearest_kernel computes (ascending dimensions, unfused).  Any point whose d64
// can be the minimum satisfies d32 - B <= min_j (d32_j + B_j), so only those candidates need
// the FP64 evaluation; ties among them are still settled by id.
//   L2:  e1 = (2d + 16) u d32                   FP32 rounding of t = x - mu32, t^2, the sum
//        e2 = delta (2 sqrt(d32 + e1) + 3 delta) mu32 instead of mu, delta = ||mu - mu32||_2
//        e3 = (d + 4) 2^-52 (d32 + e1 + e2)     the FP64 evaluation itself
//   IP:  e1 = (d + 4) u 1.01 a + u (1 + |s|)    a = sum |x mu32|, s = sum x mu32
//        e2 = 1.00001 ||x|| delta
//        e3 = (d + 4) 2^-52 (a + ||x|| delta + 1) + 2^-53 (1 + |s|)
//   B = 1.1 (e1 + e2 + e3) + 1e-30, u = 2^-24, and the bound itself rounded upward.
template <int METRIC>
__device__ __forceinline__ void entry_d32(const float* __restrict__ x, int d, const float* __restrict__ mu32,
                                          float delta, float& lo, float& hi) {
  const int lane = threadIdx.x & 31;
  float s = 0.0f, a = 0.0f, xx = 0.0f;
  for (int k = lane; k < d; k += 32) {
    const float xv = x[k], m = mu32[k];
    if (METRIC == 0) {
      const float t = xv - m;
      s = fmaf(t, t, s);
    } else {
      s = fmaf(xv, m, s);
      a = fmaf(fabsf(xv), fabsf(m), a);
      xx = fmaf(xv, xv, xx);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    if (METRIC != 0) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      xx += __shfl_xor_sync(0xffffffffu, xx, o);
    }
  }
  const float u = 5.9604645e-08f;  // 2^-24
  float d32, B;
  if (METRIC == 0) {
    d32 = fmaxf(s, 0.0f);
    const float e1 = __fmul_ru(__fmul_ru((float)(2 * d + 16), u), d32);
    const float e2 = __fmul_ru(delta, __fadd_ru(__fmul_ru(2.0f, __fsqrt_ru(__fadd_ru(d32, e1))), __fmul_ru(3.0f, delta)));
    const float e3 = __fmul_ru(__fmul_ru((float)(d + 4), 2.220446e-16f), __fadd_ru(__fadd_ru(d32, e1), e2));
    B = __fadd_ru(__fmul_ru(1.1f, __fadd_ru(__fadd_ru(e1, e2), e3)), 1e-30f);
  } else {
    d32 = 1.0f - s;
    const float as = fabsf(s);
    const float e1 = __fadd_ru(__fmul_ru(__fmul_ru((float)(d + 4) * 1.01f, u), a), __fmul_ru(u, __fadd_ru(1.0f, as)));
    const float xn = __fmul_ru(__fsqrt_ru(xx), 1.00001f);
    const float e2 = __fmul_ru(xn, delta);
    const float e3 = __fadd_ru(__fmul_ru(__fmul_ru((float)(d + 4), 2.220446e-16f), __fadd_ru(__fadd_ru(a, e2), 1.0f)),
                               __fmul_ru(1.110223e-16f, __fadd_ru(1.0f, as)));
    B = __fadd_ru(__fmul_ru(1.1f, __fadd_ru(__fadd_ru(e1, e2), e3)), 1e-30f);
  }
  lo = __fsub_rd(d32, B);
  hi = __fadd_ru(d32, B);
}

// mu32 = FP32 rounding of the FP64 mean and delta = ||mu - mu32||_2 rounded upward (one block).
__global__ void mean32_kernel(const double* __restrict__ mu, int d, float* __restrict__ mu32,
                              float* __restrict__ delta) {
  __shared__ double red[256];
  double e = 0.0;
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    const float m = __double2float_rn(mu[k]);
    mu32[k] = m;
    const double t = mu[k] - (double)m;
    e += t * t;
  }
  red[threadIdx.x] = e;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *delta = __double2float_ru(sqrt(red[0] * (1.0 + 1e-12)) * (1.0 + 1e-12));
}

// Per block: the smallest upper end d32 + B of its points (warp per point).
template <int METRIC>
__global__ void __launch_bounds__(256) entry_upper_kernel(const float* __restrict__ X, int64_t n, int d, int ld,
                                                          const float* __restrict__ mu32,
                                                          const float* __restrict__ delta,
                                                          float* __restrict__ bmin) {
  __shared__ float wmin[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float dl = *delta;
  float best = FLT_MAX;
  for (int64_t i = (int64_t)blockIdx.x * 8 + warp; i < n; i += (int64_t)gridDim.x * 8) {
    float lo, hi;
    entry_d32<METRIC>(X + i * ld, d, mu32, dl, lo, hi);
    best = fminf(best, hi);
  }
  if (lane == 0) wmin[warp] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = wmin[0];
    for (int w = 1; w < 8; ++w) b = fminf(b, wmin[w]);
    bmin[blockIdx.x] = b;
  }
}

// Per block: (FP64 distance, id) minimum over the candidate points only: those whose lower
// end d32 - B is at most the smallest upper end over all points.
template <int METRIC>
__global__ void __launch_bounds__(256) nearest_kernel(const float* __restrict__ X, int64_t n, int d,
                                                      int ld, const double* __restrict__ mu,
                                                      const float* __restrict__ mu32,
                                                      const float* __restrict__ delta,
                                                      const float* __restrict__ bmin, int nbmin,
                                                      double* __restrict__ bd,
                                                      int32_t* __restrict__ bi) {
  __shared__ double sd[256];
  __shared__ int32_t si[256];
  __shared__ float s_up;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    float u = FLT_MAX;
    for (int b = 0; b < nbmin; ++b) u = fminf(u, bmin[b]);
    s_up = u;
  }
  __syncthreads();
  const float up = s_up, dl = *delta;
  double best = DBL_MAX;
  int32_t bid = INT32_MAX;
  for (int64_t i = (int64_t)blockIdx.x * 8 + warp; i < n; i += (int64_t)gridDim.x * 8) {
    const float* x = X + i * ld;
    float lo, hi;
    entry_d32<METRIC>(x, d, mu32, dl, lo, hi);
    if (lo > up) continue;  // cannot be the nearest point (warp-uniform)
    if (lane == 0) {  // the FP64 value, exactly as defined: ascending dimensions, unfused
      double s = 0.0;
      for (int k = 0; k < d; ++k) {
        if (METRIC == 0) {
          const double t = __dsub_rn((double)x[k], mu[k]);
          s = __dadd_rn(s, __dmul_rn(t, t));
        } else {
          s = __dadd_rn(s, __dmul_rn((double)x[k], mu[k]));
        }
      }
      if (METRIC != 0) s = __dsub_rn(1.0, s);
      if (dl_less(s, (int32_t)i, best, bid)) {
        best = s;
        bid = (int32_t)i;
      }
    }
  }
  sd[threadIdx.x] = best;
  si[threadIdx.x] = bid;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o && dl_less(sd[threadIdx.x + o], si[threadIdx.x + o], sd[threadIdx.x], si[threadIdx.x])) {
      sd[threadIdx.x] = sd[threadIdx.x + o];
      si[threadIdx.x] = si[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bd[blockIdx.x] = sd[0];
    bi[blockIdx.x] = si[0];
  }
}

__global__ void nearest_final_kernel(const double* __restrict__ bd, const int32_t* __restrict__ bi,
                                     int nb, int32_t* __restrict__ entry) {
  if (threadIdx.x != 0) return;
  double best = DBL_MAX;
  int32_t id = INT32_MAX;
  for (int b = 0; b < nb; ++b)
    if (dl_less(bd[b], bi[b], best, id)) {
      best = bd[b];
      id = bi[b];
    }
  *entry = id;
}

size_t entry_workspace_bytes(int64_t n, int d) {
  (void)n;
  return al256((size_t)kEntryBlocks * d * 8) + al256((size_t)d * 8) + al256(kEntryBlocks * 8) +
         al256(kEntryBlocks * 4);
}

cudaError_t launch_entry(const float* X, int64_t n, int d, int ld, int metric, int32_t* entry,
                         void* ws, size_t ws_bytes, cudaStream_t st) {
  if (ws_bytes < entry_workspace_bytes(n, d)) return cudaErrorInvalidValue;
  char* p = static_cast<char*>(ws);
  double* partial = reinterpret_cast<double*>(p);
  p += al256((size_t)kEntryBlocks * d * 8);
  double* mu = reinterpret_cast<double*>(p);
  p += al256((size_t)d * 8);
  double* bd = reinterpret_cast<double*>(p);
  p += al256(kEntryBlocks * 8);
  int32_t* bi = reinterpret_cast<int32_t*>(p);
  // once the mean is formed, the column sums' region holds the FP32 mean, its distance to the
  // FP64 mean and the per-block upper ends (d + 256 + 512 floats <= 512 d doubles)
  float* mu32 = reinterpret_cast<float*>(partial);
  float* delta = mu32 + al256((size_t)d * 4) / 4;
  float* bmin = delta + 64;
  const int64_t rpb = ceil_div(n, kEntryBlocks);
  const int nb = (int)ceil_div(n, rpb);
  const int nb2 = (int)std::min<int64_t>(kEntryBlocks, ceil_div(n, 8));
  ProfScope ps("entry", st);
  colsum_kernel<<<nb, 256, 0, st>>>(X, n, d, ld, rpb, partial);
  mean_kernel<<<(unsigned)ceil_div(d, 256), 256, 0, st>>>(partial, nb, d, n, mu);
  mean32_kernel<<<1, 256, 0, st>>>(mu, d, mu32, delta);
  if (metric == 0) {
    entry_upper_kernel<0><<<nb2, 256, 0, st>>>(X, n, d, ld, mu32, delta, bmin);
    nearest_kernel<0><<<nb2, 256, 0, st>>>(X, n, d, ld, mu, mu32, delta, bmin, nb2, bd, bi);
  } else {
    entry_upper_kernel<1><<<nb2, 256, 0, st>>>(X, n, d, ld, mu32, delta, bmin);
    nearest_kernel<1><<<nb2, 256, 0, st>>>(X, n, d, ld, mu, mu32, delta, bmin, nb2, bd, bi);
  }
  nearest_final_kernel<<<1, 32, 0, st>>>(bd, bi, nb2, entry);
  return cudaGetLastError();
}

// ---- search entries of a batch of builds: the same arithmetic as launch_entry, per build --
// Build b covers rows [off[b], off[b+1]); its column sums use the same row blocks as a
// single build of those rows (rpb = ceil(n_b / 512) rows per block, blocks in order), so the
// mean, and therefore the entry, is the one launch_entry computes for the build alone.
__global__ void seg_colsum_kernel(const float* __restrict__ X, int ld, int d, const int64_t* __restrict__ off,
                                  int nbuild, double* __restrict__ partial) {
  const int64_t total = (int64_t)nbuild * kEntryBlocks * d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % d);
    const int64_t bj = t / d;
    const int b = (int)(bj / kEntryBlocks), j = (int)(bj % kEntryBlocks);
    const int64_t lo = off[b], nb = off[b + 1] - lo;
    const int64_t rpb = (nb + kEntryBlocks - 1) / kEntryBlocks;
    const int64_t r0 = lo + (int64_t)j * rpb, r1 = std::min<int64_t>(lo + nb, r0 + rpb);
    if (r0 >= r1) continue;
    double s = 0.0;
    for (int64_t r = r0; r < r1; ++r) s = __dadd_rn(s, (double)X[r * ld + k]);
    partial[bj * d + k] = s;
  }
}

__global__ void seg_mean_kernel(const double* __restrict__ partial, int d, const int64_t* __restrict__ off,
                                int nbuild, double* __restrict__ mu) {
  const int64_t total = (int64_t)nbuild * d;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / d), k = (int)(t % d);
    const int64_t nb = off[b + 1] - off[b];
    const int64_t rpb = (nb + kEntryBlocks - 1) / kEntryBlocks;
    const int blocks = (int)((nb + rpb - 1) / rpb);
    double s = 0.0;
    for (int j = 0; j < blocks; ++j) s = __dadd_rn(s, partial[((int64_t)b * kEntryBlocks + j) * d + k]);
    mu[t] = __ddiv_rn(s, (double)nb);
  }
}

template <int METRIC>
__global__ void seg_nearest_kernel(const float* __restrict__ X, int ld, int d, const int64_t* __restrict__ off,
                                   const double* __restrict__ mu, int32_t* __restrict__ entry) {
  __shared__ double sd[256];
  __shared__ int32_t si[256];
  const int b = blockIdx.x;
  const int64_t lo = off[b], nb = off[b + 1] - lo;
  const double* m = mu + (int64_t)b * d;
  double best = DBL_MAX;
  int32_t bid = INT32_MAX;
  for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) {
    const float* x = X + (lo + i) * ld;
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
      if (METRIC == 0) {
        const double t = __dsub_rn((double)x[k], m[k]);
        s = __dadd_rn(s, __dmul_rn(t, t));
      } else {
        s = __dadd_rn(s, __dmul_rn((double)x[k], m[k]));
      }
    }
    if (METRIC != 0) s = __dsub_rn(1.0, s);
    if (dl_less(s, (int32_t)i, best, bid)) {
      best = s;
      bid = (int32_t)i;
    }
  }
  sd[threadIdx.x] = best;
  si[threadIdx.x] = bid;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o && dl_less(sd[threadIdx.x + o], si[threadIdx.x + o], sd[threadIdx.x], si[threadIdx.x])) {
      sd[threadIdx.x] = sd[threadIdx.x + o];
      si[threadIdx.x] = si[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) entry[b] = si[0];
}

size_t entry_batch_workspace_bytes(int32_t nbuild, int d) {
  return al256((size_t)nbuild * kEntryBlocks * d * 8) + al256((size_t)nbuild * d * 8);
}

cudaError_t launch_entry_batch(const float* X, int d, int ld, int metric, const int64_t* off_dev, int32_t nbuild,
                               int32_t* entries, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (ws_bytes < entry_batch_workspace_bytes(nbuild, d)) return cudaErrorInvalidValue;
  char* p = static_cast<char*>(ws);
  double* partial = reinterpret_cast<double*>(p);
  p += al256((size_t)nbuild * kEntryBlocks * d * 8);
  double* mu = reinterpret_cast<double*>(p);
  ProfScope ps("entry", st);
  const int64_t t1 = (int64_t)nbuild * kEntryBlocks * d, t2 = (int64_t)nbuild * d;
  seg_colsum_kernel<<<(unsigned)std::min<int64_t>(ceil_div(t1, 256), (int64_t)sm_count() * 32), 256, 0, st>>>(
      X, ld, d, off_dev, nbuild, partial);
  seg_mean_kernel<<<(unsigned)std::min<int64_t>(ceil_div(t2, 256), (int64_t)sm_count() * 8), 256, 0, st>>>(
      partial, d, off_dev, nbuild, mu);
  if (metric == 0)
    seg_nearest_kernel<0><<<(unsigned)nbuild, 256, 0, st>>>(X, ld, d, off_dev, mu, entries);
  else
    seg_nearest_kernel<1><<<(unsigned)nbuild, 256, 0, st>>>(X, ld, d, off_dev, mu, entries);
  return cudaGetLastError();
}

// ---- candidate-list search -----------------------------------------------------------------
// One warp per query.  The candidate list C (ascending keys; bit 0 = expanded) lives in
// shared memory.  A small direct-mapped cache of evaluated ids skips re-evaluations; a
// cache miss re-evaluates a vertex, which cannot change C: C only ever holds the best
// `beam` distinct evaluated vertices, so a vertex evaluated before is either still in C
// (found by the membership test) or worse than every entry of C.
namespace {
constexpr int SW = 4;          // warps per block
constexpr int kMaxBeam = 256;
constexpr int kCache = 1024;
constexpr int kMaxD = 1024;
}

template <int METRIC>
__device__ __forceinline__ float warp_qdist(const float* __restrict__ q, const float* __restrict__ x,
                                            int d) {
  const int lane = threadIdx.x & 31;
  float acc = 0.0f;
  for (int k = lane; k < d; k += 32) acc = dist_step<METRIC>(acc, q[k], __ldg(x + k));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  acc = __shfl_sync(0xffffffffu, acc, 0);
  return dist_finish<METRIC>(acc);
}

template <int METRIC>
__global__ void __launch_bounds__(SW * 32) search_kernel(
    const float* __restrict__ X, int64_t n, int d, int ld, const int32_t* __restrict__ gids,
    const int32_t* __restrict__ gdeg, int R, int entry, const float* __restrict__ Q, int64_t nq,
    int ldq, int k, int beam, int32_t* __restrict__ ids_out, float* __restrict__ dists_out) {
  __shared__ float qs[SW][kMaxD];
  __shared__ uint64_t cl[SW][kMaxBeam];
  __shared__ int32_t cache[SW][kCache];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* q = qs[warp];
  uint64_t* C = cl[warp];
  int32_t* cc = cache[warp];
  const int nchunk = (beam + 31) >> 5;
  for (int64_t qi = (int64_t)blockIdx.x * SW + warp; qi < nq; qi += (int64_t)gridDim.x * SW) {
    for (int t = lane; t < d; t += 32) q[t] = Q[qi * ldq + t];
    for (int t = lane; t < kCache; t += 32) cc[t] = -1;
    __syncwarp();
    int sz = 1;
    {
      const float de = warp_qdist<METRIC>(q, X + (int64_t)entry * ld, d);
      if (lane == 0) {
        C[0] = make_key(de, (uint32_t)entry, 0u);
        cc[((uint32_t)entry * 2654435761u) >> 22] = entry;
      }
    }
    __syncwarp();
    for (int64_t it = 0; it <= n; ++it) {
      int first = -1;
      for (int ch = 0; ch < nchunk && first < 0; ++ch) {
        const int e = ch * 32 + lane;
        const unsigned b = __ballot_sync(0xffffffffu, e < sz && !(C[e] & 1ull));
        if (b) first = ch * 32 + __ffs(b) - 1;
      }
      if (first < 0) break;  // every candidate expanded
      const uint64_t ck = C[first];
      __syncwarp();
      if (lane == 0) C[first] = ck | 1ull;
      const int u = (int)key_id(ck);
      const int du = gdeg[u];
      for (int base = 0; base < du; base += 32) {
        const int j = base + lane;
        const int w = j < du ? gids[(int64_t)u * R + j] : -1;
        bool todo = false;
        if (w >= 0) {
          const uint32_t slot = ((uint32_t)w * 2654435761u) >> 22;
          todo = cc[slot] != w;
          __syncwarp(__activemask());
          if (todo) cc[slot] = w;
        }
        unsigned pend = __ballot_sync(0xffffffffu, todo);
        __syncwarp();
        while (pend) {
          const int l = __ffs(pend) - 1;
          pend &= pend - 1;
          const int ww = __shfl_sync(0xffffffffu, w, l);
          const float dw = warp_qdist<METRIC>(q, X + (int64_t)ww * ld, d);
          const uint64_t key = make_key(dw, (uint32_t)ww, 0u);
          if (sz == beam && (key >> 1) >= (C[beam - 1] >> 1)) continue;
          bool present = false;
          int pos = 0;
          for (int ch = 0; ch < nchunk; ++ch) {
            const int e = ch * 32 + lane;
            const bool in = e < sz;
            const uint64_t ce = in ? C[e] : kEmpty;
            present |= __any_sync(0xffffffffu, in && key_id(ce) == (uint32_t)ww);
            pos += __popc(__ballot_sync(0xffffffffu, in && (ce >> 1) < (key >> 1)));
          }
          if (present) continue;
          // shift C[pos .. sz-1] one place right (the last entry drops when full)
          uint64_t hold[kMaxBeam / 32];
#pragma unroll
          for (int ch = 0; ch < kMaxBeam / 32; ++ch) {
            const int e = ch * 32 + lane;
            hold[ch] = (ch < nchunk && e >= pos && e < sz && e + 1 < beam) ? C[e] : 0ull;
          }
          __syncwarp();
#pragma unroll
          for (int ch = 0; ch < kMaxBeam / 32; ++ch) {
            const int e = ch * 32 + lane;
            if (ch < nchunk && e >= pos && e < sz && e + 1 < beam) C[e + 1] = hold[ch];
          }
          __syncwarp();
          if (lane == 0) C[pos] = key;
          sz = sz < beam ? sz + 1 : beam;
          __syncwarp();
        }
      }
    }
    for (int j = lane; j < k; j += 32) {
      const bool ok = j < sz;
      ids_out[qi * k + j] = ok ? (int32_t)key_id(C[j]) : -1;
      if (dists_out) dists_out[qi * k + j] = ok ? key_dist(C[j]) : __int_as_float(0x7f800000);
    }
    __syncwarp();
  }
}

cudaError_t launch_search(const float* X, int64_t n, int d, int ld, int metric,
                          const int32_t* gids, const int32_t* gdeg, int R, int entry,
                          const float* Q, int64_t nq, int ldq, int k, int beam, int32_t* ids_out,
                          float* dists_out, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  if (d > kMaxD || beam > kMaxBeam) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(nq, SW), (int64_t)sm_count() * 8);
  ProfScope ps("search", st);
  if (metric == 0)
    search_kernel<0><<<blocks, SW * 32, 0, st>>>(X, n, d, ld, gids, gdeg, R, entry, Q, nq, ldq, k,
                                                 beam, ids_out, dists_out);
  else
    search_kernel<1><<<blocks, SW * 32, 0, st>>>(X, n, d, ld, gids, gdeg, R, entry, Q, nq, ldq, k,
                                                 beam, ids_out, dists_out);
  return cudaGetLastError();
}

// ---- exact k-NN (ground truth) -----------------------------------------------------------
// Block: 32 queries x tiles of 64 points; each thread a 2 x 4 register tile accumulating
// the canonical distance over dimension chunks of 64; then each warp folds the tile into
// the running top-k of 4 queries.
namespace {
constexpr int BQ = 32, BP = 64, BD = 64, BS = BD + 1, KMAX = 32;
}

template <int METRIC>
__global__ void __launch_bounds__(256) brute_knn_kernel(const float* __restrict__ X, int64_t n,
                                                        int d, int ld, const float* __restrict__ Q,
                                                        int64_t nq, int ldq, int k,
                                                        int32_t* __restrict__ ids_out,
                                                        float* __restrict__ dists_out) {
  __shared__ float qs[BQ][BS];
  __shared__ float ps[BP][BS];
  __shared__ float dt[BQ][BP + 1];
  __shared__ uint64_t tk[BQ][KMAX];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t q0 = (int64_t)blockIdx.x * BQ;
  const int qp = tid >> 4, pg = tid & 15;  // queries 2qp, 2qp+1; points pg + 16i
  for (int t = tid; t < BQ * KMAX; t += 256) tk[t / KMAX][t % KMAX] = kEmpty;
  __syncthreads();
  for (int64_t p0 = 0; p0 < n; p0 += BP) {
    float acc[2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
    for (int c0 = 0; c0 < d; c0 += BD) {
      const int cl = min(BD, d - c0);
      for (int t = tid; t < BQ * BD; t += 256) {
        const int r = t / BD, c = t % BD;
        qs[r][c] = (q0 + r < nq && c < cl) ? Q[(q0 + r) * ldq + c0 + c] : 0.0f;
      }
      for (int t = tid; t < BP * BD; t += 256) {
        const int r = t / BD, c = t % BD;
        ps[r][c] = (p0 + r < n && c < cl) ? X[(p0 + r) * ld + c0 + c] : 0.0f;
      }
      __syncthreads();
      for (int c = 0; c < cl; ++c) {
        const float qa = qs[2 * qp][c], qb = qs[2 * qp + 1][c];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float x = ps[pg + 16 * b][c];
          acc[0][b] = dist_step<METRIC>(acc[0][b], qa, x);
          acc[1][b] = dist_step<METRIC>(acc[1][b], qb, x);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) dt[2 * qp + a][pg + 16 * b] = dist_finish<METRIC>(acc[a][b]);
    __syncthreads();
    for (int qq = warp * 4; qq < warp * 4 + 4; ++qq) {
      if (q0 + qq >= nq) break;
      uint64_t* L = tk[qq];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int pj = h * 32 + lane;
        const bool valid = p0 + pj < n;
        const uint64_t key = valid ? make_key(dt[qq][pj], (uint32_t)(p0 + pj), 0u) : kEmpty;
        unsigned pend = __ballot_sync(0xffffffffu, valid && key < L[k - 1]);
        while (pend) {
          const int l = __ffs(pend) - 1;
          pend &= pend - 1;
          const uint64_t kk = __shfl_sync(0xffffffffu, key, l);
          const uint64_t cur = lane < k ? L[lane] : kEmpty;
          if (kk >= L[k - 1]) continue;
          const int pos = __popc(__ballot_sync(0xffffffffu, lane < k && cur < kk));
          __syncwarp();
          if (lane >= pos && lane + 1 < k) L[lane + 1] = cur;
          __syncwarp();
          if (lane == 0) L[pos] = kk;
          __syncwarp();
        }
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < BQ * k; t += 256) {
    const int r = t / k, j = t % k;
    if (q0 + r >= nq) continue;
    const uint64_t key = tk[r][j];
    ids_out[(q0 + r) * k + j] = key == kEmpty ? -1 : (int32_t)key_id(key);
    if (dists_out) dists_out[(q0 + r) * k + j] = key == kEmpty ? __int_as_float(0x7f800000) : key_dist(key);
  }
}

cudaError_t launch_brute_knn(const float* X, int64_t n, int d, int ld, int metric, const float* Q,
                             int64_t nq, int ldq, int k, int32_t* ids_out, float* dists_out,
                             cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  if (k < 1 || k > KMAX) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)ceil_div(nq, BQ);
  ProfScope ps("brute_knn", st);
  if (metric == 0)
    brute_knn_kernel<0><<<blocks, 256, 0, st>>>(X, n, d, ld, Q, nq, ldq, k, ids_out, dists_out);
  else
    brute_knn_kernel<1><<<blocks, 256, 0, st>>>(X, n, d, ld, Q, nq, ldq, k, ids_out, dists_out);
  return cudaGetLastError();
}

// ---- self-test of the bounded waits -------------------------------------------------------
// One thread waits, with the same bounded mbarrier wait as the join kernels, on a barrier
// that expects one arrival and gets none: the wait gives up after `limit` tries and the
// outcome goes to the status word, as in a join.  Nothing is copied, so nothing is left in
// flight when the thread returns.
__device__ int32_t g_wait_selftest_status;

__global__ void wait_selftest_kernel(uint32_t limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  const bool ok = mbar_wait(&bar, 0u, limit);
  g_wait_selftest_status = ok ? 0 : kErrTimeout;
}

cudaError_t launch_wait_selftest(uint32_t limit, int32_t* status, cudaStream_t st) {
  const int32_t unset = -1;
  cudaError_t e = cudaMemcpyToSymbolAsync(g_wait_selftest_status, &unset, 4, 0, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  wait_selftest_kernel<<<1, 32, 0, st>>>(limit);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyFromSymbolAsync(status, g_wait_selftest_status, 4, 0, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  return cudaStreamSynchronize(st);
}

}  // namespace grnnd
