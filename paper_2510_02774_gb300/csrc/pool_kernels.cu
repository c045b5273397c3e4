// GRNND pool kernels for sm_103a: rnd_init, rnd_join (gather + dist_tile + rng_prune),
// reverse sampling and rev_merge (bucket by target + per-target top-R select).
//
//   rnd_init    Alg 3, INITIAL_NEIGHBORS
//   rnd_join    Alg 4 (pair loop) with the pair rule of Eq 2 and the distance of Alg 5
//   rev_merge   the end state of WARP_INSERT (Alg 6) over fixed-capacity pools (Sec 3.5)
//   reverse     reverse-edge sampling (Sec 3.6)
#include <cstdio>

#include "common.cuh"
#include "internal.h"

namespace grnnd {

namespace {

constexpr uint32_t kWaitLimit = 1u << 24;

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

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
  const unsigned below = (1u << lane) - 1u;
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
// rnd_join: one CTA per vertex at a time (persistent over vertices).
//
//  1. load pool1[v]; a vertex without new entries has only old x old pairs, which never
//     fire (design reading C10), so it re-proposes its pool unchanged and gathers nothing;
//  2. visit order pi: rank of (h(seed,t1,t2,v,id), id) (or the ascending / descending
//     key order);
//  3. rows of the pool are staged in shared memory with one bulk copy per row (TMA
//     engine, completion on an mbarrier), new rows first so that the pairs to evaluate
//     -- every pair with at least one new side -- form a dense list;
//  4. dist_tile: one thread per pair, canonical FP32 accumulation over d (chunks of DC
//     dimensions; partial sums stay in shared memory between chunks);
//  5. rng_prune: fire bits F[b] = {a < b : d(a,b) < max(d(v,a), d(v,b))} in pi order;
//     the sequential pair scan of Alg 4 is then resolved column by column with 64-bit
//     masks: in column b the live firing a's below the first a that makes b the far
//     side become bottom, and b becomes bottom if such an a exists;
//  6. every entry emits one proposal: survivors back to v (old), bottom entries to
//     their absorber with distance d(close, far) (new).
// =====================================================================================
namespace {

constexpr int JT = 128;            // threads per CTA
constexpr int DC = 128;            // dimensions per staged chunk
constexpr int RS = DC + 4;         // row stride in floats: rows fall on different banks
constexpr int MAXP = kMaxR * (kMaxR - 1) / 2;

struct __align__(16) JoinSmem {
  float rows[kMaxR][RS];
  float pd[MAXP];               // pair partial sums, then pair distances
  uint64_t pkey[kMaxR];         // pool key by pi position
  uint64_t hk[kMaxR];           // order key by storage slot
  uint64_t skey[kMaxR];         // pool key by storage slot
  uint64_t fire[kMaxR];         // fire bits per pi column
  uint64_t bfar[kMaxR];         // bits a < b with key(a) < key(b)
  int32_t pid[kMaxR];           // id by pi position
  int32_t killer[kMaxR];        // pi position of the absorber, -1 if none
  int32_t rowoff[kMaxR + 1];    // first pair index of new row i
  int16_t pos_of_slot[kMaxR];
  int16_t row_of_pos[kMaxR];
  int16_t pos_of_row[kMaxR];
  uint64_t bar;
  uint64_t alive;
  uint64_t mask2;
};

struct JoinArgs {
  const float* X;
  int64_t n;
  int d, ld, R;
  const uint64_t* keys_in;
  const int32_t* deg_in;
  uint64_t seed;
  int t1, t2, order, mode;
  int32_t* prop_tgt;
  uint64_t* prop_key;
  int prop_stride;
  int32_t* count;
  uint64_t* out_keys;
  int32_t* out_deg;
  int64_t* stats;
  int32_t* err;
};

__device__ __forceinline__ uint64_t bits_below(int i) { return i == 0 ? 0ull : (~0ull >> (64 - i)); }

template <int METRIC>
__global__ void __launch_bounds__(JT) rnd_join_kernel(JoinArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  JoinSmem& s = *reinterpret_cast<JoinSmem*>(smem_raw);
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&s.bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  long long st_vert = 0, st_rows = 0, st_pairs = 0, st_fired = 0, st_props = 0;
  const int R = a.R;

  for (int64_t v = blockIdx.x; v < a.n; v += gridDim.x) {
    const int m = a.deg_in[v];
    const uint64_t kk = (tid < m) ? a.keys_in[v * R + tid] : kEmpty;
    const int k_new = __syncthreads_count(tid < m && !key_old(kk));
    const int npairs = k_new * (m - 1) - k_new * (k_new - 1) / 2;

    if (npairs == 0) {  // nothing can fire: every entry survives unchanged
      if (a.mode == 0) {
        if (tid < R) {
          a.prop_tgt[v * a.prop_stride + tid] = tid < m ? (int32_t)v : -1;
          a.prop_key[v * a.prop_stride + tid] = tid < m ? (kk | 1ull) : kEmpty;
        }
        if (tid == 0 && m > 0) atomicAdd(&a.count[v], m);
      } else {
        if (tid < R) a.out_keys[v * R + tid] = tid < m ? (kk | 1ull) : kEmpty;
        if (tid == 0) a.out_deg[v] = m;
      }
      if (tid == 0) st_props += m;
      continue;
    }

    // ---- 2. visit order ------------------------------------------------------------
    if (tid < m) {
      const uint32_t id = key_id(kk);
      s.skey[tid] = kk;
      s.hk[tid] = (a.order == 0)   ? counter_hash(a.seed, (uint64_t)a.t1, (uint64_t)a.t2,
                                                  (uint64_t)v, (uint64_t)id)
                  : (a.order == 1) ? (uint64_t)tid
                                   : (uint64_t)(m - 1 - tid);
    }
    __syncthreads();
    if (tid < m) {
      const uint64_t h = s.hk[tid];
      const uint32_t id = key_id(kk);
      int p = 0;
      for (int j = 0; j < m; ++j) {
        const uint64_t hj = s.hk[j];
        p += (hj < h) || (hj == h && key_id(s.skey[j]) < id);
      }
      s.pos_of_slot[tid] = (int16_t)p;
      s.pkey[p] = kk;
      s.pid[p] = (int32_t)id;
    }
    __syncthreads();
    if (tid < 64) {
      const bool nw = tid < m && !key_old(s.pkey[tid]);
      const unsigned b = __ballot_sync(0xffffffffu, nw);
      if ((tid & 31) == 0) reinterpret_cast<uint32_t*>(&s.mask2)[tid >> 5] = b;
    }
    __syncthreads();
    const uint64_t newm = s.mask2;
    const uint64_t valid = (m >= 64) ? ~0ull : ((1ull << m) - 1ull);
    if (tid < m) {
      const uint64_t lo = bits_below(tid);
      const int row = ((newm >> tid) & 1ull) ? __popcll(newm & lo)
                                             : k_new + __popcll(~newm & valid & lo);
      s.row_of_pos[tid] = (int16_t)row;
      s.pos_of_row[row] = (int16_t)tid;
      const uint64_t kb = s.pkey[tid] >> 1;
      uint64_t bf = 0;
      for (int q = 0; q < tid; ++q) bf |= ((s.pkey[q] >> 1) < kb ? 1ull : 0ull) << q;
      s.bfar[tid] = bf;
      s.fire[tid] = 0;
      s.killer[tid] = -1;
    }
    if (tid <= k_new) s.rowoff[tid] = tid * (m - 1) - tid * (tid - 1) / 2;
    __syncthreads();

    // ---- 3./4. gather rows chunk by chunk and accumulate pair distances --------------
    const int nchunks = (a.d + DC - 1) / DC;
    for (int c = 0; c < nchunks; ++c) {
      const int c0 = c * DC;
      const int clen = min(DC, a.d - c0);
      const int clen4 = (clen + 3) & ~3;
      if (tid == 0) {
        mbar_expect_tx(&s.bar, (uint32_t)(m * clen4 * 4));
        for (int p = 0; p < m; ++p)
          bulk_g2s(&s.rows[s.row_of_pos[p]][0], a.X + (int64_t)s.pid[p] * a.ld + c0,
                   (uint32_t)(clen4 * 4), &s.bar);
      }
      const bool ok = mbar_wait(&s.bar, phase, kWaitLimit);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        // a bounded wait gave up: report, let in-flight copies land, and stop.
        if (tid == 0) atomicExch(a.err, kErrTimeout);
        if (!ok) mbar_wait(&s.bar, phase ^ 1u, kWaitLimit);
        return;
      }
      int i = 0;
      for (int q = tid; q < npairs; q += JT) {
        while (s.rowoff[i + 1] <= q) ++i;
        const int j = i + 1 + (q - s.rowoff[i]);
        const float* ra = &s.rows[i][0];
        const float* rb = &s.rows[j][0];
        float acc = (c == 0) ? 0.0f : s.pd[q];
        int t = 0;
        for (; t + 4 <= clen; t += 4)
          acc = dist_step4<METRIC>(acc, *reinterpret_cast<const float4*>(ra + t),
                                   *reinterpret_cast<const float4*>(rb + t));
        for (; t < clen; ++t) acc = dist_step<METRIC>(acc, ra[t], rb[t]);
        s.pd[q] = acc;
      }
      __syncthreads();
    }

    // ---- 5. rng_prune ---------------------------------------------------------------
    {
      int i = 0;
      for (int q = tid; q < npairs; q += JT) {
        while (s.rowoff[i + 1] <= q) ++i;
        const int j = i + 1 + (q - s.rowoff[i]);
        const int pa = s.pos_of_row[i], pb = s.pos_of_row[j];
        const int lo = min(pa, pb), hi = max(pa, pb);
        const float dab = dist_finish<METRIC>(s.pd[q]);
        s.pd[q] = dab;
        const float mx = fmaxf(key_dist(s.pkey[lo]), key_dist(s.pkey[hi]));
        if (dab < mx) atomicOr(reinterpret_cast<unsigned long long*>(&s.fire[hi]), 1ull << lo);
      }
    }
    __syncthreads();
    if (tid == 0) {
      uint64_t alive = valid;
      for (int b = 1; b < m; ++b) {
        const uint64_t cand = s.fire[b] & alive;
        if (!cand) continue;
        const uint64_t x = cand & s.bfar[b];
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
      st_vert += 1;
      st_rows += m;
      st_pairs += npairs;
      st_fired += m - __popcll(alive);
      st_props += m;
    }
    __syncthreads();

    // ---- 6. emit ---------------------------------------------------------------------
    const uint64_t alive = s.alive;
    if (a.mode == 0) {
      if (tid < R) {
        int32_t tgt = -1;
        uint64_t key = kEmpty;
        if (tid < m) {
          if ((alive >> tid) & 1ull) {
            tgt = (int32_t)v;
            key = s.pkey[tid] | 1ull;
          } else {
            const int cpos = s.killer[tid];
            const int ri = s.row_of_pos[cpos], rj = s.row_of_pos[tid];
            const int i = min(ri, rj), j = max(ri, rj);
            const float dd = s.pd[s.rowoff[i] + (j - i - 1)];
            tgt = s.pid[cpos];
            key = make_key(dd, (uint32_t)s.pid[tid], 0u);
          }
          atomicAdd(&a.count[tgt], 1);
        }
        a.prop_tgt[v * a.prop_stride + tid] = tgt;
        a.prop_key[v * a.prop_stride + tid] = key;
      }
    } else {
      __syncthreads();
      if (tid < 64) {
        const bool al = tid < m && ((alive >> s.pos_of_slot[tid]) & 1ull);
        const unsigned b = __ballot_sync(0xffffffffu, al);
        if ((tid & 31) == 0) reinterpret_cast<uint32_t*>(&s.mask2)[tid >> 5] = b;
      }
      __syncthreads();
      const uint64_t sm = s.mask2;
      const int cnt = __popcll(sm);
      if (tid < m && ((sm >> tid) & 1ull)) a.out_keys[v * R + __popcll(sm & bits_below(tid))] = kk | 1ull;
      if (tid >= cnt && tid < R) a.out_keys[v * R + tid] = kEmpty;
      if (tid == 0) a.out_deg[v] = cnt;
    }
  }
  if (tid == 0 && a.stats) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[0]), (unsigned long long)st_vert);
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[1]), (unsigned long long)st_rows);
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[2]), (unsigned long long)st_pairs);
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[3]), (unsigned long long)st_fired);
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[4]), (unsigned long long)st_props);
  }
}

}  // namespace

cudaError_t launch_join(const float* X, int64_t n, int d, int ld, int metric, int R,
                        const uint64_t* keys_in, const int32_t* deg_in, uint64_t seed, int t1,
                        int t2, int order, int mode, const Workspace& ws, uint64_t* out_keys,
                        int32_t* out_deg, int64_t* stats, cudaStream_t st) {
  JoinArgs a;
  a.X = X;
  a.n = n;
  a.d = d;
  a.ld = ld;
  a.R = R;
  a.keys_in = keys_in;
  a.deg_in = deg_in;
  a.seed = seed;
  a.t1 = t1;
  a.t2 = t2;
  a.order = order;
  a.mode = mode;
  a.prop_tgt = ws.prop_tgt;
  a.prop_key = ws.prop_key;
  a.prop_stride = R;
  a.count = ws.count;
  a.out_keys = out_keys;
  a.out_deg = out_deg;
  a.stats = stats;
  a.err = ws.err;
  const size_t smem = sizeof(JoinSmem);
  static bool attr_set[2] = {false, false};
  auto kern = metric == 0 ? rnd_join_kernel<0> : rnd_join_kernel<1>;
  if (!attr_set[metric]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set[metric] = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, JT, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t blocks = std::min<int64_t>(n, (int64_t)sm_count() * per_sm);
  ProfScope ps(mode == 0 ? "rnd_join" : "final_prune", st);
  kern<<<(unsigned)blocks, JT, smem, st>>>(a);
  return cudaGetLastError();
}

// =====================================================================================
// Reverse-edge sampling (Sec 3.6): each vertex re-proposes its own pool and proposes
// itself to the first floor(rho * deg) entries of its row (the closest ones).
// =====================================================================================
__global__ void reverse_propose_kernel(int64_t n, int R, float rho,
                                       const uint64_t* __restrict__ keys,
                                       const int32_t* __restrict__ deg,
                                       int32_t* __restrict__ tgt, uint64_t* __restrict__ pk,
                                       int32_t* __restrict__ count) {
  const int64_t total = n * R;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / R;
    const int j = (int)(i - v * R);
    const int k = deg[v];
    const int r = (int)floor((double)rho * (double)k);
    const uint64_t key = keys[i];
    const int64_t base = v * 2 * R;
    tgt[base + j] = j < k ? (int32_t)v : -1;
    pk[base + j] = j < k ? key : kEmpty;
    if (j == 0 && k > 0) atomicAdd(&count[v], k);
    int32_t t1 = -1;
    uint64_t k1 = kEmpty;
    if (j < r) {
      t1 = (int32_t)key_id(key);
      k1 = (key & 0xFFFFFFFF00000000ull) | ((uint64_t)v << 1);
      atomicAdd(&count[t1], 1);
    }
    tgt[base + R + j] = t1;
    pk[base + R + j] = k1;
  }
}

cudaError_t launch_reverse_propose(int64_t n, int R, float rho, const uint64_t* keys,
                                   const int32_t* deg, const Workspace& ws, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>(ceil_div(n * R, 256), (int64_t)sm_count() * 32);
  ProfScope ps("reverse_propose", st);
  reverse_propose_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, R, rho, keys, deg, ws.prop_tgt,
                                                          ws.prop_key, ws.count);
  return cudaGetLastError();
}

// =====================================================================================
// rev_merge: exclusive scan of the per-target counts, scatter of the proposal keys into
// per-target buckets, and a per-target select of the R smallest distinct ids.
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
                               int64_t nslots, const int64_t* __restrict__ off,
                               int32_t* __restrict__ count, uint64_t* __restrict__ bucket) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nslots;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = tgt[i];
    if (t < 0) continue;
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

__global__ void __launch_bounds__(256) select_kernel(const uint64_t* __restrict__ bucket,
                                                     const int64_t* __restrict__ off, int64_t n,
                                                     int R, uint64_t* __restrict__ keys_out,
                                                     int32_t* __restrict__ deg_out,
                                                     int64_t* __restrict__ round_new,
                                                     int64_t* __restrict__ stats) {
  __shared__ uint64_t bufs[8][128];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t* buf = bufs[warp];
  long long n_new = 0, n_in = 0;
  for (int64_t u = (int64_t)blockIdx.x * 8 + warp; u < n; u += (int64_t)gridDim.x * 8) {
    const int64_t b0 = off[u];
    const int64_t c = off[u + 1] - b0;
    n_in += c;
    uint64_t out0, out1;
    if (c <= 64) {
      uint64_t x[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int e = j * 32 + lane;
        x[j] = e < c ? bucket[b0 + e] : kEmpty;
      }
      if (c > 1) select_pass<2>(x, buf);
      out0 = x[0];
      out1 = x[1];
    } else {
      // running top-R (elements 0..63) plus 64 incoming per pass
      uint64_t x[4] = {kEmpty, kEmpty, kEmpty, kEmpty};
      for (int64_t done = 0; done < c; done += 64) {
#pragma unroll
        for (int j = 2; j < 4; ++j) {
          const int64_t e = done + (j - 2) * 32 + lane;
          x[j] = e < c ? bucket[b0 + e] : kEmpty;
        }
        select_pass<4>(x, buf);
        x[2] = kEmpty;
        x[3] = kEmpty;
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
    if (lane < R) keys_out[u * R + lane] = out0;
    if (lane + 32 < R) keys_out[u * R + 32 + lane] = out1;
    if (lane == 0) deg_out[u] = __popc(v0) + __popc(v1);
    n_new += __popc(w0) + __popc(w1);
  }
  if (lane == 0) {
    if (n_new) atomicAdd(reinterpret_cast<unsigned long long*>(round_new), (unsigned long long)n_new);
    if (stats && n_in) atomicAdd(reinterpret_cast<unsigned long long*>(&stats[6]), (unsigned long long)n_in);
  }
}

}  // namespace

cudaError_t launch_merge(const Workspace& ws, int stride, uint64_t* keys_out, int32_t* deg_out,
                         int64_t* stats, cudaStream_t st) {
  const int64_t n = ws.n;
  const int64_t nb = ceil_div(n, SCAN_TILE);
  {
    ProfScope ps("scan", st);
    scan_reduce_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(ws.count, n, ws.bsum);
    scan_blocks_kernel<<<1, 1024, 0, st>>>(ws.bsum, nb, ws.off + n);
    scan_apply_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(ws.count, n, ws.bsum, ws.off);
  }
  const int64_t nslots = n * stride;
  const int64_t sblocks = std::min<int64_t>(ceil_div(nslots, 256), (int64_t)sm_count() * 32);
  {
    ProfScope ps("scatter", st);
    scatter_kernel<<<(unsigned)sblocks, 256, 0, st>>>(ws.prop_tgt, ws.prop_key, nslots, ws.off,
                                                     ws.count, ws.bucket);
  }
  cudaMemsetAsync(ws.round_new, 0, sizeof(int64_t), st);
  const int64_t blocks = std::min<int64_t>(ceil_div(n, 8), (int64_t)sm_count() * 16);
  {
    ProfScope ps("select", st);
    select_kernel<<<(unsigned)blocks, 256, 0, st>>>(ws.bucket, ws.off, n, ws.R, keys_out, deg_out,
                                                   ws.round_new, stats);
  }
  return cudaGetLastError();
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
  const size_t slots = (size_t)n * 2 * R;
  const size_t nb = (size_t)ceil_div(n, SCAN_TILE) + 1;
  return al256(slots * 4) + al256(slots * 8) + al256(slots * 8) + al256((size_t)n * 4) +
         al256(((size_t)n + 1) * 8) + al256(nb * 8) + al256(4) + al256(8);
}

bool carve_workspace(void* base, size_t bytes, int64_t n, int R, Workspace* ws) {
  if (!base || bytes < workspace_bytes(n, R)) return false;
  if (((uintptr_t)base & 255u) != 0) return false;
  const size_t slots = (size_t)n * 2 * R;
  const size_t nb = (size_t)ceil_div(n, SCAN_TILE) + 1;
  char* p = static_cast<char*>(base);
  ws->n = n;
  ws->R = R;
  ws->prop_tgt = reinterpret_cast<int32_t*>(p);
  p += al256(slots * 4);
  ws->prop_key = reinterpret_cast<uint64_t*>(p);
  p += al256(slots * 8);
  ws->bucket = reinterpret_cast<uint64_t*>(p);
  p += al256(slots * 8);
  ws->count = reinterpret_cast<int32_t*>(p);
  p += al256((size_t)n * 4);
  ws->off = reinterpret_cast<int64_t*>(p);
  p += al256(((size_t)n + 1) * 8);
  ws->bsum = reinterpret_cast<int64_t*>(p);
  p += al256(nb * 8);
  ws->err = reinterpret_cast<int32_t*>(p);
  p += al256(4);
  ws->round_new = reinterpret_cast<int64_t*>(p);
  return true;
}

}  // namespace grnnd
