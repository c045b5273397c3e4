// Wide pools (R > 64) for sm_103a: the join of pools of 65..256 entries and the per-target
// merge of rows longer than 64 entries.
//
//   rnd_join_wide   Alg 4's pair loop with the rule of Eq 2 for one vertex per CTA
//                   (256 threads, thread t owns storage slot t):
//     order   rank of (h(seed,t1,t2,v,id), id) among the m entries (or the key order);
//     tile    the canonical FP32 distance of every pair with a new side, as 64 x 64 tiles of
//             local rows (new entries first), staged 32 dimensions at a time, each thread
//             holding 4 x 4 pairs with their four partial sums; a pair that fires sets its
//             bit in the later position's fire mask (four 64-bit words per position);
//     chain   the sequential outcome of the pair scan over the fire masks as a fixed point,
//             one column (pi position) per thread, with a block-wide prefix OR per round;
//     emit    survivors rewritten in place as old; each bottom entry one redirect to its
//             absorber, with the canonical distance of the pair that fired.
//   The tiles use the FP32 rows in every precision form, so every decision and every
//   recorded distance of these pools is the canonical FP32 one.
//
//   select_wide     per target, the merge rule of Sec 3.5 / Alg 6's end state: the R
//                   smallest distinct ids of (the row, the target's bucket), a duplicate
//                   keeping its smallest distance and old if any copy is old; done as two
//                   block-wide sorts (by (id, dist) to drop duplicates, then by key) in
//                   shared memory, 2,048 entries at a time.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "kernels.cuh"

namespace grnnd {

namespace {

constexpr int XW = 256;    // threads per wide join CTA = largest pool
constexpr int XT = 64;     // local rows per tile side
constexpr int XDC = 32;    // dimensions per staged chunk
constexpr int XRED = kRedChunk;  // redirect slots a CTA reserves at a time
static_assert(XW == kMaxRWide, "one thread per pool entry");

struct __align__(16) WideSmem {
  float sa[XDC][XT + 4];     // staged chunk of the tile's first rows, dimension-major
  float sb[XDC][XT + 4];     // ... and of its second rows
  uint64_t fire[XW][4];      // by pi position b: positions a < b whose pair with b fires
  uint64_t closer[XW][4];    // by pi position b: positions whose entry is closer to v than b's
  uint64_t hk[XW];           // visit-order key by storage slot
  uint32_t hid[XW];          // id by storage slot (ties of the order key)
  int32_t rowid[XW];         // point id by local row (new entries first, each part in slot order)
  float rowdv[XW];           // recorded distance to v by local row
  uint16_t rowpos[XW];       // pi position by local row
  uint16_t posslot[XW];      // storage slot by pi position
  int16_t killer[XW];        // by pi position: the absorbing position (-1: survives)
  uint64_t wtot[2][8][4];    // chain rounds: per warp, the OR of its columns' kill sets
  uint32_t wnew[8], wsurv[8];
  unsigned long long red_next, red_end, red_b0, red_b1;
  int32_t red_avail;
};

__device__ __forceinline__ uint64_t word_of(const uint64_t (&x)[4], int i) {
  return i < 64 ? x[0] : (i < 128 ? x[1] : (i < 192 ? x[2] : x[3]));
}
// bits of positions below f in word w (all of them when f < 0)
__device__ __forceinline__ uint64_t below_in_word(int f, int w) {
  if (f < 0) return ~0ull;
  const int fw = f >> 6;
  if (w < fw) return ~0ull;
  if (w > fw) return 0ull;
  const int r = f & 63;
  return r == 0 ? 0ull : (~0ull >> (64 - r));
}
__device__ __forceinline__ unsigned lanes_below() { return (1u << (threadIdx.x & 31)) - 1u; }

// Stages dimensions [c0, c0 + XDC) of local rows [r0, r0 + XT) into st (zero past d or m).
__device__ __forceinline__ void wide_stage(float (*st)[XT + 4], const WideSmem& s, int r0, int m, int c0,
                                           const JoinArgs& a) {
  const int t = threadIdx.x, r = t >> 2, q = t & 3;  // row r, dimensions 8q .. 8q + 7
  const int row = r0 + r;
  const float* src = nullptr;
  if (row < m && in_bounds((uint32_t)s.rowid[row] < (uint64_t)a.n, a.err))
    src = a.P.X + (int64_t)s.rowid[row] * a.P.ld;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int k = c0 + 8 * q + 4 * h;
    float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (src && k < a.P.d) {
      g = __ldg(reinterpret_cast<const float4*>(src + k));
      if (k + 4 > a.P.d) g = mask4(g, a.P.d - k);
    }
    st[8 * q + 4 * h + 0][r] = g.x;
    st[8 * q + 4 * h + 1][r] = g.y;
    st[8 * q + 4 * h + 2][r] = g.z;
    st[8 * q + 4 * h + 3][r] = g.w;
  }
}

template <int METRIC>
__global__ void __launch_bounds__(XW) rnd_join_wide_kernel(JoinArgs a) {
  __shared__ WideSmem s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t cnt = a.list_n[4];  // records of the widest size class
  if ((int64_t)blockIdx.x >= cnt || *(volatile int32_t*)a.err) return;
  const int R = a.R, W = a.rec_w[4];
  const uint64_t head = hash_head(a.seed, (uint64_t)a.t1, (uint64_t)a.t2);
  if (tid == 0) s.red_next = s.red_end = 0;
  long long st_vert = 0, st_rows = 0, st_pairs = 0, st_fired = 0;

  for (int64_t p = blockIdx.x; p < cnt; p += gridDim.x) {
    const uint64_t* rec = a.rec[4] + p * W;
    const int64_t v = (int64_t)(rec[0] & 0xffffffffull);
    const uint32_t lo = (uint32_t)(rec[0] >> 32);  // first id of the vertex's build
    const int m = (int)rec[1];
    const bool has = tid < m;
    const uint64_t key = (has && in_bounds((uint64_t)v < (uint64_t)a.n, a.err)) ? a.keys_in[v * R + tid] : kEmpty;
    const uint32_t idl = key_id(key);
    // ---- visit order and local rows ---------------------------------------------------
    uint64_t h = ~0ull;
    if (has)
      h = (a.order == 0)   ? hash_tail(head, (uint64_t)(v - lo), (uint64_t)(idl - lo))
          : (a.order == 1) ? (uint64_t)tid
                           : (uint64_t)(m - 1 - tid);
    s.hk[tid] = h;
    s.hid[tid] = has ? idl : 0xffffffffu;
    const bool isnew = has && !key_old(key);
    const unsigned bn = __ballot_sync(0xffffffffu, isnew);
    if (lane == 0) s.wnew[warp] = bn;
    __syncthreads();
    int k = 0, newbefore = __popc(bn & lanes_below());
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const int c = __popc(s.wnew[w]);
      k += c;
      if (w < warp) newbefore += c;
    }
    // rows: the new entries first, then the old ones, each part in storage-slot order
    const int row = isnew ? newbefore : k + (tid - newbefore);
    int pi = 0;
    if (has)
      for (int f = 0; f < m; ++f) {
        const uint64_t hf = s.hk[f];
        pi += (hf < h) || (hf == h && s.hid[f] < idl);
      }
    if (has) {
      s.rowid[row] = (int32_t)idl;
      s.rowdv[row] = key_dist(key);
      s.rowpos[row] = (uint16_t)pi;
      s.posslot[pi] = (uint16_t)tid;
    }
#pragma unroll
    for (int w = 0; w < 4; ++w) s.fire[tid][w] = 0ull;
    s.killer[tid] = -1;
    // "closer to v" is storage-slot order (rows hold their keys in ascending order): the
    // closer mask of a position is the OR of the position bits of the slots before its own
    {
      uint64_t inc[4];
#pragma unroll
      for (int w = 0; w < 4; ++w) inc[w] = (has && (pi >> 6) == w) ? (1ull << (pi & 63)) : 0ull;
#pragma unroll
      for (int w = 0; w < 4; ++w)
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
          const uint64_t y = __shfl_up_sync(0xffffffffu, inc[w], dd);
          if (lane >= dd) inc[w] |= y;
        }
      if (lane == 31)
#pragma unroll
        for (int w = 0; w < 4; ++w) s.wtot[0][warp][w] = inc[w];
      __syncthreads();
      uint64_t pre[4];
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        uint64_t x = __shfl_up_sync(0xffffffffu, inc[w], 1);
        if (lane == 0) x = 0ull;
        for (int q = 0; q < warp; ++q) x |= s.wtot[0][q][w];
        pre[w] = x;
      }
      if (has)
#pragma unroll
        for (int w = 0; w < 4; ++w) s.closer[pi][w] = pre[w];
    }
    __syncthreads();

    // ---- tiles: canonical FP32 distance of every pair (i < k, i < j < m) of local rows ----
    const int np = k * (m - 1) - k * (k - 1) / 2;
    const int ti = tid >> 4, tj = tid & 15;
    const int nblk = (m + XT - 1) / XT, kblk = (k + XT - 1) / XT;
    for (int I = 0; I < kblk; ++I)
      for (int J = I; J < nblk; ++J) {
        float4 acc[4][4];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int c0 = 0; c0 < a.P.d; c0 += XDC) {
          __syncthreads();  // the previous chunk has been read
          wide_stage(s.sa, s, I * XT, m, c0, a);
          wide_stage(s.sb, s, J * XT, m, c0, a);
          __syncthreads();
          // dimensions in ascending order, dimension c0 + kk + q into partial sum q: the
          // canonical four-accumulator evaluation
#pragma unroll 2
          for (int kk = 0; kk < XDC; kk += 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 av = *reinterpret_cast<const float4*>(&s.sa[kk + q][ti * 4]);
              const float4 bv = *reinterpret_cast<const float4*>(&s.sb[kk + q][tj * 4]);
              const float ax[4] = {av.x, av.y, av.z, av.w}, bx[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
              for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                  float& c = q == 0 ? acc[x][y].x : (q == 1 ? acc[x][y].y : (q == 2 ? acc[x][y].z : acc[x][y].w));
                  c = dist_step<METRIC>(c, ax[x], bx[y]);
                }
            }
          }
        }
        // fire decisions of the tile's pairs
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            const int i = I * XT + ti * 4 + x, j = J * XT + tj * 4 + y;
            if (i < k && j > i && j < m) {
              const float dab = dist_finish4<METRIC>(acc[x][y]);
              if (dab < fmaxf(s.rowdv[i], s.rowdv[j])) {
                const int pa = s.rowpos[i], pb = s.rowpos[j];
                const int lo2 = min(pa, pb), hi2 = max(pa, pb);
                atomicOr(reinterpret_cast<unsigned long long*>(&s.fire[hi2][lo2 >> 6]), 1ull << (lo2 & 63));
              }
            }
          }
      }
    __syncthreads();

    // ---- prune: the chain's outcome, one column (pi position) per thread ------------------
    // Column b of the sequential pair scan kills K_b: its live firing partners before the
    // first closer one f, then b itself (absorbed by f); all of them when none is closer.
    // Its live partners are the valid positions that no column c < b killed (b itself is
    // alive when its column starts: earlier columns involve only earlier positions), so the
    // outcome is the fixed point of K_b = rule(fire[b] & valid & ~OR_{c<b} K_c).  Rounds that
    // apply the rule to every column at once from K = 0 reach it: after round r the columns
    // 0..r are final; the first round whose prefix ORs repeat the ones it used ends the loop.
    uint64_t K[4] = {0ull, 0ull, 0ull, 0ull};
    int f = -1;
    {
      const int b = tid;
      uint64_t fb[4], cb[4], valid[4], pre[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        fb[w] = s.fire[b][w];
        cb[w] = s.closer[b][w];
        const int lo3 = w * 64;
        valid[w] = m >= lo3 + 64 ? ~0ull : (m <= lo3 ? 0ull : (~0ull >> (64 - (m - lo3))));
      }
      for (int r = 0;; ++r) {
        uint64_t cand[4];
        f = -1;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          cand[w] = (b < m) ? (fb[w] & valid[w] & ~pre[w]) : 0ull;
          const uint64_t x = cand[w] & cb[w];
          if (f < 0 && x) f = w * 64 + __ffsll((long long)x) - 1;
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          K[w] = cand[w] & below_in_word(f, w);
          if (f >= 0 && (b >> 6) == w) K[w] |= 1ull << (b & 63);
        }
        uint64_t inc[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          inc[w] = K[w];
#pragma unroll
          for (int dd = 1; dd < 32; dd <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, inc[w], dd);
            if (lane >= dd) inc[w] |= y;
          }
        }
        const int buf = r & 1;
        if (lane == 31)
#pragma unroll
          for (int w = 0; w < 4; ++w) s.wtot[buf][warp][w] = inc[w];
        __syncthreads();
        bool changed = false;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          uint64_t x = __shfl_up_sync(0xffffffffu, inc[w], 1);
          if (lane == 0) x = 0ull;
          for (int q = 0; q < warp; ++q) x |= s.wtot[buf][q][w];
          changed |= (x != pre[w]);
          pre[w] = x;
        }
        if (!__syncthreads_or(changed) || r >= XW) break;
      }
      // absorbers: b for the partners it kills, f for b itself
      if (b < m) {
#pragma unroll
        for (int w = 0; w < 4; ++w)
          for (uint64_t kb = K[w] & ~(((b >> 6) == w) ? (1ull << (b & 63)) : 0ull); kb; kb &= kb - 1)
            s.killer[w * 64 + __ffsll((long long)kb) - 1] = (int16_t)b;
        if (f >= 0) s.killer[b] = (int16_t)f;
      }
    }
    __syncthreads();

    // ---- emit ----------------------------------------------------------------------------
    const bool surv = has && s.killer[pi] < 0;
    const unsigned sb = __ballot_sync(0xffffffffu, surv);
    if (lane == 0) s.wsurv[warp] = sb;
    __syncthreads();
    int nkeep = 0, survbefore = __popc(sb & lanes_below());
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const int c = __popc(s.wsurv[w]);
      nkeep += c;
      if (w < warp) survbefore += c;
    }
    const int ndead = m - nkeep;
    if (a.emit_redirects && tid == 0 && ndead > 0) {
      // fill the CTA's chunk to its end, then continue in a fresh one (ndead < XRED)
      const unsigned long long base = s.red_next;
      unsigned long long b1 = base, next = base + (unsigned long long)ndead;
      int avail = ndead;
      if (next > s.red_end) {
        avail = (int)(s.red_end - base);
        b1 = atomicAdd(a.red_n, (unsigned long long)XRED);
        next = b1 + (unsigned long long)(ndead - avail);
        s.red_end = b1 + XRED;
      }
      s.red_next = next;
      s.red_b0 = base;
      s.red_b1 = b1;
      s.red_avail = avail;
    }
    __syncthreads();
    const bool vok = in_bounds((uint64_t)v < (uint64_t)a.n, a.err);
    if (surv && vok) a.keys_out[v * R + survbefore] = key | 1ull;
    // in place, the slots past m are empty already (pool rows end in empty slots)
    const int pend = a.keys_out == a.keys_in ? m : R;
    for (int t = nkeep + tid; vok && t < pend; t += XW) a.keys_out[v * R + t] = kEmpty;
    if (tid == 0 && vok) a.deg_out[v] = nkeep;
    if (a.emit_redirects && has && !surv) {
      const int kp = s.killer[pi];
      const int32_t tgt = (int32_t)s.hid[s.posslot[kp]];
      const int g = tid - survbefore;  // bottom entries in the slots before this one
      const unsigned long long sl =
          g < s.red_avail ? s.red_b0 + (unsigned long long)g : s.red_b1 + (unsigned long long)(g - s.red_avail);
      if (in_bounds(sl < (unsigned long long)a.red_cap && (uint64_t)(uint32_t)tgt < (uint64_t)a.n &&
                        (uint64_t)idl < (uint64_t)a.n,
                    a.err)) {
        // the canonical distance of the pair that fired (the tiles' value, bit for bit)
        const float dd = row_dist<METRIC>(a.P.X + (int64_t)tgt * a.P.ld, a.P.X + (int64_t)idl * a.P.ld, a.P.d);
        a.red_tgt[sl] = tgt;
        a.red_key[sl] = make_key(dd, idl, 0u);
        atomicAdd(&a.count[tgt], 1);
      }
    }
    if (tid == 0) {
      st_vert += 1;
      st_rows += m;
      st_pairs += np;
      st_fired += ndead;
    }
    __syncthreads();
  }
  if (a.emit_redirects)
    for (unsigned long long i = s.red_next + tid; i < s.red_end; i += XW) a.red_tgt[i] = -1;
  if (a.stats && tid == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[0]), (unsigned long long)st_vert);
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[1]), (unsigned long long)st_rows);
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[2]), (unsigned long long)st_pairs);
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[3]), (unsigned long long)st_fired);
  }
}

// ---- merge of rows of more than 64 entries ---------------------------------------------
constexpr int SWT = 256;    // threads per CTA
constexpr int SWN = 2048;   // entries sorted at a time (the row and a chunk of proposals)
constexpr int SWH = 512;    // slots of the hash of the row's old ids

// (id, dist, old) order: equal ids meet, the nearest copy first
__device__ __forceinline__ uint64_t to_idkey(uint64_t k) {
  return ((uint64_t)key_id(k) << 33) | ((k >> 32) << 1) | (k & 1ull);
}
__device__ __forceinline__ uint64_t from_idkey(uint64_t x) {
  return (((x >> 1) & 0xffffffffull) << 32) | ((x >> 33) << 1) | (x & 1ull);
}
__device__ __forceinline__ uint32_t old_slot(uint32_t id) { return (id * 0x9E3779B1u) >> 23; }

// Ascending bitonic sort of buf[0, P) (P a power of two) by the block.
__device__ void block_sort(uint64_t* buf, int P) {
  for (int kk = 2; kk <= P; kk <<= 1)
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += SWT) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const uint64_t x = buf[i], y = buf[ixj];
          const bool up = (i & kk) == 0;
          if ((x > y) == up) {
            buf[i] = y;
            buf[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
}

__global__ void __launch_bounds__(SWT) select_wide_kernel(SelectArgs a) {
  __shared__ uint64_t buf[SWN];
  __shared__ uint32_t oid[SWH];
  __shared__ int s_cnt, s_new;
  const int tid = threadIdx.x;
  const int R = a.R;
  if (*a.err) return;
  const bool in_place = a.keys_out == a.keys_in;
  long long n_new = 0, n_in = 0;
  for (int64_t u = blockIdx.x; u < a.n; u += gridDim.x) {
    int64_t b0 = 0, c = 0;
    if (a.bucket) {
      b0 = a.off[u];
      c = a.off[u + 1] - b0;
    }
    const bool kept = in_place || (a.active && a.active[u]);
    if (c == 0 && kept) {  // nothing proposed and the row is in place: final already
      if (a.next_active && a.next_active_all && tid == 0) a.next_active[u] = 0;
      continue;
    }
    if (!in_bounds(b0 >= 0 && c >= 0 && b0 + c <= a.n * R, a.err)) continue;
    const uint64_t* base = kept ? a.keys_out + u * R : a.keys_in + u * R;
    const int na = kept ? a.deg_out[u] : a.deg_in[u];
    for (int i = tid; i < SWH; i += SWT) oid[i] = 0xffffffffu;
    __syncthreads();
    for (int i = tid; i < na; i += SWT) {
      const uint64_t x = base[i];
      buf[i] = x;
      if (x & 1ull) {  // the row's ids are distinct: each insert finds a free slot
        const uint32_t id = key_id(x);
        uint32_t sl = old_slot(id);
        for (int probe = 0; probe < SWH; ++probe) {
          if (atomicCAS(&oid[sl], 0xffffffffu, id) == 0xffffffffu) break;
          sl = (sl + 1) & (SWH - 1);
        }
      }
    }
    __syncthreads();
    n_in += c;
    int cur = na;
    for (int64_t done = 0; done < c;) {
      const int take = (int)std::min<int64_t>(c - done, (int64_t)(SWN - cur));
      // proposals are new; an id is old in the result iff the row held it as old, which an
      // earlier chunk may have pushed out of the row: each proposal takes its id's old bit
      for (int i = tid; i < take; i += SWT) {
        uint64_t x = a.bucket[b0 + done + i];
        const uint32_t id = key_id(x);
        uint32_t sl = old_slot(id);
        for (int probe = 0; probe < SWH; ++probe) {
          const uint32_t hv = oid[sl];
          if (hv == id) {
            x |= 1ull;
            break;
          }
          if (hv == 0xffffffffu) break;
          sl = (sl + 1) & (SWH - 1);
        }
        buf[cur + i] = x;
      }
      done += take;
      const int tot = cur + take;
      int P = 2;
      while (P < tot) P <<= 1;
      __syncthreads();
      for (int i = tid; i < P; i += SWT) buf[i] = i < tot ? to_idkey(buf[i]) : ~0ull;
      __syncthreads();
      block_sort(buf, P);
      // one copy per id: the first of its run (the nearest; every copy of an id the row
      // held as old carries the old bit)
      uint64_t keep[SWN / SWT];
#pragma unroll
      for (int q = 0; q < SWN / SWT; ++q) {
        const int i = tid + q * SWT;
        keep[q] = kEmpty;
        if (i < tot) {
          const uint64_t x = buf[i];
          if (i == 0 || (buf[i - 1] >> 33) != (x >> 33)) keep[q] = from_idkey(x);
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < SWN / SWT; ++q) {
        const int i = tid + q * SWT;
        if (i < P) buf[i] = keep[q];
      }
      if (tid == 0) s_cnt = 0;
      __syncthreads();
      int mine = 0;
#pragma unroll
      for (int q = 0; q < SWN / SWT; ++q) mine += keep[q] != kEmpty;
      if (mine) atomicAdd(&s_cnt, mine);
      block_sort(buf, P);  // by key: the distinct ids nearest first, then the empties
      cur = min(R, s_cnt);
      __syncthreads();
    }
    if (tid == 0) s_new = 0;
    __syncthreads();
    int fresh = 0;
    for (int i = tid; i < R; i += SWT) {
      const uint64_t x = i < cur ? buf[i] : kEmpty;
      a.keys_out[u * R + i] = x;
      fresh += (x != kEmpty && !(x & 1ull));
    }
    if (fresh) atomicAdd(&s_new, fresh);
    __syncthreads();
    if (tid == 0) {
      a.deg_out[u] = cur;
      n_new += s_new;
      if (a.next_active) a.next_active[u] = s_new > 0 ? 1 : 0;
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n_new) atomicAdd(reinterpret_cast<unsigned long long*>(a.round_new), (unsigned long long)n_new);
    if (a.stats && n_in) atomicAdd(reinterpret_cast<unsigned long long*>(&a.stats[6]), (unsigned long long)n_in);
  }
}

}  // namespace

cudaError_t launch_join_wide(const JoinArgs& a, int metric, cudaStream_t st, const char* name) {
  const int64_t blocks = std::min<int64_t>((int64_t)sm_count() * 4, kMaxJoinGrid);
  ProfScope ps(name, st);
  if (metric == 0)
    rnd_join_wide_kernel<0><<<(unsigned)blocks, XW, 0, st>>>(a);
  else
    rnd_join_wide_kernel<1><<<(unsigned)blocks, XW, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_select_wide(const SelectArgs& a, cudaStream_t st) {
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(a.n, (int64_t)sm_count() * 8));
  ProfScope ps("select_wide", st);
  select_wide_kernel<<<(unsigned)blocks, SWT, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace grnnd
