// Host-side declarations shared by the GRNND translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <memory>
#include <string>
#include <cuda_runtime.h>

#include "grnnd.h"

namespace grnnd {

// Device workspace of one round, final pass or reverse step for n vertices of capacity R.
struct Workspace {
  int64_t n = 0;
  int R = 0;
  int32_t* red_tgt = nullptr;              // redirect / reverse-proposal targets (-1: unused)
  int64_t red_cap = 0;                     // slots of red_tgt / red_key
  uint64_t* red_key = nullptr;             // n*R their keys
  uint64_t* bucket = nullptr;              // n*R keys bucketed by target
  int32_t* count = nullptr;                // n proposals per target (zeroed per step)
  int64_t* off = nullptr;                  // n+1 exclusive prefix of count
  int64_t* bsum = nullptr;                 // scan block sums
  uint8_t* active = nullptr;               // n flags: the vertex is in the list
  uint8_t* next_active = nullptr;          // n flags written by an in-place merge: the row holds
                                           // a new entry (read by the next step's prep)
  uint64_t* rec[5] = {};                   // work records by pool-size class (entries <= 8,
  int rec_w[5] = {};                       // <= 16, <= 32, <= 64, more): n records of rec_w[c]
  int rec_cap[5] = {};                     // words each, holding up to rec_cap[c] entries (the
                                           // last class exists only when R > 64)
  int32_t* list_n = nullptr;               // [5] records per class
  unsigned long long* red_n = nullptr;     // number of redirects / reverse proposals
  unsigned int* work_q = nullptr;          // [3] next work item of the warp and team joins (third word spare)
  int32_t* err = nullptr;                  // device status word (bounded waits)
  int64_t* round_new = nullptr;            // new entries written by the last merge
};

// Each quantized row ends in a 32-byte tail holding (norm^2 of the quantized row, residual
// norm) as two floats, then zeros: 16 BF16 elements or 32 e4m3 bytes, which keeps every row
// on a 32-byte sector boundary.  The row stride is the padded dimension count (16 BF16 / 32
// e4m3 elements) plus the tail; the joins copy the tail's first kTailCopy bytes with a row.
constexpr int kRowTail16 = 16;
constexpr int kRowTail8 = 32;
constexpr int kTailCopy = 16;

// The points as the pool kernels read them.  precision 0: FP32 rows only; 1: also a
// BF16 copy (row stride ldb = d rounded up to 16, plus the tail), per-row (norm^2, residual)
// and dataset flags; 2: an FP8-e4m3 copy (ldb = d rounded up to 32, plus the tail) with the
// same per-row terms, the row's scale exponent in the low byte of the residual.
// bytes from src to dst on stream st, either side device or host memory.  When one side is
// pinned (page-locked, mapped) host memory, both are 16-byte aligned and bytes is a multiple
// of 16, a kernel moves them with 16-byte loads and stores over the host link instead of the
// copy engine: the same rate (about 210 GB/s up, 190 GB/s down), without the copy engine's
// periodic stalls between builds (copies of 10-25 ms instead of 1.3-2.4 ms, about every
// 0.5 s).  Otherwise cudaMemcpyAsync.
cudaError_t copy_bytes(void* dst, const void* src, size_t bytes, cudaStream_t st);

// n rows of d floats into rows of ld >= d floats.  Rows that need no padding go as one
// contiguous copy (copy_bytes), not as a pitched copy.
inline cudaError_t copy_rows(float* dst, int ld, const float* src, int d, int64_t n, cudaMemcpyKind kind,
                             cudaStream_t st) {
  if (ld == d) return copy_bytes(dst, src, (size_t)n * d * 4, st);
  return cudaMemcpy2DAsync(dst, (size_t)ld * 4, src, (size_t)d * 4, (size_t)d * 4, (size_t)n, kind, st);
}

struct PointsSet {
  const float* X = nullptr;
  int ld = 0;
  const void* Xb = nullptr;
  int ldb = 0;
  const float2* aux = nullptr;
  const unsigned* qflags = nullptr;
  int d = 0, metric = 0, precision = 0;
  // Batched builds: per vertex (first id, number of points) of the build it belongs to;
  // null for one build.  Random draws and visit orders use ids local to the build.
  const int2* vseg = nullptr;
  // Join launch shape (grnnd_tuning): lane-group routing by pool size, CTAs per SM caps.
  int group_max[3] = {8, 16, 32};
  int warp_ctas = 0, team_ctas = 0;
  int row_copies = 0;  // quantized rows of the warp join: 1 one bulk copy per row, 2 gather4 (where
                       // possible), 0 gather4 for BF16 rows of at most 128 dimensions, else 1
};

// Where a build's device memory comes from: cudaMalloc / cudaFree (pool == nullptr), or
// stream-ordered allocations from `pool` on the build's stream, the graph's own memory being
// released on `free_stream` (the serving loop: builds on different streams then never wait
// on the implicit device synchronisation of cudaFree).
struct AllocMode {
  cudaMemPool_t pool = nullptr;
  cudaStream_t free_stream = nullptr;
  // the graph's memory may still be read by the caller's own work on any stream when it is
  // freed: synchronise the device first (the memory cache of grnnd_set_memory_cache)
  bool sync_before_free = false;
};

size_t workspace_bytes(int64_t n, int R);
bool carve_workspace(void* base, size_t bytes, int64_t n, int R, Workspace* ws);

// Xb16 / ldb / qflags (optional): the BF16 copy of the rows and its dataset flags; when every
// value is exact in BF16 the drawn rows are read from it (same values, half the bytes).
cudaError_t launch_pool_init(const float* X, int64_t n, int d, int ld, int metric, int S, int R,
                             uint64_t seed, uint64_t* keys, int32_t* deg, cudaStream_t st,
                             const int2* vseg = nullptr, const void* Xb16 = nullptr, int ldb = 0,
                             const unsigned* qflags = nullptr);

// Batched builds: subtracts each row's build base from its ids (-1 stays -1).
cudaError_t launch_localize_ids(int64_t n, int R, int32_t* ids, const int2* vseg, cudaStream_t st);

// precision 1: BF16 rows (ldb = d rounded up to 16 elements, plus the tail); 2: e4m3 rows
// with a power-of-two scale per row (ldb = d rounded up to 32 bytes, plus the tail).
cudaError_t launch_quantize(const float* X, int64_t n, int d, int ld, void* Xb, int ldb,
                            float2* aux, unsigned* qflags, int precision, cudaStream_t st);

// One-time launch set-up of the join kernels that points P will use (shared-memory opt-in,
// occupancy); launches inside a stream capture rely on it having run.
cudaError_t prepare_join_kernels(const PointsSet& P);

// One round of Alg 4: prep + rnd_join + scan + scatter + select (keys_out == keys_in: in
// place).  use_hint: the last step on these pools was an in-place round or reverse step with
// the same workspace, so its per-row new-entry flags replace prep's scan of the keys.
// keys_canonical: every distance in the pools came from the library's own arithmetic (a
// whole build), so the merge may find duplicate ids by their keys.
cudaError_t launch_round(const PointsSet& P, int64_t n, int R, const uint64_t* keys_in,
                         const int32_t* deg_in, uint64_t seed, int t1, int t2, int order,
                         const Workspace& ws, uint64_t* keys_out, int32_t* deg_out, int64_t* stats,
                         cudaStream_t st, bool use_hint = false, bool keys_canonical = false);

// Final prune-only pass: survivors only, no redirects (use_hint as for launch_round).
cudaError_t launch_final(const PointsSet& P, int64_t n, int R, const uint64_t* keys_in,
                         const int32_t* deg_in, uint64_t seed, int t1, int order,
                         const Workspace& ws, uint64_t* keys_out, int32_t* deg_out, cudaStream_t st,
                         bool use_hint = false);

// Reverse-edge sampling + merge.
cudaError_t launch_reverse(int64_t n, int R, float rho, const uint64_t* keys_in,
                           const int32_t* deg_in, const Workspace& ws, uint64_t* keys_out,
                           int32_t* deg_out, int64_t* stats, cudaStream_t st);

cudaError_t launch_keys_to_graph(int64_t n, int R, const uint64_t* keys, int32_t* ids,
                                 float* dists, int32_t* deg, cudaStream_t st);

cudaError_t launch_pair_dist(const float* X, int d, int ld, int metric, const int32_t* pairs,
                             int64_t np, float* out, cudaStream_t st);

cudaError_t launch_check_finite(const float* X, int64_t n, int d, int ld, int32_t* flag,
                                cudaStream_t st);

size_t entry_workspace_bytes(int64_t n, int d);
// Search entries of nbuild builds whose rows are [off[b], off[b+1]) of X (off: device
// int64[nbuild + 1]); entries[b] = the entry launch_entry gives for build b alone (local id).
size_t entry_batch_workspace_bytes(int32_t nbuild, int d);
cudaError_t launch_entry_batch(const float* X, int d, int ld, int metric, const int64_t* off_dev, int32_t nbuild,
                               int32_t* entries, void* ws, size_t ws_bytes, cudaStream_t st);
cudaError_t launch_entry(const float* X, int64_t n, int d, int ld, int metric, int32_t* entry,
                         void* ws, size_t ws_bytes, cudaStream_t st);

cudaError_t launch_search(const float* X, int64_t n, int d, int ld, int metric,
                          const int32_t* gids, const int32_t* gdeg, int R, int entry,
                          const float* Q, int64_t nq, int ldq, int k, int beam, int32_t* ids_out,
                          float* dists_out, cudaStream_t st);

cudaError_t launch_brute_knn(const float* X, int64_t n, int d, int ld, int metric, const float* Q,
                             int64_t nq, int ldq, int k, int32_t* ids_out, float* dists_out,
                             cudaStream_t st);

// Self-test of the bounded device waits: *status (host) = 1 when a wait that nothing
// completes gave up after `limit` tries, 0 if it completed (never).  Synchronises `st`.
cudaError_t launch_wait_selftest(uint32_t limit, int32_t* status, cudaStream_t st);

int sm_count();

// Sets the thread-local message returned by grnnd_last_error.
void set_last_error(const std::string& msg);

// Per-kernel event profiler of the calling thread (no-ops unless enabled).
void prof_start(const char* name, cudaStream_t st);
bool prof_on();  // the per-kernel event profiler is recording
void prof_stop(cudaStream_t st);

struct ProfScope {
  cudaStream_t st;
  ProfScope(const char* name, cudaStream_t s) : st(s) { prof_start(name, s); }
  ~ProfScope() { prof_stop(st); }
};

}  // namespace grnnd

// Device memory of one build call; the graphs of a batched build share it, and it is freed
// with the last of them (stream-ordered when it came from a memory pool).
struct GraphBlock {
  void* points = nullptr;
  void* graph = nullptr;
  bool pooled = false;
  bool sync_before_free = false;
  cudaStream_t free_stream = nullptr;
  ~GraphBlock() {
    if (pooled && sync_before_free && (points || graph)) cudaDeviceSynchronize();
    for (void* q : {points, graph})
      if (q) {
        if (pooled)
          cudaFreeAsync(q, free_stream);
        else
          cudaFree(q);
      }
  }
};

struct grnnd_graph {
  int64_t n = 0;
  int32_t d = 0, ld = 0, R = 0, metric = 0, entry = 0;
  float* points = nullptr;   // n x ld, zero padded
  int32_t* ids = nullptr;    // n x R
  float* dists = nullptr;    // n x R
  int32_t* deg = nullptr;    // n
  int64_t stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  std::shared_ptr<GraphBlock> mem;
};

namespace grnnd {
// grnnd_build_ex's argument checks (GRNND_OK or GRNND_EINVAL with the message set).
int validate_build(const float* points, int64_t n, int32_t d, const grnnd_params* p);
// Whole build with the allocation mode of the caller (grnnd_build_ex's validation first).
int build_with(const float* points, int64_t n, int32_t d, const grnnd_params* p, const AllocMode& am,
               grnnd_graph** graph_out);
// Device bytes a single build of n x d points with params p allocates: *resident of them stay
// with the graph (points + rows), the rest is scratch released when the build returns.
size_t build_device_bytes(int64_t n, int32_t d, const grnnd_params* p, size_t* resident);
}  // namespace grnnd
