// Host-side declarations shared by the GRNND translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

namespace grnnd {

// Device workspace of one round / reverse step for n vertices of capacity R.
// Proposal slots: 2R per vertex (a round uses R, reverse sampling 2R).
struct Workspace {
  int64_t n = 0;
  int R = 0;
  int32_t* prop_tgt = nullptr;   // n*2R target vertex or -1
  uint64_t* prop_key = nullptr;  // n*2R pool key of the proposal
  uint64_t* bucket = nullptr;    // n*2R keys bucketed by target
  int32_t* count = nullptr;      // n proposals per target (zero between steps)
  int64_t* off = nullptr;        // n+1 exclusive prefix of count
  int64_t* bsum = nullptr;       // scan block sums
  int32_t* err = nullptr;        // device status word (bounded waits)
  int64_t* round_new = nullptr;  // new entries written by the last merge
};

size_t workspace_bytes(int64_t n, int R);
bool carve_workspace(void* base, size_t bytes, int64_t n, int R, Workspace* ws);

cudaError_t launch_pool_init(const float* X, int64_t n, int d, int ld, int metric, int S, int R,
                             uint64_t seed, uint64_t* keys, int32_t* deg, cudaStream_t st);

// mode 0: emit proposals of a round into ws; mode 1: final prune into out_keys/out_deg.
cudaError_t launch_join(const float* X, int64_t n, int d, int ld, int metric, int R,
                        const uint64_t* keys_in, const int32_t* deg_in, uint64_t seed, int t1,
                        int t2, int order, int mode, const Workspace& ws, uint64_t* out_keys,
                        int32_t* out_deg, int64_t* stats, cudaStream_t st);

cudaError_t launch_reverse_propose(int64_t n, int R, float rho, const uint64_t* keys,
                                   const int32_t* deg, const Workspace& ws, cudaStream_t st);

// scan + scatter + per-target select of the proposals in ws (stride slots per vertex).
cudaError_t launch_merge(const Workspace& ws, int stride, uint64_t* keys_out, int32_t* deg_out,
                         int64_t* stats, cudaStream_t st);

cudaError_t launch_keys_to_graph(int64_t n, int R, const uint64_t* keys, int32_t* ids,
                                 float* dists, int32_t* deg, cudaStream_t st);

cudaError_t launch_pair_dist(const float* X, int d, int ld, int metric, const int32_t* pairs,
                             int64_t np, float* out, cudaStream_t st);

cudaError_t launch_check_finite(const float* X, int64_t n, int d, int ld, int32_t* flag,
                                cudaStream_t st);

size_t entry_workspace_bytes(int64_t n, int d);
cudaError_t launch_entry(const float* X, int64_t n, int d, int ld, int metric, int32_t* entry,
                         void* ws, size_t ws_bytes, cudaStream_t st);

cudaError_t launch_search(const float* X, int64_t n, int d, int ld, int metric,
                          const int32_t* gids, const int32_t* gdeg, int R, int entry,
                          const float* Q, int64_t nq, int ldq, int k, int beam, int32_t* ids_out,
                          float* dists_out, cudaStream_t st);

cudaError_t launch_brute_knn(const float* X, int64_t n, int d, int ld, int metric, const float* Q,
                             int64_t nq, int ldq, int k, int32_t* ids_out, float* dists_out,
                             cudaStream_t st);

int sm_count();

// Sets the thread-local message returned by grnnd_last_error.
void set_last_error(const std::string& msg);

// Per-kernel event profiler of the calling thread (no-ops unless enabled).
void prof_start(const char* name, cudaStream_t st);
void prof_stop(cudaStream_t st);

struct ProfScope {
  cudaStream_t st;
  ProfScope(const char* name, cudaStream_t s) : st(s) { prof_start(name, s); }
  ~ProfScope() { prof_stop(st); }
};

}  // namespace grnnd
