// Launch arguments shared by the translation units that hold the pool kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace grnnd {

// Work records of a round are sorted into size classes by pool size m: m <= 8, <= 16, <= 32
// (the warp join's lane groups), <= 64 (the two-warp team join, or the batched join for FP32
// rows longer than 128) and 65..R (the wide join; only allocated when R > 64).
constexpr int kNumClasses = 5;
constexpr int kTeamMaxM = 64;     // largest pool of classes 0..3 (one 64-bit prune mask)
constexpr int kMaxRWide = 256;    // largest pool capacity R of the library
constexpr int kRedChunk = 1024;   // redirect slots a join CTA reserves at a time, at most
constexpr int64_t kMaxJoinGrid = 2048;  // CTAs of one join kernel at most (sizes the redirect slack)

// A TMA tensor map: the driver's 128-byte, 64-byte aligned descriptor, passed to a kernel by
// value (as a __grid_constant__ parameter) and named to the copy by its address.
struct alignas(64) TmaMap {
  unsigned long long w[16];
};

struct PointsDev {
  const float* X;
  int ld;
  const void* Xb;  // quantized rows: bfloat16 (BF16 form) or e4m3 bytes (FP8 form)
  int ldb;
  const float2* aux;
  const unsigned* qflags;
  int d;
};

struct JoinArgs {
  // the quantized rows as a 2-D tensor (ldb columns x n rows; boxes of one 128-column chunk
  // plus the first 16 bytes after it, one row high) for the warp join's gather4 copies
  TmaMap rows_map;
  int rows_tma;  // 1: the warp join stages quantized rows by gather4 copies through rows_map
  PointsDev P;
  int64_t n;
  int R;
  const uint64_t* keys_in;
  const int32_t* deg_in;
  const int32_t* list_n;             // records per pool-size class
  const uint64_t* rec[kNumClasses];  // work records by class
  int rec_w[kNumClasses];            // words per record
  int rec_cap[kNumClasses];          // entries a record holds
  uint64_t seed;
  int t1, t2, order;
  uint64_t* keys_out;  // survivors (in place for the round, final graph for the last pass)
  int32_t* deg_out;
  int emit_redirects;
  int32_t* red_tgt;
  uint64_t* red_key;
  unsigned long long* red_n;
  int64_t red_cap;          // redirect slots in red_tgt / red_key
  int32_t* count;
  int64_t* stats;
  int32_t* err;
  unsigned int* work_q;      // [3] device work queues of the warp and team joins, one spare (zeroed per step)
  int warp_ctas, team_ctas;  // launch caps (host side only; 0: as many as fit)
};

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
  int32_t* err;            // nonzero: a wait of this round gave up, leave every pool as it is
  uint8_t* next_active;    // per target: its output row holds a new entry (prep's hint), or null
  int next_active_all;     // 1: write the flag of every target (a round: rows the merge leaves
                           // alone hold no new entry); 0: only of merged targets (a reverse step)
  // Copies of one id proposed to one target can differ in distance only when the recorded
  // distances are not canonical FP32 (quantized tiles outside their exact mode); then the
  // merge first gives each proposal the old bit its id has in the row.  old_pass 1: always;
  // 0: when qflags (the quantized rows' dataset flags, null for FP32 rows) show that the
  // tiles of d-dimensional rows are not exact.
  int old_pass;
  const unsigned* qflags;
  int d;
  // 1: every distance recorded in the pools came from this library's own canonical arithmetic
  // (a whole build), so copies of one id carry equal keys up to the old bit and duplicates
  // can be found by comparing keys; 0 (step calls on caller-supplied pools): by id
  int keys_canonical;
};

// The join of pools of 65..R entries (records of class 4), every precision form, and the
// merge of rounds and reverse steps when R > 64 (wide_kernels.cu).
cudaError_t launch_join_wide(const JoinArgs& a, int metric, cudaStream_t st, const char* name);
cudaError_t launch_select_wide(const SelectArgs& a, cudaStream_t st);

}  // namespace grnnd
