// Host driver and C ABI of the GRNND library (declarations in include/grnnd.h).
//
// grnnd_build_ex runs Alg 3 on one GPU: rnd_init, then T1 outer iterations of T2 rounds
// (rnd_join + rev_merge into the other pool buffer, then a pointer swap: Sec 3.5), with
// reverse-edge sampling (Sec 3.6) after every outer iteration but the last, then the
// optional final prune, the export to (ids, dists) rows and the search entry.
#include <algorithm>
#include <cstddef>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "grnnd.h"
#include "internal.h"

namespace {

thread_local std::string g_err;
// The calling thread's current stream (grnnd_set_stream); null = the legacy default stream.
thread_local cudaStream_t g_stream = nullptr;

// NVTX range over a host scope (shown by profilers that attach; no cost otherwise).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

// The status word of a step: 1 = a bounded device wait gave up; 2 = an index outside its buffer
// (only the checked build, -DGRNND_CHECKS=1, tests for it).
int status_fail(int32_t word) {
  if (word == 2) return fail(GRNND_ECUDA, "a device bounds check failed (checked build)");
  return fail(GRNND_ETIMEOUT, "a device-side wait reached its iteration limit");
}

#define GR_CU(call)                                                                         \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      cudaGetLastError();                                                                   \
      return fail(GRNND_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
    }                                                                                       \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// A pointer that kernels can dereference for p, or null: device memory as it is, pinned host
// memory through its mapped device address; *host tells which.  Pageable and managed memory
// give null (the copy engine moves those).
const void* kernel_ptr(const void* p, bool* host) {
  cudaPointerAttributes at;
  *host = false;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice) return p;
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    *host = true;
    return at.devicePointer;
  }
  return nullptr;
}

__global__ void host_copy_kernel(uint4* __restrict__ dst, const uint4* __restrict__ src, int64_t n16) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

int32_t round4(int32_t d) { return (d + 3) & ~3; }
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Layout of the quantized copy of n x d points (BF16 or FP8 form), shared by the builds and
// grnnd_quantize: rows of ldb elements of qelem bytes (each ending in its (norm^2, residual)
// tail), then the per-row terms once more as an array, then the two dataset flags; each
// region 256-byte aligned.
struct QLayout {
  int32_t ldb = 0;
  size_t qelem = 0, rows_b = 0, aux_b = 0, total = 0;
};
QLayout q_layout(int64_t n, int32_t d, int32_t precision) {
  QLayout q;
  if (precision != GRNND_BF16 && precision != GRNND_FP8) return q;
  // padded dimensions, then the row's 16-byte tail of (norm^2, residual)
  q.ldb = precision == GRNND_FP8 ? ((d + 31) & ~31) + grnnd::kRowTail8 : ((d + 15) & ~15) + grnnd::kRowTail16;
  q.qelem = precision == GRNND_FP8 ? 1 : 2;
  q.rows_b = al256((size_t)n * q.ldb * q.qelem);
  q.aux_b = al256((size_t)n * 8);
  q.total = q.rows_b + q.aux_b + 256;
  return q;
}
// The point set of a step call: FP32 rows, plus the quantized copy in a precision form.
int step_points(const float* points, int64_t n, int32_t d, int32_t ld, int32_t metric, int32_t precision,
                const void* qpoints, size_t qbytes, grnnd::PointsSet* P) {
  P->X = points;
  P->ld = ld;
  P->d = d;
  P->metric = metric;
  if (precision == GRNND_FP32) return GRNND_OK;
  if (precision != GRNND_BF16 && precision != GRNND_FP8) return fail(GRNND_EINVAL, "unknown precision");
  const QLayout q = q_layout(n, d, precision);
  if (!qpoints || ((uintptr_t)qpoints & 255u) != 0 || qbytes < q.total)
    return fail(GRNND_EINVAL, "quantized points: need a 256-byte aligned buffer of grnnd_quantized_size bytes");
  const char* b = static_cast<const char*>(qpoints);
  P->precision = precision;
  P->Xb = b;
  P->ldb = q.ldb;
  P->aux = reinterpret_cast<const float2*>(b + q.rows_b);
  P->qflags = reinterpret_cast<const unsigned*>(b + q.rows_b + q.aux_b);
  return GRNND_OK;
}

// Owned device allocation released on scope exit: cudaMalloc / cudaFree, or stream-ordered
// from a memory pool on the given stream.
struct DevMem {
  void* p = nullptr;
  cudaMemPool_t pool = nullptr;
  cudaStream_t st = nullptr;
  DevMem() = default;
  DevMem(const grnnd::AllocMode& am, cudaStream_t s) : pool(am.pool), st(s) {}
  ~DevMem() {
    if (p) {
      if (pool)
        cudaFreeAsync(p, st);
      else
        cudaFree(p);
    }
  }
  cudaError_t alloc(size_t bytes) {
    if (!bytes) bytes = 16;
    return pool ? cudaMallocFromPoolAsync(&p, bytes, pool, st) : cudaMalloc(&p, bytes);
  }
  void* release() {
    void* q = p;
    p = nullptr;
    return q;
  }
};

int check_step_points(const float* points, int64_t n, int32_t d, int32_t ld, int32_t metric) {
  if (!points) return fail(GRNND_EINVAL, "points is NULL");
  if (n < 1 || n > 0x7FFFFFFELL) return fail(GRNND_EINVAL, "n out of range");
  if (d < 1 || ld < d || (ld & 3) != 0) return fail(GRNND_EINVAL, "need d >= 1, ld >= d, ld % 4 == 0");
  if (((uintptr_t)points & 15u) != 0) return fail(GRNND_EINVAL, "points must be 16-byte aligned");
  if (metric != GRNND_L2SQ && metric != GRNND_IP) return fail(GRNND_EINVAL, "unknown metric");
  return GRNND_OK;
}

int check_R(int32_t R) {
  if (R < 2 || R > 256) return fail(GRNND_EINVAL, "R must be in [2, 256]");
  return GRNND_OK;
}

// ---- per-kernel event profiler (thread-local) ------------------------------------------
struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
};
struct Profiler {
  bool on = false;
  std::vector<std::string> only;  // kernel names to time (empty: every kernel)
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  const char* open_name = nullptr;
  cudaEvent_t open_ev = nullptr;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};
thread_local Profiler g_prof;

}  // namespace

namespace grnnd {
void set_last_error(const std::string& msg) { g_err = msg; }
bool prof_on() { return g_prof.on; }

void prof_start(const char* name, cudaStream_t st) {
  if (!g_prof.on) return;
  if (!g_prof.only.empty()) {
    bool hit = false;
    for (const auto& o : g_prof.only) hit = hit || o == name;
    if (!hit) return;  // not timed: no events around this launch
  }
  g_prof.open_name = name;
  g_prof.open_ev = g_prof.get();
  cudaEventRecord(g_prof.open_ev, st);
}
void prof_stop(cudaStream_t st) {
  if (!g_prof.on || !g_prof.open_ev) return;
  cudaEvent_t b = g_prof.get();
  cudaEventRecord(b, st);
  g_prof.recs.push_back({g_prof.open_name, g_prof.open_ev, b});
  g_prof.open_ev = nullptr;
}

cudaError_t copy_bytes(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (!bytes) return cudaSuccess;
  bool dh = false, sh = false;
  void* kd = const_cast<void*>(kernel_ptr(dst, &dh));
  const void* ks = kernel_ptr(src, &sh);
  const bool aligned = ((reinterpret_cast<uintptr_t>(kd) | reinterpret_cast<uintptr_t>(ks) | bytes) & 15u) == 0;
  if (!kd || !ks || !(dh || sh) || !aligned) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st);
  const int64_t n16 = (int64_t)(bytes / 16);
  const int64_t blocks = std::min<int64_t>((n16 + 255) / 256, (int64_t)sm_count() * 16);
  ProfScope ps("host_copy", st);
  host_copy_kernel<<<(unsigned)blocks, 256, 0, st>>>(static_cast<uint4*>(kd), static_cast<const uint4*>(ks), n16);
  return cudaGetLastError();
}
}  // namespace grnnd

extern "C" {

const char* grnnd_last_error(void) { return g_err.c_str(); }

void grnnd_set_stream(void* stream) { g_stream = (cudaStream_t)stream; }
void* grnnd_get_stream(void) { return (void*)g_stream; }

int grnnd_profile_begin(void) {
  for (auto& r : g_prof.recs) {
    g_prof.pool.push_back(r.a);
    g_prof.pool.push_back(r.b);
  }
  g_prof.recs.clear();
  g_prof.only.clear();
  g_prof.on = true;
  return GRNND_OK;
}

int grnnd_profile_begin_only(const char* names) {
  grnnd_profile_begin();
  if (names) {
    const std::string all(names);
    size_t a = 0;
    while (a <= all.size()) {
      size_t b = all.find(',', a);
      if (b == std::string::npos) b = all.size();
      if (b > a) g_prof.only.push_back(all.substr(a, b - a));
      a = b + 1;
    }
  }
  return GRNND_OK;
}

int grnnd_profile_end(grnnd_kernel_time* out, int32_t max_entries, int32_t* n_entries) {
  g_prof.on = false;
  std::vector<grnnd_kernel_time> acc;
  for (auto& r : g_prof.recs) {
    float ms = 0.0f;
    GR_CU(cudaEventSynchronize(r.b));
    GR_CU(cudaEventElapsedTime(&ms, r.a, r.b));
    size_t i = 0;
    while (i < acc.size() && std::strcmp(acc[i].name, r.name) != 0) ++i;
    if (i == acc.size()) {
      grnnd_kernel_time t;
      std::memset(&t, 0, sizeof(t));
      std::strncpy(t.name, r.name, sizeof(t.name) - 1);
      acc.push_back(t);
    }
    acc[i].launches += 1;
    acc[i].ms += ms;
  }
  for (auto& r : g_prof.recs) {
    g_prof.pool.push_back(r.a);
    g_prof.pool.push_back(r.b);
  }
  g_prof.recs.clear();
  if (n_entries) *n_entries = (int32_t)acc.size();
  if (out)
    for (int32_t i = 0; i < max_entries && i < (int32_t)acc.size(); ++i) out[i] = acc[i];
  return GRNND_OK;
}

void grnnd_params_default(grnnd_params* p) {
  if (!p) return;
  p->S = 16;
  p->R = 32;
  p->T1 = 4;
  p->T2 = 8;
  p->rho = 0.6f;
  p->seed = 0;
  p->metric = GRNND_L2SQ;
  p->precision = GRNND_FP32;
  p->order = GRNND_ORDER_RANDOM;
  p->final_prune = 1;
  p->stream = nullptr;
  p->hbm_budget = 0;
  p->tuning = nullptr;
}

size_t grnnd_workspace_size(int64_t n, int32_t R) {
  if (n < 1 || R < 1) return 0;
  return grnnd::workspace_bytes(n, R);
}

size_t grnnd_entry_workspace_size(int64_t n, int32_t d) {
  if (n < 1 || d < 1) return 0;
  return grnnd::entry_workspace_bytes(n, d);
}

int grnnd_pool_init(const float* points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                    int32_t S, int32_t R, uint64_t seed, uint64_t* keys, int32_t* deg,
                    void* stream) {
  int rc = check_step_points(points, n, d, ld, metric);
  if (rc) return rc;
  if ((rc = check_R(R))) return rc;
  if (n < 2 || S < 1 || S > R || (int64_t)S > n - 1)
    return fail(GRNND_EINVAL, "need n >= 2 and 1 <= S <= min(R, n-1)");
  if (!keys || !deg) return fail(GRNND_EINVAL, "keys/deg is NULL");
  GR_CU(grnnd::launch_pool_init(points, n, d, ld, metric, S, R, seed, keys, deg,
                                (cudaStream_t)stream));
  return GRNND_OK;
}

int grnnd_join_round_q(const float* points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                       int32_t precision, const void* qpoints, size_t qpoints_bytes, int32_t R,
                       const uint64_t* keys_in, const int32_t* deg_in, uint64_t seed, int32_t t1,
                       int32_t t2, int32_t order, uint64_t* keys_out, int32_t* deg_out, void* workspace,
                       size_t workspace_bytes, int64_t* stats, void* stream) {
  int rc = check_step_points(points, n, d, ld, metric);
  if (rc) return rc;
  if ((rc = check_R(R))) return rc;
  if (!keys_in || !deg_in || !keys_out || !deg_out) return fail(GRNND_EINVAL, "pool buffer is NULL");
  if ((keys_in == keys_out) != (deg_in == deg_out))
    return fail(GRNND_EINVAL, "keys and degrees must both be in place or both separate");
  if (order < 0 || order > 2) return fail(GRNND_EINVAL, "unknown order");
  grnnd::PointsSet P;
  if ((rc = step_points(points, n, d, ld, metric, precision, qpoints, qpoints_bytes, &P))) return rc;
  grnnd::Workspace ws;
  if (!grnnd::carve_workspace(workspace, workspace_bytes, n, R, &ws))
    return fail(GRNND_EINVAL, "workspace too small or not 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  GR_CU(grnnd::launch_round(P, n, R, keys_in, deg_in, seed, t1, t2, order, ws, keys_out, deg_out,
                            stats, st));
  if (stats) GR_CU(cudaMemcpyAsync(stats + 5, ws.round_new, 8, cudaMemcpyDeviceToDevice, st));
  return GRNND_OK;
}

int grnnd_join_round(const float* points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                     int32_t R, const uint64_t* keys_in, const int32_t* deg_in, uint64_t seed,
                     int32_t t1, int32_t t2, int32_t order, uint64_t* keys_out, int32_t* deg_out,
                     void* workspace, size_t workspace_bytes, int64_t* stats, void* stream) {
  return grnnd_join_round_q(points, n, d, ld, metric, GRNND_FP32, nullptr, 0, R, keys_in, deg_in, seed, t1,
                            t2, order, keys_out, deg_out, workspace, workspace_bytes, stats, stream);
}

size_t grnnd_quantized_size(int64_t n, int32_t d, int32_t precision) {
  if (n < 1 || d < 1) return 0;
  return q_layout(n, d, precision).total;
}

int grnnd_quantize(const float* points, int64_t n, int32_t d, int32_t ld, int32_t precision, void* qpoints,
                   size_t qpoints_bytes, void* stream) {
  int rc = check_step_points(points, n, d, ld, GRNND_L2SQ);
  if (rc) return rc;
  if (precision != GRNND_BF16 && precision != GRNND_FP8)
    return fail(GRNND_EINVAL, "precision must be GRNND_BF16 or GRNND_FP8");
  grnnd::PointsSet P;
  if ((rc = step_points(points, n, d, ld, GRNND_L2SQ, precision, qpoints, qpoints_bytes, &P))) return rc;
  GR_CU(grnnd::launch_quantize(points, n, d, ld, const_cast<void*>(P.Xb), P.ldb, const_cast<float2*>(P.aux),
                               const_cast<unsigned*>(P.qflags), precision, (cudaStream_t)stream));
  return GRNND_OK;
}

int grnnd_selftest_bounded_wait(uint32_t limit, void* stream) {
  if (limit < 1 || limit > (1u << 20)) return fail(GRNND_EINVAL, "limit must be in [1, 2^20]");
  int32_t status = -1;
  GR_CU(grnnd::launch_wait_selftest(limit, &status, (cudaStream_t)stream));
  if (status == 0) return GRNND_OK;
  if (status == 1) return fail(GRNND_ETIMEOUT, "the self-test wait gave up after its iteration limit");
  return fail(GRNND_ECUDA, "the self-test kernel did not report");
}

int grnnd_workspace_status(const void* workspace, size_t workspace_bytes, int64_t n, int32_t R,
                           void* stream) {
  if (n < 1 || n > 0x7FFFFFFELL) return fail(GRNND_EINVAL, "n out of range");
  int rc = check_R(R);
  if (rc) return rc;
  grnnd::Workspace ws;
  if (!grnnd::carve_workspace(const_cast<void*>(workspace), workspace_bytes, n, R, &ws))
    return fail(GRNND_EINVAL, "workspace too small or not 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  int32_t h = 0;
  GR_CU(cudaMemcpyAsync(&h, ws.err, 4, cudaMemcpyDeviceToHost, st));
  GR_CU(cudaStreamSynchronize(st));
  if (h) return status_fail(h);
  return GRNND_OK;
}

int grnnd_reverse_sample(int64_t n, int32_t R, float rho, const uint64_t* keys_in,
                         const int32_t* deg_in, uint64_t* keys_out, int32_t* deg_out,
                         void* workspace, size_t workspace_bytes, int64_t* stats, void* stream) {
  int rc = check_R(R);
  if (rc) return rc;
  if (n < 1) return fail(GRNND_EINVAL, "n out of range");
  if (!(rho >= 0.0f && rho <= 1.0f)) return fail(GRNND_EINVAL, "rho must be in [0, 1]");
  if (!keys_in || !deg_in || !keys_out || !deg_out) return fail(GRNND_EINVAL, "pool buffer is NULL");
  if ((keys_in == keys_out) != (deg_in == deg_out))
    return fail(GRNND_EINVAL, "keys and degrees must both be in place or both separate");
  grnnd::Workspace ws;
  if (!grnnd::carve_workspace(workspace, workspace_bytes, n, R, &ws))
    return fail(GRNND_EINVAL, "workspace too small or not 256-byte aligned");
  GR_CU(grnnd::launch_reverse(n, R, rho, keys_in, deg_in, ws, keys_out, deg_out, stats,
                              (cudaStream_t)stream));
  return GRNND_OK;
}

int grnnd_final_prune_q(const float* points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                        int32_t precision, const void* qpoints, size_t qpoints_bytes, int32_t R,
                        const uint64_t* keys_in, const int32_t* deg_in, uint64_t seed, int32_t t1,
                        int32_t order, uint64_t* keys_out, int32_t* deg_out, void* workspace,
                        size_t workspace_bytes, void* stream) {
  int rc = check_step_points(points, n, d, ld, metric);
  if (rc) return rc;
  if ((rc = check_R(R))) return rc;
  if (!keys_in || !deg_in || !keys_out || !deg_out) return fail(GRNND_EINVAL, "pool buffer is NULL");
  if (keys_in == keys_out || deg_in == deg_out)
    return fail(GRNND_EINVAL, "output pool must not alias the input pool");
  if (order < 0 || order > 2) return fail(GRNND_EINVAL, "unknown order");
  grnnd::PointsSet P;
  if ((rc = step_points(points, n, d, ld, metric, precision, qpoints, qpoints_bytes, &P))) return rc;
  grnnd::Workspace ws;
  if (!grnnd::carve_workspace(workspace, workspace_bytes, n, R, &ws))
    return fail(GRNND_EINVAL, "workspace too small or not 256-byte aligned");
  GR_CU(grnnd::launch_final(P, n, R, keys_in, deg_in, seed, t1, order, ws, keys_out, deg_out,
                            (cudaStream_t)stream));
  return GRNND_OK;
}

int grnnd_final_prune(const float* points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                      int32_t R, const uint64_t* keys_in, const int32_t* deg_in, uint64_t seed,
                      int32_t t1, int32_t order, uint64_t* keys_out, int32_t* deg_out,
                      void* workspace, size_t workspace_bytes, void* stream) {
  return grnnd_final_prune_q(points, n, d, ld, metric, GRNND_FP32, nullptr, 0, R, keys_in, deg_in, seed, t1,
                             order, keys_out, deg_out, workspace, workspace_bytes, stream);
}

int grnnd_pair_dist(const float* points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                    const int32_t* pairs, int64_t np, float* out, void* stream) {
  int rc = check_step_points(points, n, d, ld, metric);
  if (rc) return rc;
  if (np < 0 || (np > 0 && (!pairs || !out))) return fail(GRNND_EINVAL, "bad pair list");
  GR_CU(grnnd::launch_pair_dist(points, d, ld, metric, pairs, np, out, (cudaStream_t)stream));
  return GRNND_OK;
}

int grnnd_entry_point(const float* points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                      int32_t* entry_out, void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_step_points(points, n, d, ld, metric);
  if (rc) return rc;
  if (!entry_out || !workspace || workspace_bytes < grnnd::entry_workspace_bytes(n, d))
    return fail(GRNND_EINVAL, "entry_out/workspace missing or too small");
  GR_CU(grnnd::launch_entry(points, n, d, ld, metric, entry_out, workspace, workspace_bytes,
                            (cudaStream_t)stream));
  return GRNND_OK;
}

int grnnd_search_graph(const float* points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                       const int32_t* gids, const int32_t* gdeg, int32_t R, int32_t entry,
                       const float* queries, int64_t nq, int32_t ldq, int32_t k, int32_t beam,
                       int32_t* ids_out, float* dists_out, void* stream) {
  int rc = check_step_points(points, n, d, ld, metric);
  if (rc) return rc;
  if (!gids || !gdeg || R < 1 || entry < 0 || entry >= n) return fail(GRNND_EINVAL, "bad graph");
  if (nq < 0 || (nq > 0 && (!queries || !ids_out)) || ldq < d)
    return fail(GRNND_EINVAL, "bad queries/ids_out");
  if (k < 1 || beam < k || beam > 256) return fail(GRNND_EINVAL, "need 1 <= k <= beam <= 256");
  if (d > 1024) return fail(GRNND_EINVAL, "search supports d <= 1024");
  GR_CU(grnnd::launch_search(points, n, d, ld, metric, gids, gdeg, R, entry, queries, nq, ldq, k,
                             beam, ids_out, dists_out, (cudaStream_t)stream));
  return GRNND_OK;
}

int grnnd_brute_knn(const float* points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                    const float* queries, int64_t nq, int32_t ldq, int32_t k, int32_t* ids_out,
                    float* dists_out, void* stream) {
  int rc = check_step_points(points, n, d, ld, metric);
  if (rc) return rc;
  if (nq < 0 || (nq > 0 && (!queries || !ids_out)) || ldq < d)
    return fail(GRNND_EINVAL, "bad queries/ids_out");
  if (k < 1 || k > 32 || k > n) return fail(GRNND_EINVAL, "need 1 <= k <= min(32, n)");
  GR_CU(grnnd::launch_brute_knn(points, n, d, ld, metric, queries, nq, ldq, k, ids_out, dists_out,
                                (cudaStream_t)stream));
  return GRNND_OK;
}

int grnnd_keys_to_graph(int64_t n, int32_t R, const uint64_t* keys, int32_t* ids, float* dists,
                        void* stream) {
  if (n < 1 || R < 1 || !keys) return fail(GRNND_EINVAL, "bad arguments");
  GR_CU(grnnd::launch_keys_to_graph(n, R, keys, ids, dists, nullptr, (cudaStream_t)stream));
  return GRNND_OK;
}

// ---------------------------------------------------------------------------------------
// Whole build
// ---------------------------------------------------------------------------------------

namespace {
// The memory cache of grnnd_set_memory_cache: one stream-ordered pool per device, keeping up
// to the set number of freed bytes for the next build instead of returning them.
constexpr int kMaxDevices = 64;
std::mutex g_cache_mu;
cudaMemPool_t g_cache_pool[kMaxDevices] = {};
uint64_t g_cache_bytes[kMaxDevices] = {};

grnnd::AllocMode cache_alloc_mode() {
  grnnd::AllocMode am;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return am;
  }
  std::lock_guard<std::mutex> lk(g_cache_mu);
  if (g_cache_bytes[dev] && g_cache_pool[dev]) {
    am.pool = g_cache_pool[dev];
    am.free_stream = nullptr;
    am.sync_before_free = true;
  }
  return am;
}
}  // namespace

int grnnd_set_memory_cache(uint64_t bytes) {
  int dev = 0;
  GR_CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(GRNND_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lk(g_cache_mu);
  if (!g_cache_pool[dev]) {
    if (!bytes) return GRNND_OK;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    GR_CU(cudaMemPoolCreate(&g_cache_pool[dev], &props));
  }
  uint64_t keep = bytes;
  GR_CU(cudaMemPoolSetAttribute(g_cache_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep));
  g_cache_bytes[dev] = bytes;
  if (!bytes) {  // off: return what the pool still keeps (graphs alive keep their memory)
    GR_CU(cudaDeviceSynchronize());
    GR_CU(cudaMemPoolTrimTo(g_cache_pool[dev], 0));
  }
  return GRNND_OK;
}

namespace {
// Pinned host slots for the per-round probe of the build driver (one pair per host thread;
// released at thread exit).
// A round's status word and new-entry counter as they lie in the workspace (the counter 256
// bytes after the status word), read back with one copy.
struct RoundProbe {
  int32_t err;
  unsigned char pad[252];
  int64_t fresh;
};
static_assert(offsetof(RoundProbe, fresh) == 256, "round probe layout");
struct ProbeHolder {
  RoundProbe* p = nullptr;
  ~ProbeHolder() {
    if (p) cudaFreeHost(p);
  }
};
RoundProbe* round_probe() {
  thread_local ProbeHolder h;
  if (!h.p) {
    void* q = nullptr;
    if (cudaHostAlloc(&q, 2 * sizeof(RoundProbe), cudaHostAllocPortable) != cudaSuccess) return nullptr;
    h.p = static_cast<RoundProbe*>(q);
  }
  return h.p;
}
}  // namespace

namespace {

int check_params(const grnnd_params* p) {
  if (!p) return fail(GRNND_EINVAL, "params is NULL");
  int rc = check_R(p->R);
  if (rc) return rc;
  if (p->S < 1 || p->S > p->R) return fail(GRNND_EINVAL, "need 1 <= S <= R");
  if (p->T1 < 1 || p->T2 < 1) return fail(GRNND_EINVAL, "T1 and T2 must be >= 1");
  if (!(p->rho >= 0.0f && p->rho <= 1.0f)) return fail(GRNND_EINVAL, "rho must be in [0, 1]");
  if (p->metric != GRNND_L2SQ && p->metric != GRNND_IP) return fail(GRNND_EINVAL, "unknown metric");
  if (p->order < 0 || p->order > 2) return fail(GRNND_EINVAL, "unknown order");
  if (p->precision != GRNND_FP32 && p->precision != GRNND_BF16 && p->precision != GRNND_FP8)
    return fail(GRNND_EINVAL, "unknown precision");
  if (const grnnd_tuning* t = p->tuning) {
    for (int c = 0; c < 3; ++c)
      if (t->group_max[c] < 0 || t->group_max[c] > (8 << c))
        return fail(GRNND_EINVAL, "tuning: need 0 <= group_max[c] <= 8 << c");
    if (t->warp_ctas_per_sm < 0 || t->team_ctas_per_sm < 0)
      return fail(GRNND_EINVAL, "tuning: CTAs per SM must be >= 0");
    if (t->row_copies < 0 || t->row_copies > 2) return fail(GRNND_EINVAL, "tuning: row_copies must be 0, 1 or 2");
  }
  return GRNND_OK;
}

// Device bytes of one build call: what stays with the graphs (points + graph) and the
// scratch released at the end (pools, round workspace, quantized rows, segments).
struct BuildSizes {
  size_t pts_b, q_b, pool_b, deg_b, ws_b, ent_b, graph_b, stats_b, seg_b, scratch_b;
};
BuildSizes build_sizes(int64_t n, int32_t d, const grnnd_params* p, bool batched, int32_t nbuild) {
  BuildSizes z;
  const int32_t R = p->R, ld = round4(d);
  // quantized forms: a BF16 copy (rows of d rounded up to 16 elements) or an e4m3 copy
  // (rows of d rounded up to 32 bytes), per-row terms and dataset flags
  z.pts_b = al256((size_t)n * ld * 4);
  z.q_b = q_layout(n, d, p->precision).total;
  z.pool_b = al256((size_t)n * R * 8);
  z.deg_b = al256((size_t)n * 4);
  z.ws_b = grnnd::workspace_bytes(n, R);
  z.ent_b = batched ? grnnd::entry_batch_workspace_bytes(nbuild, d) : grnnd::entry_workspace_bytes(n, d);
  z.graph_b = al256((size_t)n * R * 4) * 2 + z.deg_b;
  z.stats_b = 256 + al256((size_t)nbuild * 4);  // counters, then one entry per build
  z.seg_b = batched ? al256((size_t)n * 8) + al256(((size_t)nbuild + 1) * 8) : 0;
  z.scratch_b = 2 * z.pool_b + 2 * z.deg_b + std::max(z.ws_b, z.ent_b) + z.stats_b + z.q_b + z.seg_b;
  return z;
}

// One build call over n points: a single build (offsets == nullptr) or nbuild independent
// builds of the rows [offsets[b], offsets[b+1]) (ids local to each build, one graph each).
// A batched call records the whole pass in one CUDA graph and launches it once.
int build_core(const float* points, int64_t n, int32_t d, const grnnd_params* p, const int64_t* offsets,
               int32_t nbuild, grnnd_graph** graphs_out, const grnnd::AllocMode& am = grnnd::AllocMode()) {
  const bool batched = offsets != nullptr;
  NvtxRange nvtx_build(batched ? "grnnd_build_batch" : "grnnd_build");
  const int32_t R = p->R, ld = round4(d);
  const bool quant = p->precision != GRNND_FP32;
  cudaStream_t st = (cudaStream_t)p->stream;

  const BuildSizes z = build_sizes(n, d, p, batched, nbuild);
  const size_t pts_b = z.pts_b, q_b = z.q_b, pool_b = z.pool_b, deg_b = z.deg_b, ws_b = z.ws_b,
               ent_b = z.ent_b, graph_b = z.graph_b, stats_b = z.stats_b, scratch_b = z.scratch_b;
  if (p->hbm_budget && pts_b + graph_b + scratch_b > p->hbm_budget)
    return fail(GRNND_ENOMEM, "build needs " + std::to_string(pts_b + graph_b + scratch_b) +
                                  " bytes, above hbm_budget " + std::to_string(p->hbm_budget));

  auto block = std::make_shared<GraphBlock>();
  DevMem mscratch(am, st);
  if (am.pool) {
    block->pooled = true;
    block->sync_before_free = am.sync_before_free;
    block->free_stream = am.free_stream;
    GR_CU(cudaMallocFromPoolAsync(&block->points, pts_b, am.pool, st));
    GR_CU(cudaMallocFromPoolAsync(&block->graph, graph_b, am.pool, st));
  } else {
    GR_CU(cudaMalloc(&block->points, pts_b));
    GR_CU(cudaMalloc(&block->graph, graph_b));
  }
  GR_CU(mscratch.alloc(scratch_b));
  float* X = static_cast<float*>(block->points);
  char* gp = static_cast<char*>(block->graph);
  int32_t* gids = reinterpret_cast<int32_t*>(gp);
  float* gd = reinterpret_cast<float*>(gp + al256((size_t)n * R * 4));
  int32_t* gdeg = reinterpret_cast<int32_t*>(gp + 2 * al256((size_t)n * R * 4));
  char* sp = static_cast<char*>(mscratch.p);
  uint64_t* poolA = reinterpret_cast<uint64_t*>(sp);
  uint64_t* poolB = reinterpret_cast<uint64_t*>(sp + pool_b);
  int32_t* degA = reinterpret_cast<int32_t*>(sp + 2 * pool_b);
  int32_t* degB = reinterpret_cast<int32_t*>(sp + 2 * pool_b + deg_b);
  int64_t* stats = reinterpret_cast<int64_t*>(sp + 2 * pool_b + 2 * deg_b);
  int32_t* d_entry = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(stats) + 256);
  void* wsp = sp + 2 * pool_b + 2 * deg_b + stats_b;
  const size_t wsp_b = std::max(ws_b, ent_b);
  char* qp = sp + 2 * pool_b + 2 * deg_b + stats_b + al256(wsp_b);
  int2* vseg = batched ? reinterpret_cast<int2*>(qp + q_b) : nullptr;
  int64_t* off_dev = batched ? reinterpret_cast<int64_t*>(qp + q_b + al256((size_t)n * 8)) : nullptr;

  // points -> padded device rows; the segment of every vertex
  const cudaMemcpyKind kind = is_device_ptr(points) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (ld != d) GR_CU(cudaMemsetAsync(X, 0, (size_t)n * ld * 4, st));
  GR_CU(grnnd::copy_rows(X, ld, points, d, n, kind, st));
  GR_CU(cudaMemsetAsync(stats, 0, 256, st));
  std::vector<int2> hseg;
  if (batched) {
    hseg.resize((size_t)n);
    for (int32_t b = 0; b < nbuild; ++b)
      for (int64_t v = offsets[b]; v < offsets[b + 1]; ++v)
        hseg[(size_t)v] = make_int2((int)offsets[b], (int)(offsets[b + 1] - offsets[b]));
    GR_CU(cudaMemcpyAsync(vseg, hseg.data(), (size_t)n * 8, cudaMemcpyHostToDevice, st));
    GR_CU(cudaMemcpyAsync(off_dev, offsets, ((size_t)nbuild + 1) * 8, cudaMemcpyHostToDevice, st));
  }
  grnnd::Workspace ws;
  if (!grnnd::carve_workspace(wsp, wsp_b, n, R, &ws)) return fail(GRNND_EINVAL, "internal workspace");
  GR_CU(cudaMemsetAsync(ws.err, 0, 4, st));
  GR_CU(grnnd::launch_check_finite(X, n, d, ld, ws.err, st));
  int32_t h_flag = 0;
  GR_CU(cudaMemcpyAsync(&h_flag, ws.err, 4, cudaMemcpyDeviceToHost, st));
  GR_CU(cudaStreamSynchronize(st));
  if (h_flag) return fail(GRNND_EINVAL, "points contain a non-finite value");

  grnnd::PointsSet P;
  P.X = X;
  P.ld = ld;
  P.d = d;
  P.metric = p->metric;
  P.vseg = vseg;
  if (const grnnd_tuning* t = p->tuning) {
    for (int c = 0; c < 3; ++c) P.group_max[c] = t->group_max[c];
    P.warp_ctas = t->warp_ctas_per_sm;
    P.team_ctas = t->team_ctas_per_sm;
    P.row_copies = t->row_copies;
  }
  if (quant && step_points(X, n, d, ld, p->metric, p->precision, qp, q_b, &P) != GRNND_OK)
    return fail(GRNND_EINVAL, "internal quantized layout");

  // A batched pass runs every round (a round after one that left no new entry is an
  // identity) and is recorded as one CUDA graph; a single build reads each round's
  // new-entry count one round late from pinned memory and stops after the first identity.
  const bool capture = batched && !grnnd::prof_on();
  GR_CU(grnnd::prepare_join_kernels(P));  // kernel set-up stays outside the capture
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cst = nullptr;  // the capture runs on a private stream (the caller's may be
                               // the legacy default stream, which cannot be captured)
  struct GraphGuard {
    cudaGraph_t* g;
    cudaGraphExec_t* x;
    cudaStream_t* s;
    ~GraphGuard() {
      if (*x) cudaGraphExecDestroy(*x);
      if (*g) cudaGraphDestroy(*g);
      if (*s) cudaStreamDestroy(*s);
    }
  } graph_guard{&graph, &gexec, &cst};
  const cudaStream_t user_st = st;
  if (capture) {
    GR_CU(cudaStreamCreateWithFlags(&cst, cudaStreamNonBlocking));
    st = cst;
    GR_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  }
  auto end_capture = [&]() {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(st, &g);
    if (g) cudaGraphDestroy(g);
  };
#define GR_CAP(call)                                                                           \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      if (capture) end_capture();                                                              \
      cudaGetLastError();                                                                      \
      return fail(GRNND_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));           \
    }                                                                                          \
  } while (0)

  if (quant)
    GR_CAP(grnnd::launch_quantize(X, n, d, ld, qp, P.ldb, const_cast<float2*>(P.aux),
                                  const_cast<unsigned*>(P.qflags), p->precision, st));
  if (p->precision == GRNND_BF16)  // the drawn rows from the BF16 copy when it is exact
    GR_CAP(grnnd::launch_pool_init(X, n, d, ld, p->metric, p->S, R, p->seed, poolA, degA, st, vseg, P.Xb, P.ldb,
                                   P.qflags));
  else
    GR_CAP(grnnd::launch_pool_init(X, n, d, ld, p->metric, p->S, R, p->seed, poolA, degA, st, vseg));
  RoundProbe* probe = nullptr;
  cudaEvent_t rev[2] = {nullptr, nullptr};
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() {
      for (int i = 0; i < 2; ++i)
        if (e[i]) cudaEventDestroy(e[i]);
    }
  } ev_guard{rev};
  if (!capture) {
    probe = round_probe();
    if (!probe) return fail(GRNND_ENOMEM, "pinned host memory for the round probe");
    for (int e = 0; e < 2; ++e) GR_CU(cudaEventCreateWithFlags(&rev[e], cudaEventDisableTiming));
  }
  int64_t rounds = 0;
  for (int32_t t1 = 1; t1 <= p->T1; ++t1) {
    int prev = -1;
    for (int32_t t2 = 1; t2 <= p->T2; ++t2) {
      // the round updates the pool in place: survivors are rewritten in their own row and
      // only rows that receive proposals are merged (the role of Sec 3.5's second buffer)
      {
        NvtxRange nvtx_round("round");
        GR_CAP(grnnd::launch_round(P, n, R, poolA, degA, p->seed, t1, t2, p->order, ws, poolA, degA,
                                   stats, st, rounds > 0, /*keys_canonical=*/true));
      }
      const int cur = (int)(rounds & 1);
      ++rounds;
      if (capture) continue;
      if (reinterpret_cast<char*>(ws.round_new) == reinterpret_cast<char*>(ws.err) + 256) {
        GR_CU(cudaMemcpyAsync(&probe[cur], ws.err, sizeof(RoundProbe), cudaMemcpyDeviceToHost, st));
      } else {
        GR_CU(cudaMemcpyAsync(&probe[cur].fresh, ws.round_new, 8, cudaMemcpyDeviceToHost, st));
        GR_CU(cudaMemcpyAsync(&probe[cur].err, ws.err, 4, cudaMemcpyDeviceToHost, st));
      }
      GR_CU(cudaEventRecord(rev[cur], st));
      if (prev >= 0) {  // the previous round's outcome, read while this one runs
        GR_CU(cudaEventSynchronize(rev[prev]));
        if (probe[prev].err) return status_fail(probe[prev].err);
        if (probe[prev].fresh == 0) break;  // no new entry anywhere: the rest are identities
      }
      prev = cur;
    }
    if (t1 != p->T1) {
      NvtxRange nvtx_rev("reverse_sample");
      GR_CAP(grnnd::launch_reverse(n, R, p->rho, poolA, degA, ws, poolA, degA, nullptr, st));
    }
  }
  uint64_t* gkeys = poolA;
  int32_t* gdg = degA;
  if (p->final_prune) {
    GR_CAP(grnnd::launch_final(P, n, R, poolA, degA, p->seed, p->T1 + 1, p->order, ws, poolB, degB, st, true));
    gkeys = poolB;
    gdg = degB;
  }
  GR_CAP(grnnd::launch_keys_to_graph(n, R, gkeys, gids, gd, nullptr, st));
  if (batched) GR_CAP(grnnd::launch_localize_ids(n, R, gids, vseg, st));
  GR_CAP(cudaMemcpyAsync(gdeg, gdg, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
  // the entry workspace reuses the (now idle) round workspace; the round status word
  // moves to the stats block first
  GR_CAP(cudaMemcpyAsync(stats + 8, ws.err, 4, cudaMemcpyDeviceToDevice, st));
  if (batched)
    GR_CAP(grnnd::launch_entry_batch(X, d, ld, p->metric, off_dev, nbuild, d_entry, wsp, wsp_b, st));
  else
    GR_CAP(grnnd::launch_entry(X, n, d, ld, p->metric, d_entry, wsp, wsp_b, st));
#undef GR_CAP
  if (capture) {
    GR_CU(cudaStreamEndCapture(st, &graph));
    st = user_st;
    GR_CU(cudaGraphInstantiate(&gexec, graph, 0));
    GR_CU(cudaGraphLaunch(gexec, st));
  }
  std::vector<int32_t> h_entry((size_t)nbuild);
  int64_t h_stats[9];
  GR_CU(cudaMemcpyAsync(h_entry.data(), d_entry, (size_t)nbuild * 4, cudaMemcpyDeviceToHost, st));
  GR_CU(cudaMemcpyAsync(h_stats, stats, 72, cudaMemcpyDeviceToHost, st));
  GR_CU(cudaStreamSynchronize(st));
  if ((int32_t)h_stats[8]) return status_fail((int32_t)h_stats[8]);

  for (int32_t b = 0; b < nbuild; ++b) {
    const int64_t lo = batched ? offsets[b] : 0, nb = batched ? offsets[b + 1] - offsets[b] : n;
    grnnd_graph* g = new grnnd_graph();
    g->n = nb;
    g->d = d;
    g->ld = ld;
    g->R = R;
    g->metric = p->metric;
    g->entry = h_entry[(size_t)b];
    g->points = X + lo * ld;
    g->ids = gids + lo * R;
    g->dists = gd + lo * R;
    g->deg = gdeg + lo;
    g->stats[0] = rounds;  // a batched call reports the counters of the whole pass
    g->stats[1] = h_stats[0];
    g->stats[2] = h_stats[1];
    g->stats[3] = h_stats[2];
    g->stats[4] = h_stats[3];
    g->stats[5] = h_stats[4];
    g->stats[6] = h_stats[6];
    g->stats[7] = h_stats[7];
    g->mem = block;
    graphs_out[b] = g;
  }
  return GRNND_OK;
}

}  // namespace

int grnnd_build_ex(const float* points, int64_t n, int32_t d, const grnnd_params* p,
                   grnnd_graph** graph_out) {
  if (p && !p->stream && g_stream) {  // no stream given: the thread's current stream
    grnnd_params q = *p;
    q.stream = (void*)g_stream;
    return grnnd::build_with(points, n, d, &q, cache_alloc_mode(), graph_out);
  }
  return grnnd::build_with(points, n, d, p, cache_alloc_mode(), graph_out);
}

int grnnd_build_batch(const float* points, const int64_t* offsets, int32_t nbuild, int32_t d,
                      const grnnd_params* p, grnnd_graph** graphs_out) {
  if (!graphs_out) return fail(GRNND_EINVAL, "graphs_out is NULL");
  if (nbuild < 1) return fail(GRNND_EINVAL, "need nbuild >= 1");
  for (int32_t b = 0; b < nbuild; ++b) graphs_out[b] = nullptr;
  int rc = check_params(p);
  if (rc) return rc;
  if (!points || !offsets) return fail(GRNND_EINVAL, "points/offsets is NULL");
  if (d < 1) return fail(GRNND_EINVAL, "d must be >= 1");
  if (offsets[0] != 0) return fail(GRNND_EINVAL, "offsets[0] must be 0");
  for (int32_t b = 0; b < nbuild; ++b) {
    const int64_t nb = offsets[b + 1] - offsets[b];
    if (nb < 2) return fail(GRNND_EINVAL, "every build needs >= 2 points");
    if ((int64_t)p->S > nb - 1) return fail(GRNND_EINVAL, "need S <= (points of every build) - 1");
  }
  if (offsets[nbuild] > 0x7FFFFFFELL) return fail(GRNND_EINVAL, "total points must be <= 2^31 - 2");
  grnnd_params q = *p;
  if (!q.stream) q.stream = (void*)g_stream;  // no stream given: the thread's current stream
  return build_core(points, offsets[nbuild], d, &q, offsets, nbuild, graphs_out, cache_alloc_mode());
}

int grnnd_autotune(const float* points, int64_t n, int32_t d, const int64_t* offsets, int32_t nbuild,
                   const grnnd_params* p, grnnd_tuning* best) {
  if (!best) return fail(GRNND_EINVAL, "best is NULL");
  int rc = check_params(p);
  if (rc) return rc;
  if (offsets && (nbuild < 1 || offsets[nbuild] != n)) return fail(GRNND_EINVAL, "offsets must end at n");
  grnnd_params q = *p;
  std::vector<grnnd_graph*> gs(offsets ? (size_t)nbuild : 1, nullptr);
  // one candidate: a build to settle allocations, then the best of two timed builds
  auto trial = [&](const grnnd_tuning& t, float* ms) -> int {
    q.tuning = &t;
    float m = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      const auto t0 = std::chrono::steady_clock::now();
      const int r = offsets ? grnnd_build_batch(points, offsets, nbuild, d, &q, gs.data())
                            : grnnd_build_ex(points, n, d, &q, gs.data());
      const auto t1 = std::chrono::steady_clock::now();
      if (r != GRNND_OK) return r;
      for (auto*& g : gs) {
        grnnd_free(g);
        g = nullptr;
      }
      if (rep > 0) m = std::min(m, std::chrono::duration<float, std::milli>(t1 - t0).count());
    }
    *ms = m;
    return GRNND_OK;
  };
  grnnd_tuning cur{{8, 16, 32}, 0, 0, 0, 0.0f};
  float cur_ms = 0.0f;
  if ((rc = trial(cur, &cur_ms))) return rc;
  const int32_t routes[4][3] = {{0, 16, 32}, {0, 0, 32}, {8, 16, 16}, {0, 16, 16}};
  grnnd_tuning base = cur;
  for (const auto& r : routes) {
    grnnd_tuning t = base;
    for (int c = 0; c < 3; ++c) t.group_max[c] = r[c];
    float ms;
    if ((rc = trial(t, &ms))) return rc;
    if (ms < cur_ms) cur = t, cur_ms = ms;
  }
  base = cur;
  for (int w = 1; w <= 3; ++w) {
    grnnd_tuning t = base;
    t.warp_ctas_per_sm = w;
    float ms;
    if ((rc = trial(t, &ms))) return rc;
    if (ms < cur_ms) cur = t, cur_ms = ms;
  }
  base = cur;
  for (int w = 2; w <= 6; w += 2) {
    grnnd_tuning t = base;
    t.team_ctas_per_sm = w;
    float ms;
    if ((rc = trial(t, &ms))) return rc;
    if (ms < cur_ms) cur = t, cur_ms = ms;
  }
  if (p->precision != GRNND_FP32) {  // quantized rows: one bulk copy per row, or gather4 copies
    base = cur;
    for (int r = 1; r <= 2; ++r) {
      grnnd_tuning t = base;
      t.row_copies = r;
      float ms;
      if ((rc = trial(t, &ms))) return rc;
      if (ms < cur_ms) cur = t, cur_ms = ms;
    }
  }
  cur.ms = cur_ms;
  *best = cur;
  return GRNND_OK;
}

int grnnd_autotune_pool(const float* points, int64_t n, int32_t d, int64_t nq, const grnnd_params* p,
                        const int32_t* R_candidates, int32_t ncand, float recall_target, int32_t k,
                        int32_t beam, int32_t* R_out, float* recall_out, float* ms_out) {
  if (!points || !p || !R_candidates) return fail(GRNND_EINVAL, "points, params and candidates must be given");
  if (ncand < 1 || ncand > 64) return fail(GRNND_EINVAL, "need 1 <= ncand <= 64");
  for (int c = 0; c < ncand; ++c)
    if (R_candidates[c] < 2 || R_candidates[c] > 256) return fail(GRNND_EINVAL, "pool candidates need 2 <= R <= 256");
  if (d < 1) return fail(GRNND_EINVAL, "need d >= 1");
  if (nq < 1 || nq > n - 3) return fail(GRNND_EINVAL, "need 1 <= nq <= n - 3 held-out query rows");
  if (k < 1 || k > 32 || beam < k || beam > 256) return fail(GRNND_EINVAL, "need 1 <= k <= 32 and k <= beam <= 256");
  if (!(recall_target > 0.0f && recall_target <= 1.0f)) return fail(GRNND_EINVAL, "need 0 < recall_target <= 1");
  const int64_t nb = n - nq;  // the built rows; the rest are the queries
  if (k > nb) return fail(GRNND_EINVAL, "need k <= n - nq");
  const cudaStream_t st = p->stream ? static_cast<cudaStream_t>(p->stream) : g_stream;
  const float* qrows = points + nb * (int64_t)d;
  // exact k nearest neighbours of the queries among the built rows, on a device copy whose
  // rows are padded to a multiple of 4 floats (the exact k-NN kernel reads 16-byte vectors)
  const int32_t ld = (d + 3) & ~3;
  DevMem mp, mi;
  GR_CU(mp.alloc((size_t)n * ld * 4));
  if (ld != d) GR_CU(cudaMemsetAsync(mp.p, 0, (size_t)n * ld * 4, st));
  GR_CU(grnnd::copy_rows(static_cast<float*>(mp.p), ld, points, d, n,
                         is_device_ptr(points) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  const float* dpts = static_cast<const float*>(mp.p);
  GR_CU(mi.alloc((size_t)nq * k * 4));
  GR_CU(grnnd::launch_brute_knn(dpts, nb, d, ld, p->metric, dpts + nb * (int64_t)ld, nq, ld, k,
                                static_cast<int32_t*>(mi.p), nullptr, st));
  std::vector<int32_t> gt((size_t)nq * k), got((size_t)nq * k);
  GR_CU(cudaMemcpyAsync(gt.data(), mi.p, gt.size() * 4, cudaMemcpyDeviceToHost, st));
  GR_CU(cudaStreamSynchronize(st));
  int best = -1;
  float best_ms = 0.0f, best_rec = -1.0f;
  for (int c = 0; c < ncand; ++c) {
    grnnd_params q = *p;
    q.R = R_candidates[c];
    q.S = std::min<int64_t>(std::min(p->S, q.R), nb - 1);
    grnnd_graph* g = nullptr;
    int rc = grnnd_build_ex(points, nb, d, &q, &g);  // settles the allocations
    if (rc != GRNND_OK) return rc;
    grnnd_free(g);
    g = nullptr;
    const auto t0 = std::chrono::steady_clock::now();
    rc = grnnd_build_ex(points, nb, d, &q, &g);
    const auto t1 = std::chrono::steady_clock::now();
    if (rc != GRNND_OK) return rc;
    const float ms = std::chrono::duration<float, std::milli>(t1 - t0).count();
    rc = grnnd_search(g, qrows, nq, k, beam, got.data());
    grnnd_free(g);
    if (rc != GRNND_OK) return rc;
    int64_t hit = 0;
    for (int64_t i = 0; i < nq; ++i)
      for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b)
          if (got[i * k + a] == gt[i * k + b] && got[i * k + a] >= 0) {
            ++hit;
            break;
          }
    const float rec = (float)((double)hit / ((double)nq * k));
    const bool ok = rec >= recall_target, best_ok = best_rec >= recall_target;
    // passing candidates by build time; while none passes, by recall (then time)
    const bool better = best < 0 || (ok && (!best_ok || ms < best_ms)) ||
                        (!ok && !best_ok && (rec > best_rec || (rec == best_rec && ms < best_ms)));
    if (better) {
      best = c;
      best_ms = ms;
      best_rec = rec;
    }
  }
  if (R_out) *R_out = R_candidates[best];
  if (recall_out) *recall_out = best_rec;
  if (ms_out) *ms_out = best_ms;
  return GRNND_OK;
}

int grnnd_build(const float* points, int64_t n, int32_t d, int32_t metric, int32_t S, int32_t R,
                int32_t T1, int32_t T2, uint64_t seed, grnnd_graph** graph_out) {
  grnnd_params p;
  grnnd_params_default(&p);
  p.metric = metric;
  p.S = S;
  p.R = R;
  p.T1 = T1;
  p.T2 = T2;
  p.seed = seed;
  return grnnd_build_ex(points, n, d, &p, graph_out);
}

int grnnd_search(const grnnd_graph* g, const float* queries, int64_t nq, int32_t k, int32_t beam,
                 int32_t* ids_out) {
  if (!g) return fail(GRNND_EINVAL, "graph is NULL");
  if (nq < 0 || (nq > 0 && (!queries || !ids_out))) return fail(GRNND_EINVAL, "bad queries/ids_out");
  if (k < 1 || beam < k || beam > 256) return fail(GRNND_EINVAL, "need 1 <= k <= beam <= 256");
  if (g->d > 1024) return fail(GRNND_EINVAL, "search supports d <= 1024");
  if (nq == 0) return GRNND_OK;
  const int32_t ldq = g->ld;
  const cudaStream_t st = g_stream;  // the thread's current stream
  DevMem mq, mo;
  GR_CU(mq.alloc((size_t)nq * ldq * 4));
  const bool out_dev = is_device_ptr(ids_out);
  int32_t* dids = ids_out;
  if (!out_dev) {
    GR_CU(mo.alloc((size_t)nq * k * 4));
    dids = static_cast<int32_t*>(mo.p);
  }
  float* dq = static_cast<float*>(mq.p);
  const cudaMemcpyKind kind = is_device_ptr(queries) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (ldq != g->d) GR_CU(cudaMemsetAsync(dq, 0, (size_t)nq * ldq * 4, st));
  GR_CU(grnnd::copy_rows(dq, ldq, queries, g->d, nq, kind, st));
  GR_CU(grnnd::launch_search(g->points, g->n, g->d, g->ld, g->metric, g->ids, g->deg, g->R, g->entry,
                             dq, nq, ldq, k, beam, dids, nullptr, st));
  if (!out_dev) GR_CU(cudaMemcpyAsync(ids_out, dids, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, st));
  GR_CU(cudaStreamSynchronize(st));
  return GRNND_OK;
}

int grnnd_graph_info(const grnnd_graph* g, int64_t* n, int32_t* d, int32_t* R, int32_t* entry) {
  if (!g) return fail(GRNND_EINVAL, "graph is NULL");
  if (n) *n = g->n;
  if (d) *d = g->d;
  if (R) *R = g->R;
  if (entry) *entry = g->entry;
  return GRNND_OK;
}

int grnnd_graph_view(const grnnd_graph* g, const int32_t** ids, const float** dists,
                     const int32_t** deg) {
  if (!g) return fail(GRNND_EINVAL, "graph is NULL");
  if (ids) *ids = g->ids;
  if (dists) *dists = g->dists;
  if (deg) *deg = g->deg;
  return GRNND_OK;
}

int grnnd_graph_copy(const grnnd_graph* g, int32_t* ids, float* dists, int32_t* deg) {
  if (!g) return fail(GRNND_EINVAL, "graph is NULL");
  const size_t nr = (size_t)g->n * g->R;
  const cudaStream_t st = g_stream;  // the thread's current stream
  if (ids) GR_CU(grnnd::copy_bytes(ids, g->ids, nr * 4, st));
  if (dists) GR_CU(grnnd::copy_bytes(dists, g->dists, nr * 4, st));
  if (deg) GR_CU(grnnd::copy_bytes(deg, g->deg, (size_t)g->n * 4, st));
  GR_CU(cudaStreamSynchronize(st));
  return GRNND_OK;
}

int grnnd_graph_stats(const grnnd_graph* g, int64_t* out, int32_t count) {
  if (!g || !out || count < 0) return fail(GRNND_EINVAL, "bad arguments");
  const int32_t c = std::min<int32_t>(count, 8);
  for (int32_t i = 0; i < c; ++i) out[i] = g->stats[i];
  return c;
}

void grnnd_free(grnnd_graph* g) {
  delete g;  // the device memory goes with the last graph that shares it
}

}  // extern "C"

namespace grnnd {
int validate_build(const float* points, int64_t n, int32_t d, const grnnd_params* p) {
  int rc = check_params(p);
  if (rc) return rc;
  if (!points) return fail(GRNND_EINVAL, "points is NULL");
  if (n < 2 || n > 0x7FFFFFFELL) return fail(GRNND_EINVAL, "n must be in [2, 2^31 - 2]");
  if (d < 1) return fail(GRNND_EINVAL, "d must be >= 1");
  if ((int64_t)p->S > n - 1) return fail(GRNND_EINVAL, "need 1 <= S <= min(R, n-1)");
  return GRNND_OK;
}

int build_with(const float* points, int64_t n, int32_t d, const grnnd_params* p, const AllocMode& am,
               grnnd_graph** graph_out) {
  if (graph_out) *graph_out = nullptr;
  if (!graph_out) return fail(GRNND_EINVAL, "graph_out is NULL");
  int rc = validate_build(points, n, d, p);
  if (rc) return rc;
  return build_core(points, n, d, p, nullptr, 1, graph_out, am);
}

size_t build_device_bytes(int64_t n, int32_t d, const grnnd_params* p, size_t* resident) {
  const BuildSizes z = build_sizes(n, d, p, false, 1);
  if (resident) *resident = z.pts_b + z.graph_b;
  return z.pts_b + z.graph_b + z.scratch_b;
}
}  // namespace grnnd
