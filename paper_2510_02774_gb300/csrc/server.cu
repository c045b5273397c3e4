// Serving loop of the GRNND library (declarations in include/grnnd.h).
//
// The paper builds one graph per run and has no serving path.  This is the request loop
// around the build and search kernels: build and search requests arrive from any host
// thread, `slots` worker threads each own a non-blocking CUDA stream, and a free worker
// admits the oldest request that fits the HBM budget (skipping ones that do not fit yet, and
// searches whose index is still being built).  A worker that admits a search also takes the
// other waiting searches of the same index, k and beam, and serves them with one launch.
// Device memory comes from a stream-ordered pool owned by the server, so requests on
// different streams never wait on each other's allocations or frees.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "grnnd.h"
#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
int32_t round4(int32_t d) { return (d + 3) & ~3; }

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int fail(int code, const std::string& msg) {
  grnnd::set_last_error(msg);
  return code;
}

struct Request {
  int64_t id = 0;
  int kind = GRNND_REQ_BUILD;
  int state = GRNND_REQ_QUEUED;
  int status = GRNND_OK;
  int batch = 0;
  int64_t index = 0;
  int64_t units = 0;
  uint64_t bytes = 0;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  std::string msg;
  // build
  const float* points = nullptr;
  int32_t d = 0;
  grnnd_params p{};
  grnnd_tuning tuning{};
  bool has_tuning = false;
  uint64_t resident = 0;
  // search
  const float* queries = nullptr;
  int32_t k = 0, beam = 0;
  int32_t* ids_out = nullptr;
};

enum { IDX_BUILDING = 0, IDX_READY = 1, IDX_FAILED = 2 };

struct Index {
  int state = IDX_BUILDING;
  int32_t d = 0;
  grnnd_graph* g = nullptr;
  uint64_t resident = 0;
  int users = 0;  // searches of it queued or running
};

// Device buffer from the server's pool, freed on the same stream.
struct PoolBuf {
  void* p = nullptr;
  cudaStream_t st;
  explicit PoolBuf(cudaStream_t s) : st(s) {}
  ~PoolBuf() {
    if (p) cudaFreeAsync(p, st);
  }
};

}  // namespace

struct grnnd_server {
  int device = 0;
  int slots = 1;
  uint64_t budget = 0, used = 0, peak = 0;
  int64_t max_batch = 65536;
  cudaMemPool_t pool = nullptr;
  cudaStream_t free_stream = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  std::deque<Request*> queue;         // queued requests, arrival order
  std::map<int64_t, Request*> reqs;   // requests not yet collected by a wait
  std::map<int64_t, Index> indices;
  int64_t next_id = 1;
  int running = 0;
  bool stop = false;
  Clock::time_point t0 = Clock::now();
  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void finish_locked(grnnd_server* S, Request* r, int status, const std::string& msg) {
  r->state = GRNND_REQ_DONE;
  r->status = status;
  r->msg = msg;
  r->t_done = S->now();
}

// Under the lock: the next request(s) a free slot runs, reserved against the budget.
// Requests that can no longer run (a build above the whole budget, a search of an index
// that failed or is gone) are completed here with their error.
bool pick_locked(grnnd_server* S, std::vector<Request*>& batch) {
  bool completed = false;
  for (auto it = S->queue.begin(); it != S->queue.end();) {
    Request* r = *it;
    if (r->kind == GRNND_REQ_BUILD) {
      if (r->bytes > S->budget) {
        finish_locked(S, r, GRNND_ENOMEM,
                      "build needs " + std::to_string(r->bytes) + " bytes, above the server's hbm_budget");
        S->indices[r->index].state = IDX_FAILED;
        it = S->queue.erase(it);
        completed = true;
        continue;
      }
      if (S->used + r->bytes <= S->budget) {
        batch.push_back(r);
        S->queue.erase(it);
        break;
      }
      ++it;
      continue;
    }
    auto ix = S->indices.find(r->index);
    if (ix == S->indices.end() || ix->second.state == IDX_FAILED) {
      if (ix != S->indices.end()) ix->second.users -= 1;
      finish_locked(S, r, GRNND_EINVAL, "index " + std::to_string(r->index) + " is not available");
      it = S->queue.erase(it);
      completed = true;
      continue;
    }
    if (ix->second.state != IDX_READY || S->used + r->bytes > S->budget) {
      ++it;
      continue;
    }
    // this search and every other waiting search of the same index, k and beam
    uint64_t tot = r->bytes;
    int64_t q = r->units;
    batch.push_back(r);
    it = S->queue.erase(it);
    for (auto jt = it; jt != S->queue.end();) {
      Request* o = *jt;
      if (o->kind == GRNND_REQ_SEARCH && o->index == r->index && o->k == r->k && o->beam == r->beam &&
          q + o->units <= S->max_batch && S->used + tot + o->bytes <= S->budget) {
        batch.push_back(o);
        tot += o->bytes;
        q += o->units;
        jt = S->queue.erase(jt);
      } else {
        ++jt;
      }
    }
    break;
  }
  if (completed) S->done_cv.notify_all();
  if (batch.empty()) return false;
  const double t = S->now();
  for (Request* r : batch) {
    S->used += r->bytes;
    r->state = GRNND_REQ_RUNNING;
    r->t_admit = t;
    r->batch = (int)batch.size();
  }
  S->peak = std::max(S->peak, S->used);
  S->running += (int)batch.size();
  return true;
}

void run_build(grnnd_server* S, Request* r, cudaStream_t st) {
  nvtxRangePushA("serve build");
  grnnd_params p = r->p;
  p.stream = st;
  p.hbm_budget = 0;
  p.tuning = r->has_tuning ? &r->tuning : nullptr;
  grnnd::AllocMode am;
  am.pool = S->pool;
  am.free_stream = S->free_stream;
  grnnd_graph* g = nullptr;
  const int rc = grnnd::build_with(r->points, r->units, r->d, &p, am, &g);
  nvtxRangePop();
  const std::string msg = rc ? std::string(grnnd_last_error()) : std::string();
  std::lock_guard<std::mutex> lk(S->mu);
  Index& ix = S->indices[r->index];
  if (rc == GRNND_OK) {
    ix.state = IDX_READY;
    ix.g = g;
    ix.resident = r->resident;
    S->used -= r->bytes - r->resident;  // the scratch is back in the pool; the index stays
  } else {
    ix.state = IDX_FAILED;
    S->used -= r->bytes;
  }
  S->running -= 1;
  finish_locked(S, r, rc, msg);
  S->work_cv.notify_all();
  S->done_cv.notify_all();
}

int search_batch(const grnnd_graph* g, const std::vector<Request*>& batch, cudaMemPool_t pool, cudaStream_t st) {
  const int32_t ld = g->ld, d = g->d, k = batch[0]->k, beam = batch[0]->beam;
  int64_t Q = 0;
  for (Request* r : batch) Q += r->units;
  PoolBuf dq(st), dout(st);
  cudaError_t e = cudaMallocFromPoolAsync(&dq.p, al256((size_t)Q * ld * 4), pool, st);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&dout.p, al256((size_t)Q * k * 4), pool, st);
  float* q = static_cast<float*>(dq.p);
  int32_t* out = static_cast<int32_t*>(dout.p);
  if (e == cudaSuccess && ld != d) e = cudaMemsetAsync(q, 0, (size_t)Q * ld * 4, st);
  int64_t off = 0;
  for (Request* r : batch) {  // the queries of every request, one after the other
    if (e != cudaSuccess) break;
    const cudaMemcpyKind kind = is_device_ptr(r->queries) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    e = grnnd::copy_rows(q + off * ld, ld, r->queries, d, r->units, kind, st);
    off += r->units;
  }
  if (e == cudaSuccess)
    e = grnnd::launch_search(g->points, g->n, g->d, g->ld, g->metric, g->ids, g->deg, g->R, g->entry, q, Q, ld, k,
                             beam, out, nullptr, st);
  off = 0;
  for (Request* r : batch) {  // each request's rows of the result
    if (e != cudaSuccess) break;
    e = cudaMemcpyAsync(r->ids_out, out + off * k, (size_t)r->units * k * 4, cudaMemcpyDefault, st);
    off += r->units;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    grnnd::set_last_error(std::string("search: ") + cudaGetErrorString(e));
    return GRNND_ECUDA;
  }
  return GRNND_OK;
}

void run_search(grnnd_server* S, const std::vector<Request*>& batch, cudaStream_t st) {
  const grnnd_graph* g = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    g = S->indices[batch[0]->index].g;  // ready, and kept while its searches run
  }
  nvtxRangePushA("serve search batch");
  const int rc = search_batch(g, batch, S->pool, st);
  nvtxRangePop();
  const std::string msg = rc ? std::string(grnnd_last_error()) : std::string();
  std::lock_guard<std::mutex> lk(S->mu);
  for (Request* r : batch) {
    S->used -= r->bytes;
    finish_locked(S, r, rc, msg);
  }
  S->indices[batch[0]->index].users -= (int)batch.size();
  S->running -= (int)batch.size();
  S->work_cv.notify_all();
  S->done_cv.notify_all();
}

void worker_main(grnnd_server* S, int slot) {
  cudaSetDevice(S->device);
  cudaStream_t st = S->streams[(size_t)slot];
  for (;;) {
    std::vector<Request*> batch;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->work_cv.wait(lk, [&] { return S->stop || pick_locked(S, batch); });
      if (batch.empty()) return;  // stopping
    }
    if (batch[0]->kind == GRNND_REQ_BUILD)
      run_build(S, batch[0], st);
    else
      run_search(S, batch, st);
  }
}

void fill_info(const Request* r, grnnd_request_info* info) {
  if (!info) return;
  std::memset(info, 0, sizeof(*info));
  info->id = r->id;
  info->kind = r->kind;
  info->state = r->state;
  info->status = r->status;
  info->batch = r->batch;
  info->index = r->index;
  info->units = r->units;
  info->bytes = r->bytes;
  info->t_submit = r->t_submit;
  info->t_admit = r->t_admit;
  info->t_done = r->t_done;
  std::strncpy(info->message, r->msg.c_str(), sizeof(info->message) - 1);
}

}  // namespace

extern "C" {

int grnnd_server_create(const grnnd_server_config* cfg, grnnd_server** out) {
  if (out) *out = nullptr;
  if (!cfg || !out) return fail(GRNND_EINVAL, "config/out is NULL");
  if (cfg->slots < 1 || cfg->slots > 64) return fail(GRNND_EINVAL, "slots must be in [1, 64]");
  if (cfg->hbm_budget == 0) return fail(GRNND_EINVAL, "hbm_budget must be > 0");
  if (cfg->max_batch_queries < 0) return fail(GRNND_EINVAL, "max_batch_queries must be >= 0");
  grnnd_server* S = new grnnd_server();
  S->slots = cfg->slots;
  S->budget = cfg->hbm_budget;
  S->max_batch = cfg->max_batch_queries ? cfg->max_batch_queries : 65536;
  auto undo = [&](const std::string& what, cudaError_t e) {
    for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
    if (S->free_stream) cudaStreamDestroy(S->free_stream);
    if (S->pool) cudaMemPoolDestroy(S->pool);
    delete S;
    cudaGetLastError();
    return fail(GRNND_ECUDA, what + ": " + cudaGetErrorString(e));
  };
  cudaError_t e = cudaGetDevice(&S->device);
  if (e != cudaSuccess) return undo("cudaGetDevice", e);
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = S->device;
  if ((e = cudaMemPoolCreate(&S->pool, &props)) != cudaSuccess) return undo("cudaMemPoolCreate", e);
  uint64_t keep = S->budget;  // freed blocks stay cached up to the budget
  if ((e = cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess)
    return undo("cudaMemPoolSetAttribute", e);
  if ((e = cudaStreamCreateWithFlags(&S->free_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return undo("cudaStreamCreate", e);
  for (int i = 0; i < S->slots; ++i) {
    cudaStream_t s = nullptr;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return undo("cudaStreamCreate", e);
    S->streams.push_back(s);
  }
  for (int i = 0; i < S->slots; ++i) S->workers.emplace_back(worker_main, S, i);
  *out = S;
  return GRNND_OK;
}

int grnnd_server_submit_build(grnnd_server* S, const float* points, int64_t n, int32_t d, const grnnd_params* p,
                              int64_t* id_out) {
  if (id_out) *id_out = -1;
  if (!S || !id_out) return fail(GRNND_EINVAL, "server/id_out is NULL");
  int rc = grnnd::validate_build(points, n, d, p);
  if (rc) return rc;
  Request* r = new Request();
  r->kind = GRNND_REQ_BUILD;
  r->points = points;
  r->units = n;
  r->d = d;
  r->p = *p;
  if (p->tuning) {
    r->tuning = *p->tuning;
    r->has_tuning = true;
  }
  size_t resident = 0;
  r->bytes = grnnd::build_device_bytes(n, d, p, &resident);
  r->resident = resident;
  std::lock_guard<std::mutex> lk(S->mu);
  r->id = S->next_id++;
  r->index = r->id;
  r->t_submit = S->now();
  Index& ix = S->indices[r->id];
  ix.state = IDX_BUILDING;
  ix.d = d;
  S->reqs[r->id] = r;
  S->queue.push_back(r);
  *id_out = r->id;
  S->work_cv.notify_one();
  return GRNND_OK;
}

int grnnd_server_submit_search(grnnd_server* S, int64_t index, const float* queries, int64_t nq, int32_t k,
                               int32_t beam, int32_t* ids_out, int64_t* id_out) {
  if (id_out) *id_out = -1;
  if (!S || !id_out) return fail(GRNND_EINVAL, "server/id_out is NULL");
  if (nq < 1 || !queries || !ids_out) return fail(GRNND_EINVAL, "need nq >= 1, queries and ids_out");
  if (k < 1 || beam < k || beam > 256) return fail(GRNND_EINVAL, "need 1 <= k <= beam <= 256");
  std::lock_guard<std::mutex> lk(S->mu);
  auto ix = S->indices.find(index);
  if (ix == S->indices.end() || ix->second.state == IDX_FAILED)
    return fail(GRNND_EINVAL, "index " + std::to_string(index) + " is not available");
  if (ix->second.d > 1024) return fail(GRNND_EINVAL, "search supports d <= 1024");
  Request* r = new Request();
  r->kind = GRNND_REQ_SEARCH;
  r->index = index;
  r->queries = queries;
  r->units = nq;
  r->k = k;
  r->beam = beam;
  r->ids_out = ids_out;
  r->bytes = al256((size_t)nq * round4(ix->second.d) * 4) + al256((size_t)nq * k * 4);
  r->id = S->next_id++;
  r->t_submit = S->now();
  ix->second.users += 1;
  S->reqs[r->id] = r;
  S->queue.push_back(r);
  *id_out = r->id;
  S->work_cv.notify_one();
  return GRNND_OK;
}

int grnnd_server_wait(grnnd_server* S, int64_t id, double timeout_s, grnnd_request_info* info) {
  if (!S) return fail(GRNND_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return fail(GRNND_EINVAL, "unknown request " + std::to_string(id));
  Request* r = it->second;
  auto done = [&] { return r->state == GRNND_REQ_DONE; };
  if (timeout_s < 0)
    S->done_cv.wait(lk, done);
  else
    S->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), done);
  fill_info(r, info);
  if (!done()) return fail(GRNND_ETIMEOUT, "request " + std::to_string(id) + " is not done");
  const int status = r->status;
  if (status != GRNND_OK) grnnd::set_last_error(r->msg);
  S->reqs.erase(it);
  delete r;
  return status;
}

int grnnd_server_index(grnnd_server* S, int64_t index, const grnnd_graph** g) {
  if (g) *g = nullptr;
  if (!S || !g) return fail(GRNND_EINVAL, "server/g is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  auto ix = S->indices.find(index);
  if (ix == S->indices.end() || ix->second.state == IDX_FAILED)
    return fail(GRNND_EINVAL, "index " + std::to_string(index) + " is not available");
  if (ix->second.state == IDX_BUILDING) return fail(GRNND_EBUSY, "index " + std::to_string(index) + " is being built");
  *g = ix->second.g;
  return GRNND_OK;
}

int grnnd_server_release(grnnd_server* S, int64_t index) {
  if (!S) return fail(GRNND_EINVAL, "server is NULL");
  grnnd_graph* g = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto ix = S->indices.find(index);
    if (ix == S->indices.end()) return fail(GRNND_EINVAL, "unknown index " + std::to_string(index));
    if (ix->second.state == IDX_BUILDING || ix->second.users > 0)
      return fail(GRNND_EBUSY, "index " + std::to_string(index) + " has work queued or running");
    g = ix->second.g;
    S->used -= ix->second.resident;
    S->indices.erase(ix);
    S->work_cv.notify_all();
  }
  grnnd_free(g);  // stream-ordered free into the server's pool
  return GRNND_OK;
}

int grnnd_server_status(grnnd_server* S, uint64_t* bytes_in_use, uint64_t* peak_bytes, int32_t* queued,
                        int32_t* running, int32_t* indices) {
  if (!S) return fail(GRNND_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  if (bytes_in_use) *bytes_in_use = S->used;
  if (peak_bytes) *peak_bytes = S->peak;
  if (queued) *queued = (int32_t)S->queue.size();
  if (running) *running = S->running;
  if (indices) {
    int32_t c = 0;
    for (auto& kv : S->indices) c += kv.second.state == IDX_READY ? 1 : 0;
    *indices = c;
  }
  return GRNND_OK;
}

void grnnd_server_destroy(grnnd_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->work_cv.notify_all();
  for (auto& t : S->workers) t.join();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (Request* r : S->queue) finish_locked(S, r, GRNND_EBUSY, "server destroyed");
    S->queue.clear();
    S->done_cv.notify_all();
  }
  for (auto& kv : S->indices)
    if (kv.second.g) grnnd_free(kv.second.g);
  S->indices.clear();
  cudaStreamSynchronize(S->free_stream);
  for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
  cudaStreamDestroy(S->free_stream);
  cudaMemPoolDestroy(S->pool);
  for (auto& kv : S->reqs) delete kv.second;
  delete S;
}

}  // extern "C"
