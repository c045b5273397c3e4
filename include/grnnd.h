/*
 * grnnd.h — C ABI of the GB300 (sm_103a) GRNND graph-construction library.
 *
 * GRNND (arXiv 2510.02774) builds a sparse proximity graph by Relative
 * NN-Descent: random initial pools (Alg 3), then rounds of disordered
 * neighbour propagation (Alg 4 with the pair rule of Eq 2) over fixed-capacity
 * double-buffered pools (Sec 3.5), with reverse-edge sampling between outer
 * iterations (Sec 3.6).  The graph is queried with a candidate-list search
 * (Sec 2.1, Sec 4.2).
 *
 * Conventions shared by every entry point
 *   - Every call returns GRNND_OK (0) or a negative grnnd_status; calls never
 *     abort.  On failure grnnd_last_error() returns a thread-local message and
 *     output handles are set to NULL.
 *   - "device" pointers are CUDA device (or managed) memory on the current
 *     device; "host or device" pointers are classified with
 *     cudaPointerGetAttributes and copied as needed.  Pinned (page-locked)
 *     host buffers that are 16-byte aligned, with a byte size that is a
 *     multiple of 16, are moved by the library's own copy kernel (16-byte loads
 *     and stores over the host link); pageable, misaligned or ragged buffers by
 *     cudaMemcpyAsync.  The bytes are the same either way.
 *   - Point matrices are row-major float32, one row per point.  Step-level
 *     calls take a leading dimension `ld` (floats per row): ld >= d, ld % 4 == 0,
 *     and the base address 16-byte aligned (rows are moved with bulk copies).
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Step-level calls are asynchronous on that stream; grnnd_build*,
 *     grnnd_search and grnnd_graph_copy are synchronous on return.  Calls that
 *     take no stream argument (grnnd_build, grnnd_search, grnnd_graph_copy), and
 *     grnnd_build_ex / grnnd_build_batch given p->stream == NULL, run on the
 *     calling thread's current stream (grnnd_set_stream).
 *   - Pool layout (step-level calls): a pool is n rows of R slots of uint64
 *     keys plus an int32 degree per row.  A key packs one entry as
 *         key = (ordered_bits(dist) << 32) | (id << 1) | old
 *     where ordered_bits maps float32 to uint32 monotonically (non-negative x:
 *     bits | 0x80000000; negative x: ~bits), so key order is (dist, id) order.
 *     `old` = 1 marks an entry that survived its own vertex's previous prune.
 *     Row v holds deg[v] keys in ascending order followed by empty slots
 *     (0xFFFFFFFFFFFFFFFF).  Ids must be < 2^31.
 *   - Distances: GRNND_L2SQ = squared Euclidean distance (the square of Alg 5's
 *     result; every decision is the same), GRNND_IP = 1 - <x, y>.  In the FP32
 *     form every recorded distance is the canonical FP32 value: one fused
 *     multiply-add per dimension in ascending dimension order, so the same
 *     pair always gets the same bits wherever it is computed.
 */
#ifndef GRNND_H
#define GRNND_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GRNND_API __attribute__((visibility("default")))
#else
#define GRNND_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GRNND_OK = 0,
    GRNND_EINVAL = -1,   /* invalid argument; nothing was launched */
    GRNND_ENOMEM = -2,   /* device allocation or HBM budget exceeded before any launch */
    GRNND_ECUDA = -3,    /* a CUDA runtime call or kernel launch failed */
    GRNND_ETIMEOUT = -4, /* a device-side wait gave up after its iteration limit */
    GRNND_EBUSY = -5     /* the object is in use by another call */
} grnnd_status;

typedef enum { GRNND_L2SQ = 0, GRNND_IP = 1 } grnnd_metric;

/* Arithmetic of the pair-distance tiles (dist_tile).  The paper states no
 * precision (Sec 3.4 computes distances with FP32 warp arithmetic).  FP32:
 * direct differences on CUDA cores (the canonical form).  BF16: Gram tiles of a
 * bfloat16 copy on the tensor cores with FP32 accumulation.  FP8: Gram tiles of
 * an e4m3 copy with one power-of-two scale per row, FP32 accumulation.  In both
 * quantized forms a fire decision whose margin is within the per-pair error
 * bound (quantization residuals of the two rows + accumulation) is re-decided
 * with the canonical FP32 distance. */
typedef enum { GRNND_FP32 = 0, GRNND_BF16 = 1, GRNND_FP8 = 2 } grnnd_precision;

/* Visit order of a pool's pairs: disordered (Sec 3.3, the paper's method),
 * ascending (dist, id) (Alg 2's serial order), or descending (Sec 4.3 ablation). */
typedef enum { GRNND_ORDER_RANDOM = 0, GRNND_ORDER_ASC = 1, GRNND_ORDER_DESC = 2 } grnnd_order;

typedef struct grnnd_graph grnnd_graph; /* opaque, library-owned */

/* Launch shape of the join (no counterpart in the paper).  A pool of m entries is joined
 * by a lane group of 8 lanes (four pools per warp) if m <= group_max[0], else of 16 lanes
 * (two per warp) if m <= group_max[1], else of 32 lanes if m <= group_max[2], else by a
 * 64-thread CTA; 0 <= group_max[c] <= 8 << c.  warp_ctas_per_sm / team_ctas_per_sm cap the
 * resident CTAs per SM of the two join kernels (0: as many as fit); row_copies picks how the
 * warp join stages quantized rows in shared memory.  Only speed depends on it: every tuning
 * gives the same graph.  Defaults {8, 16, 32}, 0, 0, 0. */
typedef struct grnnd_tuning {
    int32_t group_max[3];
    int32_t warp_ctas_per_sm;
    int32_t team_ctas_per_sm;
    int32_t row_copies;   /* BF16 / FP8 rows of the warp join: 1 = one bulk copy per row,
                             2 = TMA gather4 copies of four rows each (where the rows' layout
                             allows: fewer copy instructions, 2-way bank conflicts in the tiles),
                             0 = gather4 for BF16 rows of at most 128 dimensions, else 1 */
    float ms;             /* grnnd_autotune: build time of the chosen tuning on the sample */
} grnnd_tuning;

/* Parameters of a build (Table 1: S, R, T1, T2, rho). */
typedef struct grnnd_params {
    int32_t S;            /* initial random neighbours per vertex, 1 <= S <= min(R, n-1) */
    int32_t R;            /* pool capacity = maximum out-degree, 2 <= R <= 256 (Sec 3.5) */
    int32_t T1;           /* outer iterations, >= 1 */
    int32_t T2;           /* inner iterations (rounds) per outer iteration, >= 1 */
    float rho;            /* reverse-edge sampling ratio in [0, 1] (Sec 3.6); default 0.6 */
    uint64_t seed;        /* seed of the counter-based hash behind every random choice */
    int32_t metric;       /* grnnd_metric */
    int32_t precision;    /* grnnd_precision */
    int32_t order;        /* grnnd_order */
    int32_t final_prune;  /* 1: return the survivors of one more prune pass; 0: the last pool */
    void *stream;         /* cudaStream_t for all work of the build; NULL = the calling
                             thread's current stream (grnnd_set_stream) */
    uint64_t hbm_budget;  /* bytes the build may allocate; 0 = no limit */
    const grnnd_tuning *tuning; /* join launch shape; NULL = defaults */
} grnnd_params;

/* Fills *p with defaults: S=16, R=32, T1=4, T2=8, rho=0.6, seed=0, L2SQ, FP32,
 * random order, final_prune=1, stream=NULL, no budget, default tuning. */
GRNND_API void grnnd_params_default(grnnd_params *p);

/* Autotuner: builds the given points (a sample of the workload to tune for: host or device
 * rows, as for grnnd_build_ex; with offsets != NULL a batch of nbuild builds, as for
 * grnnd_build_batch) once per candidate tuning and writes the fastest to *best (with its
 * time in best->ms).  Candidates: the lane-group routing {8,16,32}, {0,16,32}, {0,0,32},
 * {8,16,16} and {0,16,16}, then 1..3 warp-kernel CTAs and 2, 4 or 6 team CTAs per SM around
 * the best, one axis at a time, then (BF16 / FP8) row_copies 1 and 2.  p->tuning is ignored.
 * Synchronous. */
GRNND_API int grnnd_autotune(const float *points, int64_t n, int32_t d, const int64_t *offsets,
                             int32_t nbuild, const grnnd_params *p, grnnd_tuning *best);

/* Pool-capacity autotuner (no counterpart in the paper): chooses the pool capacity R of a
 * build -- the candidate that builds fastest among those whose graph reaches recall@k >=
 * recall_target, or the one of highest recall when none does.  The last nq rows of `points`
 * (n rows of d floats, host or device, as for grnnd_build_ex) are held out as queries; each
 * candidate R builds the first n - nq rows with p's parameters but R and S = min(p->S, R),
 * once to settle allocations and once timed, and its graph is searched (grnnd_search with
 * k and beam) against the exact k nearest neighbours of the built rows (grnnd_brute_knn).
 * The candidates are tried in the order given.  Writes the chosen R, its recall and its
 * build time (ms) to *R_out, *recall_out and *ms_out (each may be NULL).  Validation:
 * 1 <= ncand <= 64, every candidate 2 <= R <= 256, 1 <= nq <= n - 3, 1 <= k <= 32,
 * k <= beam <= 256, 0 < recall_target <= 1.  Synchronous. */
GRNND_API int grnnd_autotune_pool(const float *points, int64_t n, int32_t d, int64_t nq,
                                  const grnnd_params *p, const int32_t *R_candidates, int32_t ncand,
                                  float recall_target, int32_t k, int32_t beam, int32_t *R_out,
                                  float *recall_out, float *ms_out);

/* Memory cache of whole builds on the current device (no counterpart in the paper).  A build
 * allocates its device memory (points, graph, pools, round workspace: about 4 GB for 1M x 128
 * with R = 64) and frees the scratch part when it returns.  With bytes > 0, grnnd_build_ex and
 * grnnd_build_batch take that memory from a stream-ordered pool owned by the library, which
 * keeps up to `bytes` freed bytes for the next build instead of returning them to the driver
 * (saving the cudaMalloc / cudaFree work of every build, a few ms at 1M points), like a
 * framework's caching allocator.  The memory of a graph returns to the pool when the graph
 * is freed (grnnd_free synchronises the device first, since the caller's own work may still
 * read the graph).  bytes = 0 (the default) turns the cache off and releases what it holds.
 * Graphs are the same either way. */
GRNND_API int grnnd_set_memory_cache(uint64_t bytes);

/* Builds a graph over n points of dimension d (Alg 3).  `points` is host or
 * device memory, n rows of d contiguous floats; every value must be finite.
 * Validation: n >= 2, d >= 1, 1 <= S <= min(R, n-1), 2 <= R <= 256, T1, T2 >= 1.
 * On success *graph_out owns a device copy of the points and the graph; free it
 * with grnnd_free.  Runs on the calling thread's current stream (grnnd_set_stream). */
GRNND_API int grnnd_build(const float *points, int64_t n, int32_t d, int32_t metric, int32_t S,
                int32_t R, int32_t T1, int32_t T2, uint64_t seed, grnnd_graph **graph_out);

/* The calling thread's current stream (no counterpart in the paper, which runs one build at a
 * time): the stream of every call that takes no stream argument and of builds whose
 * p->stream is NULL.  A framework binding sets it to its own current stream before a call
 * (the Python binding passes PyTorch's).  Initially NULL, the legacy default stream; the
 * setting is per host thread. */
GRNND_API void grnnd_set_stream(void *stream);
GRNND_API void *grnnd_get_stream(void);

/* Same as grnnd_build with every parameter of grnnd_params. */
GRNND_API int grnnd_build_ex(const float *points, int64_t n, int32_t d, const grnnd_params *p,
                   grnnd_graph **graph_out);

/* Batched form (no counterpart in the paper, which builds one graph per call): nbuild
 * independent builds in one pass.  Build b takes the rows points[offsets[b] ..
 * offsets[b+1]) (d floats each, host or device memory, as for grnnd_build_ex) and gets
 * graphs_out[b]: the graph grnnd_build_ex returns for those rows alone with the same
 * params, ids local to the build.  Every build shares p.  Each round runs all builds in the
 * same kernels (random draws and visit orders use ids local to each build); the pass runs
 * all T1 x T2 rounds (a round after one that left no new entry is an identity, so the
 * result is the same), is recorded as one CUDA graph and launched once on p->stream.  The
 * graphs share one device allocation, released with the last of them (grnnd_free each).
 * offsets: host int64[nbuild + 1], offsets[0] = 0, every build >= max(2, S + 1) points,
 * total <= 2^31 - 2.  Graph stats hold the counters of the whole pass.  On failure every
 * graphs_out[b] is NULL. */
GRNND_API int grnnd_build_batch(const float *points, const int64_t *offsets, int32_t nbuild,
                                int32_t d, const grnnd_params *p, grnnd_graph **graphs_out);

/* Candidate-list search (Sec 4.2): best-first expansion from the entry point
 * (the point nearest the dataset mean) with a candidate list of `beam`
 * entries; stops when every listed candidate is expanded and writes the k
 * nearest found ids per query, ascending by (dist, id), -1 padded.
 * `queries` (nq x d floats) and `ids_out` (nq x k int32) are host or device.
 * 1 <= k <= beam <= 256. */
GRNND_API int grnnd_search(const grnnd_graph *g, const float *queries, int64_t nq, int32_t k,
                 int32_t beam, int32_t *ids_out);

/* Sizes of a graph: n, d, R (row capacity) and the search entry id.  Any
 * output pointer may be NULL. */
GRNND_API int grnnd_graph_info(const grnnd_graph *g, int64_t *n, int32_t *d, int32_t *R,
                     int32_t *entry);

/* Device pointers into the graph (valid until grnnd_free): ids n x R int32
 * (-1 padded), dists n x R float32 (+inf padded), deg n int32.  Row v lists
 * its deg[v] neighbours ascending by (dist, id). */
GRNND_API int grnnd_graph_view(const grnnd_graph *g, const int32_t **ids, const float **dists,
                     const int32_t **deg);

/* Copies the graph into caller buffers (host or device; any may be NULL). */
GRNND_API int grnnd_graph_copy(const grnnd_graph *g, int32_t *ids, float *dists, int32_t *deg);

/* Counters of the build of g: [0] rounds run, [1] vertex prunes with a new
 * entry, [2] candidate rows gathered, [3] pair distances evaluated, [4] pairs
 * fired, [5] proposals of the rounds (every pool entry once per round), [6]
 * redirects and reverse proposals merged, [7] BF16 decisions re-taken in FP32.
 * `out` is host memory of `count` int64 slots; returns the number written (at
 * most 8). */
GRNND_API int grnnd_graph_stats(const grnnd_graph *g, int64_t *out, int32_t count);

GRNND_API void grnnd_free(grnnd_graph *g);

/* Thread-local message of the last failed call on this thread ("" if none). */
GRNND_API const char *grnnd_last_error(void);

/* Per-kernel timing (tracing).  Between grnnd_profile_begin and
 * grnnd_profile_end every kernel that the calling thread launches through this
 * library is bracketed by two CUDA events recorded on its launching stream.
 * grnnd_profile_end synchronises those events and writes one entry per kernel
 * name (launch count and summed event time in ms) into `out` (host memory,
 * max_entries slots); *n_entries receives the number of distinct names. */
typedef struct grnnd_kernel_time {
    char name[32];
    int64_t launches;
    double ms;
} grnnd_kernel_time;
GRNND_API int grnnd_profile_begin(void);
/* grnnd_profile_begin that times only the kernels named in `names` (host string, a
 * comma-separated list such as "rnd_join_warp,rnd_join_team"; NULL or "" times every
 * kernel): the other launches get no events, so the timing perturbs them not at all. */
GRNND_API int grnnd_profile_begin_only(const char *names);
GRNND_API int grnnd_profile_end(grnnd_kernel_time *out, int32_t max_entries, int32_t *n_entries);

/* ------------------------------------------------------------------------- */
/* Serving loop (no counterpart in the paper, which builds one graph per run)  */
/* ------------------------------------------------------------------------- */

/* A request loop on the current device.  Build requests (each makes one resident
 * index: a graph and its points) and search requests against resident indices are
 * submitted from any host thread as they arrive.  `slots` worker threads each own a
 * non-blocking CUDA stream, and every admitted request runs on a free slot, so requests
 * that arrive while others run overlap with them on the device.
 *   Admission: requests are considered in arrival order; one is admitted when a slot is
 *   free and its device bytes fit the HBM budget beside the resident indices and the
 *   requests in flight (a build: points, graph and scratch, as grnnd_build_ex allocates;
 *   a search: its queries and results).  A request that does not fit yet, or a search
 *   whose index is still being built, waits without holding back later requests.  A
 *   build larger than the whole budget fails with GRNND_ENOMEM.
 *   Continuous batching of searches: a slot that takes a search also takes every other
 *   waiting search of the same index with the same k and beam (up to max_batch_queries
 *   queries together) and serves them with one search launch.  Each query's result does
 *   not depend on the other queries, so it is the same alone and in any mix.
 *   Memory: builds and searches allocate from the server's own stream-ordered memory pool,
 *   so one request's allocations and frees never wait on another request's kernels.
 * Every entry point is thread-safe.  Buffers passed to a submit call (points, queries,
 * ids_out; host or device memory) must stay valid until the request is done. */
typedef struct grnnd_server grnnd_server; /* opaque */

typedef struct grnnd_server_config {
    int32_t slots;              /* requests on the device at once, 1..64 */
    uint64_t hbm_budget;        /* device bytes for resident indices + requests in flight, > 0 */
    int64_t max_batch_queries;  /* queries one search launch may merge; 0 = 65536 */
} grnnd_server_config;

typedef enum { GRNND_REQ_BUILD = 0, GRNND_REQ_SEARCH = 1 } grnnd_request_kind;
typedef enum { GRNND_REQ_QUEUED = 0, GRNND_REQ_RUNNING = 1, GRNND_REQ_DONE = 2 } grnnd_request_state;

typedef struct grnnd_request_info {
    int64_t id;          /* request id; a build's id is also the id of the index it makes */
    int32_t kind;        /* grnnd_request_kind */
    int32_t state;       /* grnnd_request_state */
    int32_t status;      /* grnnd_status of the request once done */
    int32_t batch;       /* search: requests served by the same launch (1 = alone) */
    int64_t index;       /* index built or searched */
    int64_t units;       /* points (build) or queries (search) */
    uint64_t bytes;      /* device bytes reserved while it ran */
    double t_submit;     /* seconds on the server's steady clock: submitted, */
    double t_admit;      /* admitted to a slot, */
    double t_done;       /* done */
    char message[128];   /* grnnd_last_error text of a failed request */
} grnnd_request_info;

/* Creates a server on the current device.  cfg: slots 1..64, hbm_budget > 0. */
GRNND_API int grnnd_server_create(const grnnd_server_config *cfg, grnnd_server **out);

/* Queues a build of n x d points (host or device) with params p (copied; p->stream and
 * p->hbm_budget are ignored: the request runs on its slot's stream under the server's
 * budget).  *id_out = the request id = the index id.  Arguments are validated as for
 * grnnd_build_ex before anything is queued. */
GRNND_API int grnnd_server_submit_build(grnnd_server *s, const float *points, int64_t n, int32_t d,
                                        const grnnd_params *p, int64_t *id_out);

/* Queues a search of nq queries (host or device rows of the index's d floats) on index
 * `index` (a build request id, possibly still queued or running); ids_out (host or
 * device, nq x k int32) receives what grnnd_search returns.  1 <= k <= beam <= 256.  A
 * search of an index that failed or was released completes with GRNND_EINVAL. */
GRNND_API int grnnd_server_submit_search(grnnd_server *s, int64_t index, const float *queries, int64_t nq,
                                         int32_t k, int32_t beam, int32_t *ids_out, int64_t *id_out);

/* Waits up to timeout_s seconds (< 0: no limit) for request `id` and fills *info (may be
 * NULL).  Returns the request's status once it is done (and then forgets the request), or
 * GRNND_ETIMEOUT if it is still queued or running (info then holds its current state).
 * An unknown id is GRNND_EINVAL. */
GRNND_API int grnnd_server_wait(grnnd_server *s, int64_t id, double timeout_s, grnnd_request_info *info);

/* The resident graph of a finished build (borrowed: valid until grnnd_server_release or
 * grnnd_server_destroy; do not grnnd_free it).  GRNND_EBUSY while the build is queued or
 * running, GRNND_EINVAL if it failed, was released or is unknown. */
GRNND_API int grnnd_server_index(grnnd_server *s, int64_t index, const grnnd_graph **g);

/* Frees a resident index.  GRNND_EBUSY while its build or a search of it is queued or
 * running. */
GRNND_API int grnnd_server_release(grnnd_server *s, int64_t index);

/* Counters (any pointer may be NULL): device bytes reserved now and at most so far
 * (resident indices + requests in flight), requests queued and running, resident indices. */
GRNND_API int grnnd_server_status(grnnd_server *s, uint64_t *bytes_in_use, uint64_t *peak_bytes,
                                  int32_t *queued, int32_t *running, int32_t *indices);

/* Finishes the requests that are running, fails the queued ones (GRNND_EBUSY), frees
 * every index and the server.  No other call on this server may run concurrently with it
 * or follow it (requests not yet collected by grnnd_server_wait go with the server). */
GRNND_API void grnnd_server_destroy(grnnd_server *s);

/* ------------------------------------------------------------------------- */
/* Step-level entry points on caller-owned device buffers                     */
/* ------------------------------------------------------------------------- */

/* rnd_init (Alg 3, INITIAL_NEIGHBORS): for each vertex v, the first S distinct
 * ids u != v drawn as r = h(seed,0,0,v,j) mod (n-1), u = r + (r >= v), for
 * j = 0, 1, ...; their canonical FP32 distances; the row sorted by key, all
 * entries new.  points: device, n x ld.  keys: device n x R (written in full).
 * deg: device n (written).  h is five chained SplitMix64 steps:
 * h = f(f(f(f(f(seed) ^ t1) ^ t2) ^ v) ^ x). */
GRNND_API int grnnd_pool_init(const float *points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                    int32_t S, int32_t R, uint64_t seed, uint64_t *keys, int32_t *deg,
                    void *stream);

/* Bytes of device workspace that grnnd_join_round and grnnd_reverse_sample
 * need for n vertices with capacity R. */
GRNND_API size_t grnnd_workspace_size(int64_t n, int32_t R);

/* One round of Alg 4: pool_in -> pool_out, i.e. rnd_join (gather + dist_tile +
 * rng_prune + proposal emission) followed by rev_merge (proposal bucketing and
 * per-target top-R selection).  For each vertex v with m = deg_in[v] entries:
 * the entries are visited in order pi (order key h(seed, t1, t2, v, id), ties
 * by id; or ascending / descending key); pairs (pi_a, pi_b), b = 1..m-1,
 * a = 0..b-1, are evaluated unless either side is already bottom or both are
 * old; a pair fires when d(a,b) < max(d(v,a), d(v,b)) (Eq 2), making the entry
 * with the larger (dist, id) bottom and proposing it to the other one with
 * distance d(a,b); every survivor is proposed back to v as old.  pool_out[u] =
 * the R smallest keys among the distinct ids proposed to u (a duplicate keeps
 * its smallest distance and is old if any copy is old).  Buffers are device
 * memory.  keys_out/deg_out either are separate buffers (Sec 3.5 double
 * buffer: the caller swaps the two pools afterwards, which is pool_swap) or
 * alias keys_in/deg_in exactly (in-place update: each vertex rewrites its own
 * row and only rows that receive proposals are merged).
 * stats (optional, device int64[8], accumulated): [0] vertices with new
 * entries, [1] rows gathered, [2] pair distances, [3] pairs fired,
 * [4] proposals (every pool entry, proposed explicitly or kept in place),
 * [5] new entries in pool_out, [6] redirects merged. */
GRNND_API int grnnd_join_round(const float *points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                     int32_t R, const uint64_t *keys_in, const int32_t *deg_in, uint64_t seed,
                     int32_t t1, int32_t t2, int32_t order, uint64_t *keys_out, int32_t *deg_out,
                     void *workspace, size_t workspace_bytes, int64_t *stats, void *stream);

/* Quantized copy of the points for the precision forms of the step calls (the
 * build calls make their own).  The paper states no precision (Sec 3.4 computes
 * FP32 distances); these are the BF16 / FP8 forms of the dist_tile step of
 * Alg 5 / Eq 2 that grnnd_precision describes.  grnnd_quantized_size returns
 * the bytes of the copy of n x d points in `precision` (GRNND_BF16 or
 * GRNND_FP8; 0 for anything else): rows rounded once to bfloat16 (round to
 * nearest even) or to e4m3 with one power-of-two scale per row, per-row
 * (squared norm of the rounded row, norm of the rounding residual) terms and
 * two dataset flags; the layout is private to the library.  grnnd_quantize
 * writes it from `points` (device n x ld floats, as for grnnd_join_round) into
 * `qpoints` (device, 256-byte aligned, >= grnnd_quantized_size bytes), which
 * the caller owns; asynchronous on `stream`.  GRNND_EINVAL for a bad
 * precision, size or alignment. */
GRNND_API size_t grnnd_quantized_size(int64_t n, int32_t d, int32_t precision);
GRNND_API int grnnd_quantize(const float *points, int64_t n, int32_t d, int32_t ld, int32_t precision,
                             void *qpoints, size_t qpoints_bytes, void *stream);

/* grnnd_join_round in a precision form: the pair distances of the prune (Eq 2)
 * come from the quantized tiles of `qpoints` (written by grnnd_quantize for
 * the same points and precision), with every decision inside the tiles' error
 * bound re-taken with the canonical FP32 distance of `points`, as in the
 * builds.  precision GRNND_FP32 ignores qpoints (NULL allowed) and equals
 * grnnd_join_round.  Other arguments, results and errors as for
 * grnnd_join_round. */
GRNND_API int grnnd_join_round_q(const float *points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                                 int32_t precision, const void *qpoints, size_t qpoints_bytes, int32_t R,
                                 const uint64_t *keys_in, const int32_t *deg_in, uint64_t seed,
                                 int32_t t1, int32_t t2, int32_t order, uint64_t *keys_out,
                                 int32_t *deg_out, void *workspace, size_t workspace_bytes,
                                 int64_t *stats, void *stream);

/* Reverse-edge sampling (Sec 3.6): for each v with k = deg_in[v], the first
 * floor((double)rho * k) entries n of its row propose (v, d(v,n), new) to n;
 * pool_out[u] = merge of pool_in[u] with the proposals to u (same rule as the
 * round).  0 <= rho <= 1.  The output may alias the input (in place). */
GRNND_API int grnnd_reverse_sample(int64_t n, int32_t R, float rho, const uint64_t *keys_in,
                         const int32_t *deg_in, uint64_t *keys_out, int32_t *deg_out,
                         void *workspace, size_t workspace_bytes, int64_t *stats, void *stream);

/* Status of the last step (grnnd_join_round, grnnd_reverse_sample or
 * grnnd_final_prune) that used this workspace, for the same n and R.  Each step
 * clears the workspace's status word when it starts; a device-side wait of the
 * step that reaches its iteration limit sets it, and the rest of that step then
 * does nothing: its output pool is incomplete (rows of vertices that were not
 * reached keep their input when the step runs in place, and are unspecified
 * otherwise).  Synchronises `stream`.  Returns GRNND_OK, GRNND_ETIMEOUT, or
 * GRNND_EINVAL / GRNND_ECUDA.  The paper has no counterpart: it is the error
 * channel of the bounded waits. */
GRNND_API int grnnd_workspace_status(const void *workspace, size_t workspace_bytes, int64_t n,
                                     int32_t R, void *stream);

/* Self-test of the device-side failure detection (no counterpart in the paper): one thread
 * waits, with the bounded mbarrier wait of the join kernels, on a barrier that nothing
 * completes; after `limit` tries (1 <= limit <= 2^20; each try is a hardware-timed
 * try_wait) it gives up and records the timeout in a status word, which this call reads.
 * Returns GRNND_ETIMEOUT (the expected outcome), never faults or hangs, copies nothing, and
 * leaves the context usable.  Synchronises `stream`. */
GRNND_API int grnnd_selftest_bounded_wait(uint32_t limit, void *stream);

/* Final prune-only pass: the prune of a round with order key t1 (t2 = 0),
 * keeping only each vertex's survivors, in key order; no redirects.
 * keys_out: device n x R (written in full, must not alias keys_in), deg_out:
 * device n; workspace as for grnnd_join_round. */
GRNND_API int grnnd_final_prune(const float *points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                      int32_t R, const uint64_t *keys_in, const int32_t *deg_in, uint64_t seed,
                      int32_t t1, int32_t order, uint64_t *keys_out, int32_t *deg_out,
                      void *workspace, size_t workspace_bytes, void *stream);

/* grnnd_final_prune in a precision form (qpoints and precision as for
 * grnnd_join_round_q). */
GRNND_API int grnnd_final_prune_q(const float *points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                                  int32_t precision, const void *qpoints, size_t qpoints_bytes, int32_t R,
                                  const uint64_t *keys_in, const int32_t *deg_in, uint64_t seed,
                                  int32_t t1, int32_t order, uint64_t *keys_out, int32_t *deg_out,
                                  void *workspace, size_t workspace_bytes, void *stream);

/* Canonical FP32 distances of np point pairs: out[i] = d(points[pairs[2i]],
 * points[pairs[2i+1]]) exactly as the pool kernels compute it.  pairs: device
 * int32 (np x 2), out: device float32 (np). */
GRNND_API int grnnd_pair_dist(const float *points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                    const int32_t *pairs, int64_t np, float *out, void *stream);

/* Search entry (reading C13 of the design notes): the id of the point nearest
 * the dataset mean, ties to the smaller id, computed in FP64.  entry_out:
 * device int32[1].  workspace: device, >= grnnd_entry_workspace_size(n, d). */
GRNND_API size_t grnnd_entry_workspace_size(int64_t n, int32_t d);
GRNND_API int grnnd_entry_point(const float *points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                      int32_t *entry_out, void *workspace, size_t workspace_bytes, void *stream);

/* Candidate-list search on a caller-provided graph: gids device n x R int32
 * (-1 padded), gdeg device n; queries device nq x ldq; ids_out device nq x k
 * (-1 padded), dists_out device nq x k (may be NULL).  entry: a vertex id. */
GRNND_API int grnnd_search_graph(const float *points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                       const int32_t *gids, const int32_t *gdeg, int32_t R, int32_t entry,
                       const float *queries, int64_t nq, int32_t ldq, int32_t k, int32_t beam,
                       int32_t *ids_out, float *dists_out, void *stream);

/* Exact k nearest neighbours by (canonical FP32 dist, id) — the ground truth
 * of Recall@k (Sec 2.1).  Device buffers; 1 <= k <= 32. */
GRNND_API int grnnd_brute_knn(const float *points, int64_t n, int32_t d, int32_t ld, int32_t metric,
                    const float *queries, int64_t nq, int32_t ldq, int32_t k, int32_t *ids_out,
                    float *dists_out, void *stream);

/* Converts pool keys to (ids, dists): ids n x R int32 (-1 for empty),
 * dists n x R float32 (+inf for empty).  Device buffers. */
GRNND_API int grnnd_keys_to_graph(int64_t n, int32_t R, const uint64_t *keys, int32_t *ids, float *dists,
                        void *stream);

/* Search entry without device allocation.  The paper has no counterpart: this
 * is a library service for callers that may not allocate device memory when
 * they need the entry point (an application that owns all GPU memory through
 * its own arena, a latency-critical loop that must not pay cudaMalloc's
 * implicit synchronisation, a plugin given buffers but no allocator).  Same
 * result as grnnd_entry_point; the scratch is one fixed device array of
 * 4,208,640 bytes inside the library (held on every GPU that loads it until
 * exit), so 1 <= d <= 1024 (larger d returns GRNND_EINVAL).  No cudaMalloc or
 * cudaFree is called.  The first call on a device looks up the array's address
 * with that device current and remembers it with the current context's id; a
 * call under a new context (after cudaDeviceReset) looks it up again.  Make the
 * first call, and the first after a reset, before any stream capture.  All calls on a
 * device share the array: calls that overlap on the GPU race, so order them on
 * one stream.  points: device n x ld (16-byte aligned, ld % 4 == 0);
 * entry_out: device int32[1]. */
GRNND_API int grnnd_entry_point_noalloc(const float *points, int64_t n, int32_t d, int32_t ld,
                                        int32_t metric, int32_t *entry_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GRNND_H */
