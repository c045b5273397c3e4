/*
 * The FP64 oracle's build (orc_build in grnnd_oracle.c) on several host threads.
 *
 * TEST INFRASTRUCTURE ONLY: the CPU-baseline leg of the benchmark times the oracle on all
 * host cores with it, and the test suite checks that it returns orc_build's graph bit for
 * bit at any thread count.  It shares nothing with the CUDA library.
 *
 * No arithmetic of the method is restated here.  Every step calls the oracle's own
 * functions in the order orc_build does (Alg 3): orc_init, then per round (Alg 4 with
 * Eq 2) orc_visit_order + orc_prune for every vertex and orc_merge of the proposals (the
 * merge rule of Sec 3.5 / C6), reverse sampling (Sec 3.6) as proposals + orc_merge, and the
 * final prune-only pass (C11).  What runs on several threads:
 *   - the per-vertex prunes of a round or of the final pass: vertices are split into
 *     contiguous ranges, one per thread; each vertex's proposals go to its own slots;
 *   - the merges: the targets are split into contiguous ranges, and each thread merges the
 *     proposals addressed to its range with orc_merge (targets rebased to the range), since
 *     the merge of one target never looks at another target's proposals.
 * orc_init stays single-threaded (its draws use the global vertex count).  The results are
 * the same at any thread count: every random choice is counter-based (C9), and each target's
 * merged pool depends only on the set of proposals addressed to it.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* the oracle's own entry points (grnnd_oracle.c) */
int orc_init(const float *X, int64_t n, int32_t d, int32_t metric, int32_t S, int32_t R,
             uint64_t seed, double tol, int32_t *ids, double *dist, uint8_t *old, int32_t *deg,
             uint8_t *flags);
void orc_visit_order(uint64_t seed, int32_t t1, int32_t t2, int64_t v, int32_t m,
                     const int32_t *ids, int32_t order, int32_t *perm);
int orc_prune(const float *X, int32_t d, int32_t metric, int32_t m, const int32_t *ids,
              const double *dist, const uint8_t *old, const int32_t *perm, int32_t skip_old,
              double tol, uint8_t *alive, int32_t *killer, double *kdist, int64_t *n_eval);
int orc_merge(int64_t n, int32_t R, int64_t np, const int32_t *target, const int32_t *id,
              const double *dist, const uint8_t *old, int32_t *ids_out, double *dist_out,
              uint8_t *old_out, int32_t *deg_out);

#define MT_EINVAL (-1)
#define MT_ENOMEM (-2)

/* Proposals in slots: slot v * W + i belongs to vertex v (target < 0: unused). */
typedef struct {
    int32_t *tgt, *id;
    double *dist;
    uint8_t *old;
    int64_t cap;
} props_t;

typedef struct {
    /* inputs */
    const float *X;
    int64_t n;
    int32_t d, metric, R, order, skip_old;
    uint64_t seed;
    int32_t t1, t2;
    float rho;
    const int32_t *ids;
    const double *dist;
    const uint8_t *old;
    const int32_t *deg;
    /* outputs */
    props_t *P;             /* per-vertex proposals (rounds, reverse) */
    int32_t *gids;          /* final pass: survivors */
    double *gdist;
    int32_t *gdeg;
    int32_t *ids_out;       /* merge */
    double *dist_out;
    uint8_t *old_out;
    int32_t *deg_out;
    /* work split */
    int64_t a, b;           /* vertex or target range */
    int kind;               /* 0 prune of a round, 1 final prune, 2 reverse proposals, 3 merge */
    int rc;
    int64_t n_eval, n_fire;
} job_t;

/* One round's prunes of vertices [a, b): orc_round's vertex loop. */
static void prune_range(job_t *j)
{
    int32_t perm[1024], killer[1024];
    uint8_t alive[1024];
    double kdist[1024];
    const int32_t R = j->R;
    for (int64_t v = j->a; v < j->b; ++v) {
        const int32_t m = j->deg[v];
        const int32_t *row = j->ids + v * R;
        const double *drow = j->dist + v * R;
        const uint8_t *orow = j->old + v * R;
        orc_visit_order(j->seed, j->t1, j->t2, v, m, row, j->order, perm);
        orc_prune(j->X, j->d, j->metric, m, row, drow, orow, perm, j->skip_old, 0.0, alive, killer,
                  kdist, &j->n_eval);
        for (int32_t i = 0; i < R; ++i) {
            const int64_t s = v * R + i;
            if (i >= m) {
                j->P->tgt[s] = -1;
                continue;
            }
            if (alive[i]) { /* survivor: back into pool2[v], marked old */
                j->P->tgt[s] = (int32_t)v;
                j->P->id[s] = row[i];
                j->P->dist[s] = drow[i];
                j->P->old[s] = 1;
            } else { /* redirect n_far into pool2[n_close] (Eq 2) */
                j->P->tgt[s] = row[killer[i]];
                j->P->id[s] = row[i];
                j->P->dist[s] = kdist[i];
                j->P->old[s] = 0;
                ++j->n_fire;
            }
        }
    }
}

/* The final prune of vertices [a, b): orc_final_prune's vertex loop. */
static void final_range(job_t *j)
{
    int32_t perm[1024], killer[1024];
    uint8_t alive[1024];
    double kdist[1024];
    const int32_t R = j->R;
    for (int64_t v = j->a; v < j->b; ++v) {
        const int32_t m = j->deg[v];
        const int32_t *row = j->ids + v * R;
        const double *drow = j->dist + v * R;
        orc_visit_order(j->seed, j->t1, 0, v, m, row, j->order, perm);
        orc_prune(j->X, j->d, j->metric, m, row, drow, j->old + v * R, perm, j->skip_old, 0.0, alive,
                  killer, kdist, NULL);
        int32_t c = 0;
        for (int32_t i = 0; i < m; ++i)
            if (alive[i]) {
                j->gids[v * R + c] = row[i];
                j->gdist[v * R + c] = drow[i];
                ++c;
            }
        for (int32_t i = c; i < R; ++i) {
            j->gids[v * R + i] = -1;
            j->gdist[v * R + i] = INFINITY;
        }
        j->gdeg[v] = c;
    }
}

/* Reverse sampling proposals of vertices [a, b): orc_reverse's proposal loop (each vertex's
 * own pool, then its first floor(rho * k) entries proposing v back), two slots per entry. */
static void reverse_range(job_t *j)
{
    const int32_t R = j->R;
    for (int64_t v = j->a; v < j->b; ++v) {
        const int32_t k = j->deg[v];
        const int32_t r = (int32_t)floor((double)j->rho * (double)k);
        for (int32_t i = 0; i < R; ++i) {
            const int64_t s = (v * R + i) * 2;
            j->P->tgt[s] = j->P->tgt[s + 1] = -1;
            if (i >= k)
                continue;
            j->P->tgt[s] = (int32_t)v;
            j->P->id[s] = j->ids[v * R + i];
            j->P->dist[s] = j->dist[v * R + i];
            j->P->old[s] = j->old[v * R + i];
            if (i < r) {
                j->P->tgt[s + 1] = j->ids[v * R + i];
                j->P->id[s + 1] = (int32_t)v;
                j->P->dist[s + 1] = j->dist[v * R + i];
                j->P->old[s + 1] = 0;
            }
        }
    }
}

/* Merge of the proposals addressed to targets [a, b), with the oracle's merge. */
static void merge_range(job_t *j)
{
    if (j->b <= j->a)
        return;
    int64_t np = 0;
    for (int64_t s = 0; s < j->P->cap; ++s)
        np += (j->P->tgt[s] >= j->a && j->P->tgt[s] < j->b);
    int32_t *t = (int32_t *)malloc((size_t)(np > 0 ? np : 1) * sizeof(int32_t));
    int32_t *id = (int32_t *)malloc((size_t)(np > 0 ? np : 1) * sizeof(int32_t));
    double *dd = (double *)malloc((size_t)(np > 0 ? np : 1) * sizeof(double));
    uint8_t *od = (uint8_t *)malloc((size_t)(np > 0 ? np : 1));
    if (!t || !id || !dd || !od) {
        j->rc = MT_ENOMEM;
    } else {
        int64_t q = 0;
        for (int64_t s = 0; s < j->P->cap; ++s) {
            const int32_t g = j->P->tgt[s];
            if (g >= j->a && g < j->b) {
                t[q] = (int32_t)(g - j->a);
                id[q] = j->P->id[s];
                dd[q] = j->P->dist[s];
                od[q] = j->P->old[s];
                ++q;
            }
        }
        const int64_t R = j->R;
        j->rc = orc_merge(j->b - j->a, j->R, np, t, id, dd, od, j->ids_out + j->a * R, j->dist_out + j->a * R,
                          j->old_out + j->a * R, j->deg_out + j->a);
    }
    free(t);
    free(id);
    free(dd);
    free(od);
}

static void *run_job(void *arg)
{
    job_t *j = (job_t *)arg;
    switch (j->kind) {
    case 0: prune_range(j); break;
    case 1: final_range(j); break;
    case 2: reverse_range(j); break;
    default: merge_range(j); break;
    }
    return NULL;
}

/* Runs `kind` over [0, n) split into `threads` contiguous ranges; returns the first error. */
static int run_split(job_t *base, int kind, int threads, int64_t *n_eval, int64_t *n_fire)
{
    pthread_t th[256];
    job_t jobs[256];
    int started[256];
    const int64_t n = base->n;
    for (int i = 0; i < threads; ++i) {
        jobs[i] = *base;
        jobs[i].kind = kind;
        jobs[i].a = n * i / threads;
        jobs[i].b = n * (i + 1) / threads;
        jobs[i].rc = 0;
        jobs[i].n_eval = jobs[i].n_fire = 0;
        started[i] = pthread_create(&th[i], NULL, run_job, &jobs[i]) == 0;
        if (!started[i])
            run_job(&jobs[i]); /* no thread: run it here */
    }
    int rc = 0;
    for (int i = 0; i < threads; ++i) {
        if (started[i])
            pthread_join(th[i], NULL);
        if (jobs[i].rc && !rc)
            rc = jobs[i].rc;
        if (n_eval)
            *n_eval += jobs[i].n_eval;
        if (n_fire)
            *n_fire += jobs[i].n_fire;
    }
    return rc;
}

/* orc_build on `threads` host threads (1..256); same arguments and results as orc_build. */
int orc_build_mt(const float *X, int64_t n, int32_t d, int32_t metric, int32_t S, int32_t R,
                 int32_t T1, int32_t T2, float rho, uint64_t seed, int32_t order, int32_t skip_old,
                 int32_t final_prune, int32_t threads, int32_t *gids, double *gdist, int32_t *gdeg,
                 int64_t *stats)
{
    if (T1 < 1 || T2 < 1 || R > 1024 || threads < 1 || threads > 256)
        return MT_EINVAL;
    const size_t slots = (size_t)(n * R);
    int32_t *ia = (int32_t *)malloc(slots * sizeof(int32_t)), *ib = (int32_t *)malloc(slots * sizeof(int32_t));
    double *da = (double *)malloc(slots * sizeof(double)), *db = (double *)malloc(slots * sizeof(double));
    uint8_t *oa = (uint8_t *)malloc(slots), *ob = (uint8_t *)malloc(slots);
    int32_t *ga = (int32_t *)malloc((size_t)n * sizeof(int32_t)), *gb = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    props_t P;
    P.cap = (int64_t)slots * 2;
    P.tgt = (int32_t *)malloc((size_t)P.cap * sizeof(int32_t));
    P.id = (int32_t *)malloc((size_t)P.cap * sizeof(int32_t));
    P.dist = (double *)malloc((size_t)P.cap * sizeof(double));
    P.old = (uint8_t *)malloc((size_t)P.cap);
    int rc = MT_ENOMEM;
    int64_t tot[3] = {0, 0, 0};
    if (!ia || !ib || !da || !db || !oa || !ob || !ga || !gb || !P.tgt || !P.id || !P.dist || !P.old)
        goto done;
    rc = orc_init(X, n, d, metric, S, R, seed, 0.0, ia, da, oa, ga, NULL);
    if (rc)
        goto done;
    job_t base;
    memset(&base, 0, sizeof(base));
    base.X = X;
    base.n = n;
    base.d = d;
    base.metric = metric;
    base.R = R;
    base.order = order;
    base.skip_old = skip_old;
    base.seed = seed;
    base.rho = rho;
    base.P = &P;
    for (int32_t t1 = 1; t1 <= T1; ++t1) {
        for (int32_t t2 = 1; t2 <= T2; ++t2) {
            base.t1 = t1;
            base.t2 = t2;
            base.ids = ia;
            base.dist = da;
            base.old = oa;
            base.deg = ga;
            P.cap = (int64_t)slots;
            int64_t ne = 0, nf = 0;
            rc = run_split(&base, 0, threads, &ne, &nf);
            if (rc)
                goto done;
            base.ids_out = ib;
            base.dist_out = db;
            base.old_out = ob;
            base.deg_out = gb;
            rc = run_split(&base, 3, threads, NULL, NULL);
            if (rc)
                goto done;
            int64_t np = 0;
            for (int64_t v = 0; v < n; ++v)
                np += ga[v];
            tot[0] += ne;
            tot[1] += nf;
            tot[2] += np;
            int32_t *ti = ia; ia = ib; ib = ti;
            double *td = da; da = db; db = td;
            uint8_t *to = oa; oa = ob; ob = to;
            int32_t *tg = ga; ga = gb; gb = tg;
        }
        if (t1 != T1) {
            base.ids = ia;
            base.dist = da;
            base.old = oa;
            base.deg = ga;
            P.cap = (int64_t)slots * 2;
            rc = run_split(&base, 2, threads, NULL, NULL);
            if (rc)
                goto done;
            base.ids_out = ib;
            base.dist_out = db;
            base.old_out = ob;
            base.deg_out = gb;
            rc = run_split(&base, 3, threads, NULL, NULL);
            if (rc)
                goto done;
            int32_t *ti = ia; ia = ib; ib = ti;
            double *td = da; da = db; db = td;
            uint8_t *to = oa; oa = ob; ob = to;
            int32_t *tg = ga; ga = gb; gb = tg;
        }
    }
    if (final_prune) {
        base.t1 = T1 + 1;
        base.ids = ia;
        base.dist = da;
        base.old = oa;
        base.deg = ga;
        base.gids = gids;
        base.gdist = gdist;
        base.gdeg = gdeg;
        rc = run_split(&base, 1, threads, NULL, NULL);
    } else {
        memcpy(gids, ia, slots * sizeof(int32_t));
        memcpy(gdist, da, slots * sizeof(double));
        memcpy(gdeg, ga, (size_t)n * sizeof(int32_t));
    }
    if (stats)
        for (int i = 0; i < 3; ++i)
            stats[i] = tot[i];
done:
    free(ia); free(ib); free(da); free(db); free(oa); free(ob); free(ga); free(gb);
    free(P.tgt); free(P.id); free(P.dist); free(P.old);
    return rc;
}
