/*
 * GRNND oracle: a plain, single-threaded, FP64 CPU statement of the
 * Relative NN-Descent build in the GRNND paper (arXiv 2510.02774).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
 * CUDA library.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or helper
 * with the CUDA path, and the CUDA path never calls it.
 *
 * Every step follows the paper's order and notation:
 *   - initialisation with S random neighbours ........ Alg 3 (INITIAL_NEIGHBORS)
 *   - one round of disordered propagation ............. Alg 4 with Eq 2
 *   - fixed-capacity double-buffered pools ............ Sec 3.5
 *   - reverse-edge sampling with ratio rho ............ Sec 3.6, Alg 3
 *   - the serial ascending update, as a special case .. Alg 2
 *   - recall@k and the candidate-list search .......... Sec 2.1, Sec 4.2
 *
 * Readings of points the paper leaves open (each one is listed with its
 * reason in the design notes of the repository):
 *   C3  "random neighbour pairs" = every unordered pair of the pool, visited
 *       as (pi_a, pi_b) for b = 1..m-1, a = 0..b-1, where pi sorts the pool by
 *       the counter hash h(seed, t1, t2, v, id) (ties by id).  With pi equal to
 *       the ascending (dist, id) order this is exactly Alg 2's greedy.
 *   C4  a pair in which either side is already marked "bottom" is skipped.
 *   C5  fire rule is strict: d(ni,nj) < max(d(v,ni), d(v,nj)) (Eq 2, Alg 4);
 *       close = smaller (d(v,.), id), far = the other.
 *   C6  pool2[u] = the R smallest (dist, id) among the distinct ids proposed
 *       to u; a duplicate id keeps its smallest distance and is "old" if any
 *       copy is old.  This is the order-free end state of WARP_INSERT (Alg 6).
 *   C7  reverse sampling takes the first floor(rho * deg(v)) entries of v's
 *       pool in (dist, id) order and proposes v to each of them.
 *   C8  L2 metric = squared Euclidean distance (Alg 5 returns the root; the
 *       square is monotone so every decision is the same); IP = 1 - <x, y>.
 *   C9  counter hash h = five chained SplitMix64 steps (Steele, Lea, Flood,
 *       OOPSLA 2014): h = f(f(f(f(f(seed) ^ t1) ^ t2) ^ v) ^ x) where
 *       f(z) is one SplitMix64 output for state z.
 *   C10 pairs whose two entries are both "old" (both survived v's previous
 *       prune together) may be skipped; the result does not change.
 *   C11 the returned graph is either the last pool or, with final_prune, the
 *       survivors of one more prune pass (order key t1 = T1 + 1, t2 = 0).
 *   C13 search enters at the point nearest the dataset mean (by (dist, id)).
 *
 * Build with -ffp-contract=off so that no multiply-add is fused: the results
 * are then identical on every IEEE-754 host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* ------------------------------------------------------------------------- */
/* C9: counter-based hash from the published SplitMix64 step                  */
/* ------------------------------------------------------------------------- */

/* One SplitMix64 output for state z: advance by the golden gamma, then the
 * 64-bit finaliser (shifts 30/27/31, the two published odd multipliers). */
uint64_t orc_splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_hash(uint64_t seed, uint64_t t1, uint64_t t2, uint64_t v, uint64_t x)
{
    uint64_t h = orc_splitmix64(seed);
    h = orc_splitmix64(h ^ t1);
    h = orc_splitmix64(h ^ t2);
    h = orc_splitmix64(h ^ v);
    h = orc_splitmix64(h ^ x);
    return h;
}

/* ------------------------------------------------------------------------- */
/* C8: distance d(x, y) in FP64                                               */
/* ------------------------------------------------------------------------- */

double orc_dist(const float *x, const float *y, int32_t d, int32_t metric)
{
    double s = 0.0;
    if (metric == 0) {
        for (int32_t k = 0; k < d; ++k) {
            double t = (double)x[k] - (double)y[k];
            s += t * t;
        }
        return s;
    }
    for (int32_t k = 0; k < d; ++k)
        s += (double)x[k] * (double)y[k];
    return 1.0 - s;
}

static int near_tie(double a, double b, double tol)
{
    if (tol <= 0.0)
        return 0;
    double m = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    if (m < 1.0)
        m = 1.0;
    return fabs(a - b) <= tol * m;
}

/* (dist, id) lexicographic "less than" */
static int dl_less(double da, int32_t ia, double db, int32_t ib)
{
    return da < db || (da == db && ia < ib);
}

/* ------------------------------------------------------------------------- */
/* Alg 3, INITIAL_NEIGHBORS: S distinct random ids != v, sorted by (dist,id)  */
/* ------------------------------------------------------------------------- */

/* Pools are flat arrays of n*R slots.  Row v holds deg[v] entries sorted by
 * (dist, id); empty slots have id -1, dist +inf, old 0. */
static void clear_row(int32_t *ids, double *dist, uint8_t *old, int32_t R, int32_t from)
{
    for (int32_t j = from; j < R; ++j) {
        ids[j] = -1;
        dist[j] = INFINITY;
        old[j] = 0;
    }
}

/* insertion sort of a row by (dist, id); returns 1 if two adjacent distances
 * of different ids are within tol (an ordering that FP32 may flip). */
static int sort_row(int32_t *ids, double *dist, uint8_t *old, int32_t m, double tol)
{
    for (int32_t i = 1; i < m; ++i) {
        int32_t id = ids[i];
        double ds = dist[i];
        uint8_t o = old[i];
        int32_t j = i - 1;
        while (j >= 0 && dl_less(ds, id, dist[j], ids[j])) {
            ids[j + 1] = ids[j];
            dist[j + 1] = dist[j];
            old[j + 1] = old[j];
            --j;
        }
        ids[j + 1] = id;
        dist[j + 1] = ds;
        old[j + 1] = o;
    }
    int flag = 0;
    for (int32_t i = 1; i < m; ++i)
        if (near_tie(dist[i - 1], dist[i], tol))
            flag = 1;
    return flag;
}

int orc_init(const float *X, int64_t n, int32_t d, int32_t metric, int32_t S, int32_t R,
             uint64_t seed, double tol, int32_t *ids, double *dist, uint8_t *old, int32_t *deg,
             uint8_t *flags)
{
    if (n < 2 || d < 1 || S < 1 || R < S || (int64_t)S > n - 1)
        return ORC_EINVAL;
    for (int64_t v = 0; v < n; ++v) {
        int32_t *row = ids + v * R;
        double *drow = dist + v * R;
        uint8_t *orow = old + v * R;
        int32_t cnt = 0;
        for (uint64_t k = 0; cnt < S; ++k) {
            uint64_t r = orc_hash(seed, 0, 0, (uint64_t)v, k) % (uint64_t)(n - 1);
            int32_t u = (int32_t)(r + (r >= (uint64_t)v ? 1 : 0));
            int dup = 0;
            for (int32_t j = 0; j < cnt; ++j)
                if (row[j] == u)
                    dup = 1;
            if (dup)
                continue;
            row[cnt] = u;
            drow[cnt] = orc_dist(X + v * d, X + (int64_t)u * d, d, metric);
            orow[cnt] = 0;
            ++cnt;
        }
        int f = sort_row(row, drow, orow, S, tol);
        clear_row(row, drow, orow, R, S);
        deg[v] = S;
        if (flags)
            flags[v] = (uint8_t)(f ? 1 : 0);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* C3: visit order pi of one pool                                             */
/* ------------------------------------------------------------------------- */

/* order 0 = disordered (hash), 1 = ascending (dist, id), 2 = descending. */
void orc_visit_order(uint64_t seed, int32_t t1, int32_t t2, int64_t v, int32_t m,
                     const int32_t *ids, int32_t order, int32_t *perm)
{
    for (int32_t i = 0; i < m; ++i)
        perm[i] = (order == 2) ? (m - 1 - i) : i;
    if (order != 0)
        return;
    uint64_t hk[1024];
    for (int32_t i = 0; i < m; ++i)
        hk[i] = orc_hash(seed, (uint64_t)t1, (uint64_t)t2, (uint64_t)v, (uint64_t)ids[i]);
    for (int32_t i = 1; i < m; ++i) {
        int32_t p = perm[i];
        int32_t j = i - 1;
        while (j >= 0 && (hk[p] < hk[perm[j]] || (hk[p] == hk[perm[j]] && ids[p] < ids[perm[j]]))) {
            perm[j + 1] = perm[j];
            --j;
        }
        perm[j + 1] = p;
    }
}

/* ------------------------------------------------------------------------- */
/* Eq 2 / Alg 4: the prune of one vertex's pool in a given visit order       */
/* ------------------------------------------------------------------------- */

/* Inputs: the m entries of pool1[v] (ids, d(v, .), old flags) and the visit
 * order perm.  Outputs per entry i: alive[i] = 1 if it survives; otherwise
 * killer[i] = the entry index of n_close that absorbs it and kdist[i] =
 * d(n_close, n_far).  Returns 1 if any evaluated comparison was within tol
 * (a decision that FP32 arithmetic could take the other way), else 0. */
int orc_prune(const float *X, int32_t d, int32_t metric, int32_t m, const int32_t *ids,
              const double *dist, const uint8_t *old, const int32_t *perm, int32_t skip_old,
              double tol, uint8_t *alive, int32_t *killer, double *kdist, int64_t *n_eval)
{
    int flagged = 0;
    for (int32_t i = 0; i < m; ++i) {
        alive[i] = 1;
        killer[i] = -1;
        kdist[i] = 0.0;
    }
    for (int32_t b = 1; b < m; ++b) {
        for (int32_t a = 0; a < b; ++a) {
            int32_t A = perm[a], B = perm[b];
            if (!alive[A] || !alive[B])
                continue; /* C4 */
            if (skip_old && old[A] && old[B])
                continue; /* C10 */
            double dab = orc_dist(X + (int64_t)ids[A] * d, X + (int64_t)ids[B] * d, d, metric);
            double mx = dist[A] > dist[B] ? dist[A] : dist[B];
            if (n_eval)
                ++*n_eval;
            if (near_tie(dab, mx, tol))
                flagged = 1;
            if (dab < mx) { /* Eq 2 fires */
                if (near_tie(dist[A], dist[B], tol))
                    flagged = 1;
                int a_close = dl_less(dist[A], ids[A], dist[B], ids[B]);
                int32_t cl = a_close ? A : B, fa = a_close ? B : A;
                alive[fa] = 0;
                killer[fa] = cl;
                kdist[fa] = dab;
            }
        }
    }
    return flagged;
}

/* ------------------------------------------------------------------------- */
/* C6: merge of proposals into fixed-capacity pools (Alg 6 end state)         */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t target, id;
    double dist;
    uint8_t old;
} orc_prop;

static int prop_cmp(const void *pa, const void *pb)
{
    const orc_prop *a = (const orc_prop *)pa, *b = (const orc_prop *)pb;
    if (a->target != b->target)
        return a->target < b->target ? -1 : 1;
    if (a->dist != b->dist)
        return a->dist < b->dist ? -1 : 1;
    if (a->id != b->id)
        return a->id < b->id ? -1 : 1;
    return (int)b->old - (int)a->old; /* old copies first */
}

/* Writes pools for every target 0..n-1 (targets with no proposal get deg 0).
 * flags (optional): bit 1 set for a target whose R-th and (R+1)-th distinct
 * keys are within tol. */
static int merge_props(orc_prop *P, int64_t np, int64_t n, int32_t R, double tol, int32_t *ids,
                       double *dist, uint8_t *old, int32_t *deg, uint8_t *flags)
{
    qsort(P, (size_t)np, sizeof(orc_prop), prop_cmp);
    int32_t *seen = NULL;
    int64_t seen_cap = 0;
    int64_t s = 0;
    for (int64_t u = 0; u < n; ++u) {
        int32_t *row = ids + u * R;
        double *drow = dist + u * R;
        uint8_t *orow = old + u * R;
        int64_t e = s;
        while (e < np && P[e].target == u)
            ++e;
        if (e - s > seen_cap) {
            seen_cap = 2 * (e - s);
            free(seen);
            seen = (int32_t *)malloc((size_t)seen_cap * sizeof(int32_t));
            if (!seen)
                return ORC_ENOMEM;
        }
        int64_t nseen = 0;
        int32_t cnt = 0;
        double next_dist = INFINITY;
        int has_next = 0;
        for (int64_t j = s; j < e; ++j) {
            int64_t q = -1;
            for (int64_t t = 0; t < nseen; ++t)
                if (seen[t] == P[j].id) {
                    q = t;
                    break;
                }
            if (q >= 0) {
                if (q < cnt && P[j].old)
                    orow[q] = 1; /* old if any copy is old */
                continue;
            }
            seen[nseen++] = P[j].id;
            if (cnt < R) {
                row[cnt] = P[j].id;
                drow[cnt] = P[j].dist;
                orow[cnt] = P[j].old;
                ++cnt;
            } else if (!has_next) {
                has_next = 1;
                next_dist = P[j].dist;
            }
        }
        clear_row(row, drow, orow, R, cnt);
        deg[u] = cnt;
        if (flags && has_next && near_tie(drow[R - 1], next_dist, tol))
            flags[u] |= 2;
        s = e;
    }
    free(seen);
    return ORC_OK;
}

/* The merge on its own, for proposals given as parallel arrays. */
int orc_merge(int64_t n, int32_t R, int64_t np, const int32_t *target, const int32_t *id,
              const double *dist, const uint8_t *old, int32_t *ids_out, double *dist_out,
              uint8_t *old_out, int32_t *deg_out)
{
    if (n < 1 || R < 1 || np < 0)
        return ORC_EINVAL;
    orc_prop *P = (orc_prop *)malloc((size_t)(np > 0 ? np : 1) * sizeof(orc_prop));
    if (!P)
        return ORC_ENOMEM;
    for (int64_t i = 0; i < np; ++i) {
        if (target[i] < 0 || target[i] >= n) {
            free(P);
            return ORC_EINVAL;
        }
        P[i].target = target[i];
        P[i].id = id[i];
        P[i].dist = dist[i];
        P[i].old = old[i];
    }
    int rc = merge_props(P, np, n, R, 0.0, ids_out, dist_out, old_out, deg_out, NULL);
    free(P);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Alg 4: one round, pool1 -> pool2, for every vertex                         */
/* ------------------------------------------------------------------------- */

/* stats (optional, 3 counters): pairs evaluated, pairs fired, proposals. */
int orc_round(const float *X, int64_t n, int32_t d, int32_t metric, int32_t R,
              const int32_t *ids, const double *dist, const uint8_t *old, const int32_t *deg,
              uint64_t seed, int32_t t1, int32_t t2, int32_t order, int32_t skip_old, double tol,
              int32_t *ids_out, double *dist_out, uint8_t *old_out, int32_t *deg_out,
              uint8_t *flags, int64_t *stats)
{
    if (n < 2 || R < 1 || R > 1024)
        return ORC_EINVAL;
    orc_prop *P = (orc_prop *)malloc((size_t)(n * R) * sizeof(orc_prop));
    if (!P)
        return ORC_ENOMEM;
    int32_t perm[1024], killer[1024];
    uint8_t alive[1024];
    double kdist[1024];
    int64_t np = 0, n_eval = 0, n_fire = 0;
    if (flags)
        memset(flags, 0, (size_t)n);
    for (int64_t v = 0; v < n; ++v) {
        int32_t m = deg[v];
        const int32_t *row = ids + v * R;
        const double *drow = dist + v * R;
        const uint8_t *orow = old + v * R;
        orc_visit_order(seed, t1, t2, v, m, row, order, perm);
        int f = orc_prune(X, d, metric, m, row, drow, orow, perm, skip_old, tol, alive, killer,
                          kdist, &n_eval);
        if (flags && f)
            flags[v] |= 1;
        for (int32_t i = 0; i < m; ++i) {
            orc_prop p;
            if (alive[i]) { /* survivor: back into pool2[v], marked old */
                p.target = (int32_t)v;
                p.id = row[i];
                p.dist = drow[i];
                p.old = 1;
            } else { /* redirect n_far into pool2[n_close] (Eq 2) */
                p.target = row[killer[i]];
                p.id = row[i];
                p.dist = kdist[i];
                p.old = 0;
                ++n_fire;
            }
            P[np++] = p;
        }
    }
    int rc = merge_props(P, np, n, R, tol, ids_out, dist_out, old_out, deg_out, flags);
    free(P);
    if (stats) {
        stats[0] = n_eval;
        stats[1] = n_fire;
        stats[2] = np;
    }
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Sec 3.6: reverse-edge sampling between outer iterations                    */
/* ------------------------------------------------------------------------- */

int orc_reverse(int64_t n, int32_t R, float rho, const int32_t *ids, const double *dist,
                const uint8_t *old, const int32_t *deg, int32_t *ids_out, double *dist_out,
                uint8_t *old_out, int32_t *deg_out, uint8_t *flags)
{
    if (n < 1 || R < 1 || !(rho >= 0.0f) || rho > 1.0f)
        return ORC_EINVAL;
    orc_prop *P = (orc_prop *)malloc((size_t)(2 * n * R) * sizeof(orc_prop));
    if (!P)
        return ORC_ENOMEM;
    int64_t np = 0;
    for (int64_t v = 0; v < n; ++v) {
        int32_t k = deg[v];
        int32_t r = (int32_t)floor((double)rho * (double)k);
        for (int32_t i = 0; i < k; ++i) { /* the pool itself */
            orc_prop p = {(int32_t)v, ids[v * R + i], dist[v * R + i], old[v * R + i]};
            P[np++] = p;
        }
        for (int32_t i = 0; i < r; ++i) { /* top rho*k: n <- v */
            orc_prop p = {ids[v * R + i], (int32_t)v, dist[v * R + i], 0};
            P[np++] = p;
        }
    }
    if (flags)
        memset(flags, 0, (size_t)n);
    int rc = merge_props(P, np, n, R, 0.0, ids_out, dist_out, old_out, deg_out, flags);
    free(P);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* C11: final prune-only pass; graph row v = survivors in (dist, id) order    */
/* ------------------------------------------------------------------------- */

int orc_final_prune(const float *X, int64_t n, int32_t d, int32_t metric, int32_t R,
                    const int32_t *ids, const double *dist, const uint8_t *old,
                    const int32_t *deg, uint64_t seed, int32_t t1, int32_t order,
                    int32_t skip_old, double tol, int32_t *gids, double *gdist, int32_t *gdeg,
                    uint8_t *flags)
{
    if (n < 2 || R < 1 || R > 1024)
        return ORC_EINVAL;
    int32_t perm[1024], killer[1024];
    uint8_t alive[1024];
    double kdist[1024];
    for (int64_t v = 0; v < n; ++v) {
        int32_t m = deg[v];
        const int32_t *row = ids + v * R;
        const double *drow = dist + v * R;
        orc_visit_order(seed, t1, 0, v, m, row, order, perm);
        int f = orc_prune(X, d, metric, m, row, drow, old + v * R, perm, skip_old, tol, alive,
                          killer, kdist, NULL);
        if (flags)
            flags[v] = (uint8_t)(f ? 1 : 0);
        int32_t c = 0;
        for (int32_t i = 0; i < m; ++i)
            if (alive[i]) {
                gids[v * R + c] = row[i];
                gdist[v * R + c] = drow[i];
                ++c;
            }
        for (int32_t j = c; j < R; ++j) {
            gids[v * R + j] = -1;
            gdist[v * R + j] = INFINITY;
        }
        gdeg[v] = c;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Alg 3: the whole build                                                     */
/* ------------------------------------------------------------------------- */

int orc_build(const float *X, int64_t n, int32_t d, int32_t metric, int32_t S, int32_t R,
              int32_t T1, int32_t T2, float rho, uint64_t seed, int32_t order, int32_t skip_old,
              int32_t final_prune, int32_t *gids, double *gdist, int32_t *gdeg, int64_t *stats)
{
    if (T1 < 1 || T2 < 1 || R > 1024)
        return ORC_EINVAL;
    size_t slots = (size_t)(n * R);
    int32_t *ia = (int32_t *)malloc(slots * sizeof(int32_t)), *ib = (int32_t *)malloc(slots * sizeof(int32_t));
    double *da = (double *)malloc(slots * sizeof(double)), *db = (double *)malloc(slots * sizeof(double));
    uint8_t *oa = (uint8_t *)malloc(slots), *ob = (uint8_t *)malloc(slots);
    int32_t *ga = (int32_t *)malloc((size_t)n * sizeof(int32_t)), *gb = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int rc = ORC_ENOMEM;
    if (!ia || !ib || !da || !db || !oa || !ob || !ga || !gb)
        goto done;
    rc = orc_init(X, n, d, metric, S, R, seed, 0.0, ia, da, oa, ga, NULL);
    if (rc)
        goto done;
    int64_t st[3], tot[3] = {0, 0, 0};
    for (int32_t t1 = 1; t1 <= T1; ++t1) {
        for (int32_t t2 = 1; t2 <= T2; ++t2) {
            rc = orc_round(X, n, d, metric, R, ia, da, oa, ga, seed, t1, t2, order, skip_old, 0.0,
                           ib, db, ob, gb, NULL, st);
            if (rc)
                goto done;
            for (int i = 0; i < 3; ++i)
                tot[i] += st[i];
            /* Alg 4 end: clear pool1 and swap the two buffers */
            int32_t *ti = ia; ia = ib; ib = ti;
            double *td = da; da = db; db = td;
            uint8_t *to = oa; oa = ob; ob = to;
            int32_t *tg = ga; ga = gb; gb = tg;
        }
        if (t1 != T1) {
            rc = orc_reverse(n, R, rho, ia, da, oa, ga, ib, db, ob, gb, NULL);
            if (rc)
                goto done;
            int32_t *ti = ia; ia = ib; ib = ti;
            double *td = da; da = db; db = td;
            uint8_t *to = oa; oa = ob; ob = to;
            int32_t *tg = ga; ga = gb; gb = tg;
        }
    }
    if (final_prune) {
        rc = orc_final_prune(X, n, d, metric, R, ia, da, oa, ga, seed, T1 + 1, order, skip_old,
                             0.0, gids, gdist, gdeg, NULL);
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
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Sec 2.1: exact k nearest neighbours (ground truth for Recall@k)            */
/* ------------------------------------------------------------------------- */

int orc_brute_knn(const float *X, int64_t n, int32_t d, int32_t metric, const float *Q, int64_t nq,
                  int32_t k, int32_t *ids_out, double *dist_out)
{
    if (k < 1 || k > 1024)
        return ORC_EINVAL;
    int32_t bi[1024];
    double bd[1024];
    for (int64_t q = 0; q < nq; ++q) {
        int32_t c = 0;
        for (int64_t i = 0; i < n; ++i) {
            double di = orc_dist(Q + q * d, X + i * d, d, metric);
            if (c == k && !dl_less(di, (int32_t)i, bd[k - 1], bi[k - 1]))
                continue;
            int32_t j = (c < k) ? c++ : k - 1;
            while (j > 0 && dl_less(di, (int32_t)i, bd[j - 1], bi[j - 1])) {
                bd[j] = bd[j - 1];
                bi[j] = bi[j - 1];
                --j;
            }
            bd[j] = di;
            bi[j] = (int32_t)i;
        }
        for (int32_t j = 0; j < k; ++j) {
            ids_out[q * k + j] = j < c ? bi[j] : -1;
            dist_out[q * k + j] = j < c ? bd[j] : INFINITY;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* C13: search entry = the point nearest the dataset mean                     */
/* ------------------------------------------------------------------------- */

int64_t orc_entry(const float *X, int64_t n, int32_t d, int32_t metric)
{
    double *mu = (double *)calloc((size_t)d, sizeof(double));
    if (!mu || n < 1)
        return -1;
    for (int32_t k = 0; k < d; ++k) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i)
            s += (double)X[i * d + k];
        mu[k] = s / (double)n;
    }
    int64_t best = 0;
    double bd = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        if (metric == 0) {
            for (int32_t k = 0; k < d; ++k) {
                double t = (double)X[i * d + k] - mu[k];
                s += t * t;
            }
        } else {
            for (int32_t k = 0; k < d; ++k)
                s += (double)X[i * d + k] * mu[k];
            s = 1.0 - s;
        }
        if (s < bd) { /* strict: the smallest id wins ties */
            bd = s;
            best = i;
        }
    }
    free(mu);
    return best;
}

/* ------------------------------------------------------------------------- */
/* Sec 4.2: best-first search with a bounded candidate list of size `beam`    */
/* ------------------------------------------------------------------------- */

int orc_search(const int32_t *gids, const int32_t *gdeg, int32_t R, const float *X, int64_t n,
               int32_t d, int32_t metric, int64_t entry, const float *Q, int64_t nq, int32_t k,
               int32_t beam, int32_t *ids_out, double *dist_out, int64_t *n_dist)
{
    if (k < 1 || beam < k || beam > 4096 || entry < 0 || entry >= n)
        return ORC_EINVAL;
    uint8_t *vis = (uint8_t *)malloc((size_t)n);
    int32_t *cid = (int32_t *)malloc((size_t)(beam + 1) * sizeof(int32_t));
    double *cd = (double *)malloc((size_t)(beam + 1) * sizeof(double));
    uint8_t *cx = (uint8_t *)malloc((size_t)(beam + 1));
    if (!vis || !cid || !cd || !cx) {
        free(vis); free(cid); free(cd); free(cx);
        return ORC_ENOMEM;
    }
    int64_t evals = 0;
    for (int64_t q = 0; q < nq; ++q) {
        const float *qv = Q + q * d;
        memset(vis, 0, (size_t)n);
        int32_t size = 1;
        cid[0] = (int32_t)entry;
        cd[0] = orc_dist(qv, X + entry * d, d, metric);
        cx[0] = 0;
        vis[entry] = 1;
        ++evals;
        for (;;) {
            int32_t i = 0;
            while (i < size && cx[i])
                ++i;
            if (i == size)
                break; /* every candidate expanded */
            cx[i] = 1;
            int32_t u = cid[i];
            for (int32_t j = 0; j < gdeg[u]; ++j) {
                int32_t w = gids[(int64_t)u * R + j];
                if (w < 0 || vis[w])
                    continue;
                vis[w] = 1;
                double dw = orc_dist(qv, X + (int64_t)w * d, d, metric);
                ++evals;
                if (size == beam && !dl_less(dw, w, cd[size - 1], cid[size - 1]))
                    continue;
                int32_t p = (size < beam) ? size++ : beam - 1;
                while (p > 0 && dl_less(dw, w, cd[p - 1], cid[p - 1])) {
                    cid[p] = cid[p - 1];
                    cd[p] = cd[p - 1];
                    cx[p] = cx[p - 1];
                    --p;
                }
                cid[p] = w;
                cd[p] = dw;
                cx[p] = 0;
            }
        }
        for (int32_t j = 0; j < k; ++j) {
            ids_out[q * k + j] = j < size ? cid[j] : -1;
            dist_out[q * k + j] = j < size ? cd[j] : INFINITY;
        }
    }
    if (n_dist)
        *n_dist = evals;
    free(vis); free(cid); free(cd); free(cx);
    return ORC_OK;
}
