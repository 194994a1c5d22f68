/*
 * louvain_omp.c -- multi-threaded CPU synchronous Louvain (OpenMP), a CPU baseline.
 *
 * Method: Forster, "Parallel Louvain Community Detection Optimized for GPUs" (arXiv
 * 1805.10904).  The paper compares its GPU code with an 8-thread CPU parallel Louvain
 * (Sec. 6); this file is this project's own parallel CPU form of the same synchronous
 * method the CUDA library runs, so that both can be timed on the same graphs with the
 * same results.  It shares no code with the CUDA library or with the oracle.
 *
 * Steps per level, each parallel over vertices or communities:
 *   - weighted degrees delta_i and 2W                                   [Sec. 2]
 *   - singleton start; degree-one vertex following at level 0 (or every level)
 *     (Lu et al.'s heuristic that Sec. 7 refers to)
 *   - synchronous sweeps: every vertex aggregates e_{i->C} over its non-loop entries
 *     [Eq. 1] in a per-thread open-addressing table, scores every neighbouring community
 *     with the exact gain [Eq. 4, Eq. 5] against the previous sweep's state, takes the best
 *     (ties to the smallest label, Sec. 3.1.2), moves only on a strictly positive gain and
 *     not as a singleton into a larger-labelled singleton (Sec. 3.1.1)      [Algorithm 1]
 *   - deg_C / size_C rebuilt after every sweep with integer atomics [Eq. 2]; Qn = (2W)^2 Q
 *     [Eq. 3] reduced in 128-bit integers; stop when nothing moved, when the gain is below
 *     theta * (2W)^2 (exact), or at the sweep cap
 *   - renumbering by a prefix sum over used labels, level recorded when it merged, outer
 *     test against the previous level's Qn                                    [Algorithm 2]
 *   - induced graph: members grouped by community, each community's entries merged in a
 *     per-thread table, rows sorted by column; a counting pass then a writing pass
 *     [Sec. 5.1.2 "Inducing new graph"]
 *
 * Arithmetic: weights, degrees and sums are int64; gains and Qn are __int128; the theta
 * tests compare 192-bit products.  Integer sums do not depend on the order in which the
 * threads add them, so the result is the same for every thread count.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 s128;
typedef unsigned __int128 u128;

enum { OMP_OK = 0, OMP_ERR_INVALID = 1, OMP_ERR_OOM = 2 };

/* ------------------------------------------------------------------ graph */

typedef struct {
    int64_t n, nnz;
    int64_t *rp;
    int32_t *col;
    int64_t *w;
} lg_graph;

static void lg_free(lg_graph *g)
{
    free(g->rp);
    free(g->col);
    free(g->w);
    g->rp = NULL;
    g->col = NULL;
    g->w = NULL;
}

/* ------------------------------------------------------------------ 192-bit compare */

typedef struct {
    uint64_t w[3]; /* little-endian 64-bit words */
} u192;

static u192 mul128x64(u128 a, uint64_t b)
{
    u128 lo = (u128)(uint64_t)a * b;
    u128 hi = (u128)(uint64_t)(a >> 64) * b + (uint64_t)(lo >> 64);
    u192 r = {{(uint64_t)lo, (uint64_t)hi, (uint64_t)(hi >> 64)}};
    return r;
}

static int lt192(u192 a, u192 b)
{
    for (int k = 2; k >= 0; k--)
        if (a.w[k] != b.w[k]) return a.w[k] < b.w[k];
    return 0;
}

/* (qn_new - qn_old) * den < num * tw^2 with tw <= 2^62, num >= 0, den > 0 */
static int gain_below(s128 qn_new, s128 qn_old, int64_t tw, int64_t num, int64_t den)
{
    s128 d = qn_new - qn_old;
    if (d < 0) return 1;
    u128 tw2 = (u128)(uint64_t)tw * (uint64_t)tw;
    return lt192(mul128x64((u128)d, (uint64_t)den), mul128x64(tw2, (uint64_t)num));
}

/* ------------------------------------------------------------------ per-thread table */

typedef struct {
    int32_t *key; /* -1 = empty */
    int64_t *sum;
    int32_t *used; /* slots in insertion order */
    int32_t *sorted; /* scratch for a row's keys in ascending order */
    int64_t cap, mask, nused;
} lg_table;

static void table_free(lg_table *t)
{
    free(t->key);
    free(t->sum);
    free(t->used);
    free(t->sorted);
    t->key = NULL;
    t->sum = NULL;
    t->used = NULL;
    t->sorted = NULL;
    t->cap = 0;
}

/* Make an empty table hold max_keys keys at a load factor of at most 1/2. */
static int table_reserve(lg_table *t, int64_t max_keys)
{
    if (2 * max_keys <= t->cap) return OMP_OK;
    int64_t cap = 16;
    while (cap < 2 * max_keys) cap <<= 1;
    table_free(t);
    t->key = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    t->sum = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    t->used = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    t->sorted = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    if (!t->key || !t->sum || !t->used || !t->sorted) {
        table_free(t);
        return OMP_ERR_OOM;
    }
    for (int64_t s = 0; s < cap; s++) t->key[s] = -1;
    t->cap = cap;
    t->mask = cap - 1;
    t->nused = 0;
    return OMP_OK;
}

static inline int64_t table_home(const lg_table *t, int32_t k)
{
    return (int64_t)((((uint64_t)(uint32_t)k * 0x9E3779B97F4A7C15ULL) >> 17) & (uint64_t)t->mask);
}

static inline void table_add(lg_table *t, int32_t k, int64_t x)
{
    for (int64_t s = table_home(t, k);; s = (s + 1) & t->mask) {
        if (t->key[s] == k) {
            t->sum[s] += x;
            return;
        }
        if (t->key[s] < 0) {
            t->key[s] = k;
            t->sum[s] = x;
            t->used[t->nused++] = (int32_t)s;
            return;
        }
    }
}

static inline int64_t table_get(const lg_table *t, int32_t k)
{
    for (int64_t s = table_home(t, k);; s = (s + 1) & t->mask)
        if (t->key[s] == k) return t->sum[s];
}

static inline void table_clear(lg_table *t)
{
    for (int64_t u = 0; u < t->nused; u++) t->key[t->used[u]] = -1;
    t->nused = 0;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------ level state */

typedef struct {
    int32_t *C, *Cn, *size, *new_id, *map;
    int64_t *delta, *deg;
} lg_state;

static void community_rebuild(int64_t n, const int32_t *C, const int64_t *delta, int64_t *deg,
                              int32_t *size)
{
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; c++) {
        deg[c] = 0;
        size[c] = 0;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int32_t c = C[i];
#pragma omp atomic
        deg[c] += delta[i];
#pragma omp atomic
        size[c] += 1;
    }
}

/* Qn = TW * sum_i (weight of i's entries inside C(i), loop included) - sum_c deg_c^2 */
static s128 modularity_qn(const lg_graph *g, const int32_t *C, const int64_t *deg, int64_t TW)
{
    int64_t n = g->n;
    int64_t internal = 0;
    s128 sq = 0;
#pragma omp parallel
    {
        int64_t in_t = 0;
        s128 sq_t = 0;
#pragma omp for schedule(dynamic, 256) nowait
        for (int64_t i = 0; i < n; i++) {
            int32_t a = C[i];
            for (int64_t k = g->rp[i]; k < g->rp[i + 1]; k++)
                if (C[g->col[k]] == a) in_t += g->w[k];
        }
#pragma omp for schedule(static) nowait
        for (int64_t c = 0; c < n; c++) sq_t += (s128)deg[c] * deg[c];
#pragma omp critical
        {
            internal += in_t;
            sq += sq_t;
        }
    }
    return (s128)TW * internal - sq;
}

/* One synchronous sweep from (C, deg, size): proposals into Cn, returns vertices moved. */
static int64_t sweep(const lg_graph *g, const lg_state *st, int64_t TW, lg_table *tables)
{
    int64_t n = g->n, moved = 0;
    const int32_t *C = st->C;
#pragma omp parallel reduction(+ : moved)
    {
        lg_table *t = &tables[omp_get_thread_num()];
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; i++) {
            int32_t a = C[i];
            for (int64_t k = g->rp[i]; k < g->rp[i + 1]; k++)
                if (g->col[k] != i) table_add(t, C[g->col[k]], g->w[k]);
            int32_t target = a;
            if (t->nused > 0) {
                int64_t di = st->delta[i];
                int64_t e_a = 0;
                int found_best = 0;
                int32_t best = 0;
                s128 g_best = 0;
                for (int64_t u = 0; u < t->nused; u++) {
                    int32_t s = t->used[u];
                    int32_t b = t->key[s];
                    if (b == a) {
                        e_a = t->sum[s];
                        continue;
                    }
                    s128 gb = (s128)TW * t->sum[s] - (s128)di * st->deg[b];
                    if (!found_best || gb > g_best || (gb == g_best && b < best)) {
                        found_best = 1;
                        g_best = gb;
                        best = b;
                    }
                }
                s128 g_stay = (s128)TW * e_a - (s128)di * (st->deg[a] - di);
                if (found_best && g_best > g_stay &&
                    !(st->size[a] == 1 && st->size[best] == 1 && best > a))
                    target = best;
                table_clear(t);
            }
            st->Cn[i] = target;
            moved += target != a;
        }
    }
    return moved;
}

/* Degree-one vertices join their neighbour's community; an isolated pair joins min(i, j). */
static void vertex_following(const lg_graph *g, int32_t *C)
{
    int64_t n = g->n;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; i++) {
        int64_t cnt = 0;
        int32_t j = -1;
        for (int64_t k = g->rp[i]; k < g->rp[i + 1]; k++)
            if (g->col[k] != i) {
                cnt++;
                j = g->col[k];
            }
        C[i] = (int32_t)i;
        if (cnt != 1) continue;
        int64_t cj = 0;
        for (int64_t k = g->rp[j]; k < g->rp[j + 1]; k++) cj += g->col[k] != j;
        C[i] = cj == 1 ? (int32_t)(i < j ? i : j) : j;
    }
}

/* new_id[c] = number of used labels below c; returns the count of used labels */
static int64_t renumber(int64_t n, const int32_t *C, int32_t *new_id)
{
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; c++) new_id[c] = 0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
#pragma omp atomic write
        new_id[C[i]] = 1;
    }
    int64_t k = 0;
    for (int64_t c = 0; c < n; c++) {
        int32_t used = new_id[c];
        new_id[c] = (int32_t)k;
        k += used;
    }
    return k;
}

/* The graph induced by the k communities: A'_ab = sum of A_uv over C(u)=a, C(v)=b. */
static int induce(const lg_graph *g, const lg_state *st, int64_t k, lg_table *tables,
                  lg_graph *out)
{
    int64_t n = g->n;
    int64_t *moff = (int64_t *)calloc((size_t)(k + 1), sizeof(int64_t));
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    int32_t *members = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *cnt = (int64_t *)calloc((size_t)(k + 1), sizeof(int64_t));
    if (!moff || !cur || !members || !cnt) goto oom;
#pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < n; u++) {
        int64_t a = st->new_id[st->C[u]];
#pragma omp atomic
        moff[a + 1] += 1;
    }
    for (int64_t a = 0; a < k; a++) moff[a + 1] += moff[a];
    memcpy(cur, moff, sizeof(int64_t) * (size_t)k);
#pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < n; u++) {
        int64_t a = st->new_id[st->C[u]], p;
#pragma omp atomic capture
        p = cur[a]++;
        members[p] = (int32_t)u;
    }
    /* pass 1: distinct neighbouring communities of every community */
    int failed = 0;
#pragma omp parallel
    {
        lg_table *t = &tables[omp_get_thread_num()];
#pragma omp for schedule(dynamic, 16)
        for (int64_t a = 0; a < k; a++) {
            int64_t entries = 0;
            for (int64_t p = moff[a]; p < moff[a + 1]; p++)
                entries += g->rp[members[p] + 1] - g->rp[members[p]];
            if (table_reserve(t, entries < k ? entries : k) != OMP_OK) {
#pragma omp atomic write
                failed = 1;
                continue;
            }
            for (int64_t p = moff[a]; p < moff[a + 1]; p++) {
                int32_t u = members[p];
                for (int64_t e = g->rp[u]; e < g->rp[u + 1]; e++)
                    table_add(t, st->new_id[st->C[g->col[e]]], g->w[e]);
            }
            cnt[a + 1] = t->nused;
            table_clear(t);
        }
    }
    if (failed) goto oom;
    for (int64_t a = 0; a < k; a++) cnt[a + 1] += cnt[a];
    out->n = k;
    out->nnz = cnt[k];
    out->rp = cnt;
    cnt = NULL;
    out->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(out->nnz > 0 ? out->nnz : 1));
    out->w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(out->nnz > 0 ? out->nnz : 1));
    if (!out->col || !out->w) goto oom;
    /* pass 2: merge again and write each row sorted by column */
#pragma omp parallel
    {
        lg_table *t = &tables[omp_get_thread_num()];
#pragma omp for schedule(dynamic, 16)
        for (int64_t a = 0; a < k; a++) {
            int64_t entries = 0;
            for (int64_t p = moff[a]; p < moff[a + 1]; p++)
                entries += g->rp[members[p] + 1] - g->rp[members[p]];
            if (table_reserve(t, entries < k ? entries : k) != OMP_OK) {
#pragma omp atomic write
                failed = 1;
                continue;
            }
            for (int64_t p = moff[a]; p < moff[a + 1]; p++) {
                int32_t u = members[p];
                for (int64_t e = g->rp[u]; e < g->rp[u + 1]; e++)
                    table_add(t, st->new_id[st->C[g->col[e]]], g->w[e]);
            }
            int64_t m = t->nused;
            for (int64_t u = 0; u < m; u++) t->sorted[u] = t->key[t->used[u]];
            qsort(t->sorted, (size_t)m, sizeof(int32_t), cmp_i32);
            int64_t base = out->rp[a];
            for (int64_t u = 0; u < m; u++) {
                out->col[base + u] = t->sorted[u];
                out->w[base + u] = table_get(t, t->sorted[u]);
            }
            table_clear(t);
        }
    }
    free(moff);
    free(cur);
    free(members);
    return failed ? OMP_ERR_OOM : OMP_OK;
oom:
    free(moff);
    free(cur);
    free(members);
    free(cnt);
    return OMP_ERR_OOM;
}

/* ------------------------------------------------------------------ result */

typedef struct {
    int32_t level, iter;
    int64_t moved;
    s128 qn;
} lg_trace;

typedef struct {
    int64_t n0, tw, edge_visits, sweeps;
    int32_t num_levels, cap_levels, hit_cap;
    int32_t *labels; /* num_levels x n0 */
    int64_t *ncomm, *n, *nnz;
    int32_t *iters;
    s128 *qn, *qn_init;
    lg_trace *trace;
    int64_t ntrace, trace_cap;
} lg_result;

static int trace_add(lg_result *r, int32_t level, int32_t iter, int64_t moved, s128 qn)
{
    if (r->ntrace == r->trace_cap) {
        int64_t cap = r->trace_cap ? 2 * r->trace_cap : 64;
        lg_trace *t = (lg_trace *)realloc(r->trace, sizeof(lg_trace) * (size_t)cap);
        if (!t) return OMP_ERR_OOM;
        r->trace = t;
        r->trace_cap = cap;
    }
    lg_trace e = {level, iter, moved, qn};
    r->trace[r->ntrace++] = e;
    return OMP_OK;
}

void lomp_free(void *h)
{
    lg_result *r = (lg_result *)h;
    if (!r) return;
    free(r->labels);
    free(r->ncomm);
    free(r->n);
    free(r->nnz);
    free(r->iters);
    free(r->qn);
    free(r->qn_init);
    free(r->trace);
    free(r);
}

/* ------------------------------------------------------------------ driver */

static int run_levels(lg_graph *g, int64_t theta_num, int64_t theta_den, int32_t max_iters,
                      int32_t max_levels, int32_t vf, int32_t vf_all, lg_result *r)
{
    int64_t n0 = g->n, N = n0 > 0 ? n0 : 1;
    int nthreads = omp_get_max_threads();
    lg_state st;
    st.C = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    st.Cn = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    st.size = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    st.new_id = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    st.map = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    st.delta = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    st.deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    lg_table *tables = (lg_table *)calloc((size_t)nthreads, sizeof(lg_table));
    int rc = OMP_OK;
    if (!st.C || !st.Cn || !st.size || !st.new_id || !st.map || !st.delta || !st.deg || !tables) {
        rc = OMP_ERR_OOM;
        goto done;
    }
    for (int64_t v = 0; v < n0; v++) st.map[v] = (int32_t)v;
    {
        s128 tw = 0;
        for (int64_t k = 0; k < g->nnz; k++) tw += g->w[k];
        if (tw > ((s128)1 << 62)) {
            rc = OMP_ERR_INVALID;
            goto done;
        }
        r->tw = (int64_t)tw;
    }
    const int64_t TW = r->tw;
    s128 qn_level_prev = 0;
    for (int32_t level = 0; level < max_levels && n0 > 0; level++) {
        int64_t n = g->n;
        int64_t longest = 1;
        for (int64_t i = 0; i < n; i++)
            if (g->rp[i + 1] - g->rp[i] > longest) longest = g->rp[i + 1] - g->rp[i];
        for (int t = 0; t < nthreads; t++)
            if (table_reserve(&tables[t], longest) != OMP_OK) {
                rc = OMP_ERR_OOM;
                goto done;
            }
#pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t i = 0; i < n; i++) {
            int64_t d = 0;
            for (int64_t k = g->rp[i]; k < g->rp[i + 1]; k++) d += g->w[k];
            st.delta[i] = d;
            st.C[i] = (int32_t)i;
        }
        if (vf && (level == 0 || vf_all)) vertex_following(g, st.C);
        community_rebuild(n, st.C, st.delta, st.deg, st.size);
        s128 qn_init = modularity_qn(g, st.C, st.deg, TW);
        s128 qn_prev = qn_init, qn = qn_init;
        int32_t iters = 0;
        for (;;) {
            int64_t moved = sweep(g, &st, TW, tables);
            iters++;
            r->sweeps++;
            r->edge_visits += g->nnz;
            int32_t *tmp = st.C;
            st.C = st.Cn;
            st.Cn = tmp;
            community_rebuild(n, st.C, st.delta, st.deg, st.size);
            qn = modularity_qn(g, st.C, st.deg, TW);
            if ((rc = trace_add(r, level, iters, moved, qn)) != OMP_OK) goto done;
            if (moved == 0 || gain_below(qn, qn_prev, TW, theta_num, theta_den)) break;
            if (iters >= max_iters) {
                r->hit_cap = 1;
                break;
            }
            qn_prev = qn;
        }
        int64_t k = renumber(n, st.C, st.new_id);
        if (k == n) break; /* nothing merged: no new level */
#pragma omp parallel for schedule(static)
        for (int64_t v = 0; v < n0; v++) st.map[v] = st.new_id[st.C[st.map[v]]];
        int32_t L = r->num_levels;
        memcpy(r->labels + (size_t)L * (size_t)n0, st.map, sizeof(int32_t) * (size_t)n0);
        r->ncomm[L] = k;
        r->qn[L] = qn;
        r->qn_init[L] = qn_init;
        r->iters[L] = iters;
        r->n[L] = n;
        r->nnz[L] = g->nnz;
        r->num_levels = L + 1;
        if (level >= 1 && gain_below(qn, qn_level_prev, TW, theta_num, theta_den)) break;
        qn_level_prev = qn;
        if (level + 1 >= max_levels) break;
        lg_graph next = {0, 0, NULL, NULL, NULL};
        if ((rc = induce(g, &st, k, tables, &next)) != OMP_OK) {
            lg_free(&next);
            goto done;
        }
        lg_free(g);
        *g = next;
    }
done:
    if (tables)
        for (int t = 0; t < nthreads; t++) table_free(&tables[t]);
    free(tables);
    free(st.C);
    free(st.Cn);
    free(st.size);
    free(st.new_id);
    free(st.map);
    free(st.delta);
    free(st.deg);
    return rc;
}

/* Full run with `threads` OpenMP threads (<= 0: the runtime's default).  Input: symmetric
 * CSR (row offsets int64, columns int32, weights int32 >= 1 or NULL for all 1).  Returns a
 * result handle or NULL with *status set (1 invalid input, 2 out of memory). */
void *lomp_run(int64_t n, const int64_t *rp, const int32_t *col, const int32_t *w,
               int64_t theta_num, int64_t theta_den, int32_t max_iters, int32_t max_levels,
               int32_t vf, int32_t vf_all, int32_t threads, int32_t *status)
{
    int st = OMP_OK;
    lg_result *r = NULL;
    lg_graph g = {0, 0, NULL, NULL, NULL};
    if (n < 0 || !rp || rp[0] != 0 || theta_den <= 0 || theta_num < 0 ||
        theta_den > INT32_MAX || theta_num > INT32_MAX || max_iters < 1 || max_levels < 1) {
        st = OMP_ERR_INVALID;
        goto fail;
    }
    for (int64_t i = 0; i < n; i++)
        if (rp[i + 1] < rp[i]) {
            st = OMP_ERR_INVALID;
            goto fail;
        }
    g.n = n;
    g.nnz = rp[n];
    g.rp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    g.col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g.nnz > 0 ? g.nnz : 1));
    g.w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(g.nnz > 0 ? g.nnz : 1));
    r = (lg_result *)calloc(1, sizeof(lg_result));
    if (!g.rp || !g.col || !g.w || !r) {
        st = OMP_ERR_OOM;
        goto fail;
    }
    memcpy(g.rp, rp, sizeof(int64_t) * (size_t)(n + 1));
    if (g.nnz > 0) memcpy(g.col, col, sizeof(int32_t) * (size_t)g.nnz);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t k = 0; k < g.nnz; k++) {
        g.w[k] = w ? w[k] : 1;
        bad |= g.w[k] < 1 || col[k] < 0 || col[k] >= n;
    }
#pragma omp parallel for schedule(dynamic, 1024) reduction(| : bad)
    for (int64_t i = 0; i < n; i++)
        for (int64_t k = rp[i] + 1; k < rp[i + 1]; k++) bad |= col[k] <= col[k - 1];
    if (bad) { /* weights >= 1, columns in range, each row sorted without repeats */
        st = OMP_ERR_INVALID;
        goto fail;
    }
    r->n0 = n;
    r->cap_levels = max_levels;
    size_t L = (size_t)max_levels;
    r->labels = (int32_t *)malloc(sizeof(int32_t) * L * (size_t)(n > 0 ? n : 1));
    r->ncomm = (int64_t *)calloc(L, sizeof(int64_t));
    r->n = (int64_t *)calloc(L, sizeof(int64_t));
    r->nnz = (int64_t *)calloc(L, sizeof(int64_t));
    r->iters = (int32_t *)calloc(L, sizeof(int32_t));
    r->qn = (s128 *)calloc(L, sizeof(s128));
    r->qn_init = (s128 *)calloc(L, sizeof(s128));
    if (!r->labels || !r->ncomm || !r->n || !r->nnz || !r->iters || !r->qn || !r->qn_init) {
        st = OMP_ERR_OOM;
        goto fail;
    }
    if (threads > 0) omp_set_num_threads(threads);
    st = run_levels(&g, theta_num, theta_den, max_iters, max_levels, vf, vf_all, r);
    if (st != OMP_OK) goto fail;
    lg_free(&g);
    if (status) *status = OMP_OK;
    return r;
fail:
    lg_free(&g);
    lomp_free(r);
    if (status) *status = st;
    return NULL;
}

static void put128(s128 v, int64_t out[2])
{
    out[0] = (int64_t)(v >> 64);
    out[1] = (int64_t)(uint64_t)v;
}

int32_t lomp_num_levels(const void *h) { return ((const lg_result *)h)->num_levels; }
int64_t lomp_tw(const void *h) { return ((const lg_result *)h)->tw; }
int64_t lomp_edge_visits(const void *h) { return ((const lg_result *)h)->edge_visits; }
int64_t lomp_sweeps(const void *h) { return ((const lg_result *)h)->sweeps; }
int32_t lomp_hit_cap(const void *h) { return ((const lg_result *)h)->hit_cap; }
int64_t lomp_trace_len(const void *h) { return ((const lg_result *)h)->ntrace; }
int32_t lomp_max_threads(void) { return omp_get_max_threads(); }

void lomp_level(const void *h, int32_t l, int32_t *labels, int64_t *ncomm, int64_t qn[2],
                int64_t qn_init[2], int32_t *iters, int64_t *n, int64_t *nnz)
{
    const lg_result *r = (const lg_result *)h;
    memcpy(labels, r->labels + (size_t)l * (size_t)r->n0, sizeof(int32_t) * (size_t)r->n0);
    *ncomm = r->ncomm[l];
    put128(r->qn[l], qn);
    put128(r->qn_init[l], qn_init);
    *iters = r->iters[l];
    *n = r->n[l];
    *nnz = r->nnz[l];
}

void lomp_trace(const void *h, int32_t *level, int32_t *iter, int64_t *moved, int64_t *qn)
{
    const lg_result *r = (const lg_result *)h;
    for (int64_t t = 0; t < r->ntrace; t++) {
        level[t] = r->trace[t].level;
        iter[t] = r->trace[t].iter;
        moved[t] = r->trace[t].moved;
        put128(r->trace[t].qn, qn + 2 * t);
    }
}
