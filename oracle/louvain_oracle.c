/*
 * louvain_oracle.c -- plain sequential CPU oracle of synchronous parallel Louvain
 * (Forster, "Parallel Louvain Community Detection Optimized for GPUs", arXiv 1805.10904).
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA path and to time a
 * CPU baseline.  Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or helper with the CUDA
 * library, and it must never be called from the product path.
 *
 * What it computes (paper section / equation in brackets):
 *   - graph model, weighted degree delta_i, total weight 2W          [Sec. 2]
 *   - e_{i->C}                                                         [Eq. 1]
 *   - deg_C                                                            [Eq. 2]
 *   - modularity Q, kept exactly as Qn = (2W)^2 * Q                    [Eq. 3]
 *   - modularity gain of moving i from C(i) to C(j)                    [Eq. 4, Sec. 3]
 *   - argmax target choice                                             [Eq. 5]
 *   - singlet minimum-label rule                                       [Sec. 3.1.1]
 *   - generalised minimum-label rule (ties -> smallest label)          [Sec. 3.1.2]
 *   - synchronous phase: every decision reads the previous iteration  [Sec. 5, Algorithm 1]
 *   - multi-level driver with outer threshold                          [Sec. 4.2, Algorithm 2]
 *   - renumbering of communities to consecutive ids                    [Sec. 5.1.2 "Renumbering nodes"]
 *   - graph induction (coarsening)                                     [Sec. 3, Sec. 5.1.2 "Inducing new graph"]
 *   - vertex following (degree-one vertices join their neighbour) -- not in the
 *     paper; it is one of the "other heuristics" of Lu et al. that Sec. 7 refers to.
 *
 * Readings taken where the paper is silent, garbled or self-contradictory:
 *   R1  2W = TW = sum_i delta_i over the symmetric adjacency; a loop A_ii is stored once
 *       and counted once in delta_i.                                          [Sec. 2]
 *   R2  weights are integers >= 1 (the paper's "weight 0 when unweighted" is replaced by
 *       "weight 1"; Sec. 5.1.2 says zero weights are always raised).
 *   R3  Eq. 4 as printed drops the -e_{i->C(i)\{i}} term and writes "mod" for deg.  The
 *       full gain, multiplied by (2W)^2/2, is G_B - G_stay with
 *           G_B    = TW * e_{i->B}        - delta_i * deg_B
 *           G_stay = TW * e_{i->A\{i}}    - delta_i * (deg_A - delta_i)
 *       (A = C(i)); the difference of two Eq. 3 evaluations equals 2*(G_B - G_stay).
 *   R4  e_{i->C} used for gains excludes i's loop (Sec. 5.1.2 sets loop weights to 0 in the
 *       move step); Eq. 3's sum includes it, so Q is preserved by coarsening.
 *   R5  target = argmax gain over neighbouring communities, ties to the smallest label;
 *       i moves only if the best gain is strictly larger than the gain of staying.
 *   R6  singlet rule as a veto: if C(i) and the chosen target are both singletons in the
 *       previous iteration's state and target > C(i), i stays.
 *   R15 post_merge (a variant): after each phase, a vertex whose non-loop neighbours all
 *       lie in one other community joins it if that move's Eq. 4 gain is positive; all
 *       decisions on the post-phase state; the level records the merged state and its Qn
 *   R14 threshold_mode 1 (a variant): the phase test is the relative one printed in
 *       Algorithm 1, |Q_curr - Q_prev| / |Q_prev| < theta, exact; Q_prev = 0 only stops on
 *       an unchanged Q; the outer test stays absolute (R9)
 *   R7  phase stop: no vertex moved, or (Qn_new - Qn_prev) * theta_den < theta_num * TW^2
 *       (absolute gain test on exact integers, theta = 1/10^6 by default, Qn_prev starts at
 *       the state before the first sweep), or the sweep cap is reached.  The state after
 *       the last applied sweep is the phase result (Algorithm 1 applies, then tests).
 *   R8  renumbering keeps the order of the old labels (prefix-sum compaction).
 *   R9  a level is recorded only if it merged something (k < n); the run stops after a
 *       level whose Qn gained less than theta over the previous level (Algorithm 2), that
 *       level still being recorded.
 *   R10 coarse weight A'_ab = sum of A_uv over C(u)=a, C(v)=b over stored entries, so an
 *       internal non-loop edge adds twice to the loop of its community and old loops once;
 *       delta and TW are preserved.
 *   R11 vertex following (level 0 only unless asked): a vertex whose only non-loop
 *       neighbour is j joins j's community (j keeps its own singleton label); an isolated
 *       pair (each the other's only neighbour) joins min(i, j).
 *   R12 zero-degree vertices stay singletons at every level.
 *   R13 a graph without vertices runs no phase (no sweep, no level).
 *   R17 coloring (a variant; Lu et al.'s colouring heuristic, which Sec. 7 names among the
 *       "other heuristics" without defining it): at every level the graph's vertices get a
 *       distance-1 colouring (Jones-Plassmann rounds: an uncoloured vertex whose priority
 *       exceeds that of every uncoloured non-loop neighbour takes the smallest colour
 *       unused by its coloured neighbours; priority = SplitMix64 output function of the
 *       vertex id).  A sweep takes the colour classes in increasing colour: the vertices of
 *       a class decide together on the current state (the rule of R5/R6), their moves are
 *       applied and deg/size rebuilt before the next class.  Stop tests, trace and levels
 *       are per sweep as without colouring.
 *
 * Arithmetic: weights, degrees and sums in int64; every product of two of them in
 * __int128.  Nothing here is floating point except the reported Q = (double)Qn / (double)TW^2
 * (two int128 -> double conversions rounded to nearest, then one division).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

#define ORACLE_OK 0
#define ORACLE_ERR_INVALID 1
#define ORACLE_ERR_OOM 2

/* ------------------------------------------------------------------------- */
/* Graph storage: CSR over the symmetric adjacency, int64 weights.           */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t n;
    int64_t nnz;
    int64_t *rp;   /* n + 1 row offsets */
    int32_t *col;  /* nnz column ids */
    int64_t *w;    /* nnz weights, all >= 1 */
} og_graph;

static void graph_free(og_graph *g)
{
    if (!g) return;
    free(g->rp);
    free(g->col);
    free(g->w);
    g->rp = NULL;
    g->col = NULL;
    g->w = NULL;
}

static int graph_alloc(og_graph *g, int64_t n, int64_t nnz)
{
    g->n = n;
    g->nnz = nnz;
    g->rp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    g->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    g->w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!g->rp || !g->col || !g->w) {
        graph_free(g);
        return ORACLE_ERR_OOM;
    }
    return ORACLE_OK;
}

/* Copy a caller CSR into oracle storage and check the input contract of Sec. 2:
 * row offsets start at 0 and never decrease, every column is a vertex id, every
 * weight is >= 1 (reading R2).  w32 or w64 may be given; both NULL means all 1. */
static int graph_from_input(og_graph *g, int64_t n, const int64_t *rp, const int32_t *col,
                            const int32_t *w32, const int64_t *w64)
{
    if (n < 0 || n > INT32_MAX || !rp) return ORACLE_ERR_INVALID;
    if (rp[0] != 0) return ORACLE_ERR_INVALID;
    for (int64_t i = 0; i < n; i++)
        if (rp[i + 1] < rp[i]) return ORACLE_ERR_INVALID;
    int64_t nnz = rp[n];
    if (nnz > 0 && !col) return ORACLE_ERR_INVALID;
    if (graph_alloc(g, n, nnz) != ORACLE_OK) return ORACLE_ERR_OOM;
    memcpy(g->rp, rp, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t k = 0; k < nnz; k++) {
        if (col[k] < 0 || (int64_t)col[k] >= n) {
            graph_free(g);
            return ORACLE_ERR_INVALID;
        }
        g->col[k] = col[k];
        int64_t wk = w64 ? w64[k] : (w32 ? (int64_t)w32[k] : 1);
        if (wk < 1) {
            graph_free(g);
            return ORACLE_ERR_INVALID;
        }
        g->w[k] = wk;
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* Sec. 2 quantities.                                                        */
/* ------------------------------------------------------------------------- */

/* delta_i = sum of the weights stored in row i, the loop included once (R1). */
static void weighted_degrees(const og_graph *g, int64_t *delta)
{
    for (int64_t i = 0; i < g->n; i++) {
        int64_t s = 0;
        for (int64_t k = g->rp[i]; k < g->rp[i + 1]; k++) s += g->w[k];
        delta[i] = s;
    }
}

/* Eq. 2: deg_c = sum of delta_i over members of community c; size_c = member count. */
static void community_degrees(int64_t n, const int32_t *C, const int64_t *delta, int64_t *deg,
                              int32_t *size)
{
    for (int64_t c = 0; c < n; c++) {
        deg[c] = 0;
        size[c] = 0;
    }
    for (int64_t i = 0; i < n; i++) {
        deg[C[i]] += delta[i];
        size[C[i]] += 1;
    }
}

/* Eq. 3 multiplied by TW^2:
 *   Qn = TW * sum_i e_{i->C(i)} - sum_c deg_c^2,
 * with e_{i->C(i)} the weight of row i's entries whose column lies in C(i), the loop
 * included (R4).  deg is recomputed here from C and delta. */
static i128 modularity_qn(const og_graph *g, const int32_t *C, const int64_t *delta, int64_t TW,
                          int64_t *deg_scratch, int32_t *size_scratch)
{
    int64_t internal = 0; /* sum_i e_{i->C(i)} <= TW, fits int64 */
    for (int64_t i = 0; i < g->n; i++)
        for (int64_t k = g->rp[i]; k < g->rp[i + 1]; k++)
            if (C[g->col[k]] == C[i]) internal += g->w[k];
    community_degrees(g->n, C, delta, deg_scratch, size_scratch);
    i128 sum_sq = 0;
    for (int64_t c = 0; c < g->n; c++) sum_sq += (i128)deg_scratch[c] * deg_scratch[c];
    return (i128)TW * internal - sum_sq;
}

/* ------------------------------------------------------------------------- */
/* Vertex following (R11).                                                   */
/* ------------------------------------------------------------------------- */

static void vertex_following(const og_graph *g, int32_t *C)
{
    int64_t n = g->n;
    int64_t *nonloop = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *other = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        nonloop[i] = 0;
        other[i] = -1;
        for (int64_t k = g->rp[i]; k < g->rp[i + 1]; k++)
            if (g->col[k] != i) {
                nonloop[i] += 1;
                other[i] = g->col[k];
            }
    }
    for (int64_t i = 0; i < n; i++) C[i] = (int32_t)i;
    for (int64_t i = 0; i < n; i++) {
        if (nonloop[i] != 1) continue;
        int32_t j = other[i];
        if (nonloop[j] == 1)
            C[i] = (int32_t)(i < j ? i : j); /* isolated pair */
        else
            C[i] = j;
    }
    free(nonloop);
    free(other);
}

/* ------------------------------------------------------------------------- */
/* One synchronous local-moving sweep (Algorithm 1 body, Eq. 4-5, Sec. 3.1). */
/* ------------------------------------------------------------------------- */

/* Reads only the snapshot (C, deg, size); writes Cnext.  Returns the number of vertices
 * whose label changed.  e, seen and touched are n-sized scratch arrays; seen must be all
 * zero on entry and is all zero again on return. */
static int64_t local_move_sweep(const og_graph *g, const int32_t *C, const int64_t *deg,
                                const int32_t *size, const int64_t *delta, int64_t TW,
                                int32_t *Cnext, int64_t *e, int64_t *seen, int32_t *touched,
                                const int32_t *color, int32_t cls)
{
    int64_t moved = 0;
    for (int64_t i = 0; i < g->n; i++) {
        int32_t a = C[i];
        int64_t m = 0;
        if (color && color[i] != cls) { /* another colour class: stays this time (R17) */
            Cnext[i] = a;
            continue;
        }
        /* Eq. 1 over the neighbours' communities, loop excluded (R4) */
        for (int64_t k = g->rp[i]; k < g->rp[i + 1]; k++) {
            int32_t j = g->col[k];
            if (j == i) continue;
            int32_t c = C[j];
            if (!seen[c]) {
                seen[c] = 1;
                e[c] = 0;
                touched[m++] = c;
            }
            e[c] += g->w[k];
        }
        int64_t e_a = seen[a] ? e[a] : 0; /* e_{i -> C(i)\{i}} */
        for (int64_t t = 0; t < m; t++) seen[touched[t]] = 0; /* e[] stays readable */
        Cnext[i] = a;
        if (m == 0) continue; /* no non-loop neighbour: i stays */

        i128 g_stay = (i128)TW * e_a - (i128)delta[i] * (deg[a] - delta[i]);

        int have = 0;
        int32_t best = -1;
        i128 g_best = 0;
        for (int64_t t = 0; t < m; t++) {
            int32_t c = touched[t];
            if (c == a) continue;
            i128 gc = (i128)TW * e[c] - (i128)delta[i] * deg[c];
            /* Eq. 5 argmax; equal gains go to the smallest label (Sec. 3.1.2) */
            if (!have || gc > g_best || (gc == g_best && c < best)) {
                have = 1;
                best = c;
                g_best = gc;
            }
        }
        if (!have || !(g_best > g_stay)) continue; /* strict gain required (R5) */
        /* singlet minimum-label rule (Sec. 3.1.1, reading R6) */
        if (size[a] == 1 && size[best] == 1 && best > a) continue;
        Cnext[i] = best;
        moved += 1;
    }
    return moved;
}

/* ------------------------------------------------------------------------- */
/* Distance-1 colouring for the colouring variant (R17).                     */
/* ------------------------------------------------------------------------- */

/* Priority of vertex v: the output function of SplitMix64 (Steele, Lea, Flood 2014) applied
 * to v, a bijection of 64-bit values, so no two vertices tie. */
static uint64_t color_priority(int64_t v)
{
    uint64_t z = (uint64_t)v + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Jones-Plassmann rounds: every uncoloured vertex whose priority is above that of each of
 * its uncoloured non-loop neighbours takes the smallest colour none of its coloured
 * neighbours has; the vertices chosen in one round are pairwise non-adjacent, so the
 * order within a round does not matter.  Returns the number of colours, -1 on OOM. */
static int32_t color_graph(const og_graph *g, int32_t *color)
{
    int64_t n = g->n;
    uint8_t *pick = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    uint8_t *used = NULL;
    int64_t used_cap = 0;
    if (!pick) return -1;
    for (int64_t v = 0; v < n; v++) color[v] = -1;
    int64_t left = n;
    int32_t ncolors = 0;
    while (left > 0) {
        for (int64_t v = 0; v < n; v++) {
            pick[v] = 0;
            if (color[v] >= 0) continue;
            uint64_t pv = color_priority(v);
            int top = 1;
            for (int64_t k = g->rp[v]; k < g->rp[v + 1] && top; k++) {
                int32_t u = g->col[k];
                if (u != v && color[u] < 0 && color_priority(u) > pv) top = 0;
            }
            pick[v] = (uint8_t)top;
        }
        for (int64_t v = 0; v < n; v++) {
            if (!pick[v]) continue;
            int64_t d = g->rp[v + 1] - g->rp[v];
            if (d + 1 > used_cap) {
                free(used);
                used_cap = d + 1;
                used = (uint8_t *)malloc((size_t)used_cap);
                if (!used) {
                    free(pick);
                    return -1;
                }
            }
            memset(used, 0, (size_t)(d + 1));
            for (int64_t k = g->rp[v]; k < g->rp[v + 1]; k++) {
                int32_t cu = color[g->col[k]];
                if (g->col[k] != v && cu >= 0 && cu <= d) used[cu] = 1;
            }
            int32_t c = 0;
            while (used[c]) c++; /* at most d colours are taken: c <= d */
            color[v] = c;
            if (c + 1 > ncolors) ncolors = c + 1;
            left--;
        }
    }
    free(pick);
    free(used);
    return ncolors;
}

/* ------------------------------------------------------------------------- */
/* Renumbering (R8) and graph induction (R10).                               */
/* ------------------------------------------------------------------------- */

static int64_t renumber(int64_t n, const int32_t *C, int32_t *new_id)
{
    for (int64_t c = 0; c < n; c++) new_id[c] = -1;
    for (int64_t i = 0; i < n; i++) new_id[C[i]] = 0; /* mark used labels */
    int64_t k = 0;
    for (int64_t c = 0; c < n; c++)
        if (new_id[c] == 0) new_id[c] = (int32_t)k++;
        else new_id[c] = -1;
    return k;
}

static int cmp_i32(const void *x, const void *y)
{
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/* A'_ab = sum over u with new(C(u)) = a and entries (u, v) with new(C(v)) = b of A_uv.
 * Rows of the result list columns in ascending order. */
static int coarsen(const og_graph *g, const int32_t *C, const int32_t *new_id, int64_t k,
                   og_graph *out)
{
    int64_t n = g->n;
    int64_t *moff = (int64_t *)calloc((size_t)(k + 1), sizeof(int64_t));
    int32_t *members = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *acc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    int64_t *stamp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k > 0 ? k : 1));
    int64_t *cursor = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    int rc = ORACLE_OK;
    if (!moff || !members || !acc || !stamp || !touched || !cursor) {
        rc = ORACLE_ERR_OOM;
        goto done;
    }
    /* members of each new community, in vertex order */
    for (int64_t u = 0; u < n; u++) moff[new_id[C[u]] + 1] += 1;
    for (int64_t a = 0; a < k; a++) moff[a + 1] += moff[a];
    for (int64_t a = 0; a < k; a++) cursor[a] = moff[a];
    for (int64_t u = 0; u < n; u++) members[cursor[new_id[C[u]]]++] = (int32_t)u;
    for (int64_t a = 0; a < k; a++) stamp[a] = -1;

    /* the coarse graph has at most as many entries as the fine one */
    if (graph_alloc(out, k, g->nnz) != ORACLE_OK) {
        rc = ORACLE_ERR_OOM;
        goto done;
    }
    int64_t pos = 0;
    out->rp[0] = 0;
    for (int64_t a = 0; a < k; a++) {
        int64_t m = 0;
        for (int64_t p = moff[a]; p < moff[a + 1]; p++) {
            int32_t u = members[p];
            for (int64_t e = g->rp[u]; e < g->rp[u + 1]; e++) {
                int32_t b = new_id[C[g->col[e]]];
                if (stamp[b] != a) {
                    stamp[b] = a;
                    acc[b] = 0;
                    touched[m++] = b;
                }
                acc[b] += g->w[e];
            }
        }
        qsort(touched, (size_t)m, sizeof(int32_t), cmp_i32);
        for (int64_t t = 0; t < m; t++) {
            out->col[pos] = touched[t];
            out->w[pos] = acc[touched[t]];
            pos++;
        }
        out->rp[a + 1] = pos;
    }
    out->nnz = pos;
done:
    free(moff);
    free(members);
    free(acc);
    free(stamp);
    free(touched);
    free(cursor);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Full multi-level run (Algorithm 2 around Algorithm 1).                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t level;
    int32_t iter;   /* 1-based sweep index inside the level */
    int64_t moved;  /* vertices that changed label in this sweep */
    i128 qn;        /* Qn of the state after this sweep */
} og_trace;

typedef struct {
    int64_t n0;
    int64_t tw;
    int32_t num_levels;
    int32_t cap_levels;
    int32_t *labels;   /* num_levels * n0 */
    int64_t *ncomm;    /* communities after each level */
    i128 *qn;          /* Qn of each recorded level */
    i128 *qn_init;     /* Qn of the state before the first sweep of each recorded level */
    int32_t *iters;    /* sweeps applied in each recorded level */
    int64_t *n_level;  /* vertices of the graph the level ran on */
    int64_t *nnz_level;/* stored entries of that graph */
    int64_t trace_len, trace_cap;
    og_trace *trace;
    int64_t edge_visits; /* sum over all phases (recorded or not) of sweeps * nnz */
    int64_t sweeps_total;
    int32_t hit_iter_cap;
} og_result;

static void result_free(og_result *r)
{
    if (!r) return;
    free(r->labels);
    free(r->ncomm);
    free(r->qn);
    free(r->qn_init);
    free(r->iters);
    free(r->n_level);
    free(r->nnz_level);
    free(r->trace);
    free(r);
}

static int trace_push(og_result *r, int32_t level, int32_t iter, int64_t moved, i128 qn)
{
    if (r->trace_len == r->trace_cap) {
        int64_t cap = r->trace_cap ? 2 * r->trace_cap : 64;
        og_trace *t = (og_trace *)realloc(r->trace, sizeof(og_trace) * (size_t)cap);
        if (!t) return ORACLE_ERR_OOM;
        r->trace = t;
        r->trace_cap = cap;
    }
    r->trace[r->trace_len].level = level;
    r->trace[r->trace_len].iter = iter;
    r->trace[r->trace_len].moved = moved;
    r->trace[r->trace_len].qn = qn;
    r->trace_len++;
    return ORACLE_OK;
}

/* Post-phase merge of Sec. 5.1.2 (a variant, reading R15).  On the post-phase state C
 * (deg, size its community degrees), every vertex i whose non-loop neighbours all lie in
 * one community c != C(i) joins c when that move has a positive Eq. 4 gain:
 *   TW * e_{i->c} - delta_i * deg_c  >  TW * e_{i->C(i)} - delta_i * (deg_{C(i)} - delta_i),
 * with e_{i->C(i)} = 0 here (no neighbour shares i's community).  All decisions read the
 * same state; the moves are written to Cnext and returned as a count. */
static int64_t post_merge(const og_graph *g, const int32_t *C, const int64_t *deg,
                          const int64_t *delta, int64_t TW, int32_t *Cnext)
{
    int64_t moved = 0;
    for (int64_t i = 0; i < g->n; i++) {
        int32_t a = C[i];
        Cnext[i] = a;
        int32_t c = -1;
        int single = 1;
        int64_t e = 0;
        for (int64_t k = g->rp[i]; k < g->rp[i + 1]; k++) {
            int32_t j = g->col[k];
            if (j == (int32_t)i) continue; /* the loop is not a neighbour */
            if (c < 0) c = C[j];
            else if (C[j] != c) single = 0;
            e += g->w[k];
        }
        if (c < 0 || !single || c == a) continue;
        i128 g_move = (i128)TW * e - (i128)delta[i] * deg[c];
        i128 g_stay = -(i128)delta[i] * (deg[a] - delta[i]);
        if (g_move > g_stay) {
            Cnext[i] = c;
            moved++;
        }
    }
    return moved;
}

/* 192-bit unsigned product of a 128-bit and a 64-bit magnitude, limbs little-endian. */
typedef struct {
    uint64_t limb[3];
} u192;

static u192 mul_u128_u64(unsigned __int128 x, uint64_t m)
{
    unsigned __int128 lo = (unsigned __int128)(uint64_t)x * m;
    unsigned __int128 hi = (unsigned __int128)(uint64_t)(x >> 64) * m;
    unsigned __int128 mid = (lo >> 64) + (uint64_t)hi;
    u192 r;
    r.limb[0] = (uint64_t)lo;
    r.limb[1] = (uint64_t)mid;
    r.limb[2] = (uint64_t)(hi >> 64) + (uint64_t)(mid >> 64);
    return r;
}

static int u192_less(u192 a, u192 b)
{
    for (int k = 2; k >= 0; k--)
        if (a.limb[k] != b.limb[k]) return a.limb[k] < b.limb[k];
    return 0;
}

/* Threshold test of readings R7 / R9, exact:
 *   (qn_new - qn_old) * den < num * TW^2,
 * with den > 0, num >= 0, TW <= 2^62 (so |qn| <= TW^2 <= 2^124 and the difference
 * fits in 126 bits); both products are formed in 192 bits. */
static int below_threshold(i128 qn_new, i128 qn_old, int64_t tw, int64_t num, int64_t den)
{
    i128 diff = qn_new - qn_old;
    if (diff < 0) return 1; /* negative left side, non-negative right side */
    unsigned __int128 tw2 = (unsigned __int128)(uint64_t)tw * (uint64_t)tw;
    return u192_less(mul_u128_u64((unsigned __int128)diff, (uint64_t)den),
                     mul_u128_u64(tw2, (uint64_t)num));
}

/* Relative form of the phase test, as printed in Algorithm 1 (reading R14):
 *   |Q_curr - Q_prev| / |Q_prev| < theta   <=>   |qn_new - qn_old| * den < num * |qn_old|,
 * exact in 192 bits (both Qn carry the same factor TW^2).  Q_prev = 0 leaves the ratio
 * undefined; the test then holds only when Q did not change. */
static int below_threshold_rel(i128 qn_new, i128 qn_old, int64_t num, int64_t den)
{
    i128 diff = qn_new - qn_old;
    unsigned __int128 ad = (unsigned __int128)(diff < 0 ? -diff : diff);
    unsigned __int128 ao = (unsigned __int128)(qn_old < 0 ? -qn_old : qn_old);
    if (ao == 0) return ad == 0;
    return u192_less(mul_u128_u64(ad, (uint64_t)den), mul_u128_u64(ao, (uint64_t)num));
}

static int louvain_run_impl(const og_graph *g0, int64_t theta_num, int64_t theta_den,
                            int32_t max_iters, int32_t max_levels, int32_t vf, int32_t vf_all,
                            int32_t rel, int32_t merge, int32_t coloring, og_result *r)
{
    int64_t n0 = g0->n;
    og_graph g = {0, 0, NULL, NULL, NULL};
    og_graph next = {0, 0, NULL, NULL, NULL};
    int rc = ORACLE_OK;
    int64_t N = n0 > 0 ? n0 : 1;
    int32_t *map0 = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *C = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *Cnext = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *new_id = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *size = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *size_tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int64_t *delta = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *deg_tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *e = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *seen = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int32_t *color = coloring ? (int32_t *)malloc(sizeof(int32_t) * (size_t)N) : NULL;
    if (!map0 || !C || !Cnext || !new_id || !size || !size_tmp || !touched || !delta || !deg ||
        !deg_tmp || !e || !seen || (coloring && !color)) {
        rc = ORACLE_ERR_OOM;
        goto done;
    }
    if (graph_alloc(&g, g0->n, g0->nnz) != ORACLE_OK) {
        rc = ORACLE_ERR_OOM;
        goto done;
    }
    memcpy(g.rp, g0->rp, sizeof(int64_t) * (size_t)(g0->n + 1));
    if (g0->nnz > 0) {
        memcpy(g.col, g0->col, sizeof(int32_t) * (size_t)g0->nnz);
        memcpy(g.w, g0->w, sizeof(int64_t) * (size_t)g0->nnz);
    }
    for (int64_t v = 0; v < n0; v++) map0[v] = (int32_t)v;

    /* 2W = sum of every stored weight (R1); it is the same at every level (R10) */
    i128 tw128 = 0;
    for (int64_t k = 0; k < g.nnz; k++) tw128 += g.w[k];
    if (tw128 > ((i128)1 << 62)) {
        rc = ORACLE_ERR_INVALID;
        goto done;
    }
    int64_t TW = (int64_t)tw128;
    r->tw = TW;

    i128 qn_prev_level = 0;
    /* an empty vertex set gives Algorithm 1 nothing to evaluate: no phase is run (R13) */
    for (int32_t level = 0; level < max_levels && n0 > 0; level++) {
        int64_t n = g.n;
        /* initStatus: singletons, delta from the level's graph (Sec. 5.1.2) */
        weighted_degrees(&g, delta);
        for (int64_t i = 0; i < n; i++) C[i] = (int32_t)i;
        if (vf && (level == 0 || vf_all)) vertex_following(&g, C);
        community_degrees(n, C, delta, deg, size);
        for (int64_t i = 0; i < n; i++) seen[i] = 0;

        i128 qn_init = modularity_qn(&g, C, delta, TW, deg_tmp, size_tmp);
        i128 qn_prev = qn_init, qn_new = qn_init;
        int32_t iters = 0;
        int32_t ncolors = 1;
        if (coloring && (ncolors = color_graph(&g, color)) < 0) {
            rc = ORACLE_ERR_OOM;
            goto done;
        }
        for (;;) {
            /* one sweep: every vertex at once, or (R17) the colour classes one after the
             * other, each deciding on the state its predecessors left */
            int64_t moved = 0;
            for (int32_t cls = 0; cls < ncolors; cls++) {
                moved += local_move_sweep(&g, C, deg, size, delta, TW, Cnext, e, seen, touched,
                                          coloring ? color : NULL, cls);
                int32_t *t = C;
                C = Cnext;
                Cnext = t;
                community_degrees(n, C, delta, deg, size);
            }
            iters += 1;
            r->edge_visits += g.nnz;
            r->sweeps_total += 1;
            qn_new = modularity_qn(&g, C, delta, TW, deg_tmp, size_tmp);
            if ((rc = trace_push(r, level, iters, moved, qn_new)) != ORACLE_OK) goto done;
            if (moved == 0) break;
            if (rel ? below_threshold_rel(qn_new, qn_prev, theta_num, theta_den)
                    : below_threshold(qn_new, qn_prev, TW, theta_num, theta_den))
                break;
            if (iters >= max_iters) {
                r->hit_iter_cap = 1;
                break;
            }
            qn_prev = qn_new;
        }
        if (merge) { /* R15: after the phase, before renumbering; Qn of the merged state */
            post_merge(&g, C, deg, delta, TW, Cnext);
            int32_t *t = C;
            C = Cnext;
            Cnext = t;
            community_degrees(n, C, delta, deg, size);
            qn_new = modularity_qn(&g, C, delta, TW, deg_tmp, size_tmp);
        }

        int64_t k = renumber(n, C, new_id);
        if (k == n) break; /* nothing merged: no new level (R9) */

        for (int64_t v = 0; v < n0; v++) map0[v] = new_id[C[map0[v]]];
        int32_t L = r->num_levels;
        if (L == r->cap_levels) {
            rc = ORACLE_ERR_INVALID;
            goto done;
        }
        memcpy(r->labels + (size_t)L * (size_t)n0, map0, sizeof(int32_t) * (size_t)n0);
        r->ncomm[L] = k;
        r->qn[L] = qn_new;
        r->qn_init[L] = qn_init;
        r->iters[L] = iters;
        r->n_level[L] = n;
        r->nnz_level[L] = g.nnz;
        r->num_levels = L + 1;

        /* Algorithm 2 outer test, from the second level on (R9) */
        if (level >= 1 && below_threshold(qn_new, qn_prev_level, TW, theta_num, theta_den)) break;
        qn_prev_level = qn_new;
        if (level + 1 >= max_levels) break;

        if ((rc = coarsen(&g, C, new_id, k, &next)) != ORACLE_OK) goto done;
        graph_free(&g);
        g = next;
        next.rp = NULL;
        next.col = NULL;
        next.w = NULL;
    }
done:
    graph_free(&g);
    graph_free(&next);
    free(map0);
    free(C);
    free(Cnext);
    free(new_id);
    free(size);
    free(size_tmp);
    free(touched);
    free(delta);
    free(deg);
    free(deg_tmp);
    free(e);
    free(seen);
    free(color);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Exported entry points (loaded by the tests through ctypes).               */
/* ------------------------------------------------------------------------- */

static void put_i128(i128 v, int64_t out[2])
{
    out[0] = (int64_t)(v >> 64);             /* high limb, signed */
    out[1] = (int64_t)(uint64_t)(v & (i128)UINT64_MAX); /* low limb, bit pattern */
}

int32_t oracle_abi_version(void) { return 1; }

/* Full run.  Returns an opaque result or NULL; *status gets ORACLE_OK / _INVALID / _OOM.
 * threshold_mode 0: absolute phase test (R7); 1: relative phase test of Algorithm 1 (R14).
 * The outer test of Algorithm 2 is absolute in both modes.  post_merge_on: the post-phase
 * merge of Sec. 5.1.2 (R15) after every phase. */
void *oracle_run_ex(int64_t n, const int64_t *rp, const int32_t *col, const int32_t *w,
                    int64_t theta_num, int64_t theta_den, int32_t max_iters, int32_t max_levels,
                    int32_t vertex_following_on, int32_t vf_all_levels, int32_t threshold_mode,
                    int32_t post_merge_on, int32_t coloring, int32_t *status)
{
    if (threshold_mode != 0 && threshold_mode != 1) {
        if (status) *status = ORACLE_ERR_INVALID;
        return NULL;
    }
    og_graph g = {0, 0, NULL, NULL, NULL};
    int rc = graph_from_input(&g, n, rp, col, w, NULL);
    if (rc != ORACLE_OK || theta_den <= 0 || theta_num < 0 || theta_den > INT32_MAX ||
        theta_num > INT32_MAX || max_iters < 1 || max_levels < 1) {
        if (rc == ORACLE_OK) rc = ORACLE_ERR_INVALID;
        graph_free(&g);
        if (status) *status = rc;
        return NULL;
    }
    og_result *r = (og_result *)calloc(1, sizeof(og_result));
    if (!r) {
        graph_free(&g);
        if (status) *status = ORACLE_ERR_OOM;
        return NULL;
    }
    r->n0 = n;
    r->cap_levels = max_levels;
    size_t L = (size_t)max_levels;
    r->labels = (int32_t *)malloc(sizeof(int32_t) * L * (size_t)(n > 0 ? n : 1));
    r->ncomm = (int64_t *)calloc(L, sizeof(int64_t));
    r->qn = (i128 *)calloc(L, sizeof(i128));
    r->qn_init = (i128 *)calloc(L, sizeof(i128));
    r->iters = (int32_t *)calloc(L, sizeof(int32_t));
    r->n_level = (int64_t *)calloc(L, sizeof(int64_t));
    r->nnz_level = (int64_t *)calloc(L, sizeof(int64_t));
    if (!r->labels || !r->ncomm || !r->qn || !r->qn_init || !r->iters || !r->n_level ||
        !r->nnz_level) {
        graph_free(&g);
        result_free(r);
        if (status) *status = ORACLE_ERR_OOM;
        return NULL;
    }
    rc = louvain_run_impl(&g, theta_num, theta_den, max_iters, max_levels, vertex_following_on,
                          vf_all_levels, threshold_mode, post_merge_on, coloring != 0, r);
    graph_free(&g);
    if (rc != ORACLE_OK) {
        result_free(r);
        r = NULL;
    }
    if (status) *status = rc;
    return r;
}

void *oracle_run(int64_t n, const int64_t *rp, const int32_t *col, const int32_t *w,
                 int64_t theta_num, int64_t theta_den, int32_t max_iters, int32_t max_levels,
                 int32_t vertex_following_on, int32_t vf_all_levels, int32_t *status)
{
    return oracle_run_ex(n, rp, col, w, theta_num, theta_den, max_iters, max_levels,
                         vertex_following_on, vf_all_levels, 0, 0, 0, status);
}

int32_t oracle_res_num_levels(const void *h) { return ((const og_result *)h)->num_levels; }
int64_t oracle_res_tw(const void *h) { return ((const og_result *)h)->tw; }
int64_t oracle_res_edge_visits(const void *h) { return ((const og_result *)h)->edge_visits; }
int64_t oracle_res_sweeps(const void *h) { return ((const og_result *)h)->sweeps_total; }
int32_t oracle_res_hit_iter_cap(const void *h) { return ((const og_result *)h)->hit_iter_cap; }

/* Level l: labels of the original vertices (n0), community count, Qn (two limbs),
 * Qn before the first sweep, sweeps, graph size the level ran on, and
 * Q = (double)Qn / (double)TW^2. */
void oracle_res_level(const void *h, int32_t l, int32_t *labels, int64_t *ncomm, int64_t qn[2],
                      int64_t qn_init[2], int32_t *iters, int64_t *n_level, int64_t *nnz_level,
                      double *q)
{
    const og_result *r = (const og_result *)h;
    if (labels)
        memcpy(labels, r->labels + (size_t)l * (size_t)r->n0, sizeof(int32_t) * (size_t)r->n0);
    if (ncomm) *ncomm = r->ncomm[l];
    if (qn) put_i128(r->qn[l], qn);
    if (qn_init) put_i128(r->qn_init[l], qn_init);
    if (iters) *iters = r->iters[l];
    if (n_level) *n_level = r->n_level[l];
    if (nnz_level) *nnz_level = r->nnz_level[l];
    if (q) {
        i128 tw2 = (i128)r->tw * r->tw;
        *q = (double)r->qn[l] / (double)tw2;
    }
}

int64_t oracle_res_trace_len(const void *h) { return ((const og_result *)h)->trace_len; }

void oracle_res_trace(const void *h, int32_t *level, int32_t *iter, int64_t *moved, int64_t *qn)
{
    const og_result *r = (const og_result *)h;
    for (int64_t t = 0; t < r->trace_len; t++) {
        level[t] = r->trace[t].level;
        iter[t] = r->trace[t].iter;
        moved[t] = r->trace[t].moved;
        put_i128(r->trace[t].qn, qn + 2 * t);
    }
}

void oracle_res_free(void *h) { result_free((og_result *)h); }

/* ---- single steps, exposed so the tests can pin each against the paper ---- */

/* Colouring of reading R17 for graph (n, rp, col): colour of every vertex into color_out;
 * returns the number of colours, or -1 on bad input. */
int32_t oracle_color(int64_t n, const int64_t *rp, const int32_t *col, int32_t *color_out)
{
    og_graph g = {0, 0, NULL, NULL, NULL};
    if (graph_from_input(&g, n, rp, col, NULL, NULL) != ORACLE_OK) return -1;
    int32_t k = color_graph(&g, color_out);
    graph_free(&g);
    return k;
}

/* Eq. 3 times TW^2 for labels C (values in [0, n)).  Returns TW, or -1 on bad input. */
int64_t oracle_modularity(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
                          const int32_t *C, int64_t qn_out[2])
{
    og_graph g = {0, 0, NULL, NULL, NULL};
    if (graph_from_input(&g, n, rp, col, NULL, w) != ORACLE_OK) return -1;
    int64_t N = n > 0 ? n : 1;
    int64_t *delta = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int32_t *size = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    weighted_degrees(&g, delta);
    int64_t TW = 0;
    for (int64_t i = 0; i < n; i++) TW += delta[i];
    i128 qn = modularity_qn(&g, C, delta, TW, deg, size);
    put_i128(qn, qn_out);
    free(delta);
    free(deg);
    free(size);
    graph_free(&g);
    return TW;
}

/* (2W)^2/2 times the Eq. 4 gain of moving vertex i from C(i) to community b != C(i):
 * G_b - G_stay (reading R3), computed from the definitions of Eq. 1-2 on state C. */
void oracle_gain(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
                 const int32_t *C, int64_t i, int32_t b, int64_t out[2])
{
    og_graph g = {0, 0, NULL, NULL, NULL};
    if (graph_from_input(&g, n, rp, col, NULL, w) != ORACLE_OK) {
        out[0] = out[1] = 0;
        return;
    }
    int64_t N = n > 0 ? n : 1;
    int64_t *delta = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int32_t *size = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    weighted_degrees(&g, delta);
    community_degrees(n, C, delta, deg, size);
    int64_t TW = 0;
    for (int64_t v = 0; v < n; v++) TW += delta[v];
    int32_t a = C[i];
    int64_t e_a = 0, e_b = 0;
    for (int64_t k = g.rp[i]; k < g.rp[i + 1]; k++) {
        int32_t j = g.col[k];
        if (j == i) continue;
        if (C[j] == a) e_a += g.w[k];
        if (C[j] == b) e_b += g.w[k];
    }
    i128 g_b = (i128)TW * e_b - (i128)delta[i] * deg[b];
    i128 g_stay = (i128)TW * e_a - (i128)delta[i] * (deg[a] - delta[i]);
    put_i128(g_b - g_stay, out);
    free(delta);
    free(deg);
    free(size);
    graph_free(&g);
}

/* One synchronous sweep from state C (deg and size derived from C).  Returns moved,
 * or -1 on bad input. */
int64_t oracle_sweep(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
                     const int32_t *C, int32_t *Cnext)
{
    og_graph g = {0, 0, NULL, NULL, NULL};
    if (graph_from_input(&g, n, rp, col, NULL, w) != ORACLE_OK) return -1;
    int64_t N = n > 0 ? n : 1;
    int64_t *delta = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int32_t *size = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int64_t *e = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *seen = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    weighted_degrees(&g, delta);
    community_degrees(n, C, delta, deg, size);
    int64_t TW = 0;
    for (int64_t v = 0; v < n; v++) TW += delta[v];
    for (int64_t v = 0; v < n; v++) seen[v] = 0;
    int64_t moved = local_move_sweep(&g, C, deg, size, delta, TW, Cnext, e, seen, touched,
                                     NULL, 0);
    free(delta);
    free(deg);
    free(size);
    free(e);
    free(seen);
    free(touched);
    graph_free(&g);
    return moved;
}

void oracle_vertex_following(int64_t n, const int64_t *rp, const int32_t *col, int32_t *C)
{
    og_graph g = {0, 0, NULL, NULL, NULL};
    if (graph_from_input(&g, n, rp, col, NULL, NULL) != ORACLE_OK) return;
    vertex_following(&g, C);
    graph_free(&g);
}

/* Exact threshold test on two Qn values given as (high, low) limbs. */
int32_t oracle_below_threshold(const int64_t qn_new[2], const int64_t qn_old[2], int64_t tw,
                               int64_t num, int64_t den)
{
    i128 a = ((i128)qn_new[0] << 64) | (i128)(uint64_t)qn_new[1];
    i128 b = ((i128)qn_old[0] << 64) | (i128)(uint64_t)qn_old[1];
    return below_threshold(a, b, tw, num, den);
}

int64_t oracle_renumber(int64_t n, const int32_t *C, int32_t *new_id)
{
    return renumber(n, C, new_id);
}

/* Coarse graph of partition C (labels in [0, n)).  Returns an opaque graph or NULL. */
void *oracle_coarsen(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *w,
                     const int32_t *C)
{
    og_graph g = {0, 0, NULL, NULL, NULL};
    if (graph_from_input(&g, n, rp, col, NULL, w) != ORACLE_OK) return NULL;
    int32_t *new_id = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t k = renumber(n, C, new_id);
    og_graph *out = (og_graph *)calloc(1, sizeof(og_graph));
    if (!out || coarsen(&g, C, new_id, k, out) != ORACLE_OK) {
        free(out);
        out = NULL;
    }
    free(new_id);
    graph_free(&g);
    return out;
}

int64_t oracle_graph_n(const void *h) { return ((const og_graph *)h)->n; }
int64_t oracle_graph_nnz(const void *h) { return ((const og_graph *)h)->nnz; }

void oracle_graph_copy(const void *h, int64_t *rp, int32_t *col, int64_t *w)
{
    const og_graph *g = (const og_graph *)h;
    memcpy(rp, g->rp, sizeof(int64_t) * (size_t)(g->n + 1));
    if (g->nnz > 0) {
        memcpy(col, g->col, sizeof(int32_t) * (size_t)g->nnz);
        memcpy(w, g->w, sizeof(int64_t) * (size_t)g->nnz);
    }
}

void oracle_graph_free(void *h)
{
    og_graph *g = (og_graph *)h;
    graph_free(g);
    free(g);
}
