/*
 * graphgen.c -- seeded synthetic graph generators (input data only).
 *
 * Produces undirected, loop-free, duplicate-free graphs as symmetric CSR with rows
 * sorted by column, int32 ids and int32 weights drawn per undirected edge.  Nothing
 * here computes any part of community detection; the generators feed both the CPU
 * oracle and the CUDA library with identical inputs.
 *
 * Randomness is counter-based: every draw is mix64(key + (ctr + 1) * golden), where
 * mix64 is the SplitMix64 output function (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) and key is derived from the seed and
 * a stream number.  Results are therefore independent of thread count and schedule.
 * Probabilities are compared as 64-bit integer thresholds; floating point is used only
 * where a model is defined by real-valued weights (Chung-Lu).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t stream_key(uint64_t seed, uint64_t stream)
{
    return mix64(mix64(seed) + stream * 0xD1B54A32D192ED03ULL);
}

static inline uint64_t cb64(uint64_t key, uint64_t ctr) { return mix64(key + (ctr + 1) * GOLDEN); }

/* threshold t with P(u < t) = p for u uniform on [0, 2^64) */
static uint64_t prob_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return UINT64_MAX;
    return (uint64_t)ldexp(p, 64);
}

enum { STREAM_PAIRS = 1, STREAM_WEIGHTS = 2, STREAM_INTER = 3 };

uint64_t gg_mix64(uint64_t z) { return mix64(z); }
uint64_t gg_cb64(uint64_t key, uint64_t ctr) { return cb64(key, ctr); }
uint64_t gg_stream_key(uint64_t seed, uint64_t stream) { return stream_key(seed, stream); }

typedef struct {
    int64_t n;
    int64_t nnz;
    int64_t *rp;
    int32_t *col;
    int32_t *w;
} gg_graph;

static int cmp_i32(const void *x, const void *y)
{
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

static void sort_small(int32_t *a, int64_t m)
{
    for (int64_t i = 1; i < m; i++) {
        int32_t x = a[i];
        int64_t j = i - 1;
        while (j >= 0 && a[j] > x) {
            a[j + 1] = a[j];
            j--;
        }
        a[j + 1] = x;
    }
}

/* weight of undirected edge {u, v}, identical for both stored directions */
static inline int32_t edge_weight(uint64_t wkey, int32_t u, int32_t v, int32_t wmin, int32_t wmax)
{
    uint32_t lo = (uint32_t)(u < v ? u : v), hi = (uint32_t)(u < v ? v : u);
    uint64_t span = (uint64_t)((int64_t)wmax - (int64_t)wmin + 1);
    return (int32_t)((int64_t)wmin + (int64_t)(cb64(wkey, ((uint64_t)lo << 32) | hi) % span));
}

/* Symmetric CSR from undirected pairs (pu[k], pv[k]); loops dropped, duplicates merged
 * (a duplicate keeps the same weight because weights depend only on the pair). */
static gg_graph *build_csr(int64_t n, int64_t npairs, const int32_t *pu, const int32_t *pv,
                           int32_t wmin, int32_t wmax, uint64_t seed)
{
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    int64_t *cnt = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    if (!g || !cnt) goto fail;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < npairs; k++) {
        if (pu[k] == pv[k]) continue;
#pragma omp atomic
        cnt[pu[k] + 1] += 1;
#pragma omp atomic
        cnt[pv[k] + 1] += 1;
    }
    for (int64_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    int64_t total = cnt[n];
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!tmp || !cur) {
        free(tmp);
        free(cur);
        goto fail;
    }
    memcpy(cur, cnt, sizeof(int64_t) * (size_t)n);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < npairs; k++) {
        int32_t u = pu[k], v = pv[k];
        if (u == v) continue;
        int64_t p, q;
#pragma omp atomic capture
        p = cur[u]++;
#pragma omp atomic capture
        q = cur[v]++;
        tmp[p] = v;
        tmp[q] = u;
    }
    free(cur);
    /* sort and dedup each row in place; row length after dedup into deg */
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!deg) {
        free(tmp);
        goto fail;
    }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; i++) {
        int32_t *row = tmp + cnt[i];
        int64_t m = cnt[i + 1] - cnt[i];
        if (m <= 32) sort_small(row, m);
        else qsort(row, (size_t)m, sizeof(int32_t), cmp_i32);
        int64_t d = 0;
        for (int64_t t = 0; t < m; t++)
            if (d == 0 || row[t] != row[d - 1]) row[d++] = row[t];
        deg[i] = d;
    }
    g->n = n;
    g->rp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!g->rp) {
        free(tmp);
        free(deg);
        goto fail;
    }
    g->rp[0] = 0;
    for (int64_t i = 0; i < n; i++) g->rp[i + 1] = g->rp[i] + deg[i];
    g->nnz = g->rp[n];
    g->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->nnz > 0 ? g->nnz : 1));
    g->w = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->nnz > 0 ? g->nnz : 1));
    if (!g->col || !g->w) {
        free(tmp);
        free(deg);
        goto fail;
    }
    uint64_t wkey = stream_key(seed, STREAM_WEIGHTS);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; i++) {
        const int32_t *row = tmp + cnt[i];
        int64_t base = g->rp[i];
        for (int64_t t = 0; t < deg[i]; t++) {
            g->col[base + t] = row[t];
            g->w[base + t] = edge_weight(wkey, (int32_t)i, row[t], wmin, wmax);
        }
    }
    free(tmp);
    free(deg);
    free(cnt);
    return g;
fail:
    free(cnt);
    if (g) {
        free(g->rp);
        free(g->col);
        free(g->w);
        free(g);
    }
    return NULL;
}

/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004): edge_factor * 2^scale sampled pairs, each
 * bit level choosing quadrant (0,0) w.p. a, (0,1) b, (1,0) c, (1,1) 1-a-b-c, most
 * significant bit first; no noise, no vertex permutation.  Symmetrised, loops and
 * duplicates dropped, weights uniform in [wmin, wmax]. */
void *gg_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c, int32_t wmin,
              int32_t wmax, uint64_t seed)
{
    if (scale < 1 || scale > 30 || edge_factor < 1 || wmin < 1 || wmax < wmin) return NULL;
    int64_t n = (int64_t)1 << scale;
    int64_t m = (int64_t)edge_factor * n;
    int32_t *pu = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    int32_t *pv = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    if (!pu || !pv) {
        free(pu);
        free(pv);
        return NULL;
    }
    uint64_t ta = (uint64_t)ldexp(a, 32), tab = (uint64_t)ldexp(a + b, 32),
             tabc = (uint64_t)ldexp(a + b + c, 32);
    uint64_t key = stream_key(seed, STREAM_PAIRS);
    int64_t per_pair = (scale + 1) / 2; /* one 64-bit draw covers two bit levels */
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m; k++) {
        uint32_t u = 0, v = 0;
        uint64_t r = 0;
        for (int32_t l = 0; l < scale; l++) {
            if ((l & 1) == 0) r = cb64(key, (uint64_t)k * (uint64_t)per_pair + (uint64_t)(l / 2));
            uint64_t x = (l & 1) ? (r >> 32) : (r & 0xFFFFFFFFULL);
            uint32_t bu, bv;
            if (x < ta) {
                bu = 0;
                bv = 0;
            } else if (x < tab) {
                bu = 0;
                bv = 1;
            } else if (x < tabc) {
                bu = 1;
                bv = 0;
            } else {
                bu = 1;
                bv = 1;
            }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        pu[k] = (int32_t)u;
        pv[k] = (int32_t)v;
    }
    gg_graph *g = build_csr(n, m, pu, pv, wmin, wmax, seed);
    free(pu);
    free(pv);
    return g;
}

/* Planted partition (stochastic block model): n vertices in consecutive blocks of
 * block_size (the last one may be shorter); each intra-block pair is an edge with
 * probability p_in.  Inter-block pairs: when n <= exact_limit every pair is an edge
 * with probability p_out; above it, round(p_out * #inter-block pairs) pairs are drawn
 * uniformly among inter-block pairs (duplicates merged). */
void *gg_sbm(int64_t n, int64_t block_size, double p_in, double p_out, int32_t wmin, int32_t wmax,
             uint64_t seed, int64_t exact_limit)
{
    if (n < 0 || n > INT32_MAX || block_size < 1 || wmin < 1 || wmax < wmin) return NULL;
    uint64_t tin = prob_threshold(p_in), tout = prob_threshold(p_out);
    uint64_t kin = stream_key(seed, STREAM_PAIRS), kout = stream_key(seed, STREAM_INTER);
    int64_t nblocks = (n + block_size - 1) / block_size;
    /* pass 1 counts accepted pairs (i < j) of each row i, pass 2 writes them */
    int64_t *cnt = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    if (!cnt) return NULL;
    int exact = n <= exact_limit;
    /* intra-block pairs (and all pairs in exact mode), row-parallel */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        int64_t bi = i / block_size;
        int64_t bend = (bi + 1) * block_size < n ? (bi + 1) * block_size : n;
        int64_t c = 0;
        int64_t jend = exact ? n : bend;
        for (int64_t j = i + 1; j < jend; j++) {
            uint64_t t = (j < bend) ? tin : tout;
            uint64_t key = (j < bend) ? kin : kout;
            if (cb64(key, (uint64_t)i * (uint64_t)n + (uint64_t)j) < t) c++;
        }
        cnt[i + 1] = c;
    }
    for (int64_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    int64_t m_intra = cnt[n];
    int64_t m_inter = 0;
    if (!exact && nblocks > 1) {
        /* number of inter-block pairs */
        double pairs = 0.0;
        for (int64_t bi = 0; bi < nblocks; bi++) {
            int64_t bend = (bi + 1) * block_size < n ? (bi + 1) * block_size : n;
            pairs += (double)(bend - bi * block_size) * (double)(n - bend);
        }
        m_inter = (int64_t)llround(p_out * pairs);
    }
    int64_t m = m_intra + m_inter;
    int32_t *pu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int32_t *pv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!pu || !pv) {
        free(pu);
        free(pv);
        free(cnt);
        return NULL;
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        int64_t bi = i / block_size;
        int64_t bend = (bi + 1) * block_size < n ? (bi + 1) * block_size : n;
        int64_t p = cnt[i];
        int64_t jend = exact ? n : bend;
        for (int64_t j = i + 1; j < jend; j++) {
            uint64_t t = (j < bend) ? tin : tout;
            uint64_t key = (j < bend) ? kin : kout;
            if (cb64(key, (uint64_t)i * (uint64_t)n + (uint64_t)j) < t) {
                pu[p] = (int32_t)i;
                pv[p] = (int32_t)j;
                p++;
            }
        }
    }
    free(cnt);
    /* inter-block pairs by uniform rejection sampling (non-exact mode only) */
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m_inter; k++) {
        uint64_t ctr = (uint64_t)k << 8;
        for (;;) {
            uint64_t r1 = cb64(kout, ctr++), r2 = cb64(kout, ctr++);
            int64_t u = (int64_t)(r1 % (uint64_t)n), v = (int64_t)(r2 % (uint64_t)n);
            if (u / block_size == v / block_size) continue;
            pu[m_intra + k] = (int32_t)u;
            pv[m_intra + k] = (int32_t)v;
            break;
        }
    }
    gg_graph *g = build_csr(n, m, pu, pv, wmin, wmax, seed);
    free(pu);
    free(pv);
    return g;
}

/* Chung-Lu power law: expected weight theta_i proportional to (i+1)^(-1/(gamma-1)),
 * scaled to mean avg_deg and capped at sqrt(sum theta); m = avg_deg * n / 2 endpoint
 * pairs, each endpoint drawn proportional to theta (inverse CDF); loops and duplicates
 * dropped. */
void *gg_chung_lu(int64_t n, double gamma, double avg_deg, int32_t wmin, int32_t wmax,
                  uint64_t seed)
{
    if (n < 2 || n > INT32_MAX || gamma <= 1.0 || avg_deg <= 0 || wmin < 1 || wmax < wmin)
        return NULL;
    double *cdf = (double *)malloc(sizeof(double) * (size_t)n);
    if (!cdf) return NULL;
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) {
        cdf[i] = pow((double)(i + 1), -1.0 / (gamma - 1.0));
        s += cdf[i];
    }
    double scale = avg_deg * (double)n / s;
    double total = 0.0;
    for (int64_t i = 0; i < n; i++) total += cdf[i] * scale;
    double cap = sqrt(total);
    double acc = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double t = cdf[i] * scale;
        if (t > cap) t = cap;
        acc += t;
        cdf[i] = acc;
    }
    int64_t m = (int64_t)llround(avg_deg * (double)n / 2.0);
    int32_t *pu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int32_t *pv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!pu || !pv) {
        free(cdf);
        free(pu);
        free(pv);
        return NULL;
    }
    uint64_t key = stream_key(seed, STREAM_PAIRS);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < 2 * m; k++) {
        double u = (double)(cb64(key, (uint64_t)k) >> 11) * 0x1.0p-53 * acc;
        int64_t lo = 0, hi = n - 1;
        while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (cdf[mid] > u) hi = mid;
            else lo = mid + 1;
        }
        if (k < m) pu[k] = (int32_t)lo;
        else pv[k - m] = (int32_t)lo;
    }
    free(cdf);
    gg_graph *g = build_csr(n, m, pu, pv, wmin, wmax, seed);
    free(pu);
    free(pv);
    return g;
}

/* CSR from caller pairs (loops dropped, duplicates merged, weights from the seed) */
void *gg_from_pairs(int64_t n, int64_t m, const int32_t *pu, const int32_t *pv, int32_t wmin,
                    int32_t wmax, uint64_t seed)
{
    if (n < 0 || n > INT32_MAX || m < 0 || wmin < 1 || wmax < wmin) return NULL;
    for (int64_t k = 0; k < m; k++)
        if (pu[k] < 0 || pu[k] >= n || pv[k] < 0 || pv[k] >= n) return NULL;
    return build_csr(n, m, pu, pv, wmin, wmax, seed);
}

int64_t gg_graph_n(const void *h) { return ((const gg_graph *)h)->n; }
int64_t gg_graph_nnz(const void *h) { return ((const gg_graph *)h)->nnz; }

void gg_graph_copy(const void *h, int64_t *rp, int32_t *col, int32_t *w)
{
    const gg_graph *g = (const gg_graph *)h;
    memcpy(rp, g->rp, sizeof(int64_t) * (size_t)(g->n + 1));
    if (g->nnz > 0) {
        memcpy(col, g->col, sizeof(int32_t) * (size_t)g->nnz);
        memcpy(w, g->w, sizeof(int32_t) * (size_t)g->nnz);
    }
}

void gg_graph_free(void *h)
{
    gg_graph *g = (gg_graph *)h;
    if (!g) return;
    free(g->rp);
    free(g->col);
    free(g->w);
    free(g);
}

int gg_openmp_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
