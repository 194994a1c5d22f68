// k_level.cu -- per-level kernels around the local-moving sweep.
//
//   validation of the input CSR (Sec. 2 graph model),
//   weighted degrees delta_i and 2W (Sec. 2, "initStatus" of Sec. 5.1.2),
//   degree-one vertex following (Lu et al.; Sec. 7 "other heuristics"),
//   degree binning of the vertices (Sec. 6.3: group vertices of similar degree),
//   the phase controller (Algorithm 1 stopping rule on exact Qn = (2W)^2 Q, Eq. 3),
//   applying a sweep's moves with deg_C / size_C updates (Sec. 5.1.2 "oneLevelKernel"),
//   renumbering by prefix-sum compaction and label composition (Sec. 5.1.2).
#include <climits>

#include "lv_common.cuh"
#include "lv_kernels.h"
#include "lv_scan.cuh"

namespace lv {

// ------------------------------------------------------------------ validation

__global__ void __launch_bounds__(kBlock) k_validate_rowptr(const int64_t *rp, int64_t n,
                                                            unsigned *err)
{
    unsigned bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i == 0 && rp[0] != 0) bad |= ERRF_ROWPTR;
        if (rp[i + 1] < rp[i]) bad |= ERRF_ROWPTR;
    }
    if (bad) atomicOr(err, bad);
}

int launch_validate_rowptr(const int64_t *rp, int64_t n, unsigned *err, cudaStream_t s,
                           const LaunchCfg &lc)
{
    if (n == 0) return 0;
    k_validate_rowptr<<<grid_for(n, kBlock, lc.max_blocks), kBlock, 0, s>>>(rp, n, err);
    return 1;
}

// Entry checks of one graph on its own (columns in [0, n), weights >= 1) and its 2W, one
// warp per row; used to vet a graph before it joins others.
__global__ void __launch_bounds__(kBlock) k_check_rows(int64_t n, const int64_t *rp,
                                                       const int32_t *col, const int32_t *w,
                                                       unsigned *err, u64 *tw)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned bad = 0;
    u64 sum = 0;
    for (int64_t i = warp; i < n; i += nwarps) {
        for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += 32) {
            const int32_t j = col[k];
            const i64 x = w ? (i64)w[k] : 1;
            if (j < 0 || (int64_t)j >= n) bad |= ERRF_INDEX;
            if (x < 1) bad |= ERRF_WEIGHT;
            sum += (u64)x;
        }
    }
    sum = sum_reduce(sum, 32);
    if (lane == 0 && sum) atomicAdd(tw, sum);
    if (bad) atomicOr(err, bad);
}

int launch_check_rows(int64_t n, const int64_t *rp, const int32_t *col, const int32_t *w,
                      unsigned *err, u64 *tw, cudaStream_t s, const LaunchCfg &lc)
{
    if (n == 0) return 0;
    k_check_rows<<<grid_for(n, kBlock / 32, lc.max_blocks), kBlock, 0, s>>>(n, rp, col, w, err,
                                                                           tw);
    return 1;
}

__global__ void k_fill_ones(int32_t *w, int64_t nnz)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        w[k] = 1;
}

int launch_fill_ones(int32_t *w, int64_t nnz, cudaStream_t s, const LaunchCfg &lc)
{
    if (nnz == 0) return 0;
    k_fill_ones<<<grid_for(nnz, kBlock, lc.max_blocks), kBlock, 0, s>>>(w, nnz);
    return 1;
}

// Largest weighted degree of the level: every table sum e_{i->c} of a sweep is at most
// delta_i, and every gain of vertex i is at most 2W * delta_i in magnitude, so this bound
// picks the narrowest exact sum and gain widths of the level's sweeps.
__global__ void __launch_bounds__(kBlock) k_max_delta(const i64 *delta, int64_t n, u64 *out)
{
    u64 m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (u64)delta[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax((unsigned long long *)out, (unsigned long long)m);
}

int launch_max_delta(const i64 *delta, int64_t n, u64 *out, cudaStream_t s, const LaunchCfg &lc)
{
    cudaMemsetAsync(out, 0, sizeof(u64), s);
    if (n == 0) return 0;
    k_max_delta<<<grid_for(n, kBlock, lc.max_blocks), kBlock, 0, s>>>(delta, n, out);
    return 1;
}

// delta_i = sum of row i's weights (loop once), 2W = sum delta; columns and weights are
// checked on the way.  Rows of bin 0 take one thread each (dense kernel), rows of bins 1-4
// one warp each, longer rows one CTA each, so a hub row never serialises on one warp.
// In a batch (vg set) 2W is per graph and a column must stay inside its row's graph.
// unsorted[g] is set when a row of graph g does not list strictly increasing columns (then
// a column may repeat, and the first sweep of its phase cannot score entries one by one).
struct RowCtx {
    int64_t n;
    const int32_t *vg;
    const int64_t *gptr;
    u64 *tw;
    unsigned *unsorted;
    __device__ __forceinline__ void flag_unsorted(int g) const
    {
        if (!*(volatile unsigned *)&unsorted[g]) atomicOr(&unsorted[g], 1u);
    }
    __device__ __forceinline__ int graph(int64_t i) const { return vg ? vg[i] : 0; }
    __device__ __forceinline__ void range(int g, int64_t &lo, int64_t &hi) const
    {
        lo = vg ? gptr[g] : 0;
        hi = vg ? gptr[g + 1] : n;
    }
};

__device__ __forceinline__ void check_entry(int32_t j, i64 x, int64_t lo, int64_t hi, unsigned &bad)
{
    if ((int64_t)j < lo || (int64_t)j >= hi) bad |= ERRF_INDEX;
    if (x < 1) bad |= ERRF_WEIGHT;
}

// 2W of one graph accumulated by a thread over the rows it visits: flushed to tw[g] when the
// graph changes (rows of a batch are grouped by graph) and at the end, so a one-graph run
// issues one atomic per thread instead of one per row.
struct TwAcc {
    int g = -1;
    u64 s = 0;
    __device__ __forceinline__ void add(const RowCtx &R, int gr, u64 x)
    {
        if (gr != g) {
            if (g >= 0 && s) atomicAdd(&R.tw[g], s);
            g = gr;
            s = 0;
        }
        s += x;
    }
    __device__ __forceinline__ void flush(const RowCtx &R)
    {
        if (g >= 0 && s) atomicAdd(&R.tw[g], s);
        g = -1;
        s = 0;
    }
    // every lane of the warp calls this: one atomic per warp when the lanes share a graph
    __device__ __forceinline__ void flush_warp(const RowCtx &R)
    {
        const int g0 = __shfl_sync(0xffffffffu, g, 0);
        if (__all_sync(0xffffffffu, g == g0 || s == 0)) {
            const u64 t = sum_reduce(s, 32);
            if ((threadIdx.x & 31) == 0 && g0 >= 0 && t) atomicAdd(&R.tw[g0], t);
            g = -1;
            s = 0;
        } else {
            flush(R);
        }
    }
};

// Rows of at most dmax (<= 8) entries, one thread each: the row's entries are loaded
// together into registers, then checked and summed.
template <typename WT>
__global__ void __launch_bounds__(kBlock) k_row_sums_thread(RowCtx R, const int64_t *rp,
                                                            const int32_t *col, const WT *w,
                                                            int64_t dmax, i64 *delta,
                                                            unsigned *err)
{
    constexpr int kMax = 8;
    unsigned bad = 0;
    TwAcc acc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rp[i], e = rp[i + 1];
        const int64_t d = e - b;
        if (d > dmax) continue;
        int32_t j[kMax];
        i64 x[kMax];
#pragma unroll
        for (int t = 0; t < kMax; t++) {
            j[t] = t < d ? ld_stream(col + b + t) : 0;
            x[t] = t < d ? (i64)ld_stream(w + b + t) : 1;
        }
        const int g = R.graph(i);
        int64_t lo, hi;
        R.range(g, lo, hi);
        u64 sum = 0;
        bool uns = false;
#pragma unroll
        for (int t = 0; t < kMax; t++) {
            if (t < d) {
                check_entry(j[t], x[t], lo, hi, bad);
                if (t > 0) uns = uns || j[t] <= j[t - 1];
                sum += (u64)x[t];
            }
        }
        delta[i] = (i64)sum;
        if (uns) R.flag_unsorted(g);
        acc.add(R, g, sum);
    }
    acc.flush_warp(R);
    if (bad) atomicOr(err, bad);
}

// One warp per row (bins 1-4), four entries in flight per lane; the previous entry of a
// lane's entry (for the order check) is its left neighbour's, or the last of the round before.
template <typename WT>
__global__ void __launch_bounds__(kBlock) k_row_sums_warp(RowCtx R, const int64_t *rp,
                                                          const int32_t *col, const WT *w,
                                                          const int32_t *rows, int64_t nrows,
                                                          i64 *delta, unsigned *err)
{
    constexpr int U = 4;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned bad = 0;
    TwAcc acc;
    for (int64_t r = warp; r < nrows; r += nwarps) {
        const int32_t i = rows[r];
        const int g = R.graph(i);
        int64_t lo, hi;
        R.range(g, lo, hi);
        const int64_t b = rp[i], e = rp[i + 1];
        u64 sum = 0;
        bool uns = false;
        int32_t last = INT_MIN;  // column of the entry before this round
        for (int64_t k0 = b + lane; k0 - lane < e; k0 += 32 * U) {
            int32_t j[U];
            i64 x[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t k = k0 + 32 * u;
                j[u] = k < e ? ld_stream(col + k) : INT_MAX;
                x[u] = k < e ? (i64)ld_stream(w + k) : 0;
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t k = k0 + 32 * u;
                int32_t prev = __shfl_up_sync(0xffffffffu, j[u], 1);
                if (lane == 0) prev = last;
                last = __shfl_sync(0xffffffffu, j[u], 31);
                if (k < e) {
                    check_entry(j[u], x[u], lo, hi, bad);
                    uns = uns || (k > b && j[u] <= prev);
                    sum += (u64)x[u];
                }
            }
        }
        if (__any_sync(0xffffffffu, uns) && lane == 0) R.flag_unsorted(g);
        sum = sum_reduce(sum, 32);
        if (lane == 0) {
            delta[i] = (i64)sum;
            acc.add(R, g, sum);
        }
    }
    if (lane == 0) acc.flush(R);
    if (bad) atomicOr(err, bad);
}

// One CTA per longer row, four entries in flight per thread.
template <typename WT>
__global__ void __launch_bounds__(kBlock) k_row_sums_cta(RowCtx R, const int64_t *rp,
                                                         const int32_t *col, const WT *w,
                                                         const int32_t *rows, int64_t nrows,
                                                         i64 *delta, unsigned *err)
{
    constexpr int U = 4;
    __shared__ u64 s_part[kBlock / 32];
    __shared__ int s_uns;
    const int lane = threadIdx.x & 31;
    unsigned bad = 0;
    TwAcc acc;
    if (threadIdx.x == 0) s_uns = 0;
    __syncthreads();
    for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int32_t i = rows[r];
        const int g = R.graph(i);
        int64_t lo, hi;
        R.range(g, lo, hi);
        const int64_t b = rp[i], e = rp[i + 1];
        u64 sum = 0;
        bool uns = false;
        for (int64_t k0 = b + threadIdx.x; k0 - threadIdx.x < e; k0 += (int64_t)kBlock * U) {
            int32_t j[U];
            i64 x[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t k = k0 + (int64_t)kBlock * u;
                j[u] = k < e ? ld_stream(col + k) : INT_MAX;
                x[u] = k < e ? (i64)ld_stream(w + k) : 0;
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t k = k0 + (int64_t)kBlock * u;
                int32_t prev = __shfl_up_sync(0xffffffffu, j[u], 1);
                if (lane == 0 && k > b && k < e) prev = col[k - 1];  // left entry in another warp
                if (k < e) {
                    check_entry(j[u], x[u], lo, hi, bad);
                    uns = uns || (k > b && j[u] <= prev);
                    sum += (u64)x[u];
                }
            }
        }
        if (uns) s_uns = 1;
        sum = sum_reduce(sum, 32);
        if (lane == 0) s_part[threadIdx.x >> 5] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            u64 t = 0;
            for (int q = 0; q < kBlock / 32; q++) t += s_part[q];
            delta[i] = (i64)t;
            acc.add(R, g, t);
            if (s_uns) R.flag_unsorted(g);
            s_uns = 0;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) acc.flush(R);
    if (bad) atomicOr(err, bad);
}

template <typename WT>
static int row_sums_impl(const DevGraph &g, const Bins &b, const RowCtx &R, i64 *delta,
                         unsigned *err, cudaStream_t s, const LaunchCfg &lc)
{
    const WT *w = (const WT *)g.w;
    int launched = 1;
    k_row_sums_thread<WT><<<grid_for(g.n, kBlock, lc.max_blocks), kBlock, 0, s>>>(
        R, g.rp, g.col, w, b.upper[0], delta, err);
    // a warp per row up to bin 4's rows, a CTA per longer row (the per-row barriers and
    // reduction of a CTA cost more than the extra rounds of a warp on rows up to 2,048)
    const int64_t nwarp = b.off[5] - b.off[1];
    if (nwarp > 0) {
        k_row_sums_warp<WT><<<grid_for(nwarp, kBlock / 32, lc.max_blocks), kBlock, 0, s>>>(
            R, g.rp, g.col, w, b.list + b.off[1], nwarp, delta, err);
        launched++;
    }
    const int64_t ncta = b.off[kNumBins] - b.off[5];
    if (ncta > 0) {
        k_row_sums_cta<WT><<<grid_for(ncta, 1, lc.max_blocks), kBlock, 0, s>>>(
            R, g.rp, g.col, w, b.list + b.off[5], ncta, delta, err);
        launched++;
    }
    return launched;
}

int launch_row_sums(const DevGraph &g, const Bins &b, const int32_t *vg, const int64_t *gptr,
                    i64 *delta, u64 *tw, unsigned *unsorted, unsigned *err, cudaStream_t s,
                    const LaunchCfg &lc)
{
    if (g.n == 0) return 0;
    RowCtx R{g.n, vg, gptr, tw, unsorted};
    if (g.wbytes == 4) return row_sums_impl<int32_t>(g, b, R, delta, err, s, lc);
    return row_sums_impl<i64>(g, b, R, delta, err, s, lc);
}

// Full input checks: every row strictly increasing (sorted, no duplicate), and every
// entry (i, j, w) has a mirror (j, i, w) found by binary search in row j.
template <typename WT>
__global__ void __launch_bounds__(kBlock) k_check_symmetry(int64_t n, const int64_t *rp,
                                                           const int32_t *col, const WT *w,
                                                           unsigned *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned bad = 0;
    for (int64_t i = warp; i < n; i += nwarps) {
        const int64_t b = rp[i], e = rp[i + 1];
        for (int64_t k = b + lane; k < e; k += 32) {
            const int32_t j = col[k];
            if ((uint32_t)j >= (uint64_t)n) {
                bad |= ERRF_INDEX;
                continue;
            }
            if (k + 1 < e && col[k + 1] <= j) bad |= ERRF_DUP;
            int64_t lo = rp[j], hi = rp[j + 1];
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                if (col[mid] < (int32_t)i) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= rp[j + 1] || col[lo] != (int32_t)i || w[lo] != w[k]) bad |= ERRF_ASYM;
        }
    }
    if (bad) atomicOr(err, bad);
}

int launch_check_symmetry(const DevGraph &g, unsigned *err, cudaStream_t s, const LaunchCfg &lc)
{
    if (g.n == 0) return 0;
    const int grid = grid_for(g.n, kBlock / 32, lc.max_blocks);
    if (g.wbytes == 4)
        k_check_symmetry<int32_t><<<grid, kBlock, 0, s>>>(g.n, g.rp, g.col,
                                                          (const int32_t *)g.w, err);
    else
        k_check_symmetry<i64><<<grid, kBlock, 0, s>>>(g.n, g.rp, g.col, (const i64 *)g.w, err);
    return 1;
}

// ------------------------------------------------------------------ phase state

// Weight d of a vertex moves from community a to community b: deg and its 32-bit copy follow
// (the copy modulo 2^32), and the flag is raised when b's degree reaches 2^32, after which
// the copy is not read.  Degrees change only here, so a final degree of 2^32 or more is always
// seen by the increment that reached it.
__device__ __forceinline__ void move_degree(i64 *deg, unsigned *deg32, unsigned *bad, int32_t a,
                                            int32_t b, i64 d)
{
    const u64 ob = atomicAdd((u64 *)&deg[b], (u64)d);
    atomicAdd((u64 *)&deg[a], (u64)(-d));
    if (deg32) {
        atomicAdd(&deg32[b], (unsigned)d);
        atomicSub(&deg32[a], (unsigned)d);
        if ((ob + (u64)d) >> 32) *bad = 1u;
    }
}

__global__ void k_init_state(int64_t n, int32_t *C, i64 *deg, int32_t *size, const i64 *delta,
                             unsigned *deg32, unsigned *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        C[i] = (int32_t)i;
        deg[i] = delta[i];
        size[i] = 1;
        if (deg32) {
            deg32[i] = (unsigned)delta[i];
            if ((u64)delta[i] >> 32) *bad = 1u;
        }
    }
}

int launch_init_state(int64_t n, const PhaseState &st, cudaStream_t s, const LaunchCfg &lc)
{
    if (n == 0) return 0;
    k_init_state<<<grid_for(n, kBlock, lc.max_blocks), kBlock, 0, s>>>(n, st.C, st.deg, st.size,
                                                                      st.delta, st.deg32,
                                                                      st.deg32_bad);
    return 1;
}

// If v has exactly one non-loop neighbour, return 1 and put it in *other.
__device__ __forceinline__ int sole_neighbour(const int64_t *rp, const int32_t *col, int32_t v,
                                              int32_t *other)
{
    const int64_t b = rp[v], len = rp[v + 1] - b;
    if (len == 1) {
        const int32_t c0 = col[b];
        if (c0 != v) {
            *other = c0;
            return 1;
        }
        return 0;
    }
    if (len == 2) {
        const int32_t c0 = col[b], c1 = col[b + 1];
        if (c0 == v && c1 != v) {
            *other = c1;
            return 1;
        }
        if (c1 == v && c0 != v) {
            *other = c0;
            return 1;
        }
    }
    return 0;
}

// Vertex following: a vertex whose only non-loop neighbour is j joins j's singleton
// community; an isolated pair joins the smaller id.  Targets never follow anyone, so
// the deg/size updates below commute.  Runs right after k_init_state.
__global__ void k_vertex_following(int64_t n, const int64_t *rp, const int32_t *col,
                                   const i64 *delta, int32_t *C, i64 *deg, int32_t *size,
                                   const int32_t *vg, const int32_t *vf_on, unsigned *deg32,
                                   unsigned *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (vg && !vf_on[vg[i]]) continue;  // that graph's level does not follow
        int32_t j;
        if (!sole_neighbour(rp, col, (int32_t)i, &j)) continue;
        int32_t j2;
        const int32_t t = sole_neighbour(rp, col, j, &j2) ? min((int32_t)i, j) : j;
        if (t == (int32_t)i) continue;
        const i64 d = delta[i];
        C[i] = t;
        move_degree(deg, deg32, bad, (int32_t)i, t, d);
        atomicAdd(&size[t], 1);
        atomicSub(&size[i], 1);
    }
}

int launch_vertex_following(const DevGraph &g, const PhaseState &st, cudaStream_t s,
                            const LaunchCfg &lc, const int32_t *vg, const int32_t *vf_on)
{
    if (g.n == 0) return 0;
    k_vertex_following<<<grid_for(g.n, kBlock, lc.max_blocks), kBlock, 0, s>>>(
        g.n, g.rp, g.col, st.delta, st.C, st.deg, st.size, vg, vf_on, st.deg32, st.deg32_bad);
    return 1;
}

// ------------------------------------------------------------------ degree bins
// Pass 1 counts rows (counts[b]) and entries (int64 at counts + 16 + 2b) per bin; pass 2
// writes each row of bins 1.. into its bin's region of the list (order within a bin is
// not specified).  counts[b] is reused as the fill cursor of bin b.
struct BinArgs {
    int64_t upper[kNumBins - 1];
    int64_t off[kNumBins + 1];
    int32_t *list;
    const int32_t *vg;      // batch: graph of every vertex (nullptr for one graph)
    const LevelCtl *gctl;   // batch: rows of graphs whose phase stopped are left out
    const int32_t *color;   // colouring variant: only vertices of colour cls are binned
    int32_t cls;
};

__device__ __forceinline__ int bin_of(int64_t d, const int64_t *upper)
{
    int b = 0;
#pragma unroll
    for (int t = 0; t < kNumBins - 1; t++) b += d > upper[t];
    return b;
}

template <bool FILL>
__global__ void __launch_bounds__(kBlock) k_bin(int64_t n, const int64_t *rp, BinArgs ba,
                                                int32_t *counts)
{
    const int lane = threadIdx.x & 31;
    __shared__ int s_fcnt[kNumBins], s_fbase[kNumBins];
    // count pass: per-thread counts and entries, reduced per warp and per CTA, so each CTA
    // adds once per bin
    int cnt[kNumBins] = {};
    u64 ent[kNumBins] = {};
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n;
         i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        int bin = -1;
        int64_t d = 0;
        if (i < n && !(ba.vg && ba.gctl[ba.vg[i]].done) && !(ba.color && ba.color[i] != ba.cls)) {
            d = rp[i + 1] - rp[i];
            bin = bin_of(d, ba.upper);
        }
        if (!FILL) {
#pragma unroll
            for (int b = 0; b < kNumBins; b++) {
                cnt[b] += bin == b;
                ent[b] += bin == b ? (u64)d : 0;
            }
            continue;
        }
        // fill pass: positions claimed once per CTA and bin, warps ranked in shared memory
        if (threadIdx.x < kNumBins) s_fcnt[threadIdx.x] = 0;
        __syncthreads();
        int rank = 0;
#pragma unroll
        for (int b = 1; b < kNumBins; b++) {
            const unsigned mask = __ballot_sync(0xffffffffu, bin == b);
            if (!mask) continue;
            const int leader = __ffs(mask) - 1;
            int wbase = 0;
            if (lane == leader) wbase = atomicAdd(&s_fcnt[b], __popc(mask));
            wbase = __shfl_sync(0xffffffffu, wbase, leader);
            if (bin == b) rank = wbase + __popc(mask & ((1u << lane) - 1u));
        }
        __syncthreads();
        if (threadIdx.x < kNumBins)
            s_fbase[threadIdx.x] =
                s_fcnt[threadIdx.x] ? atomicAdd(&counts[threadIdx.x], s_fcnt[threadIdx.x]) : 0;
        __syncthreads();
        if (bin >= 1) ba.list[ba.off[bin] + s_fbase[bin] + rank] = (int32_t)i;
        __syncthreads();  // counts read before the next round resets them
    }
    if (!FILL) {
        __shared__ int s_cnt[kNumBins];
        __shared__ unsigned long long s_ent[kNumBins];
        if (threadIdx.x < kNumBins) {
            s_cnt[threadIdx.x] = 0;
            s_ent[threadIdx.x] = 0;
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < kNumBins; b++) {
            const int c = sum_reduce(cnt[b], 32);
            const u64 e = sum_reduce(ent[b], 32);
            if (lane == 0 && c) {
                atomicAdd(&s_cnt[b], c);
                atomicAdd(&s_ent[b], (unsigned long long)e);
            }
        }
        __syncthreads();
        if (threadIdx.x < kNumBins && s_cnt[threadIdx.x]) {
            atomicAdd(&counts[threadIdx.x], s_cnt[threadIdx.x]);
            atomicAdd((u64 *)(counts + 16 + 2 * threadIdx.x), (u64)s_ent[threadIdx.x]);
        }
    }
}

static BinArgs bin_args(const Bins &b, const int32_t *vg, const LevelCtl *gctl,
                        const int32_t *color, int32_t cls)
{
    BinArgs ba;
    ba.vg = vg;
    ba.gctl = gctl;
    ba.color = color;
    ba.cls = cls;
    for (int t = 0; t < kNumBins - 1; t++) ba.upper[t] = b.upper[t];
    for (int t = 0; t <= kNumBins; t++) ba.off[t] = b.off[t];
    ba.list = b.list;
    return ba;
}

int launch_bin_count(const DevGraph &g, Bins &b, cudaStream_t s, const LaunchCfg &lc,
                     const int32_t *vg, const LevelCtl *gctl, const int32_t *color, int32_t cls)
{
    cudaMemsetAsync(b.counts, 0, sizeof(int32_t) * (16 + 2 * kNumBins), s);
    if (g.n == 0) return 0;
    k_bin<false><<<grid_for(g.n, kBlock, lc.max_blocks), kBlock, 0, s>>>(
        g.n, g.rp, bin_args(b, vg, gctl, color, cls), b.counts);
    return 1;
}

int launch_bin_fill(const DevGraph &g, Bins &b, cudaStream_t s, const LaunchCfg &lc,
                    const int32_t *vg, const LevelCtl *gctl, const int32_t *color, int32_t cls)
{
    cudaMemsetAsync(b.counts, 0, sizeof(int32_t) * 16, s);
    if (g.n == 0) return 0;
    k_bin<true><<<grid_for(g.n, kBlock, lc.max_blocks), kBlock, 0, s>>>(
        g.n, g.rp, bin_args(b, vg, gctl, color, cls), b.counts);
    return 1;
}

// Chunked rows: chunk counts and, for multi-chunk rows, the number of hash partitions of the
// row's keys (a power of two keeping the expected distinct keys per partition, at most
// min(d, n) in all, at or below part_keys; 2^kMaxPartLog2 at most).
__global__ void k_big_prep(int nb, const int32_t *bverts, const int64_t *rp, int64_t n, int chunk,
                           int part_keys, int32_t *nch, int32_t *plog2)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const int32_t v = bverts[b];
        const int64_t d = rp[v + 1] - rp[v];
        const int64_t c = (d + chunk - 1) / chunk;
        nch[b] = (int32_t)c;
        int pl = 0;
        if (c > 1) {
            const int64_t keys = d < n ? d : n;  // distinct keys of the row at most
            while (pl < kMaxPartLog2 && ((int64_t)part_keys << pl) < keys) pl++;
        }
        plog2[b] = pl;
    }
}

// histogram block of multi-chunk row b: nch * (P + 1) partition offsets
struct HistIn {
    const int32_t *nch;
    const int32_t *plog2;
    __device__ __forceinline__ int64_t operator()(int64_t b) const
    {
        return nch[b] > 1 ? (int64_t)nch[b] * ((1 << plog2[b]) + 1) : 0;
    }
};

int launch_big_prep(const DevGraph &g, Bins &b, int64_t *scratch64, int32_t *scratch32,
                    cudaStream_t s, const LaunchCfg &lc)
{
    const int nb = b.nlist[kChunkedBin];
    if (nb == 0) return 0;
    k_big_prep<<<grid_for(nb, kBlock, lc.max_blocks), kBlock, 0, s>>>(
        nb, b.rows(kChunkedBin), g.rp, g.n, b.chunk, b.part_keys, b.nch, b.plog2);
    int k = 1;
    k += exclusive_scan<int32_t>(ArrayIn<int32_t>{b.nch}, nb, b.chunk_first, scratch32, s);
    k += exclusive_scan<int64_t>(HistIn{b.nch, b.plog2}, nb, b.hoff, scratch64, s);
    return k;
}

__global__ void k_big_fill(int nb, const int32_t *nch, const int32_t *chunk_first, int32_t *chunk_b)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int b = warp; b < nb; b += nwarps)
        for (int q = lane; q < nch[b]; q += 32) chunk_b[chunk_first[b] + q] = b;
}

int launch_big_fill(Bins &b, cudaStream_t s, const LaunchCfg &lc)
{
    const int nb = b.nlist[kChunkedBin];
    if (nb == 0) return 0;
    k_big_fill<<<grid_for(nb, kBlock / 32, lc.max_blocks), kBlock, 0, s>>>(nb, b.nch,
                                                                           b.chunk_first, b.chunk_b);
    return 1;
}

// Decision work items of the multi-chunk rows: one per partition of the row's keys; soff is
// their exclusive scan and slice_row the row of every item.
struct HugeSlicesIn {
    const int32_t *nch;
    const int32_t *plog2;
    __device__ __forceinline__ int64_t operator()(int64_t b) const
    {
        return nch[b] > 1 ? (int64_t)1 << plog2[b] : 0;
    }
};

int launch_huge_slices(Bins &b, int64_t *scratch64, cudaStream_t s)
{
    const int nb = b.nlist[kChunkedBin];
    if (nb == 0) return 0;
    return exclusive_scan<int64_t>(HugeSlicesIn{b.nch, b.plog2}, nb, b.soff, scratch64, s);
}

__global__ void k_huge_slice_fill(int nb, const int64_t *soff, int32_t *slice_row)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int b = warp; b < nb; b += nwarps)
        for (int64_t q = soff[b] + lane; q < soff[b + 1]; q += 32) slice_row[q] = b;
}

int launch_huge_slice_fill(Bins &b, cudaStream_t s, const LaunchCfg &lc)
{
    const int nb = b.nlist[kChunkedBin];
    if (nb == 0) return 0;
    k_huge_slice_fill<<<grid_for(nb, kBlock / 32, lc.max_blocks), kBlock, 0, s>>>(nb, b.soff,
                                                                                 b.slice_row);
    return 1;
}

// ------------------------------------------------------------------ phase controller

// (qn_new - qn_old) * den < num * tw^2, exact: both sides formed in 192 bits.
__device__ bool dev_below_threshold(i128 qn_new, i128 qn_old, i64 tw, i64 num, i64 den)
{
    const i128 diff = qn_new - qn_old;
    if (diff < 0) return true;
    const u128 tw2 = (u128)(u64)tw * (u64)tw;
    const u128 x = (u128)diff;
    // x * den and tw2 * num as (high 64, low 128)
    const u128 xl = (u128)(u64)x * (u64)den, xh = (u128)(u64)(x >> 64) * (u64)den;
    const u128 yl = (u128)(u64)tw2 * (u64)num, yh = (u128)(u64)(tw2 >> 64) * (u64)num;
    const u128 xmid = (xl >> 64) + (u64)xh, ymid = (yl >> 64) + (u64)yh;
    const u64 x2 = (u64)(xh >> 64) + (u64)(xmid >> 64), y2 = (u64)(yh >> 64) + (u64)(ymid >> 64);
    const u64 x1 = (u64)xmid, y1 = (u64)ymid, x0 = (u64)xl, y0 = (u64)yl;
    if (x2 != y2) return x2 < y2;
    if (x1 != y1) return x1 < y1;
    return x0 < y0;
}

// 192-bit a * m for a 128-bit magnitude a and a 64-bit m: (top 64, middle 64, low 64)
__device__ __forceinline__ void mul192(u128 a, u64 m, u64 &t2, u64 &t1, u64 &t0)
{
    const u128 lo = (u128)(u64)a * m, hi = (u128)(u64)(a >> 64) * m;
    const u128 mid = (lo >> 64) + (u64)hi;
    t2 = (u64)(hi >> 64) + (u64)(mid >> 64);
    t1 = (u64)mid;
    t0 = (u64)lo;
}

// Relative phase test printed in Algorithm 1: |qn_new - qn_old| * den < num * |qn_old|
// (both Qn carry the factor (2W)^2); Q_prev = 0 stops only on an unchanged Q.
__device__ bool dev_below_threshold_rel(i128 qn_new, i128 qn_old, i64 num, i64 den)
{
    const i128 diff = qn_new - qn_old;
    const u128 ad = (u128)(diff < 0 ? -diff : diff);
    const u128 ao = (u128)(qn_old < 0 ? -qn_old : qn_old);
    if (ao == 0) return ad == 0;
    u64 x2, x1, x0, y2, y1, y0;
    mul192(ad, (u64)den, x2, x1, x0);
    mul192(ao, (u64)num, y2, y1, y0);
    if (x2 != y2) return x2 < y2;
    if (x1 != y1) return x1 < y1;
    return x0 < y0;
}

// Runs after sweep k (1-based) on state C_{k-1}; the sweep measured Qn(C_{k-1}) and
// proposed C_k.  Stopping rule (Algorithm 1 with the absolute threshold on exact Qn):
//   k >= 2: stop with C_{k-1} if Qn(C_{k-1}) - Qn(C_{k-2}) is below theta, or if k-1
//           sweeps reached the cap;
//   stop with C_{k-1} = C_k if sweep k moved nobody.
// Otherwise the proposal is applied by k_apply.  The trace gets (moved, Qn) of every
// applied sweep.  Thread g runs the controller of graph g of a batch (G = 1: one graph).
__global__ void k_decide(SweepStats *sts, LevelCtl *ctls, int G, i64 *tr_moved, i64 *tr_qn,
                         u64 *cand_total, int *ndone)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    SweepStats *st = sts + g;
    LevelCtl *ctl = ctls + g;
    if (!ctl->done) {
        const i128 sq = (i128)(((u128)st->sq_hi << 64) | (u128)st->sq_lo);
        const i128 qn = (i128)ctl->tw * (i128)(i64)st->internal - sq;
        const int k = ctl->sweep + 1;
        const i64 moved = (i64)st->moved;
        bool stop = false;
        int iters = 0;
        if (k == 1) {
            i128_to(qn, ctl->qn_init);
        } else {
            const int t = k - 2;
            if (t < ctl->max_iters + 1) {
                tr_moved[(size_t)t * G + g] = ctl->moved_last;
                i128_to(qn, &tr_qn[2 * ((size_t)t * G + g)]);
            }
            const i128 qp = i128_from(ctl->qn_prev);
            if (ctl->rel ? dev_below_threshold_rel(qn, qp, ctl->theta_num, ctl->theta_den)
                         : dev_below_threshold(qn, qp, ctl->tw, ctl->theta_num, ctl->theta_den)) {
                stop = true;
                iters = k - 1;
            } else if (k - 1 >= ctl->max_iters) {
                stop = true;
                iters = k - 1;
                ctl->hit_cap = 1;
            }
        }
        if (!stop && moved == 0) {
            const int t = k - 1;
            if (t < ctl->max_iters + 1) {
                tr_moved[(size_t)t * G + g] = 0;
                i128_to(qn, &tr_qn[2 * ((size_t)t * G + g)]);
            }
            stop = true;
            iters = k;
        }
        if (stop) {
            ctl->done = 1;
            ctl->iters = iters;
            i128_to(qn, ctl->qn_final);
            atomicAdd(ndone, 1);
        } else {
            i128_to(qn, ctl->qn_prev);
            ctl->moved_last = moved;
            ctl->sweep = k;
        }
    }
    st->internal = 0;
    st->sq_lo = 0;
    st->sq_hi = 0;
    st->moved = 0;
    if (g == 0) {
        for (int b = 0; b < 16; b++) {
            cand_total[b] += st->cand[b];
            st->cand[b] = 0;
        }
    }
}

int launch_decide(SweepStats *st, LevelCtl *ctl, int G, i64 *tr_moved, i64 *tr_qn,
                  u64 *cand_total, int *ndone, cudaStream_t s)
{
    k_decide<<<(G + 127) / 128, 128, 0, s>>>(st, ctl, G, tr_moved, tr_qn, cand_total, ndone);
    return 1;
}

// Condition of the device-side sweep loop (a CUDA graph while node): go on while some
// controller is still running, fewer than `quota` graphs stopped since the loop was
// launched (a batch then returns to the host to drop their rows from the bins), and the
// loop has run fewer than `cap` sweeps (a bound the controllers never reach).
__global__ void k_loop_ctl(cudaGraphConditionalHandle handle, LoopCtl *lc, const int *ndone,
                           int G)
{
    const int it = ++lc->iters;
    const int nd = *(volatile const int *)ndone;
    const bool go = nd < G && nd - lc->nd0 < lc->quota && it < lc->cap;
    cudaGraphSetConditional(handle, go ? 1u : 0u);
}

int launch_loop_ctl(cudaGraphConditionalHandle handle, LoopCtl *lc, const int *ndone, int G,
                    cudaStream_t s)
{
    k_loop_ctl<<<1, 1, 0, s>>>(handle, lc, ndone, G);
    return 1;
}

// Apply the sweep's proposal (unless the controller of the vertex's graph stopped the
// phase): deg_C and size_C follow the moved vertices (the paper's remove / insert with
// atomics), then C <- C_next.
__global__ void __launch_bounds__(kBlock) k_apply(int64_t n, int32_t *C, const int32_t *Cnext,
                                                  i64 *deg, int32_t *size, const i64 *delta,
                                                  const LevelCtl *ctl, const int32_t *vg,
                                                  unsigned *deg32, unsigned *bad)
{
    if (!vg && ctl && *(volatile const int *)&ctl->done) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = C[i], b = Cnext[i];
        if (a == b) continue;
        if (vg && ctl && ctl[vg[i]].done) continue;
        move_degree(deg, deg32, bad, a, b, delta[i]);
        atomicAdd(&size[b], 1);
        atomicSub(&size[a], 1);
        C[i] = b;
    }
}

int launch_apply(int64_t n, const PhaseState &st, const LevelCtl *ctl, const int32_t *vg,
                 cudaStream_t s, const LaunchCfg &lc)
{
    if (n == 0) return 0;
    k_apply<<<grid_for(n, kBlock, lc.max_blocks), kBlock, 0, s>>>(n, st.C, st.Cnext, st.deg,
                                                                 st.size, st.delta, ctl, vg,
                                                                 st.deg32, st.deg32_bad);
    return 1;
}

// ------------------------------------------------------------------ post-phase merge
// Sec. 5.1.2 pushes the vertices that have a single neighbouring community into it once the
// iterations are done (reading: only when the move's Eq. 4 gain is positive).  One warp per
// vertex: the smallest and largest community among the non-loop neighbours decide whether
// there is exactly one, the weight into it is their sum; the decision reads the post-phase
// state only and is written to Cnext.
template <typename WT, typename GT>
__global__ void __launch_bounds__(kBlock) k_post_merge(int64_t n, const int64_t *rp,
                                                       const int32_t *col, const WT *w,
                                                       const int32_t *C, const i64 *deg,
                                                       const i64 *delta, const int32_t *vg,
                                                       const i64 *gtw, i64 tw1, int32_t *Cnext)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nwarps) {
        const int32_t a = C[i];
        int cmin = INT_MAX, cmax = -1;
        u64 e = 0;
        for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += 32) {
            const int32_t j = col[k];
            if (j == (int32_t)i) continue;
            const int c = C[j];
            cmin = min(cmin, c);
            cmax = max(cmax, c);
            e += (u64)w[k];
        }
        cmin = __reduce_min_sync(0xffffffffu, cmin);
        cmax = __reduce_max_sync(0xffffffffu, cmax);
        e = sum_reduce(e, 32);
        if (lane == 0) {
            int32_t target = a;
            if (cmax >= 0 && cmin == cmax && cmin != a) {
                const i64 tw = vg ? gtw[vg[i]] : tw1;
                const i64 dl = delta[i];
                const GT g_move = (GT)tw * (GT)(i64)e - (GT)dl * (GT)deg[cmin];
                const GT g_stay = -((GT)dl * (GT)(deg[a] - dl));
                if (g_move > g_stay) target = cmin;
            }
            Cnext[i] = target;
        }
    }
}

// Exact Qn of the merged state: sum_i e_{i->C(i)} (loops included) per graph, one warp per
// vertex; sum_c deg_c^2 per graph, one thread per label; then Qn = 2W * S - sum deg^2 into
// every controller's qn_final.
template <typename WT>
__global__ void __launch_bounds__(kBlock) k_qn_rows(int64_t n, const int64_t *rp,
                                                    const int32_t *col, const WT *w,
                                                    const int32_t *C, const int32_t *vg,
                                                    SweepStats *st)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    u64 acc = 0;
    for (int64_t i = warp; i < n; i += nwarps) {
        const int32_t a = C[i];
        u64 e = 0;
        for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += 32)
            if (C[col[k]] == a) e += (u64)w[k];
        e = sum_reduce(e, 32);
        if (vg) {
            if (lane == 0 && e) atomicAdd(&st[vg[i]].internal, e);
        } else {
            acc += e;
        }
    }
    if (!vg && lane == 0 && acc) atomicAdd(&st[0].internal, acc);
}

__global__ void __launch_bounds__(kBlock) k_qn_squares(int64_t n, const i64 *deg,
                                                       const int32_t *vg, SweepStats *st)
{
    u128 acc = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        const u64 d = (u64)deg[c];
        if (!d) continue;
        const u128 sq = (u128)d * d;
        if (vg) atomic_add_u128(&st[vg[c]].sq_lo, &st[vg[c]].sq_hi, sq);
        else acc += sq;
    }
    if (!vg) {
        acc = sum_reduce(acc, 32);
        if ((threadIdx.x & 31) == 0 && acc) atomic_add_u128(&st[0].sq_lo, &st[0].sq_hi, acc);
    }
}

__global__ void k_qn_finalize(int G, SweepStats *sts, LevelCtl *ctls)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    SweepStats *st = sts + g;
    const i128 sq = (i128)(((u128)st->sq_hi << 64) | (u128)st->sq_lo);
    const i128 qn = (i128)ctls[g].tw * (i128)(i64)st->internal - sq;
    i128_to(qn, ctls[g].qn_final);
    st->internal = 0;
    st->sq_lo = 0;
    st->sq_hi = 0;
    st->moved = 0;
}

template <typename WT>
static int post_merge_impl(const DevGraph &g, const PhaseState &st, const int32_t *vg,
                           const i64 *gtw, i64 tw, bool wide, SweepStats *stats, LevelCtl *ctl,
                           int G, cudaStream_t s, const LaunchCfg &lc)
{
    const WT *w = (const WT *)g.w;
    const int grid = grid_for(g.n, kBlock / 32, lc.max_blocks);
    if (wide)
        k_post_merge<WT, i128><<<grid, kBlock, 0, s>>>(g.n, g.rp, g.col, w, st.C, st.deg,
                                                       st.delta, vg, gtw, tw, st.Cnext);
    else
        k_post_merge<WT, i64><<<grid, kBlock, 0, s>>>(g.n, g.rp, g.col, w, st.C, st.deg,
                                                      st.delta, vg, gtw, tw, st.Cnext);
    int k = 1;
    k += launch_apply(g.n, st, nullptr, vg, s, lc);
    k_qn_rows<WT><<<grid, kBlock, 0, s>>>(g.n, g.rp, g.col, w, st.C, vg, stats);
    k_qn_squares<<<grid_for(g.n, kBlock, lc.max_blocks), kBlock, 0, s>>>(g.n, st.deg, vg, stats);
    k_qn_finalize<<<(G + 127) / 128, 128, 0, s>>>(G, stats, ctl);
    return k + 3;
}

// ------------------------------------------------------------------ colouring variant
// Lu et al.'s colouring heuristic (named, not defined, in Sec. 7 of the paper): a
// distance-1 colouring by Jones-Plassmann rounds, then sweeps that take the colour classes
// one after the other.  The priority of vertex v is the output function of SplitMix64
// (Steele, Lea and Flood 2014) applied to v, a bijection of 64-bit values, so no two
// vertices tie.
__device__ __forceinline__ u64 color_priority(int64_t v)
{
    u64 z = (u64)v + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One warp per uncoloured vertex: picked when no uncoloured non-loop neighbour has a higher
// priority.  Picks of one round are pairwise non-adjacent, so assigning their colours in the
// next kernel reads only colours of earlier rounds.
__global__ void __launch_bounds__(kBlock) k_color_pick(int64_t n, const int64_t *rp,
                                                       const int32_t *col, const int32_t *color,
                                                       int32_t *pick, u64 *counts)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    u64 unc = 0, picked = 0;
    for (int64_t v = warp; v < n; v += nwarps) {
        if (color[v] >= 0) {
            if (lane == 0) pick[v] = 0;
            continue;
        }
        const u64 pv = color_priority(v);
        bool beaten = false;
        for (int64_t k = rp[v] + lane; k < rp[v + 1] && !beaten; k += 32) {
            const int32_t u = col[k];
            beaten = u != (int32_t)v && color[u] < 0 && color_priority(u) > pv;
        }
        const bool top = !__any_sync(0xffffffffu, beaten);
        if (lane == 0) {
            pick[v] = top;
            unc += 1;
            picked += top;
        }
    }
    if (lane == 0) {
        if (unc) atomicAdd(&counts[0], unc);
        if (picked) atomicAdd(&counts[1], picked);
    }
}

// One warp per picked vertex: the smallest colour missing among its neighbours, found 64
// colours at a time (a vertex of d entries needs at most d + 1 colours).
__global__ void __launch_bounds__(kBlock) k_color_assign(int64_t n, const int64_t *rp,
                                                         const int32_t *col, int32_t *color,
                                                         const int32_t *pick, int32_t *ncolors)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int top = 0;
    for (int64_t v = warp; v < n; v += nwarps) {
        if (!pick[v]) continue;
        for (int base = 0;; base += 64) {
            u64 used = 0;
            for (int64_t k = rp[v] + lane; k < rp[v + 1]; k += 32) {
                const int32_t u = col[k];
                const int c = u != (int32_t)v ? color[u] - base : -1;
                if (c >= 0 && c < 64) used |= (u64)1 << c;
            }
            const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)used);
            const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(used >> 32));
            const u64 all = ((u64)hi << 32) | lo;
            if (all != ~(u64)0) {
                const int c = base + __ffsll((long long)~all) - 1;
                if (lane == 0) color[v] = c;
                top = max(top, c + 1);
                break;
            }
        }
    }
    if (lane == 0 && top) atomicMax(ncolors, top);
}

int launch_color_pick(const DevGraph &g, const int32_t *color, int32_t *pick, u64 *counts,
                      cudaStream_t s, const LaunchCfg &lc)
{
    cudaMemsetAsync(counts, 0, 2 * sizeof(u64), s);
    if (g.n == 0) return 0;
    k_color_pick<<<grid_for(g.n, kBlock / 32, lc.max_blocks), kBlock, 0, s>>>(g.n, g.rp, g.col,
                                                                             color, pick, counts);
    return 1;
}

int launch_color_assign(const DevGraph &g, int32_t *color, const int32_t *pick, int32_t *ncolors,
                        cudaStream_t s, const LaunchCfg &lc)
{
    if (g.n == 0) return 0;
    k_color_assign<<<grid_for(g.n, kBlock / 32, lc.max_blocks), kBlock, 0, s>>>(
        g.n, g.rp, g.col, color, pick, ncolors);
    return 1;
}

// Moves of the vertices of one colour class: deg / size follow (remove / insert with
// atomics), then C <- C_next for them.
__global__ void __launch_bounds__(kBlock) k_apply_class(int64_t n, int32_t *C, const int32_t *Cnext,
                                                        i64 *deg, int32_t *size, const i64 *delta,
                                                        const int32_t *color, int32_t cls,
                                                        u64 *moved, unsigned *deg32, unsigned *bad)
{
    u64 mv = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (color[i] != cls) continue;
        const int32_t a = C[i], b = Cnext[i];
        if (a == b) continue;
        move_degree(deg, deg32, bad, a, b, delta[i]);
        atomicAdd(&size[b], 1);
        atomicSub(&size[a], 1);
        C[i] = b;
        mv++;
    }
    mv = sum_reduce(mv, 32);
    if ((threadIdx.x & 31) == 0 && mv) atomicAdd(moved, mv);
}

int launch_apply_class(int64_t n, const PhaseState &st, u64 *moved, cudaStream_t s,
                       const LaunchCfg &lc)
{
    if (n == 0) return 0;
    k_apply_class<<<grid_for(n, kBlock, lc.max_blocks), kBlock, 0, s>>>(
        n, st.C, st.Cnext, st.deg, st.size, st.delta, st.color, st.cls, moved, st.deg32,
        st.deg32_bad);
    return 1;
}

template <typename WT>
static int qn_one_impl(const DevGraph &g, const PhaseState &st, SweepStats *stats, LevelCtl *ctl,
                       cudaStream_t s, const LaunchCfg &lc)
{
    k_qn_rows<WT><<<grid_for(g.n, kBlock / 32, lc.max_blocks), kBlock, 0, s>>>(
        g.n, g.rp, g.col, (const WT *)g.w, st.C, nullptr, stats);
    k_qn_squares<<<grid_for(g.n, kBlock, lc.max_blocks), kBlock, 0, s>>>(g.n, st.deg, nullptr,
                                                                         stats);
    k_qn_finalize<<<1, 128, 0, s>>>(1, stats, ctl);
    return 3;
}

int launch_qn_one(const DevGraph &g, const PhaseState &st, SweepStats *stats, LevelCtl *ctl,
                  cudaStream_t s, const LaunchCfg &lc)
{
    if (g.n == 0) return 0;
    if (g.wbytes == 4) return qn_one_impl<int32_t>(g, st, stats, ctl, s, lc);
    return qn_one_impl<i64>(g, st, stats, ctl, s, lc);
}

int launch_post_merge(const DevGraph &g, const PhaseState &st, const int32_t *vg, const i64 *gtw,
                      i64 tw, bool wide, SweepStats *stats, LevelCtl *ctl, int G, cudaStream_t s,
                      const LaunchCfg &lc)
{
    if (g.n == 0) return 0;
    if (g.wbytes == 4) return post_merge_impl<int32_t>(g, st, vg, gtw, tw, wide, stats, ctl, G, s, lc);
    return post_merge_impl<i64>(g, st, vg, gtw, tw, wide, stats, ctl, G, s, lc);
}

// ------------------------------------------------------------------ renumber / compose

struct UsedIn {  // 1 for a used label whose graph is kept
    const int32_t *size;
    const int32_t *vg;
    const int32_t *keep;
    __device__ __forceinline__ int32_t operator()(int64_t c) const
    {
        return size[c] > 0 && (!keep || keep[vg ? vg[c] : 0]) ? 1 : 0;
    }
};

// new_id[c] = number of used labels below c; new_id[n] = their count.  Labels of one graph
// are contiguous, so a batch's labels are renumbered graph by graph by the same scan.
int launch_renumber(int64_t n, const int32_t *size, const int32_t *vg, const int32_t *keep,
                    int32_t *new_id, int32_t *scratch, cudaStream_t s)
{
    return exclusive_scan<int32_t>(UsedIn{size, vg, keep}, n, new_id, scratch, s);
}

__global__ void k_gather64(const int64_t *a, const int64_t *idx, int cnt, int64_t *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
        out[i] = a[idx[i]];
}

__global__ void k_gather_ids(const int32_t *a, const int64_t *idx, int cnt, int64_t *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
        out[i] = (int64_t)a[idx[i]];
}

int launch_gather64(const int64_t *a, const int64_t *idx, int cnt, int64_t *out, cudaStream_t s)
{
    if (cnt <= 0) return 0;
    k_gather64<<<(cnt + 255) / 256, 256, 0, s>>>(a, idx, cnt, out);
    return 1;
}

int launch_gather_ids(const int32_t *a, const int64_t *idx, int cnt, int64_t *out, cudaStream_t s)
{
    if (cnt <= 0) return 0;
    k_gather_ids<<<(cnt + 255) / 256, 256, 0, s>>>(a, idx, cnt, out);
    return 1;
}

// vg[v] = the graph g with gptr[g] <= v < gptr[g+1] (empty graphs own no vertex).
__global__ void k_graph_ids(int64_t n, const int64_t *gptr, int G, int32_t *vg)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = G;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (gptr[mid] <= v) lo = mid;
            else hi = mid;
        }
        vg[v] = lo;
    }
}

int launch_graph_ids(int64_t n, const int64_t *gptr, int G, int32_t *vg, cudaStream_t s,
                     const LaunchCfg &lc)
{
    if (n == 0) return 0;
    k_graph_ids<<<grid_for(n, kBlock, lc.max_blocks), kBlock, 0, s>>>(n, gptr, G, vg);
    return 1;
}

// ------------------------------------------------------------------ stacking graphs
// Rows of a source CSR (int32 weights, or all 1) appended at vertex v_base / entry e_base of
// a stacked CSR, with its columns shifted to the stacked numbering and its weights widened.
template <typename WD>
__global__ void k_append_rows(int64_t n_src, int64_t nnz_src, const int64_t *src_rp,
                              const int32_t *src_col, const int32_t *src_w, int64_t v_base,
                              int64_t e_base, int64_t *dst_rp, int32_t *dst_col, WD *dst_w)
{
    const int64_t tot = n_src > nnz_src ? n_src : nnz_src;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n_src) dst_rp[v_base + t] = src_rp[t] + e_base;
        if (t < nnz_src) {
            dst_col[e_base + t] = src_col[t] + (int32_t)v_base;
            dst_w[e_base + t] = src_w ? (WD)src_w[t] : (WD)1;
        }
    }
}

int launch_append_rows(int64_t n_src, int64_t nnz_src, const int64_t *src_rp,
                       const int32_t *src_col, const int32_t *src_w, int64_t v_base,
                       int64_t e_base, int64_t *dst_rp, int32_t *dst_col, void *dst_w, int wbytes,
                       cudaStream_t s, const LaunchCfg &lc)
{
    const int64_t tot = n_src > nnz_src ? n_src : nnz_src;
    if (tot == 0) return 0;
    if (wbytes == 4)
        k_append_rows<int32_t><<<grid_for(tot, kBlock, lc.max_blocks), kBlock, 0, s>>>(
            n_src, nnz_src, src_rp, src_col, src_w, v_base, e_base, dst_rp, dst_col,
            (int32_t *)dst_w);
    else
        k_append_rows<i64><<<grid_for(tot, kBlock, lc.max_blocks), kBlock, 0, s>>>(
            n_src, nnz_src, src_rp, src_col, src_w, v_base, e_base, dst_rp, dst_col,
            (i64 *)dst_w);
    return 1;
}

// slot m with off[m] <= o < off[m+1] (empty slots own nothing)
__device__ __forceinline__ int slot_of(const int64_t *off, int M, int64_t o)
{
    int lo = 0, hi = M;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= o) lo = mid;
        else hi = mid;
    }
    return lo;
}

// maps[m][k] = vbase[m] + k for the k < off[m+1] - off[m] original vertices of graph m:
// a graph entering at level 0 is its own level-0 graph.
__global__ void k_map_init(int64_t tot, int M, const int64_t *off, int32_t *const *maps,
                           const int64_t *vbase)
{
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < tot;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int m = slot_of(off, M, o);
        const int64_t k = o - off[m];
        maps[m][k] = (int32_t)(vbase[m] + k);
    }
}

int launch_map_init(int64_t tot, int M, const int64_t *off, int32_t *const *maps,
                    const int64_t *vbase, cudaStream_t s, const LaunchCfg &lc)
{
    if (tot == 0) return 0;
    k_map_init<<<grid_for(tot, kBlock, lc.max_blocks), kBlock, 0, s>>>(tot, M, off, maps, vbase);
    return 1;
}

// Labels of the original vertices (Sec. 5.1.2: a vertex's community at level l is the
// community of the level-l vertex it was merged into).  Original vertex o belongs to
// graph m (off[m] <= o < off[m+1]); v = maps[m][o - off[m]] is its vertex at this level.
// For recorded graphs out[o] = new_id1[C[v]] - base1[m]; for kept graphs maps[m] moves on
// to the next level's vertex new_id2[C[v]].
__global__ void k_compose(int64_t n0, int M, const int64_t *off, int32_t *const *maps,
                          const int32_t *rec, const int32_t *keep, const int32_t *C,
                          const int32_t *new_id1, const int64_t *base1, const int32_t *new_id2,
                          int32_t *out)
{
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n0;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int m = slot_of(off, M, o);
        if (!rec[m]) continue;
        int32_t *map = maps[m] + (o - off[m]);
        const int32_t c = C[*map];
        out[o] = new_id1[c] - (int32_t)base1[m];
        if (keep[m]) *map = new_id2[c];
    }
}

int launch_compose(int64_t n0, int M, const int64_t *off, int32_t *const *maps,
                   const int32_t *rec, const int32_t *keep, const int32_t *C,
                   const int32_t *new_id1, const int64_t *base1, const int32_t *new_id2,
                   int32_t *out, cudaStream_t s, const LaunchCfg &lc)
{
    if (n0 == 0) return 0;
    k_compose<<<grid_for(n0, kBlock, lc.max_blocks), kBlock, 0, s>>>(
        n0, M, off, maps, rec, keep, C, new_id1, base1, new_id2, out);
    return 1;
}

}  // namespace lv
