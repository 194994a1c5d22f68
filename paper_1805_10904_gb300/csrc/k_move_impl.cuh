// k_move_impl.cuh -- one synchronous local-moving sweep (arXiv 1805.10904, Algorithm 1 body).
//
// For every vertex i, using only the previous iteration's state (C, deg_C, size_C):
//   e_{i->c} = sum of the weights from i into community c over non-loop entries (Eq. 1;
//              the loop is left out of the move decision as in Sec. 5.1.2),
//   G_c      = 2W * e_{i->c} - delta_i * deg_c          for c != C(i),
//   G_stay   = 2W * e_{i->C(i)} - delta_i * (deg_{C(i)} - delta_i),
// which are the Eq. 4 gains scaled by (2W)^2 / 2 with the term dropped from Eq. 4 as
// printed restored; target = argmax G_c with ties to the smaller label (Eq. 5,
// Sec. 3.1.2); i moves iff G_target > G_stay, except that a singleton never moves into
// a singleton community with a larger label (Sec. 3.1.1).
//
// The same pass also accumulates, for the state it reads, sum_i e_{i->C(i)} with loops
// (the first term of Eq. 3) and sum_c deg_c^2, so the phase controller gets the exact
// Qn = (2W)^2 Q of that state without a separate pass over the edges.
//
// Work is binned by row length (Sec. 6.3 suggests grouping vertices by degree):
//   bin 0    one thread per vertex, neighbours aggregated in registers (dense over all i),
//   bin 1-2  8-lane groups / whole warps, one shared-memory hash table per group,
//   bin 3-5  one CTA per row with a shared-memory table sized for the bin (up to 16K slots),
//   bin 6-9  a thread-block cluster of 2-16 CTAs per row; the table is partitioned over the
//            cluster's distributed shared memory by key hash (inserts are DSMEM atomics),
//            each CTA scans its own part, and rank 0 combines the partial argmaxes,
//   bin 10   CTA-sized chunks of a row, each aggregated in shared memory; a row spanning
//            several chunks has its chunks' distinct (community, weight) pairs grouped by a
//            hash partition, every partition merged in shared memory by a work item of its
//            own, and the partial argmaxes combined by the item finishing the row last.
// The first sweep of a phase (FIRST) scores entries without tables (see below).
// Table values are 32-bit when 2W < 2^32 (every e_{i->c} <= delta_i <= 2W fits), else 64-bit.
#pragma once
#include <algorithm>
#include <climits>

#include <cooperative_groups.h>

#include "lv_common.cuh"
#include "lv_kernels.h"

namespace lv {

constexpr int kSmallMax = 8;  // register slots of the thread-per-vertex kernel
constexpr int kUnroll = 4;    // independent row entries in flight per thread
// bin 5 runs 512-thread CTAs when its table has at most 2^kHalfCtaLog2 slots (rows of at
// most 6,144 entries) with 32-bit sums (two such tables fit an SM), else 1024-thread CTAs
constexpr int kHalfCtaLog2 = 13;

template <typename WT>
struct MoveArgs {
    int64_t n;
    const int64_t *rp;
    const int32_t *col;
    const WT *w;
    const int32_t *C;
    const i64 *deg;
    const int32_t *size;
    const i64 *delta;
    i64 tw;               // 2W of the graph (one graph)
    int32_t *Cnext;
    SweepStats *st;       // per graph (one entry for one graph)
    unsigned *err;
    const int32_t *vg;    // graph of every vertex in a batch of graphs, nullptr for one graph
    const i64 *gtw;       // 2W of every graph of the batch
    const LevelCtl *gctl; // phase controller of every graph; rows of finished graphs are frozen
    const int32_t *color;  // colouring variant: only colour `cls` decides (nullptr: all)
    int32_t cls;
    const unsigned *deg32;      // 32-bit copy of deg (nullptr: none)
    const unsigned *deg32_bad;  // nonzero once a community degree reached 2^32
};

// Community degrees as the candidate scans read them: the 32-bit copy (half the bytes, so
// more of it stays in L2) while every community degree fits it, else the 64-bit deg.  The
// stay gain and the sums of squares always read deg.
struct DegRead {
    const i64 *d64;
    const unsigned *d32;
    __device__ __forceinline__ i64 operator[](int32_t c) const
    {
        return d32 ? (i64)d32[c] : d64[c];
    }
};

template <typename WT>
__device__ __forceinline__ DegRead deg_read(const MoveArgs<WT> &A)
{
    const bool ok = A.deg32 && *(volatile const unsigned *)A.deg32_bad == 0;
    return DegRead{A.deg, ok ? A.deg32 : nullptr};
}

// Graph context of vertex i: its graph, that graph's 2W, and whether its phase has stopped.
// BT (a batch) is a template flag, so the one-graph kernels carry none of this.
template <bool BT, typename WT>
__device__ __forceinline__ int graph_of(const MoveArgs<WT> &A, int64_t i)
{
    if constexpr (BT) return A.vg[i];
    else return 0;
}
template <bool BT, typename WT>
__device__ __forceinline__ i64 tw_of(const MoveArgs<WT> &A, int g)
{
    if constexpr (BT) return A.gtw[g];
    else return A.tw;
}
template <bool BT, typename WT>
__device__ __forceinline__ bool frozen(const MoveArgs<WT> &A, int g)
{
    if constexpr (BT) return *(volatile const int *)&A.gctl[g].done;
    else return false;
}

// Per-row statistics of a batch of graphs go straight to the row's graph.
__device__ __forceinline__ void row_stats(SweepStats *st, int g, i64 internal, bool moved)
{
    if (internal) atomicAdd(&st[g].internal, (u64)internal);
    if (moved) atomicAdd(&st[g].moved, 1ull);
}

// Decision of Algorithm 1 for vertex i in community a (Eq. 4-5, Sec. 3.1).
template <typename GT>
__device__ __forceinline__ int32_t choose_target(int32_t a, int32_t best, GT gbest, i64 e_a,
                                                 i64 dl, i64 tw, const i64 *deg,
                                                 const int32_t *size)
{
    if (best == INT_MAX) return a;
    const GT gstay = (GT)tw * (GT)e_a - (GT)dl * (GT)(deg[a] - dl);
    if (!(gbest > gstay)) return a;
    if (size[a] == 1 && size[best] == 1 && best > a) return a;  // singlet minimum-label rule
    return best;
}

// One candidate community c with weight e from vertex (a, dl): updates the running argmax
// or records e_{i->a}.
template <typename GT>
__device__ __forceinline__ void consider(int32_t c, i64 e, int32_t a, i64 dl, i64 tw,
                                         DegRead deg, GT &gbest, int32_t &best, i64 &e_a)
{
    if (c == a) {
        e_a = e;
        return;
    }
    const GT g = (GT)tw * (GT)e - (GT)dl * (GT)deg[c];
    if (better(g, c, gbest, best)) {
        gbest = g;
        best = c;
    }
}

// consider() with the community degree dc = deg[c] already read (unused for c == a).
template <typename GT>
__device__ __forceinline__ void consider_deg(int32_t c, i64 e, i64 dc, int32_t a, i64 dl, i64 tw,
                                             GT &gbest, int32_t &best, i64 &e_a)
{
    if (c == a) {
        e_a = e;
        return;
    }
    const GT g = (GT)tw * (GT)e - (GT)dl * (GT)dc;
    if (better(g, c, gbest, best)) {
        gbest = g;
        best = c;
    }
}

// Candidate scan of a row's claim list: list positions first, first + step, ... below m,
// scored and cleared.  kScanBatch candidates are read at a time and their community degrees
// gathered together before any is scored, so those random reads overlap instead of each
// waiting for the previous one.
constexpr int kScanBatch = 4;

template <typename GT, typename VT>
__device__ __forceinline__ void scan_list(int *keys, VT *vals, const int *list, int m, int first,
                                          int step, int32_t a, i64 dl, i64 tw, DegRead deg,
                                          GT &gbest, int32_t &best, i64 &e_a)
{
    for (int p0 = first; p0 < m; p0 += kScanBatch * step) {
        int sl[kScanBatch];
        int32_t cc[kScanBatch];
        i64 dc[kScanBatch];
#pragma unroll
        for (int u = 0; u < kScanBatch; u++) {
            const int p = p0 + u * step;
            sl[u] = p < m ? list[p] : -1;
            cc[u] = sl[u] >= 0 ? keys[sl[u]] : -1;
        }
#pragma unroll
        for (int u = 0; u < kScanBatch; u++) dc[u] = (cc[u] >= 0 && cc[u] != a) ? deg[cc[u]] : 0;
#pragma unroll
        for (int u = 0; u < kScanBatch; u++) {
            if (sl[u] < 0) continue;
            const i64 e = (i64)vals[sl[u]];
            keys[sl[u]] = -1;
            vals[sl[u]] = 0;
            consider_deg<GT>(cc[u], e, dc[u], a, dl, tw, gbest, best, e_a);
        }
    }
}

// The same over a whole table segment of cap slots (tables without a claim list): slots
// first, first + step, ...; returns the occupied slots this thread saw.
template <typename GT, typename VT>
__device__ __forceinline__ i64 scan_slots(int *keys, VT *vals, int cap, int first, int step,
                                          int32_t a, i64 dl, i64 tw, DegRead deg, GT &gbest,
                                          int32_t &best, i64 &e_a)
{
    i64 seen = 0;
    for (int s0 = first; s0 < cap; s0 += kScanBatch * step) {
        int32_t cc[kScanBatch];
        i64 dc[kScanBatch];
#pragma unroll
        for (int u = 0; u < kScanBatch; u++) {
            const int sl = s0 + u * step;
            cc[u] = sl < cap ? keys[sl] : -1;
        }
#pragma unroll
        for (int u = 0; u < kScanBatch; u++) dc[u] = (cc[u] >= 0 && cc[u] != a) ? deg[cc[u]] : 0;
#pragma unroll
        for (int u = 0; u < kScanBatch; u++) {
            if (cc[u] < 0) continue;
            const int sl = s0 + u * step;
            const i64 e = (i64)vals[sl];
            keys[sl] = -1;
            vals[sl] = 0;
            seen++;
            consider_deg<GT>(cc[u], e, dc[u], a, dl, tw, gbest, best, e_a);
        }
    }
    return seen;
}

// Helpers of the first sweep of a phase (kernels and the reason they hold below).
__device__ __forceinline__ u64 first_cand(u64 cnt)
{
    return (cnt & 0xffffffffull) + ((cnt >> 32) != 0 ? 1 : 0);
}

// Score of one non-loop entry with community c and weight x (first sweep).
template <typename GT>
__device__ __forceinline__ void first_entry(int32_t c, i64 x, i64 dc, int32_t a, i64 dl, i64 tw,
                                            GT &gbest, int32_t &best, i64 &e_a, u64 &cnt)
{
    if (c == a) {
        e_a += x;
        cnt += (u64)1 << 32;
        return;
    }
    cnt += 1;
    const GT g = (GT)tw * (GT)x - (GT)dl * (GT)dc;
    if (better(g, c, gbest, best)) {
        gbest = g;
        best = c;
    }
}

// CTA-wide argmax and sums; results valid in thread 0.  Warp 0 combines the per-warp
// partials with shuffles.  Ends with a barrier.
template <typename GT>
__device__ __forceinline__ void block_argmax(GT &g, int32_t &c, i64 &e_a, i64 &loop)
{
    __shared__ GT s_g[32];
    __shared__ int32_t s_c[32];
    __shared__ i64 s_e[32], s_l[32];
    argmax_reduce(g, c, 32);
    e_a = sum_reduce(e_a, 32);
    loop = sum_reduce(loop, 32);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_g[warp] = g;
        s_c[warp] = c;
        s_e[warp] = e_a;
        s_l[warp] = loop;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (int)(blockDim.x >> 5);
        g = lane < nw ? s_g[lane] : gain_min<GT>();
        c = lane < nw ? s_c[lane] : INT_MAX;
        e_a = lane < nw ? s_e[lane] : 0;
        loop = lane < nw ? s_l[lane] : 0;
        argmax_reduce(g, c, 32);
        e_a = sum_reduce(e_a, 32);
        loop = sum_reduce(loop, 32);
    }
    __syncthreads();
}

// CTA-wide argmax and sums including the entry counter; results valid in thread 0.
template <typename GT>
__device__ __forceinline__ void block_argmax_cnt(GT &g, int32_t &c, i64 &e_a, i64 &loop, u64 &cnt)
{
    __shared__ GT s_g[32];
    __shared__ int32_t s_c[32];
    __shared__ i64 s_e[32], s_l[32];
    __shared__ u64 s_n[32];
    argmax_reduce(g, c, 32);
    e_a = sum_reduce(e_a, 32);
    loop = sum_reduce(loop, 32);
    cnt = sum_reduce(cnt, 32);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_g[warp] = g;
        s_c[warp] = c;
        s_e[warp] = e_a;
        s_l[warp] = loop;
        s_n[warp] = cnt;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (int)(blockDim.x >> 5);
        g = lane < nw ? s_g[lane] : gain_min<GT>();
        c = lane < nw ? s_c[lane] : INT_MAX;
        e_a = lane < nw ? s_e[lane] : 0;
        loop = lane < nw ? s_l[lane] : 0;
        cnt = lane < nw ? s_n[lane] : 0;
        argmax_reduce(g, c, 32);
        e_a = sum_reduce(e_a, 32);
        loop = sum_reduce(loop, 32);
        cnt = sum_reduce(cnt, 32);
    }
    __syncthreads();
}

// ------------------------------------------------------------------ bin 0
// Dense over every vertex: also adds deg[i]^2 of label i to sum_c deg_c^2.  The loop is
// uniform across each warp so a batch of graphs can combine a warp's statistics when all
// its vertices belong to one graph.
// FIRST: the first sweep of a phase, whose non-own candidates are pairwise distinct (see
// the first-sweep kernels below), so entries are scored without the pairwise merge.
template <typename WT, typename GT, bool BT, bool FIRST>
__global__ void __launch_bounds__(kBlock) k_move_small(MoveArgs<WT> A, int small_max)
{
    u64 internal = 0, moved = 0, cand = 0;
    const DegRead dg = deg_read(A);
    u128 sq = 0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < A.n;
         i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        u64 v_int = 0, v_mov = 0;
        u128 v_sq = 0;
        int g = -1;
        if (i < A.n) {
            g = graph_of<BT>(A, i);
            const i64 di = A.deg[i];
            v_sq = (u128)(u64)di * (u64)di;
            const int64_t rb = A.rp[i];
            const int64_t d = A.rp[i + 1] - rb;
            // frozen graph, or a vertex of another colour class: it keeps its label
            const bool fz = frozen<BT>(A, g) || (A.color && A.color[i] != A.cls);
            if (d <= small_max && !fz) {
                const i64 tw = tw_of<BT>(A, g);
                const int32_t a = A.C[i];
                int32_t lab[kSmallMax];
                i64 wt[kSmallMax];
#pragma unroll
                for (int t = 0; t < kSmallMax; t++) {
                    lab[t] = -1;
                    wt[t] = 0;
                    if (t < d) {
                        lab[t] = ld_stream(A.col + rb + t);
                        wt[t] = (i64)ld_stream(A.w + rb + t);
                    }
                }
                i64 loop = 0;
#pragma unroll
                for (int t = 0; t < kSmallMax; t++) {
                    if (t < d) {
                        if (lab[t] == (int32_t)i) {
                            loop += wt[t];
                            lab[t] = -1;
                        } else {
                            lab[t] = A.C[lab[t]];
                        }
                    }
                }
                const i64 dl = A.delta[i];
                i64 e_a = 0;
                GT gbest = gain_min<GT>();
                int32_t best = INT_MAX;
                int m = 0;
                if constexpr (FIRST) {
                    u64 cnt = 0;
#pragma unroll
                    for (int t = 0; t < kSmallMax; t++) {
                        const int32_t c = lab[t];
                        if (c >= 0)
                            first_entry<GT>(c, wt[t], c == a ? 0 : dg[c], a, dl, tw, gbest,
                                            best, e_a, cnt);
                    }
                    m = (int)first_cand(cnt);
                } else {
#pragma unroll
                    for (int t = 0; t < kSmallMax; t++) {
                        const int32_t c = lab[t];
                        bool first = c >= 0;
#pragma unroll
                        for (int u = 0; u < t; u++) first = first && (lab[u] != c);
                        if (first) {
                            i64 e = 0;
#pragma unroll
                            for (int u = t; u < kSmallMax; u++) e += (lab[u] == c) ? wt[u] : 0;
                            m++;
                            consider<GT>(c, e, a, dl, tw, dg, gbest, best, e_a);
                        }
                    }
                }
                const int32_t target = choose_target<GT>(a, best, gbest, e_a, dl, tw, A.deg, A.size);
                A.Cnext[i] = target;
                v_mov = target != a;
                v_int = (u64)(e_a + loop);
                cand += (u64)m;
            } else if (d <= small_max) {
                A.Cnext[i] = A.C[i];  // frozen graph or other class: nothing moves
            }
        }
        if constexpr (!BT) {
            internal += v_int;
            moved += v_mov;
            sq += v_sq;
            continue;
        }
        // batch of graphs: one atomic per warp when the warp's vertices share a graph
        const int g0 = __shfl_sync(0xffffffffu, g, 0);
        if (__all_sync(0xffffffffu, g == g0 || g < 0)) {
            const u64 wi = sum_reduce(v_int, 32), wm = sum_reduce(v_mov, 32);
            const u128 ws = sum_reduce(v_sq, 32);
            if ((threadIdx.x & 31) == 0 && g0 >= 0) {
                if (wi) atomicAdd(&A.st[g0].internal, wi);
                if (wm) atomicAdd(&A.st[g0].moved, wm);
                if (ws) atomic_add_u128(&A.st[g0].sq_lo, &A.st[g0].sq_hi, ws);
            }
        } else if (g >= 0) {
            if (v_int) atomicAdd(&A.st[g].internal, v_int);
            if (v_mov) atomicAdd(&A.st[g].moved, v_mov);
            if (v_sq) atomic_add_u128(&A.st[g].sq_lo, &A.st[g].sq_hi, v_sq);
        }
    }
    block_flush_stats(A.st, 0, internal, moved, cand, sq);
}

// ------------------------------------------------------------------ bins 1-2
// G lanes per vertex (G <= 32), each group with a 2^LOG2CAP-slot shared table.  The
// outer loop is uniform across the block so every lane reaches the shuffles.
template <int G, int LOG2CAP, typename WT, typename GT, typename VT, bool BT>
__global__ void __launch_bounds__(kBlock) k_move_group(MoveArgs<WT> A, const int32_t *verts,
                                                       int nverts, int slot)
{
    constexpr int CAP = 1 << LOG2CAP;
    constexpr int NG = kBlock / G;
    __shared__ int s_keys[NG * CAP];
    __shared__ VT s_vals[NG * CAP];
    __shared__ int s_list[NG * CAP];
    __shared__ int s_cnt[NG];
    for (int s = threadIdx.x; s < NG * CAP; s += kBlock) {
        s_keys[s] = -1;
        s_vals[s] = 0;
    }
    if (threadIdx.x < NG) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    int *keys = s_keys + g * CAP;
    VT *vals = s_vals + g * CAP;
    int *list = s_list + g * CAP;
    int *cnt = &s_cnt[g];
    u64 internal = 0, moved = 0, cand = 0;
    const DegRead dg = deg_read(A);
    for (int base = blockIdx.x * NG; base < nverts; base += gridDim.x * NG) {
        const int vi = base + g;
        const bool valid = vi < nverts;
        int32_t i = 0, a = 0;
        int64_t rb = 0, re = 0;
        i64 dl = 0, tw = 0;
        int gr = 0;
        bool fz = false;
        if (valid) {
            i = verts[vi];
            gr = graph_of<BT>(A, i);
            tw = tw_of<BT>(A, gr);
            fz = frozen<BT>(A, gr);
            rb = A.rp[i];
            re = fz ? rb : A.rp[i + 1];  // a frozen row inserts nothing and stays
            a = A.C[i];
            dl = A.delta[i];
        }
        i64 loop = 0;
        // kUnroll entries per lane in flight: columns and weights, then their labels
        for (int64_t k0 = rb + lane; k0 < re; k0 += (int64_t)G * kUnroll) {
            int32_t j[kUnroll], c[kUnroll];
            i64 x[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                const int64_t k = k0 + (int64_t)G * u;
                j[u] = k < re ? ld_stream(A.col + k) : -1;
                x[u] = k < re ? (i64)ld_stream(A.w + k) : 0;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; u++) c[u] = (j[u] >= 0 && j[u] != i) ? A.C[j[u]] : -1;
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                if (j[u] == i) loop += x[u];
                else if (c[u] >= 0)
                    tbl_insert<false, VT>(keys, vals, list, cnt, LOG2CAP, c[u], (VT)x[u], A.err);
            }
        }
        __syncwarp();
        const int m = valid ? *(volatile int *)cnt : 0;
        GT gbest = gain_min<GT>();
        int32_t best = INT_MAX;
        i64 e_a = 0;
        scan_list<GT, VT>(keys, vals, list, m, lane, G, a, dl, tw, dg, gbest, best, e_a);
        argmax_reduce(gbest, best, G);
        e_a = sum_reduce(e_a, G);
        loop = sum_reduce(loop, G);
        if (lane == 0) {
            if (valid) {
                const int32_t target =
                    choose_target<GT>(a, best, gbest, e_a, dl, tw, A.deg, A.size);
                A.Cnext[i] = target;
                if constexpr (!BT) {
                    moved += target != a;
                    internal += (u64)(e_a + loop);
                } else if (!fz) {
                    row_stats(A.st, gr, e_a + loop, target != a);
                }
                cand += (u64)m;
            }
            *cnt = 0;
        }
        __syncwarp();
    }
    block_flush_stats(A.st, slot, internal, moved, cand, 0);
}

// ------------------------------------------------------------------ bins 3-5
// Table insert of one chunk entry (key -1 = loop or absent entry: nothing to insert).
template <typename VT, typename Ins>
__device__ __forceinline__ void chunk_insert(int32_t key, i64 x, Ins ins)
{
    if (key >= 0) ins(key, (VT)x);
}

// Loads of one chunk of a row: entries base + u * BLOCK, u < kUnroll, below re.
template <int BLOCK, typename WT>
__device__ __forceinline__ void load_chunk(const MoveArgs<WT> &A, int64_t base, int64_t re,
                                           int32_t (&j)[kUnroll], i64 (&x)[kUnroll])
{
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
        const int64_t k = base + (int64_t)u * BLOCK;
        j[u] = -1;
        x[u] = 0;
        if (k < re) {
            j[u] = ld_stream(A.col + k);
            x[u] = (i64)ld_stream(A.w + k);
        }
    }
}

// Label gathers of a loaded chunk of row i: community of each non-loop entry, -1 otherwise.
template <typename WT>
__device__ __forceinline__ void gather_chunk(const MoveArgs<WT> &A, int32_t i,
                                             const int32_t (&j)[kUnroll], int32_t (&c)[kUnroll])
{
#pragma unroll
    for (int u = 0; u < kUnroll; u++) c[u] = (j[u] >= 0 && j[u] != i) ? A.C[j[u]] : -1;
}

// One CTA per row, table of 2^log2cap slots in dynamic shared memory (vals, keys, list).
// Software pipeline over the CTA's rows: while row v finishes (barrier, candidate scan,
// argmax), the next row's vertex id, entry range, first chunk of columns / weights and its
// label gathers are already in flight, issued stage by stage so no load waits on another.
// 128-thread CTAs are held to 64 registers a thread, so 8 rows are in flight on an SM (6
// otherwise; 12% faster at R-MAT 26); two 512-thread CTAs fit.  The same cap on 256-thread
// CTAs (4 rows instead of 3) made them twice as slow at R-MAT 26 and is not applied.
template <int BLOCK, typename WT, typename GT, typename VT, bool BT>
__global__ void __launch_bounds__(BLOCK, BLOCK == 128 ? 8 : (BLOCK == 512 ? 2 : 1))
    k_move_cta(MoveArgs<WT> A, const int32_t *verts, int nverts, int log2cap, int slot)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int cap = 1 << log2cap;
    VT *vals = (VT *)smem;
    int *keys = (int *)(vals + cap);
    int *list = keys + cap;
    __shared__ int s_cnt;
    for (int s = threadIdx.x; s < cap; s += BLOCK) {
        keys[s] = -1;
        vals[s] = 0;
    }
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    // the kUnroll entries of a thread go into the table together (tbl_insert_batch); the
    // loops around it are uniform across each warp
    auto ins = [&](const int32_t (&key)[kUnroll], const i64 (&x)[kUnroll]) {
        VT v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; u++) v[u] = (VT)x[u];
        tbl_insert_batch<kUnroll, VT>(keys, vals, list, &s_cnt, log2cap, key, v, A.err);
    };
    u64 internal = 0, moved = 0, cand = 0;
    const DegRead dg = deg_read(A);
    // prologue: the first row completely prefetched
    int v = blockIdx.x;
    int32_t nx_i = -1;
    int64_t nx_rb = 0, nx_re = 0;
    if (v < nverts) {
        nx_i = verts[v];
        nx_rb = A.rp[nx_i];
        nx_re = A.rp[nx_i + 1];
    }
    int32_t nj[kUnroll], nc[kUnroll];
    i64 nw[kUnroll];
    load_chunk<BLOCK>(A, nx_rb + threadIdx.x, nx_re, nj, nw);
    gather_chunk(A, nx_i, nj, nc);
    for (; v < nverts; v += gridDim.x) {
        const int32_t i = nx_i;
        const int64_t rb = nx_rb, re = nx_re;
        // stage 1: next row's vertex id; this row's own community and degree
        const int vn = v + gridDim.x;
        const int32_t i_next = vn < nverts ? verts[vn] : -1;
        const int32_t a = A.C[i];
        const i64 dl = A.delta[i];
        const int gr = graph_of<BT>(A, i);
        const i64 tw = tw_of<BT>(A, gr);
        const bool fz = frozen<BT>(A, gr);  // a frozen row inserts nothing and stays
        // the prefetched first chunk, then the rest of the row
        i64 loop = 0;
        if (!fz) {  // fz is the same for the whole CTA (one row)
#pragma unroll
            for (int u = 0; u < kUnroll; u++)
                if (nj[u] == i) loop += nw[u];
            ins(nc, nw);
        }
        for (int64_t k0 = rb + threadIdx.x + (int64_t)kUnroll * BLOCK;
             !fz && __any_sync(0xffffffffu, k0 < re); k0 += (int64_t)kUnroll * BLOCK) {
            int32_t j[kUnroll], c[kUnroll];
            i64 x[kUnroll];
            load_chunk<BLOCK>(A, k0, re, j, x);
            gather_chunk(A, i, j, c);
#pragma unroll
            for (int u = 0; u < kUnroll; u++)
                if (j[u] == i) loop += x[u];
            ins(c, x);
        }
        // stage 2: next row's entry range; this row's community degree and size
        int64_t rb_next = 0, re_next = 0;
        if (i_next >= 0) {
            rb_next = A.rp[i_next];
            re_next = A.rp[i_next + 1];
        }
        const i64 deg_a = A.deg[a];
        const int32_t size_a = A.size[a];
        __syncthreads();
        const int m = s_cnt;
        // stage 3: next row's first chunk of columns and weights
        load_chunk<BLOCK>(A, rb_next + threadIdx.x, re_next, nj, nw);
        GT gbest = gain_min<GT>();
        int32_t best = INT_MAX;
        i64 e_a = 0;
        // one candidate at a time here: the batched scan (scan_list) needs registers that the
        // next row's prefetched chunk holds, and made bins 3-4 slower (R-MAT 26: 93.7 -> 113.3
        // ms per run for 256-thread CTAs) while it speeds up the group and cluster kernels
        for (int p = threadIdx.x; p < m; p += BLOCK) {
            const int s = list[p];
            const int32_t cc = keys[s];
            const i64 e = (i64)vals[s];
            keys[s] = -1;
            vals[s] = 0;
            consider<GT>(cc, e, a, dl, tw, dg, gbest, best, e_a);
        }
        // stage 4: next row's label gathers
        gather_chunk(A, i_next, nj, nc);
        block_argmax(gbest, best, e_a, loop);
        if (threadIdx.x == 0) {
            int32_t target = a;
            if (best != INT_MAX) {
                const GT gstay = (GT)tw * (GT)e_a - (GT)dl * (GT)(deg_a - dl);
                if (gbest > gstay && !(size_a == 1 && best > a && A.size[best] == 1))
                    target = best;
            }
            A.Cnext[i] = target;
            if constexpr (!BT) {
                moved += target != a;
                internal += (u64)(e_a + loop);
            } else if (!fz) {
                row_stats(A.st, gr, e_a + loop, target != a);
            }
            cand += (u64)m;
            s_cnt = 0;
        }
        nx_i = i_next;
        nx_rb = rb_next;
        nx_re = re_next;
        __syncthreads();
    }
    block_flush_stats(A.st, slot, internal, moved, cand, 0);
}

// ------------------------------------------------------------------ bins 6-9
namespace cg = cooperative_groups;

template <int CL>
struct Log2Of {
    static constexpr int v = CL <= 1 ? 0 : 1 + Log2Of<CL / 2>::v;
};
template <>
struct Log2Of<1> {
    static constexpr int v = 0;
};

template <int CL, typename WT, typename GT, typename VT, bool BT>
__global__ void __launch_bounds__(1024) k_move_cluster(MoveArgs<WT> A, const int32_t *verts,
                                                       int nverts, int log2cap, int slot)
{
    constexpr int BLOCK = 1024;
    constexpr int LOG2CL = Log2Of<CL>::v;
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    extern __shared__ __align__(16) unsigned char smem[];
    const int cap = 1 << log2cap;
    VT *vals = (VT *)smem;
    int *keys = (int *)(vals + cap);
    __shared__ GT p_g;
    __shared__ int32_t p_c;
    __shared__ i64 p_e, p_l, p_m;
    for (int s = threadIdx.x; s < cap; s += BLOCK) {
        keys[s] = -1;
        vals[s] = 0;
    }
    cluster.sync();
    const int cid = blockIdx.x / CL, ncl = gridDim.x / CL;
    const int64_t stride = (int64_t)CL * BLOCK;
    u64 internal = 0, moved = 0, cand = 0;
    // the 64-bit degrees here: these kernels are bound by their remote atomics, and reading the
    // 32-bit copy made them slower (R-MAT 26: clusters of 2 and 8, 52.3 -> 54.8, 42.9 -> 44.1 ms)
    const DegRead dg{A.deg, nullptr};
    for (int v = cid; v < nverts; v += ncl) {
        const int32_t i = verts[v];
        const int gr = graph_of<BT>(A, i);
        const i64 tw = tw_of<BT>(A, gr);
        const bool fz = frozen<BT>(A, gr);  // a frozen row inserts nothing and stays
        const int64_t rb = A.rp[i], re = fz ? rb : A.rp[i + 1];
        i64 loop = 0;
        for (int64_t k0 = rb + (int64_t)rank * BLOCK + threadIdx.x;
             __any_sync(0xffffffffu, k0 < re); k0 += (int64_t)kUnroll * stride) {
            int32_t j[kUnroll];
            i64 x[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                const int64_t k = k0 + (int64_t)u * stride;
                j[u] = -1;
                x[u] = 0;
                if (k < re) {
                    j[u] = ld_stream(A.col + k);
                    x[u] = (i64)ld_stream(A.w + k);
                }
            }
            int32_t c[kUnroll];
            VT cv[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                c[u] = (j[u] >= 0 && j[u] != i) ? A.C[j[u]] : -1;
                cv[u] = (VT)x[u];
            }
#pragma unroll
            for (int u = 0; u < kUnroll; u++)
                if (j[u] == i) loop += x[u];
            cluster_insert_batch<kUnroll, VT>(cluster, keys, vals, LOG2CL, log2cap, c, cv, A.err);
        }
        cluster.sync();  // every insert of this row has landed
        const int32_t a = A.C[i];
        const i64 dl = A.delta[i];
        GT gbest = gain_min<GT>();
        int32_t best = INT_MAX;
        i64 e_a = 0;
        i64 mloc = scan_slots<GT, VT>(keys, vals, cap, threadIdx.x, BLOCK, a, dl, tw, dg, gbest,
                                      best, e_a);
        mloc = sum_reduce(mloc, 32);  // per-warp count, folded into the CTA sum below
        block_argmax(gbest, best, e_a, loop);
        __shared__ i64 s_mw[32];
        if ((threadIdx.x & 31) == 0) s_mw[threadIdx.x >> 5] = mloc;
        __syncthreads();
        if (threadIdx.x == 0) {
            i64 m = 0;
            for (int w = 0; w < BLOCK / 32; w++) m += s_mw[w];
            p_g = gbest;
            p_c = best;
            p_e = e_a;
            p_l = loop;
            p_m = m;
        }
        cluster.sync();  // partial results of every CTA published
        if (rank == 0 && threadIdx.x == 0) {
            GT g = p_g;
            int32_t c = p_c;
            i64 ea = p_e, lp = p_l, mm = p_m;
#pragma unroll 1
            for (int r = 1; r < CL; r++) {
                const GT g2 = *cluster.map_shared_rank(&p_g, r);
                const int32_t c2 = *cluster.map_shared_rank(&p_c, r);
                if (better(g2, c2, g, c)) {
                    g = g2;
                    c = c2;
                }
                ea += *cluster.map_shared_rank(&p_e, r);
                lp += *cluster.map_shared_rank(&p_l, r);
                mm += *cluster.map_shared_rank(&p_m, r);
            }
            const int32_t target = choose_target<GT>(a, c, g, ea, dl, tw, A.deg, A.size);
            A.Cnext[i] = target;
            if constexpr (!BT) {
                moved += target != a;
                internal += (u64)(ea + lp);
            } else if (!fz) {
                row_stats(A.st, gr, ea + lp, target != a);
            }
            cand += (u64)mm;
        }
        cluster.sync();  // partials read before the next row overwrites them
    }
    block_flush_stats(A.st, slot, internal, moved, cand, 0);
}

// ------------------------------------------------------------------ bin 10
constexpr int kHugeBlock = 512;

struct BigArgs {
    const int32_t *bverts;
    const int32_t *chunk_b;
    const int32_t *chunk_first;
    const int32_t *nch;
    u64 *gloop;        // loop weight of every multi-chunk row
    int chunk;
    int nchunks;
    // partials of multi-chunk rows: one per partition (table sweeps) or chunk (first sweeps)
    void *pgain;
    int32_t *pbest;
    i64 *pea;
    u64 *pcnt;
    int32_t *sdone;    // partials finished per row
    const int64_t *soff;
    const int32_t *slice_row;
    int64_t nslices;
    // partitioned aggregation (table sweeps)
    const int32_t *plog2;
    const int64_t *hoff;
    int32_t *hofs;
    int32_t *pkeys;
    void *pvals;
};

inline BigArgs big_args(const Bins &b)
{
    BigArgs B;
    B.bverts = b.rows(kChunkedBin);
    B.chunk_b = b.chunk_b;
    B.chunk_first = b.chunk_first;
    B.nch = b.nch;
    B.gloop = b.gloop;
    B.chunk = b.chunk;
    B.nchunks = b.nchunks;
    B.pgain = b.pgain;
    B.pbest = b.pbest;
    B.pea = b.pea;
    B.pcnt = b.pcnt;
    B.sdone = b.sdone;
    B.soff = b.soff;
    B.slice_row = b.slice_row;
    B.nslices = b.nslices;
    B.plog2 = b.plog2;
    B.hoff = b.hoff;
    B.hofs = b.hofs;
    B.pkeys = b.pkeys;
    B.pvals = b.pvals;
    return B;
}

template <typename WT, typename GT, typename VT, bool BT>
__global__ void __launch_bounds__(kHugeBlock) k_move_huge(MoveArgs<WT> A, BigArgs B)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int log2cap = 31 - __clz(2 * B.chunk);  // 2 * chunk slots
    const int cap = 1 << log2cap;
    VT *vals = (VT *)smem;
    int *keys = (int *)(vals + cap);
    int *list = keys + cap;
    __shared__ int s_cnt;
    __shared__ int s_hist[(1 << kMaxPartLog2) + 1];
    for (int s = threadIdx.x; s < cap; s += kHugeBlock) {
        keys[s] = -1;
        vals[s] = 0;
    }
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    u64 internal = 0, moved = 0, cand = 0;
    const DegRead dg = deg_read(A);
    for (int c = blockIdx.x; c < B.nchunks; c += gridDim.x) {
        const int b = B.chunk_b[c];
        const int32_t i = B.bverts[b];
        const int q = c - B.chunk_first[b];
        const int nch = B.nch[b];
        const int64_t rb = A.rp[i], re = A.rp[i + 1];
        const int64_t cb = rb + (int64_t)q * B.chunk;
        const int64_t ce = min(re, cb + (int64_t)B.chunk);
        const int32_t a = A.C[i];
        const i64 dl = A.delta[i];
        const int gr = graph_of<BT>(A, i);
        const i64 tw = tw_of<BT>(A, gr);
        if (frozen<BT>(A, gr)) {  // a frozen row stays; its first chunk records that
            if (q == 0 && threadIdx.x == 0) A.Cnext[i] = a;
            continue;
        }
        i64 loop = 0;
        for (int64_t k0 = cb + threadIdx.x; k0 < ce; k0 += (int64_t)kUnroll * kHugeBlock) {
            int32_t j[kUnroll];
            i64 x[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                const int64_t k = k0 + (int64_t)u * kHugeBlock;
                j[u] = -1;
                x[u] = 0;
                if (k < ce) {
                    j[u] = ld_stream(A.col + k);
                    x[u] = (i64)ld_stream(A.w + k);
                }
            }
            int32_t cc[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; u++) cc[u] = (j[u] >= 0 && j[u] != i) ? A.C[j[u]] : -1;
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                if (j[u] == i) loop += x[u];
                else if (cc[u] >= 0)
                    tbl_insert<false, VT>(keys, vals, list, &s_cnt, log2cap, cc[u], (VT)x[u], A.err);
            }
        }
        __syncthreads();
        const int m = s_cnt;
        if (nch == 1) {
            GT gbest = gain_min<GT>();
            int32_t best = INT_MAX;
            i64 e_a = 0;
            for (int p = threadIdx.x; p < m; p += kHugeBlock) {
                const int s = list[p];
                const int32_t k2 = keys[s];
                const i64 e = (i64)vals[s];
                keys[s] = -1;
                vals[s] = 0;
                consider<GT>(k2, e, a, dl, tw, dg, gbest, best, e_a);
            }
            block_argmax(gbest, best, e_a, loop);
            if (threadIdx.x == 0) {
                const int32_t target =
                    choose_target<GT>(a, best, gbest, e_a, dl, tw, A.deg, A.size);
                A.Cnext[i] = target;
                if constexpr (!BT) {
                    moved += target != a;
                    internal += (u64)(e_a + loop);
                } else {
                    row_stats(A.st, gr, e_a + loop, target != a);
                }
                cand += (u64)m;
            }
        } else {
            // partitioned aggregation: the chunk's distinct keys, grouped by partition, go to
            // the chunk's own region of the pair buffer, with the partitions' offsets;
            // k_move_huge_decide merges each partition of the row over all its chunks
            const int lp = B.plog2[b];
            const int P = 1 << lp;
            for (int p = threadIdx.x; p <= P; p += kHugeBlock) s_hist[p] = 0;
            __syncthreads();
            for (int r = threadIdx.x; r < m; r += kHugeBlock)
                atomicAdd(&s_hist[part_of(keys[list[r]], lp)], 1);
            __syncthreads();
            cta_excl_scan_smem<kHugeBlock>(s_hist, P);
            int32_t *ho = B.hofs + B.hoff[b] + (int64_t)q * (P + 1);
            for (int p = threadIdx.x; p <= P; p += kHugeBlock) ho[p] = s_hist[p];
            __syncthreads();  // offsets published before they turn into cursors
            int32_t *pk = B.pkeys + (int64_t)c * B.chunk;
            VT *pv = (VT *)B.pvals + (int64_t)c * B.chunk;
            for (int r = threadIdx.x; r < m; r += kHugeBlock) {
                const int s = list[r];
                const int32_t k2 = keys[s];
                const VT e = vals[s];
                keys[s] = -1;
                vals[s] = 0;
                const int pos = atomicAdd(&s_hist[part_of(k2, lp)], 1);
                pk[pos] = k2;
                pv[pos] = e;
            }
            loop = sum_reduce(loop, 32);
            if ((threadIdx.x & 31) == 0 && loop) atomicAdd(&B.gloop[b], (u64)loop);
        }
        __syncthreads();
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
    }
    block_flush_stats(A.st, kChunkedBin, internal, moved, cand, 0);
}

// Decision of the rows spread over several chunks, after k_move_huge wrote their chunks'
// pairs: one work item per partition of a row merges that partition's pairs of every chunk
// in a shared table (merge_partition, split into residue classes if its keys would crowd
// the table) and scores its keys (partial argmax); the CTA finishing a row's last partition
// combines the partials and decides the row.
template <typename WT, typename GT, typename VT, bool BT>
__global__ void __launch_bounds__(kHugeBlock) k_move_huge_decide(MoveArgs<WT> A, BigArgs B)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int log2cap = kPartTableLog2;
    constexpr int cap = 1 << log2cap;
    constexpr int thresh = cap - 2 * kHugeBlock;
    VT *vals = (VT *)smem;
    int *keys = (int *)(vals + cap);
    int *list = keys + cap;
    __shared__ int s_last;
    for (int s = threadIdx.x; s < cap; s += kHugeBlock) {
        keys[s] = -1;
        vals[s] = 0;
    }
    __syncthreads();
    GT *pg = (GT *)B.pgain;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    u64 internal = 0, moved = 0, cand = 0;
    const DegRead dg = deg_read(A);
    for (int64_t q = blockIdx.x; q < B.nslices; q += gridDim.x) {
        const int b = B.slice_row[q];
        const int32_t i = B.bverts[b];
        const int gr = graph_of<BT>(A, i);
        if (frozen<BT>(A, gr)) continue;  // its first chunk kept it in place
        const int64_t s0 = B.soff[b];
        const int ns = (int)(B.soff[b + 1] - s0);
        const int p = (int)(q - s0);
        const int P = 1 << B.plog2[b];
        const int nch = B.nch[b];
        const int64_t c0 = B.chunk_first[b];
        const int32_t *ho = B.hofs + B.hoff[b];
        const int32_t a = A.C[i];
        const i64 dl = A.delta[i];
        const i64 tw = tw_of<BT>(A, gr);
        GT gbest = gain_min<GT>();
        int32_t best = INT_MAX;
        i64 e_a = 0, lz = 0;
        u64 mm = 0;
        // partition p of every chunk: warps take chunks in turn, lanes the chunk's pairs
        auto for_pairs = [&](auto f) {
            for (int t = warp; t < nch; t += kHugeBlock / 32) {
                const int lo = ho[(int64_t)t * (P + 1) + p];
                const int hi = ho[(int64_t)t * (P + 1) + p + 1];
                const int32_t *pk = B.pkeys + (c0 + t) * B.chunk;
                const VT *pv = (const VT *)B.pvals + (c0 + t) * B.chunk;
                for (int r = lo + lane; r < hi; r += 32) f(pk[r], pv[r]);
            }
        };
        auto emit = [&](int m) {
            for (int r = threadIdx.x; r < m; r += kHugeBlock) {
                const int s = list[r];
                const int32_t k2 = keys[s];
                const i64 e = (i64)vals[s];
                keys[s] = -1;
                vals[s] = 0;
                consider<GT>(k2, e, a, dl, tw, dg, gbest, best, e_a);
            }
            if (threadIdx.x == 0) mm += (u64)m;
        };
        merge_partition<kHugeBlock, VT>(keys, vals, list, log2cap, thresh, A.err, for_pairs, emit);
        block_argmax_cnt(gbest, best, e_a, lz, mm);
        if (threadIdx.x == 0) {
            pg[q] = gbest;
            B.pbest[q] = best;
            B.pea[q] = e_a;
            B.pcnt[q] = mm;
            __threadfence();
            s_last = atomicAdd(&B.sdone[b], 1) == ns - 1;
        }
        __syncthreads();
        if (s_last) {  // every partition of row b is in: combine and decide
            __threadfence();
            GT g = gain_min<GT>();
            int32_t cb = INT_MAX;
            i64 ea = 0, l0 = 0;
            u64 n = 0;
            for (int t = threadIdx.x; t < ns; t += kHugeBlock) {
                const GT gt = *(volatile const GT *)&pg[s0 + t];  // bypasses L1
                const int32_t ct = __ldcg(&B.pbest[s0 + t]);
                if (better(gt, ct, g, cb)) {
                    g = gt;
                    cb = ct;
                }
                ea += __ldcg(&B.pea[s0 + t]);
                n += __ldcg(&B.pcnt[s0 + t]);
            }
            block_argmax_cnt(g, cb, ea, l0, n);
            if (threadIdx.x == 0) {
                const i64 lp = (i64)__ldcg(&B.gloop[b]);
                const int32_t target = choose_target<GT>(a, cb, g, ea, dl, tw, A.deg, A.size);
                A.Cnext[i] = target;
                if constexpr (!BT) {
                    moved += target != a;
                    internal += (u64)(ea + lp);
                } else {
                    row_stats(A.st, gr, ea + lp, target != a);
                }
                cand += n;
                B.gloop[b] = 0;
                B.sdone[b] = 0;
            }
        }
        __syncthreads();  // s_last read before the next item sets it
    }
    block_flush_stats(A.st, kChunkedBin, internal, moved, cand, 0);
}

// ------------------------------------------------------------------ first sweep of a phase
// Every phase starts from singleton communities, plus, at vertex-following levels,
// degree-one vertices placed in their only neighbour's community.  On a graph whose rows
// list every column at most once, the communities of row i's entries other than C(i) are
// then pairwise distinct: a non-loop neighbour j either keeps its own label j, or it
// follows, and then its only neighbour is i and C(j) = C(i) (an isolated pair shares
// min(i, j)).  So each candidate c != C(i) comes from a single entry, e_{i->c} = A_ij, and
// the first sweep scores the entries directly, without any table; e_{i->C(i)} sums the
// entries labelled C(i).  The distinct neighbouring communities of a row (the candidate
// statistic) are its entries labelled c != C(i), plus one when some entry is labelled C(i):
// the counters carry (entries labelled C(i)) << 32 | (other entries).
// G lanes per row (bins 1-2): each lane scores its entries, then the group reduces.
template <int G, typename WT, typename GT, bool BT>
__global__ void __launch_bounds__(kBlock) k_move_group_first(MoveArgs<WT> A, const int32_t *verts,
                                                             int nverts, int slot)
{
    constexpr int NG = kBlock / G;
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    u64 internal = 0, moved = 0, cand = 0;
    const DegRead dg = deg_read(A);
    for (int base = blockIdx.x * NG; base < nverts; base += gridDim.x * NG) {
        const int vi = base + g;
        const bool valid = vi < nverts;
        int32_t i = 0, a = 0;
        int64_t rb = 0, re = 0;
        i64 dl = 0, tw = 0;
        int gr = 0;
        bool fz = false;
        if (valid) {
            i = verts[vi];
            gr = graph_of<BT>(A, i);
            tw = tw_of<BT>(A, gr);
            fz = frozen<BT>(A, gr);
            rb = A.rp[i];
            re = fz ? rb : A.rp[i + 1];
            a = A.C[i];
            dl = A.delta[i];
        }
        i64 loop = 0, e_a = 0;
        u64 cnt = 0;
        GT gbest = gain_min<GT>();
        int32_t best = INT_MAX;
        for (int64_t k0 = rb + lane; k0 < re; k0 += (int64_t)G * kUnroll) {
            int32_t j[kUnroll], c[kUnroll];
            i64 x[kUnroll], dc[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                const int64_t k = k0 + (int64_t)G * u;
                j[u] = k < re ? ld_stream(A.col + k) : -1;
                x[u] = k < re ? (i64)ld_stream(A.w + k) : 0;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; u++) c[u] = (j[u] >= 0 && j[u] != i) ? A.C[j[u]] : -1;
#pragma unroll
            for (int u = 0; u < kUnroll; u++) dc[u] = (c[u] >= 0 && c[u] != a) ? dg[c[u]] : 0;
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                if (j[u] == i) loop += x[u];
                else if (c[u] >= 0)
                    first_entry<GT>(c[u], x[u], dc[u], a, dl, tw, gbest, best, e_a, cnt);
            }
        }
        argmax_reduce(gbest, best, G);
        e_a = sum_reduce(e_a, G);
        loop = sum_reduce(loop, G);
        cnt = sum_reduce(cnt, G);
        if (lane == 0 && valid) {
            const int32_t target = choose_target<GT>(a, best, gbest, e_a, dl, tw, A.deg, A.size);
            A.Cnext[i] = target;
            if constexpr (!BT) {
                moved += target != a;
                internal += (u64)(e_a + loop);
            } else if (!fz) {
                row_stats(A.st, gr, e_a + loop, target != a);
            }
            cand += first_cand(cnt);
        }
    }
    block_flush_stats(A.st, slot, internal, moved, cand, 0);
}

// One CTA per row (bins 3-9): kUnroll entries in flight per thread, each scored after its
// label and community-degree gathers; no shared table, so many CTAs fit on an SM.
template <int BLOCK, typename WT, typename GT, bool BT>
__global__ void __launch_bounds__(BLOCK) k_move_cta_first(MoveArgs<WT> A, const int32_t *verts,
                                                          int nverts, int slot)
{
    u64 internal = 0, moved = 0, cand = 0;
    const DegRead dg = deg_read(A);
    for (int v = blockIdx.x; v < nverts; v += gridDim.x) {
        const int32_t i = verts[v];
        const int gr = graph_of<BT>(A, i);
        const i64 tw = tw_of<BT>(A, gr);
        const bool fz = frozen<BT>(A, gr);
        const int64_t rb = A.rp[i];
        const int64_t re = fz ? rb : A.rp[i + 1];
        const int32_t a = A.C[i];
        const i64 dl = A.delta[i];
        i64 loop = 0, e_a = 0;
        u64 cnt = 0;
        GT gbest = gain_min<GT>();
        int32_t best = INT_MAX;
        for (int64_t k0 = rb + threadIdx.x; k0 < re; k0 += (int64_t)kUnroll * BLOCK) {
            int32_t j[kUnroll], c[kUnroll];
            i64 x[kUnroll], dc[kUnroll];
            load_chunk<BLOCK>(A, k0, re, j, x);
            gather_chunk(A, i, j, c);
#pragma unroll
            for (int u = 0; u < kUnroll; u++) dc[u] = (c[u] >= 0 && c[u] != a) ? dg[c[u]] : 0;
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                if (j[u] == i) loop += x[u];
                else if (c[u] >= 0) first_entry<GT>(c[u], x[u], dc[u], a, dl, tw, gbest, best, e_a, cnt);
            }
        }
        block_argmax_cnt(gbest, best, e_a, loop, cnt);
        if (threadIdx.x == 0) {
            const int32_t target = choose_target<GT>(a, best, gbest, e_a, dl, tw, A.deg, A.size);
            A.Cnext[i] = target;
            if constexpr (!BT) {
                moved += target != a;
                internal += (u64)(e_a + loop);
            } else if (!fz) {
                row_stats(A.st, gr, e_a + loop, target != a);
            }
            cand += first_cand(cnt);
        }
    }
    block_flush_stats(A.st, slot, internal, moved, cand, 0);
}

// Bin 10 in the first sweep: each CTA chunk of a row scores its entries; a single-chunk
// row is decided at once, otherwise the chunk's partial argmax, e_{i->C(i)} and counters go
// to its slot (index = chunk) and the CTA that finishes the row's last chunk combines them.
template <typename WT, typename GT, bool BT>
__global__ void __launch_bounds__(kHugeBlock) k_move_huge_first(MoveArgs<WT> A, BigArgs B)
{
    __shared__ int s_last;
    GT *pg = (GT *)B.pgain;
    u64 internal = 0, moved = 0, cand = 0;
    const DegRead dg = deg_read(A);
    for (int c = blockIdx.x; c < B.nchunks; c += gridDim.x) {
        const int b = B.chunk_b[c];
        const int32_t i = B.bverts[b];
        const int c0 = B.chunk_first[b];
        const int q = c - c0;
        const int nch = B.nch[b];
        const int64_t rb = A.rp[i], re = A.rp[i + 1];
        const int64_t cb = rb + (int64_t)q * B.chunk;
        const int64_t ce = min(re, cb + (int64_t)B.chunk);
        const int32_t a = A.C[i];
        const i64 dl = A.delta[i];
        const int gr = graph_of<BT>(A, i);
        const i64 tw = tw_of<BT>(A, gr);
        if (frozen<BT>(A, gr)) {  // a frozen row stays; its first chunk records that
            if (q == 0 && threadIdx.x == 0) A.Cnext[i] = a;
            continue;
        }
        i64 loop = 0, e_a = 0;
        u64 cnt = 0;
        GT gbest = gain_min<GT>();
        int32_t best = INT_MAX;
        for (int64_t k0 = cb + threadIdx.x; k0 < ce; k0 += (int64_t)kUnroll * kHugeBlock) {
            int32_t j[kUnroll], cc[kUnroll];
            i64 x[kUnroll], dc[kUnroll];
            load_chunk<kHugeBlock>(A, k0, ce, j, x);
            gather_chunk(A, i, j, cc);
#pragma unroll
            for (int u = 0; u < kUnroll; u++)
                dc[u] = (cc[u] >= 0 && cc[u] != a) ? dg[cc[u]] : 0;
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                if (j[u] == i) loop += x[u];
                else if (cc[u] >= 0)
                    first_entry<GT>(cc[u], x[u], dc[u], a, dl, tw, gbest, best, e_a, cnt);
            }
        }
        block_argmax_cnt(gbest, best, e_a, loop, cnt);
        if (nch == 1) {
            if (threadIdx.x == 0) {
                const int32_t target =
                    choose_target<GT>(a, best, gbest, e_a, dl, tw, A.deg, A.size);
                A.Cnext[i] = target;
                if constexpr (!BT) {
                    moved += target != a;
                    internal += (u64)(e_a + loop);
                } else {
                    row_stats(A.st, gr, e_a + loop, target != a);
                }
                cand += first_cand(cnt);
            }
        } else {
            if (threadIdx.x == 0) {
                pg[c] = gbest;
                B.pbest[c] = best;
                B.pea[c] = e_a;
                B.pcnt[c] = cnt;
                if (loop) atomicAdd(&B.gloop[b], (u64)loop);
                __threadfence();
                s_last = atomicAdd(&B.sdone[b], 1) == nch - 1;
            }
            __syncthreads();
            if (s_last) {  // every chunk of row b is in: combine and decide
                __threadfence();
                GT g = gain_min<GT>();
                int32_t cbest = INT_MAX;
                i64 ea = 0, l0 = 0;
                u64 n = 0;
                for (int t = threadIdx.x; t < nch; t += kHugeBlock) {
                    const GT gt = *(volatile const GT *)&pg[c0 + t];  // bypasses L1
                    const int32_t ct = __ldcg(&B.pbest[c0 + t]);
                    if (better(gt, ct, g, cbest)) {
                        g = gt;
                        cbest = ct;
                    }
                    ea += __ldcg(&B.pea[c0 + t]);
                    n += __ldcg(&B.pcnt[c0 + t]);
                }
                block_argmax_cnt(g, cbest, ea, l0, n);
                if (threadIdx.x == 0) {
                    const i64 lp = (i64)__ldcg(&B.gloop[b]);
                    const int32_t target =
                        choose_target<GT>(a, cbest, g, ea, dl, tw, A.deg, A.size);
                    A.Cnext[i] = target;
                    if constexpr (!BT) {
                        moved += target != a;
                        internal += (u64)(ea + lp);
                    } else {
                        row_stats(A.st, gr, ea + lp, target != a);
                    }
                    cand += first_cand(n);
                    B.gloop[b] = 0;
                    B.sdone[b] = 0;
                }
            }
        }
        __syncthreads();  // s_last read before the next chunk sets it
    }
    block_flush_stats(A.st, kChunkedBin, internal, moved, cand, 0);
}

// ------------------------------------------------------------------ launch

// shared table bytes: keys + values, plus a claim list when `with_list`
template <typename VT>
inline size_t table_bytes(int log2cap, bool with_list = false)
{
    return ((size_t)1 << log2cap) * (sizeof(VT) + (with_list ? 8 : 4));
}

// Grid of a persistent CTA-per-row kernel: the CTAs that can be resident at once (threads,
// registers and shared memory all counted), at most one per row.  A larger grid would leave
// CTAs waiting for a slot that only frees when a resident CTA has finished all its rows.
template <typename K>
static int launch_cta_kernel(K kernel, int block, size_t smem, int nrows, cudaStream_t s,
                             const LaunchCfg &lc, const char *name)
{
    (void)s;
    set_dyn_smem(kernel, smem, name);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int maxg = lc.num_sms * per_sm;
    return nrows < maxg ? nrows : maxg;
}

// Launch a cluster kernel with CL CTAs per cluster over nrows rows.  Returns 0 if no
// cluster of that size can be resident (then the caller reports an error).
template <int CL, typename K, typename... Args>
static int launch_cluster_kernel(K kernel, size_t smem, int nrows, cudaStream_t s,
                                 const char *name, Args... args)
{
    set_dyn_smem(kernel, smem, name);
    if (CL > 8) cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(1024, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(CL, 1, 1);
    int maxc = 0;
    if (cudaOccupancyMaxActiveClusters(&maxc, kernel, &cfg) != cudaSuccess || maxc < 1) {
        cudaGetLastError();
        if (!launch_site()) launch_site() = name;
        return 0;
    }
    const int nclusters = nrows < maxc ? nrows : maxc;
    cfg.gridDim = dim3((unsigned)(nclusters * CL), 1, 1);
    cudaLaunchKernelEx(&cfg, kernel, args...);
    note_launch(name);
    return 1;
}

// Bins 1-9 with shared / distributed shared tables.  Returns the kernels launched.
template <typename WT, typename GT, typename VT, bool BT>
static int launch_bin_table(const MoveArgs<WT> &A, const Bins &b, const BinSpec &sp,
                            const int32_t *rows, int nr, int bin, cudaStream_t bs,
                            const LaunchCfg &lc)
{
    if (sp.kind == BIN_GROUP8) {
        k_move_group<8, 6, WT, GT, VT, BT>
            <<<grid_for(nr, kBlock / 8, lc.max_blocks), kBlock, 0, bs>>>(A, rows, nr, bin);
        note_launch("k_move_group<8>");
        return 1;
    }
    if (sp.kind == BIN_WARP) {
        k_move_group<32, 8, WT, GT, VT, BT>
            <<<grid_for(nr, kBlock / 32, lc.max_blocks), kBlock, 0, bs>>>(A, rows, nr, bin);
        note_launch("k_move_group<32>");
        return 1;
    }
    const int l2 = cta_log2cap(b, bin);
    if (sp.kind == BIN_CTA) {
        const size_t smem = table_bytes<VT>(l2, true);
        if (sp.block == 128) {
            const int grid = launch_cta_kernel(k_move_cta<128, WT, GT, VT, BT>, 128, smem, nr, bs,
                                               lc, "k_move_cta<128>");
            k_move_cta<128, WT, GT, VT, BT><<<grid, 128, smem, bs>>>(A, rows, nr, l2, bin);
        } else if (sp.block == 256) {
            const int grid = launch_cta_kernel(k_move_cta<256, WT, GT, VT, BT>, 256, smem, nr, bs,
                                               lc, "k_move_cta<256>");
            k_move_cta<256, WT, GT, VT, BT><<<grid, 256, smem, bs>>>(A, rows, nr, l2, bin);
        } else if (l2 <= kHalfCtaLog2 && sizeof(VT) == 4) {
            // rows of at most 6,144 entries: 512 threads and an 8K-slot table, so that two
            // rows are in flight on an SM where the 16K-slot table leaves room for one
            const int grid = launch_cta_kernel(k_move_cta<512, WT, GT, VT, BT>, 512, smem, nr,
                                               bs, lc, "k_move_cta<512>");
            k_move_cta<512, WT, GT, VT, BT><<<grid, 512, smem, bs>>>(A, rows, nr, l2, bin);
        } else {
            const int grid = launch_cta_kernel(k_move_cta<1024, WT, GT, VT, BT>, 1024, smem, nr,
                                               bs, lc, "k_move_cta<1024>");
            k_move_cta<1024, WT, GT, VT, BT><<<grid, 1024, smem, bs>>>(A, rows, nr, l2, bin);
        }
        note_launch("k_move_cta");
        return 1;
    }
    const size_t smem = table_bytes<VT>(l2);
    switch (sp.cluster) {
    case 2:
        return launch_cluster_kernel<2>(k_move_cluster<2, WT, GT, VT, BT>, smem, nr, bs,
                                        "k_move_cluster<2>", A, rows, nr, l2, bin);
    case 4:
        return launch_cluster_kernel<4>(k_move_cluster<4, WT, GT, VT, BT>, smem, nr, bs,
                                        "k_move_cluster<4>", A, rows, nr, l2, bin);
    case 8:
        return launch_cluster_kernel<8>(k_move_cluster<8, WT, GT, VT, BT>, smem, nr, bs,
                                        "k_move_cluster<8>", A, rows, nr, l2, bin);
    default:
        return launch_cluster_kernel<16>(k_move_cluster<16, WT, GT, VT, BT>, smem, nr, bs,
                                         "k_move_cluster<16>", A, rows, nr, l2, bin);
    }
}

// Bins 1-9 of the first sweep of a phase: entries scored without tables.
template <typename WT, typename GT, bool BT>
static int launch_bin_first(const MoveArgs<WT> &A, const BinSpec &sp, const int32_t *rows, int nr,
                            int bin, cudaStream_t bs, const LaunchCfg &lc)
{
    if (sp.kind == BIN_GROUP8) {
        k_move_group_first<8, WT, GT, BT>
            <<<grid_for(nr, kBlock / 8, lc.max_blocks), kBlock, 0, bs>>>(A, rows, nr, bin);
        note_launch("k_move_group_first<8>");
    } else if (sp.kind == BIN_WARP) {
        k_move_group_first<32, WT, GT, BT>
            <<<grid_for(nr, kBlock / 32, lc.max_blocks), kBlock, 0, bs>>>(A, rows, nr, bin);
        note_launch("k_move_group_first<32>");
    } else if (sp.kind == BIN_CTA && sp.block == 128) {
        const int grid = launch_cta_kernel(k_move_cta_first<128, WT, GT, BT>, 128, 0, nr, bs, lc,
                                           "k_move_cta_first<128>");
        k_move_cta_first<128, WT, GT, BT><<<grid, 128, 0, bs>>>(A, rows, nr, bin);
        note_launch("k_move_cta_first");
    } else if (sp.kind == BIN_CTA && sp.block == 256) {
        const int grid = launch_cta_kernel(k_move_cta_first<256, WT, GT, BT>, 256, 0, nr, bs, lc,
                                           "k_move_cta_first<256>");
        k_move_cta_first<256, WT, GT, BT><<<grid, 256, 0, bs>>>(A, rows, nr, bin);
        note_launch("k_move_cta_first");
    } else {  // bin 5 and the cluster bins: one 1024-thread CTA per row
        const int grid = launch_cta_kernel(k_move_cta_first<1024, WT, GT, BT>, 1024, 0, nr, bs, lc,
                                           "k_move_cta_first<1024>");
        k_move_cta_first<1024, WT, GT, BT><<<grid, 1024, 0, bs>>>(A, rows, nr, bin);
        note_launch("k_move_cta_first");
    }
    return 1;
}

// Bin 10 in the first sweep: chunks scored without tables, combined per row.
template <typename WT, typename GT, bool BT>
static int launch_huge_first(const MoveArgs<WT> &A, const Bins &b, cudaStream_t bs,
                             const LaunchCfg &lc)
{
    const BigArgs B = big_args(b);
    const int grid = launch_cta_kernel(k_move_huge_first<WT, GT, BT>, kHugeBlock, 0, b.nchunks,
                                       bs, lc, "k_move_huge_first");
    k_move_huge_first<WT, GT, BT><<<grid, kHugeBlock, 0, bs>>>(A, B);
    note_launch("k_move_huge_first");
    return 1;
}

// Bin 10: chunk tables, then the per-partition merge and decision of rows spanning several
// chunks.
template <typename WT, typename GT, typename VT, bool BT>
static int launch_huge(const MoveArgs<WT> &A, const Bins &b, cudaStream_t bs, const LaunchCfg &lc)
{
    const BigArgs B = big_args(b);
    const int l2 = 31 - __builtin_clz(2 * b.chunk);
    const size_t smem = table_bytes<VT>(l2, true);
    const int grid = launch_cta_kernel(k_move_huge<WT, GT, VT, BT>, kHugeBlock, smem, b.nchunks, bs,
                                       lc, "k_move_huge");
    k_move_huge<WT, GT, VT, BT><<<grid, kHugeBlock, smem, bs>>>(A, B);
    note_launch("k_move_huge");
    int launched = 1;
    if (b.nslices > 0) {  // some rows span several chunks
        const size_t dsmem = table_bytes<VT>(kPartTableLog2, true);
        const int dgrid = launch_cta_kernel(k_move_huge_decide<WT, GT, VT, BT>, kHugeBlock, dsmem,
                                            (int)std::min<int64_t>(b.nslices, INT_MAX), bs, lc,
                                            "k_move_huge_decide");
        k_move_huge_decide<WT, GT, VT, BT><<<dgrid, kHugeBlock, dsmem, bs>>>(A, B);
        note_launch("k_move_huge_decide");
        launched++;
    }
    return launched;
}

// FIRST: the first sweep of a phase on a graph without repeated columns in a row; every bin
// then scores entries directly (k_move_group_first / k_move_cta_first / k_move_huge_first).
template <typename WT, typename GT, typename VT, bool BT, bool FIRST>
static int sweep_impl(const DevGraph &g, const PhaseState &st, const Bins &b, i64 tw,
                      SweepStats *stats, unsigned *err, cudaStream_t s, const LaunchCfg &lc,
                      SweepTimers *tm, const BatchCtx &bc)
{
    MoveArgs<WT> A{g.n,   g.rp,     g.col,  (const WT *)g.w, st.C,  st.deg,  st.size,
                   st.delta, tw,    st.Cnext, stats,         err,   bc.vg,   bc.gtw,
                   bc.gctl};
    A.color = st.color;
    A.cls = st.cls;
    A.deg32 = st.deg32;
    A.deg32_bad = st.deg32_bad;
    const bool timed = tm && tm->on;
    int launched = 0;
    // the bins read the same snapshot and write disjoint rows: with a stream set they run
    // concurrently (fork from s, join back into s), so one bin's last wave overlaps the next
    const SweepStreams *ss = bc.ss;
    if (ss) {
        cudaEventRecord(ss->fork, s);
        for (int q = 0; q < ss->k; q++) cudaStreamWaitEvent(ss->aux[q], ss->fork, 0);
    }
    for (int bin = 0; bin < kNumBins; bin++) {
        const cudaStream_t bs = ss ? ss->aux[bin % ss->k] : s;
        if (timed) cudaEventRecord(tm->ev[2 * bin], bs);
        const BinSpec sp = kBinSpec[bin];
        const int nr = b.nlist[bin];
        const int32_t *rows = b.rows(bin);
        if (sp.kind == BIN_THREAD) {
            if (g.n > 0) {  // dense over every vertex: also sums deg_c^2 over all labels
                k_move_small<WT, GT, BT, FIRST>
                    <<<grid_for(g.n, kBlock, lc.max_blocks), kBlock, 0, bs>>>(A, (int)b.upper[0]);
                note_launch("k_move_small");
                launched++;
            }
        } else if (sp.kind == BIN_CHUNKED) {
            if (b.nchunks > 0) {
                if constexpr (FIRST) launched += launch_huge_first<WT, GT, BT>(A, b, bs, lc);
                else launched += launch_huge<WT, GT, VT, BT>(A, b, bs, lc);
            }
        } else if (nr > 0) {
            if constexpr (FIRST) launched += launch_bin_first<WT, GT, BT>(A, sp, rows, nr, bin, bs, lc);
            else launched += launch_bin_table<WT, GT, VT, BT>(A, b, sp, rows, nr, bin, bs, lc);
        }
        if (timed) cudaEventRecord(tm->ev[2 * bin + 1], bs);
    }
    if (ss) {
        for (int q = 0; q < ss->k; q++) {
            cudaEventRecord(ss->join[q], ss->aux[q]);
            cudaStreamWaitEvent(s, ss->join[q], 0);
        }
    }
    return launched;
}

template <bool BT, bool FIRST>
int sweep_typed(const DevGraph &g, const PhaseState &st, const Bins &b, i64 tw, bool wide,
                 bool narrow, SweepStats *stats, unsigned *err, cudaStream_t s,
                 const LaunchCfg &lc, SweepTimers *tm, const BatchCtx &bc)
{
    typedef unsigned int u32;
    if (g.wbytes == 4) {
        if (wide)
            return narrow ? sweep_impl<int32_t, i128, u32, BT, FIRST>(g, st, b, tw, stats, err, s, lc, tm, bc)
                          : sweep_impl<int32_t, i128, u64, BT, FIRST>(g, st, b, tw, stats, err, s, lc, tm, bc);
        return narrow ? sweep_impl<int32_t, i64, u32, BT, FIRST>(g, st, b, tw, stats, err, s, lc, tm, bc)
                      : sweep_impl<int32_t, i64, u64, BT, FIRST>(g, st, b, tw, stats, err, s, lc, tm, bc);
    }
    if (wide)
        return narrow ? sweep_impl<i64, i128, u32, BT, FIRST>(g, st, b, tw, stats, err, s, lc, tm, bc)
                      : sweep_impl<i64, i128, u64, BT, FIRST>(g, st, b, tw, stats, err, s, lc, tm, bc);
    return narrow ? sweep_impl<i64, i64, u32, BT, FIRST>(g, st, b, tw, stats, err, s, lc, tm, bc)
                  : sweep_impl<i64, i64, u64, BT, FIRST>(g, st, b, tw, stats, err, s, lc, tm, bc);
}

}  // namespace lv
