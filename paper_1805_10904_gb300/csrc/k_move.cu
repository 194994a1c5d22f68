// k_move.cu -- one synchronous local-moving sweep (arXiv 1805.10904, Algorithm 1 body).
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
//   short rows   -> one thread per vertex, neighbours aggregated in registers,
//   medium rows  -> 8-lane groups or whole warps with a shared-memory hash table each,
//   long rows    -> CTA-sized chunks with a shared-memory hash table; a row spanning
//                   several chunks merges its chunks into a global-memory hash table and
//                   the last chunk to finish takes the decision.
#include <climits>

#include "lv_common.cuh"
#include "lv_kernels.h"

namespace lv {

constexpr int kSmallMax = 8;  // register slots of the thread-per-vertex kernel

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
    i64 tw;
    int32_t *Cnext;
    SweepStats *st;
    unsigned *err;
};

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

// ------------------------------------------------------------------ short rows
// Dense over every vertex: also adds deg[i]^2 of label i to sum_c deg_c^2.
template <typename WT, typename GT>
__global__ void __launch_bounds__(kBlock) k_move_small(MoveArgs<WT> A, int small_max)
{
    u64 internal = 0, moved = 0, cand = 0;
    u128 sq = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const i64 dg = A.deg[i];
        sq += (u128)(u64)dg * (u64)dg;
        const int64_t rb = A.rp[i];
        const int64_t d = A.rp[i + 1] - rb;
        if (d > small_max) continue;
        const int32_t a = A.C[i];
        int32_t lab[kSmallMax];
        i64 wt[kSmallMax];
#pragma unroll
        for (int t = 0; t < kSmallMax; t++) {
            lab[t] = -1;
            wt[t] = 0;
            if (t < d) {
                lab[t] = A.col[rb + t];
                wt[t] = (i64)A.w[rb + t];
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
                if (c == a) {
                    e_a = e;
                } else {
                    const GT g = (GT)A.tw * (GT)e - (GT)dl * (GT)A.deg[c];
                    if (better(g, c, gbest, best)) {
                        gbest = g;
                        best = c;
                    }
                }
            }
        }
        const int32_t target = choose_target<GT>(a, best, gbest, e_a, dl, A.tw, A.deg, A.size);
        A.Cnext[i] = target;
        moved += target != a;
        internal += (u64)(e_a + loop);
        cand += (u64)m;
    }
    block_flush_stats(A.st, 0, internal, moved, cand, sq);
}

// ------------------------------------------------------------------ medium rows
// G lanes per vertex (G <= 32), each group with a 2^LOG2CAP-slot shared table.  The
// outer loop is uniform across the block so every lane reaches the shuffles.
template <int G, int LOG2CAP, typename WT, typename GT>
__global__ void __launch_bounds__(kBlock) k_move_group(MoveArgs<WT> A, const int32_t *verts,
                                                       int nverts, int slot)
{
    constexpr int CAP = 1 << LOG2CAP;
    constexpr int NG = kBlock / G;
    __shared__ int s_keys[NG * CAP];
    __shared__ u64 s_vals[NG * CAP];
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
    u64 *vals = s_vals + g * CAP;
    int *list = s_list + g * CAP;
    int *cnt = &s_cnt[g];
    u64 internal = 0, moved = 0, cand = 0;
    for (int base = blockIdx.x * NG; base < nverts; base += gridDim.x * NG) {
        const int vi = base + g;
        const bool valid = vi < nverts;
        int32_t i = 0, a = 0;
        int64_t rb = 0, re = 0;
        i64 dl = 0;
        if (valid) {
            i = verts[vi];
            rb = A.rp[i];
            re = A.rp[i + 1];
            a = A.C[i];
            dl = A.delta[i];
        }
        i64 loop = 0;
        for (int64_t k = rb + lane; k < re; k += G) {
            const int32_t j = A.col[k];
            const i64 x = (i64)A.w[k];
            if (j == i) loop += x;
            else sh_insert<LOG2CAP>(keys, vals, list, cnt, A.C[j], (u64)x, A.err);
        }
        __syncwarp();
        const int m = valid ? *(volatile int *)cnt : 0;
        GT gbest = gain_min<GT>();
        int32_t best = INT_MAX;
        i64 e_a = 0;
        for (int p = lane; p < m; p += G) {
            const int s = list[p];
            const int32_t c = keys[s];
            const i64 e = (i64)vals[s];
            keys[s] = -1;
            vals[s] = 0;
            if (c == a) {
                e_a = e;
            } else {
                const GT gc = (GT)A.tw * (GT)e - (GT)dl * (GT)A.deg[c];
                if (better(gc, c, gbest, best)) {
                    gbest = gc;
                    best = c;
                }
            }
        }
        argmax_reduce(gbest, best, G);
        e_a = sum_reduce(e_a, G);
        loop = sum_reduce(loop, G);
        if (lane == 0) {
            if (valid) {
                const int32_t target =
                    choose_target<GT>(a, best, gbest, e_a, dl, A.tw, A.deg, A.size);
                A.Cnext[i] = target;
                moved += target != a;
                internal += (u64)(e_a + loop);
                cand += (u64)m;
            }
            *cnt = 0;
        }
        __syncwarp();
    }
    block_flush_stats(A.st, slot, internal, moved, cand, 0);
}

// ------------------------------------------------------------------ long rows
struct BigArgs {
    const int32_t *bverts;
    const int32_t *chunk_b;
    const int32_t *chunk_first;
    const int32_t *nch;
    const int64_t *goff;
    const int32_t *glog2;
    int32_t *gcnt;
    int32_t *gdone;
    u64 *gloop;
    int32_t *gkeys;
    u64 *gvals;
    int32_t *glist;
    int chunk;
    int nchunks;
};

// Shared table with a run-time power-of-two size.
__device__ __forceinline__ void shr_insert(int *keys, u64 *vals, int *list, int *cnt, int log2cap,
                                           int key, u64 val, unsigned *err)
{
    const unsigned cap = 1u << log2cap;
    unsigned h = hash_slot(key, log2cap);
#pragma unroll 1
    for (unsigned probe = 0; probe < cap; probe++) {
        int k = ((volatile int *)keys)[h];
        if (k == key) {
            atomicAdd(&vals[h], val);
            return;
        }
        if (k == -1) {
            int old = atomicCAS(&keys[h], -1, key);
            if (old == -1) {
                int p = atomicAdd(cnt, 1);
                list[p] = (int)h;
                atomicAdd(&vals[h], val);
                return;
            }
            if (old == key) {
                atomicAdd(&vals[h], val);
                return;
            }
        }
        h = (h + 1) & (cap - 1);
    }
    atomicOr(err, ERRF_HASH_FULL);
}

// CTA argmax / sums; results valid in thread 0.
template <typename GT>
__device__ __forceinline__ void block_argmax(GT &g, int32_t &c, i64 &e_a, i64 &loop)
{
    __shared__ GT s_g[kBlock / 32];
    __shared__ int32_t s_c[kBlock / 32];
    __shared__ i64 s_e[kBlock / 32], s_l[kBlock / 32];
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
    if (threadIdx.x == 0) {
        for (int w = 1; w < kBlock / 32; w++) {
            if (better(s_g[w], s_c[w], g, c)) {
                g = s_g[w];
                c = s_c[w];
            }
            e_a += s_e[w];
            loop += s_l[w];
        }
    }
    __syncthreads();
}

template <typename WT, typename GT>
__global__ void __launch_bounds__(kBlock) k_move_big(MoveArgs<WT> A, BigArgs B)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int log2cap = 31 - __clz(2 * B.chunk);  // 2 * chunk slots
    const int cap = 1 << log2cap;
    u64 *vals = (u64 *)smem;
    int *keys = (int *)(vals + cap);
    int *list = keys + cap;
    __shared__ int s_cnt;
    __shared__ int s_last;
    for (int s = threadIdx.x; s < cap; s += kBlock) {
        keys[s] = -1;
        vals[s] = 0;
    }
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    u64 internal = 0, moved = 0, cand = 0;
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
        i64 loop = 0;
        for (int64_t k = cb + threadIdx.x; k < ce; k += kBlock) {
            const int32_t j = A.col[k];
            const i64 x = (i64)A.w[k];
            if (j == i) loop += x;
            else shr_insert(keys, vals, list, &s_cnt, log2cap, A.C[j], (u64)x, A.err);
        }
        __syncthreads();
        const int m = s_cnt;
        if (nch == 1) {
            GT gbest = gain_min<GT>();
            int32_t best = INT_MAX;
            i64 e_a = 0;
            for (int p = threadIdx.x; p < m; p += kBlock) {
                const int s = list[p];
                const int32_t cc = keys[s];
                const i64 e = (i64)vals[s];
                keys[s] = -1;
                vals[s] = 0;
                if (cc == a) {
                    e_a = e;
                } else {
                    const GT g = (GT)A.tw * (GT)e - (GT)dl * (GT)A.deg[cc];
                    if (better(g, cc, gbest, best)) {
                        gbest = g;
                        best = cc;
                    }
                }
            }
            block_argmax(gbest, best, e_a, loop);
            if (threadIdx.x == 0) {
                const int32_t target =
                    choose_target<GT>(a, best, gbest, e_a, dl, A.tw, A.deg, A.size);
                A.Cnext[i] = target;
                moved += target != a;
                internal += (u64)(e_a + loop);
                cand += (u64)m;
            }
        } else {
            const int64_t off = B.goff[b];
            const int l2 = B.glog2[b];
            int32_t *gk = B.gkeys + off;
            u64 *gv = B.gvals + off;
            int32_t *gl = B.glist + off;
            for (int p = threadIdx.x; p < m; p += kBlock) {
                const int s = list[p];
                const int32_t cc = keys[s];
                const u64 e = vals[s];
                keys[s] = -1;
                vals[s] = 0;
                g_insert(gk, gv, gl, &B.gcnt[b], l2, cc, e, A.err);
            }
            loop = sum_reduce(loop, 32);
            if ((threadIdx.x & 31) == 0 && loop) atomicAdd(&B.gloop[b], (u64)loop);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                const int t = atomicAdd(&B.gdone[b], 1);
                s_last = (t == nch - 1);
            }
            __syncthreads();
            if (s_last) {
                __threadfence();
                const int gm = __ldcg(&B.gcnt[b]);
                GT gbest = gain_min<GT>();
                int32_t best = INT_MAX;
                i64 e_a = 0, lz = 0;
                for (int p = threadIdx.x; p < gm; p += kBlock) {
                    const int s = __ldcg(gl + p);
                    const int32_t cc = __ldcg(gk + s);
                    const i64 e = (i64)__ldcg(gv + s);
                    gk[s] = -1;
                    gv[s] = 0;
                    if (cc == a) {
                        e_a = e;
                    } else {
                        const GT g = (GT)A.tw * (GT)e - (GT)dl * (GT)A.deg[cc];
                        if (better(g, cc, gbest, best)) {
                            gbest = g;
                            best = cc;
                        }
                    }
                }
                block_argmax(gbest, best, e_a, lz);
                if (threadIdx.x == 0) {
                    const i64 lp = (i64)__ldcg(&B.gloop[b]);
                    const int32_t target =
                        choose_target<GT>(a, best, gbest, e_a, dl, A.tw, A.deg, A.size);
                    A.Cnext[i] = target;
                    moved += target != a;
                    internal += (u64)(e_a + lp);
                    cand += (u64)gm;
                    B.gcnt[b] = 0;
                    B.gdone[b] = 0;
                    B.gloop[b] = 0;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
    }
    block_flush_stats(A.st, 3, internal, moved, cand, 0);
}

// ------------------------------------------------------------------ launch

inline size_t big_smem_bytes(int chunk) { return (size_t)(2 * chunk) * 16; }

template <typename WT, typename GT>
static int sweep_impl(const DevGraph &g, const PhaseState &st, const Bins &b, i64 tw,
                      SweepStats *stats, unsigned *err, cudaStream_t s, const LaunchCfg &lc,
                      SweepTimers *tm)
{
    MoveArgs<WT> A{g.n, g.rp, g.col, (const WT *)g.w, st.C, st.deg, st.size, st.delta,
                   tw, st.Cnext, stats, err};
    const bool timed = tm && tm->on;
    int launched = 0;
    if (timed) cudaEventRecord(tm->ev[0], s);
    if (g.n > 0) {
        k_move_small<WT, GT><<<grid_for(g.n, kBlock, lc.max_blocks), kBlock, 0, s>>>(
            A, b.small_max);
        launched++;
    }
    if (timed) cudaEventRecord(tm->ev[1], s);
    if (timed) cudaEventRecord(tm->ev[2], s);
    if (b.nlist[0] > 0) {
        k_move_group<8, 6, WT, GT><<<grid_for(b.nlist[0], kBlock / 8, lc.max_blocks), kBlock, 0,
                                     s>>>(A, b.list[0], b.nlist[0], 1);
        launched++;
    }
    if (timed) cudaEventRecord(tm->ev[3], s);
    if (timed) cudaEventRecord(tm->ev[4], s);
    if (b.nlist[1] > 0) {
        k_move_group<32, 8, WT, GT><<<grid_for(b.nlist[1], kBlock / 32, lc.max_blocks), kBlock,
                                      0, s>>>(A, b.list[1], b.nlist[1], 2);
        launched++;
    }
    if (timed) cudaEventRecord(tm->ev[5], s);
    if (timed) cudaEventRecord(tm->ev[6], s);
    if (b.nchunks > 0) {
        BigArgs B{b.list[2], b.chunk_b, b.chunk_first, b.nch,   b.goff,  b.glog2, b.gcnt,
                  b.gdone,   b.gloop,   b.gkeys,       b.gvals, b.glist, b.chunk, b.nchunks};
        const size_t smem = big_smem_bytes(b.chunk);
        const int grid = b.nchunks < lc.max_blocks ? b.nchunks : lc.max_blocks;
        k_move_big<WT, GT><<<grid, kBlock, smem, s>>>(A, B);
        launched++;
    }
    if (timed) cudaEventRecord(tm->ev[7], s);
    return launched;
}

template <typename WT, typename GT>
static void set_big_smem(int chunk)
{
    cudaFuncSetAttribute(k_move_big<WT, GT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)big_smem_bytes(chunk));
}

int launch_sweep(const DevGraph &g, const PhaseState &st, const Bins &b, i64 tw, bool wide,
                 SweepStats *stats, unsigned *err, cudaStream_t s, const LaunchCfg &lc,
                 SweepTimers *tm)
{
    if (b.nchunks > 0 && big_smem_bytes(b.chunk) > 48 * 1024) {
        if (g.wbytes == 4) {
            if (wide) set_big_smem<int32_t, i128>(b.chunk);
            else set_big_smem<int32_t, i64>(b.chunk);
        } else {
            if (wide) set_big_smem<i64, i128>(b.chunk);
            else set_big_smem<i64, i64>(b.chunk);
        }
    }
    if (g.wbytes == 4)
        return wide ? sweep_impl<int32_t, i128>(g, st, b, tw, stats, err, s, lc, tm)
                    : sweep_impl<int32_t, i64>(g, st, b, tw, stats, err, s, lc, tm);
    return wide ? sweep_impl<i64, i128>(g, st, b, tw, stats, err, s, lc, tm)
                : sweep_impl<i64, i64>(g, st, b, tw, stats, err, s, lc, tm);
}

}  // namespace lv
