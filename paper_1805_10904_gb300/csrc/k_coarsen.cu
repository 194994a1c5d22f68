// k_coarsen.cu -- graph induction between levels (arXiv 1805.10904, Sec. 3 and Sec. 5.1.2
// "Inducing new graph").
//
// With a = new_id[C(u)] the renumbered community of u, the next level's graph is
//     A'_ab = sum over stored entries (u, v) with new_id[C(u)] = a, new_id[C(v)] = b of A_uv,
// so an internal edge adds to the loop of its community from both of its stored
// directions, old loops once, and delta and 2W are preserved.  The paper sorts
// (source, target) keys and reduces by key; here every community's entries are
// aggregated directly in a hash table keyed by the target community:
//   1. community sizes and next-level delta (= deg of the old community),
//   2. member lists by counting sort, flattened entry offsets of each community,
//   3. per community: a warp or a CTA with a shared-memory table, or (communities above
//      the largest CTA table, which take no thread-block clusters here) CTA chunks each
//      aggregated in shared memory whose
//      distinct (target, sum) pairs are then grouped by a hash partition of the target and
//      merged partition by partition in shared memory,
//   4. row offsets by prefix sum, then compaction into the next CSR.
// Rows of the induced graph are not sorted; nothing downstream depends on their order.
#include <climits>

#include "lv_common.cuh"
#include "lv_kernels.h"
#include "lv_scan.cuh"

namespace lv {

// A community c of a kept graph (keep[vg[c]], or every community for one graph) becomes
// vertex a = new_id[c] of the next level.
__device__ __forceinline__ bool kept(const int32_t *vg, const int32_t *keep, int64_t v)
{
    return !vg || keep[vg[v]];
}

__global__ void k_coarsen_prep(int64_t n, const int32_t *size, const i64 *deg,
                               const int32_t *new_id, const int32_t *vg, const int32_t *keep,
                               int32_t *csize, i64 *delta_next, int32_t *vg_next)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (size[c] > 0 && kept(vg, keep, c)) {
            const int32_t a = new_id[c];
            csize[a] = size[c];
            delta_next[a] = deg[c];
            if (vg_next) vg_next[a] = vg[c];
        }
    }
}

// members[p] = u and, for the aggregation, the first entry of u's row mrow[p] = rp[u]
__global__ void k_coarsen_scatter(int64_t n, const int32_t *C, const int32_t *new_id,
                                  const int32_t *vg, const int32_t *keep, const int32_t *moff,
                                  const int64_t *rp, int32_t *cursor, int32_t *members,
                                  int64_t *mrow)
{
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (!kept(vg, keep, u)) continue;
        const int32_t a = new_id[C[u]];
        const int32_t p = moff[a] + atomicAdd(&cursor[a], 1);
        members[p] = (int32_t)u;
        mrow[p] = rp[u];
    }
}

struct MemberDegIn {
    const int32_t *members;
    const int64_t *rp;
    __device__ __forceinline__ int64_t operator()(int64_t p) const
    {
        const int32_t u = members[p];
        return rp[u + 1] - rp[u];
    }
};

// community entry count E_a = mpre[moff[a+1]] - mpre[moff[a]]
__device__ __forceinline__ int64_t comm_entries(const int32_t *moff, const int64_t *mpre, int32_t a)
{
    return mpre[moff[a + 1]] - mpre[moff[a]];
}

// Communities binned by entry count with the sweep's thresholds (communities of bin 0 join
// the 8-lane groups of bin 1).  Count pass: counts[b]; fill pass: list regions.
struct CBinArgs {
    int64_t upper[kNumBins - 1];
    int64_t off[kNumBins + 1];
    int32_t *list;
};

template <bool FILL>
__global__ void __launch_bounds__(kBlock) k_coarsen_bin(int64_t k, const int32_t *moff,
                                                        const int64_t *mpre, CBinArgs ba,
                                                        int32_t *counts)
{
    const int lane = threadIdx.x & 31;
    __shared__ int s_cnt[kNumBins], s_base[kNumBins];
    int cnt[kNumBins] = {};
    for (int64_t a0 = (int64_t)blockIdx.x * blockDim.x; a0 < k; a0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = a0 + threadIdx.x;
        int bin = -1;
        if (a < k) {
            const int64_t e = comm_entries(moff, mpre, (int32_t)a);
            int b = 0;
#pragma unroll
            for (int t = 0; t < kNumBins - 1; t++) b += e > ba.upper[t];
            bin = b < 1 ? 1 : b;  // bin-0 communities join the 8-lane groups of bin 1
        }
        if (!FILL) {  // count pass: per thread, added once per CTA and bin at the end
#pragma unroll
            for (int b = 1; b < kNumBins; b++) cnt[b] += bin == b;
            continue;
        }
        // fill pass: positions claimed once per CTA and bin, warps ranked in shared memory
        if (threadIdx.x < kNumBins) s_cnt[threadIdx.x] = 0;
        __syncthreads();
        int rank = 0;
#pragma unroll
        for (int b = 1; b < kNumBins; b++) {
            const unsigned mask = __ballot_sync(0xffffffffu, bin == b);
            if (!mask) continue;
            const int leader = __ffs(mask) - 1;
            int wbase = 0;
            if (lane == leader) wbase = atomicAdd(&s_cnt[b], __popc(mask));
            wbase = __shfl_sync(0xffffffffu, wbase, leader);
            if (bin == b) rank = wbase + __popc(mask & ((1u << lane) - 1u));
        }
        __syncthreads();
        if (threadIdx.x < kNumBins)
            s_base[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(&counts[threadIdx.x], s_cnt[threadIdx.x]) : 0;
        __syncthreads();
        if (bin >= 1) ba.list[ba.off[bin] + s_base[bin] + rank] = (int32_t)a;
        __syncthreads();  // s_cnt / s_base read before the next round resets them
    }
    if (!FILL) {
        if (threadIdx.x < kNumBins) s_cnt[threadIdx.x] = 0;
        __syncthreads();
#pragma unroll
        for (int b = 1; b < kNumBins; b++) {
            const int c = sum_reduce(cnt[b], 32);
            if (lane == 0 && c) atomicAdd(&s_cnt[b], c);
        }
        __syncthreads();
        if (threadIdx.x < kNumBins && s_cnt[threadIdx.x])
            atomicAdd(&counts[threadIdx.x], s_cnt[threadIdx.x]);
    }
}

// A multi-chunk community's pairs are split over 2^l hash partitions of the target, 2^l the
// smallest power of two leaving at most kCPartPairs of its entries per partition on average
// (its pairs never outnumber its entries), at most 2^kCMaxPartLog2.
constexpr int64_t kCPartPairs = 4096;
constexpr int kCMaxPartLog2 = 20;

__global__ void k_cbig_prep(int nb, const int32_t *blist, const int32_t *moff, const int64_t *mpre,
                            int64_t k, int chunk, int32_t *nch, int64_t *gcap, int32_t *glog2)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const int64_t e = comm_entries(moff, mpre, blist[b]);
        const int64_t c = (e + chunk - 1) / chunk;
        nch[b] = (int32_t)c;
        int l = 0;
        if (c > 1)
            while (l < kCMaxPartLog2 && (kCPartPairs << l) < e) l++;
        gcap[b] = c > 1 ? (int64_t)1 << l : 0;
        glog2[b] = l;
    }
}

// Community of every partition: warp b fills partitions goff[b] .. goff[b + 1].
__global__ void k_cpart_fill(int nb, const int64_t *goff, int32_t *partb)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = warp; b < nb; b += nwarps)
        for (int64_t q = goff[b] + lane; q < goff[b + 1]; q += 32) partb[q] = (int32_t)b;
}

template <typename WT>
struct CoarsenArgs {
    const int64_t *rp;
    const int32_t *col;
    const WT *w;
    const int32_t *C;       // renumbered label of every vertex, new_id[C(v)]
    const int32_t *new_id;
    const int32_t *moff;
    const int64_t *mrow;  // first entry of every member's row
    const int64_t *mpre;
    int32_t *ccnt;
    int32_t *tmp_col;
    void *tmp_w;  // VT per entry (the aggregation's sum width)
    unsigned *err;
};

// largest p in [lo, hi) with mpre[p] <= t (mpre non-decreasing, mpre[lo] <= t)
__device__ __forceinline__ int32_t find_member(const int64_t *mpre, int32_t lo, int32_t hi, int64_t t)
{
    while (hi - lo > 1) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (mpre[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Entry t of community a's flattened member rows: returns (target community, weight); p is
// the member index of the previous call (advanced monotonically).
template <typename WT>
__device__ __forceinline__ void flat_entry(const CoarsenArgs<WT> &A, int32_t &p, int32_t pe,
                                           int64_t t, int32_t &key, i64 &wv)
{
    if (A.mpre[p + 1] <= t) {
        // the member holding t lies a few members on: gallop (p + 2, p + 4, p + 8, ...) to a
        // member past it, then bisect that span, instead of bisecting all members up to pe
        int32_t lo = p + 1, hi = pe;
#pragma unroll 1
        for (int32_t step = 1; lo + step < pe; step <<= 1) {
            if (A.mpre[lo + step] > t) {
                hi = lo + step;
                break;
            }
            lo += step;
        }
        p = find_member(A.mpre, lo, hi, t);
    }
    const int64_t kk = A.mrow[p] + (t - A.mpre[p]);
    key = A.C[ld_stream(A.col + kk)];  // A.C holds the renumbered labels new_id[C[v]]
    wv = (i64)ld_stream(A.w + kk);
}

// G lanes per community with few entries (8 for at most 32 entries, a warp for at most
// 128): a 2^LOG2CAP-slot shared table per group.
template <int G, int LOG2CAP, typename WT, typename VT>
__global__ void __launch_bounds__(kBlock) k_coarsen_group(CoarsenArgs<WT> A, const int32_t *clist,
                                                          int ncl)
{
    constexpr int CAP = 1 << LOG2CAP, NG = kBlock / G;
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
    // the next community's list entry, member range and entry range are loaded stage by stage
    // while the current one is merged, so no load of that chain waits at the loop's top
    const int step = gridDim.x * NG;
    int base = blockIdx.x * NG;
    int32_t na = 0, npb = 0, npe = 0;
    int64_t ntb = 0, nte = 0;
    if (base + g < ncl) {
        na = clist[base + g];
        npb = A.moff[na];
        npe = A.moff[na + 1];
        ntb = A.mpre[npb];
        nte = A.mpre[npe];
    }
    for (; base < ncl; base += step) {
        const bool valid = base + g < ncl;
        const int32_t a = na, pb = npb, pe = npe;
        const int64_t tb = ntb, te = nte;
        const bool next = base + step + g < ncl;
        if (next) na = clist[base + step + g];
        int32_t p = pb;
        for (int64_t t = tb + lane; t < te; t += G) {
            int32_t key;
            i64 wv;
            flat_entry(A, p, pe, t, key, wv);
            tbl_insert<false, VT>(keys, vals, list, cnt, LOG2CAP, key, (VT)wv, A.err);
        }
        if (next) {
            npb = A.moff[na];
            npe = A.moff[na + 1];
        }
        __syncwarp();
        const int m = valid ? *(volatile int *)cnt : 0;
        if (next) {
            ntb = A.mpre[npb];
            nte = A.mpre[npe];
        } else {  // this group has no community in the next round: an empty range
            npb = npe = 0;
            ntb = nte = 0;
        }
        for (int q = lane; q < m; q += G) {
            const int s = list[q];
            st_stream(A.tmp_col + tb + q, keys[s]);
            st_stream((VT *)A.tmp_w + tb + q, vals[s]);
            keys[s] = -1;
            vals[s] = 0;
        }
        __syncwarp();  // every lane has read the count before it is reset
        if (lane == 0) {
            if (valid) A.ccnt[a] = m;
            *cnt = 0;
        }
        __syncwarp();
    }
}

// One CTA per community with a 2^log2cap-slot table in dynamic shared memory.
template <int BLOCK, typename WT, typename VT>
__global__ void __launch_bounds__(BLOCK) k_coarsen_cta(CoarsenArgs<WT> A, const int32_t *clist,
                                                       int ncl, int log2cap)
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
    // the next community's list entry, member range and entry range are loaded stage by stage
    // while the current one is merged, so no load of that chain waits at the loop's top
    int v = blockIdx.x;
    int32_t na = 0, npb = 0, npe = 0;
    int64_t ntb = 0, nte = 0;
    if (v < ncl) {
        na = clist[v];
        npb = A.moff[na];
        npe = A.moff[na + 1];
        ntb = A.mpre[npb];
        nte = A.mpre[npe];
    }
    for (; v < ncl; v += gridDim.x) {
        const int32_t a = na, pb = npb, pe = npe;
        const int64_t tb = ntb, te = nte;
        const bool next = v + (int)gridDim.x < ncl;
        if (next) na = clist[v + gridDim.x];
        int32_t p = pb;
        for (int64_t t = tb + threadIdx.x; t < te; t += BLOCK) {
            int32_t key;
            i64 wv;
            flat_entry(A, p, pe, t, key, wv);
            tbl_insert<false, VT>(keys, vals, list, &s_cnt, log2cap, key, (VT)wv, A.err);
        }
        if (next) {
            npb = A.moff[na];
            npe = A.moff[na + 1];
        }
        __syncthreads();
        const int m = s_cnt;
        if (next) {
            ntb = A.mpre[npb];
            nte = A.mpre[npe];
        }
        for (int q = threadIdx.x; q < m; q += BLOCK) {
            const int s = list[q];
            st_stream(A.tmp_col + tb + q, keys[s]);
            st_stream((VT *)A.tmp_w + tb + q, vals[s]);
            keys[s] = -1;
            vals[s] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            A.ccnt[a] = m;
            s_cnt = 0;
        }
        __syncthreads();
    }
}

struct CBigArgs {
    const int32_t *blist;
    const int32_t *chunk_b;
    const int32_t *chunk_first;
    const int32_t *nch;
    const int64_t *pbase;   // first partition of every community (goff)
    const int32_t *plog2;   // log2 of its partition count
    int32_t *pcnt;          // pairs per partition
    const int64_t *poff;    // exclusive scan of pcnt
    int32_t *pcur;          // scatter cursor per partition
    const int32_t *partb;   // community of every partition
    int64_t nparts;
    int32_t *chm;           // distinct pairs of every chunk
    int32_t *pk;            // pairs grouped by partition
    void *pv;
    int chunk;
    int nchunks;
    const int32_t *mem0;    // member holding the first entry of every chunk
};

constexpr int kCHugeBlock = 512;

// The member holding the first entry of every chunk, found for all chunks at once (one
// thread per chunk) instead of by a search over the community's members at the start of
// each chunk's CTA.
__global__ void __launch_bounds__(kBlock) k_chunk_member0(int nchunks, const int32_t *chunk_b,
                                                          const int32_t *chunk_first,
                                                          const int32_t *blist, const int32_t *moff,
                                                          const int64_t *mpre, int chunk,
                                                          int32_t *mem0)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += gridDim.x * blockDim.x) {
        const int b = chunk_b[c];
        const int32_t a = blist[b];
        const int32_t pb = moff[a], pe = moff[a + 1];
        const int64_t tb = mpre[pb];
        const int64_t cb = tb + (int64_t)(c - chunk_first[b]) * chunk;
        mem0[c] = cb > tb ? find_member(mpre, pb, pe, cb) : pb;
    }
}

// Communities with the most entries, phase A: CTA chunks of `chunk` flattened entries, each
// aggregated in a shared table.  A one-chunk community writes its row directly.  A chunk of
// a multi-chunk community leaves its distinct (target, sum) pairs in its own slice of the
// community's temporary row and counts them per hash partition of the target.
template <typename WT, typename VT>
__global__ void __launch_bounds__(kCHugeBlock) k_coarsen_huge(CoarsenArgs<WT> A, CBigArgs B)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int log2cap = 31 - __clz(2 * B.chunk);
    const int cap = 1 << log2cap;
    VT *vals = (VT *)smem;
    int *keys = (int *)(vals + cap);
    int *list = keys + cap;
    __shared__ int s_cnt;
    for (int s = threadIdx.x; s < cap; s += kCHugeBlock) {
        keys[s] = -1;
        vals[s] = 0;
    }
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int c = blockIdx.x; c < B.nchunks; c += gridDim.x) {
        const int b = B.chunk_b[c];
        const int32_t a = B.blist[b];
        const int q = c - B.chunk_first[b];
        const int nch = B.nch[b];
        const int32_t pb = A.moff[a], pe = A.moff[a + 1];
        const int64_t tb = A.mpre[pb], te = A.mpre[pe];
        const int64_t cb = tb + (int64_t)q * B.chunk;
        const int64_t ce = min(te, cb + (int64_t)B.chunk);
        int32_t p = B.mem0[c];  // the member holding entry cb
        for (int64_t t = cb + threadIdx.x; t < ce; t += kCHugeBlock) {
            int32_t key;
            i64 wv;
            flat_entry(A, p, pe, t, key, wv);
            tbl_insert<false, VT>(keys, vals, list, &s_cnt, log2cap, key, (VT)wv, A.err);
        }
        __syncthreads();
        const int m = s_cnt;
        const int64_t out = nch == 1 ? tb : cb;  // a one-chunk community: its row
        const int pl = B.plog2[b];
        int32_t *pc = nch == 1 ? nullptr : B.pcnt + B.pbase[b];
        for (int r = threadIdx.x; r < m; r += kCHugeBlock) {
            const int s = list[r];
            const int32_t key = keys[s];
            A.tmp_col[out + r] = key;
            ((VT *)A.tmp_w)[out + r] = vals[s];
            keys[s] = -1;
            vals[s] = 0;
            if (pc) atomicAdd(&pc[part_of(key, pl)], 1);
        }
        __syncthreads();  // every thread has read the count before it is reset
        if (threadIdx.x == 0) {
            if (nch == 1) A.ccnt[a] = m;
            else B.chm[c] = m;
            if (nch > 1 && q == 0) A.ccnt[a] = 0;  // phase C counts the merged row
            s_cnt = 0;
        }
        __syncthreads();
    }
}

// Phase B: every chunk's pairs to their partition's place in (pk, pv).
template <typename VT>
__global__ void __launch_bounds__(kCHugeBlock) k_coarsen_huge_scatter(CBigArgs B,
                                                                      const int32_t *moff,
                                                                      const int64_t *mpre,
                                                                      const int32_t *tmp_col,
                                                                      const void *tmp_w)
{
    for (int c = blockIdx.x; c < B.nchunks; c += gridDim.x) {
        const int b = B.chunk_b[c];
        if (B.nch[b] == 1) continue;
        const int32_t a = B.blist[b];
        const int q = c - B.chunk_first[b];
        const int64_t cb = mpre[moff[a]] + (int64_t)q * B.chunk;
        const int m = B.chm[c];
        const int pl = B.plog2[b];
        const int64_t base = B.pbase[b];
        for (int r = threadIdx.x; r < m; r += kCHugeBlock) {
            const int32_t key = tmp_col[cb + r];
            const int64_t part = base + part_of(key, pl);
            const int64_t pos = B.poff[part] + atomicAdd(&B.pcur[part], 1);
            B.pk[pos] = key;
            ((VT *)B.pv)[pos] = ((const VT *)tmp_w)[cb + r];
        }
    }
}

// Phase C: one CTA per partition merges its pairs in a shared table (merge_partition splits a
// crowded partition into residue classes) and appends the distinct targets with their sums to
// its community's row; the order of a row's entries is left open.
template <typename WT, typename VT>
__global__ void __launch_bounds__(kCHugeBlock) k_coarsen_huge_merge(CoarsenArgs<WT> A, CBigArgs B)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int log2cap = kPartTableLog2;
    constexpr int cap = 1 << log2cap;
    constexpr int thresh = cap - 2 * kCHugeBlock;
    VT *vals = (VT *)smem;
    int *keys = (int *)(vals + cap);
    int *list = keys + cap;
    __shared__ int s_base;
    for (int s = threadIdx.x; s < cap; s += kCHugeBlock) {
        keys[s] = -1;
        vals[s] = 0;
    }
    __syncthreads();
    for (int64_t q = blockIdx.x; q < B.nparts; q += gridDim.x) {
        const int64_t lo = B.poff[q], hi = B.poff[q + 1];
        if (lo == hi) continue;
        const int32_t a = B.blist[B.partb[q]];
        const int64_t tb = A.mpre[A.moff[a]];
        auto for_pairs = [&](auto f) {
            for (int64_t r = lo + threadIdx.x; r < hi; r += kCHugeBlock)
                f(B.pk[r], ((const VT *)B.pv)[r]);
        };
        auto emit = [&](int m) {
            if (threadIdx.x == 0) s_base = atomicAdd(&A.ccnt[a], m);
            __syncthreads();
            const int64_t o = tb + s_base;
            for (int r = threadIdx.x; r < m; r += kCHugeBlock) {
                const int s = list[r];
                st_stream(A.tmp_col + o + r, keys[s]);
                st_stream((VT *)A.tmp_w + o + r, vals[s]);
                keys[s] = -1;
                vals[s] = 0;
            }
            __syncthreads();  // s_base is read before the next class sets it
        };
        merge_partition<kCHugeBlock, VT>(keys, vals, list, log2cap, thresh, A.err, for_pairs,
                                         emit);
    }
}

// Compaction into the next CSR, balanced by output entries: each warp copies a slice of
// kCompactSlice consecutive output entries; the community of an entry is found by a
// binary search over the new row offsets and then advanced monotonically.
constexpr int kCompactSlice = 1024;

__device__ __forceinline__ int64_t row_of(const int64_t *rp, int64_t lo, int64_t hi, int64_t o)
{
    // largest a in [lo, hi) with rp[a] <= o
    while (hi - lo > 1) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (rp[mid] <= o) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <typename WO, typename VT>
__global__ void __launch_bounds__(kBlock) k_coarsen_compact(int64_t k, int64_t nnz_next,
                                                            const int32_t *moff,
                                                            const int64_t *mpre,
                                                            const int64_t *rp_next,
                                                            const int32_t *tmp_col,
                                                            const VT *tmp_w, int32_t *col_next,
                                                            WO *w_next)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t o0 = warp * kCompactSlice; o0 < nnz_next; o0 += nwarps * kCompactSlice) {
        const int64_t o1 = min(nnz_next, o0 + kCompactSlice);
        int64_t a = row_of(rp_next, 0, k, o0);
        // the lane's current row: its end and the shift from output to source index, reloaded
        // only when the lane's entry crosses into a later row
        int64_t end = rp_next[a + 1];
        int64_t shift = mpre[moff[a]] - rp_next[a];
        for (int64_t o = o0 + lane; o < o1; o += 32) {
            if (end <= o) {  // gallop from the next row, then bisect
                int64_t lo = a + 1, step = 1;
                while (lo + step < k && rp_next[lo + step] <= o) {
                    lo += step;
                    step <<= 1;
                }
                a = row_of(rp_next, lo, lo + step < k ? lo + step : k, o);
                end = rp_next[a + 1];
                shift = mpre[moff[a]] - rp_next[a];
            }
            st_stream(col_next + o, ld_stream(tmp_col + o + shift));
            st_stream(w_next + o, (WO)ld_stream(tmp_w + o + shift));
        }
    }
}

struct I32AsI64In {
    const int32_t *a;
    __device__ __forceinline__ int64_t operator()(int64_t i) const { return (int64_t)a[i]; }
};

// ------------------------------------------------------------------ launchers

static CBinArgs cbin_args(const Bins &b)
{
    CBinArgs ba;
    // no cluster bins in the induction: a community above the bin-5 bound goes to bin 10
    for (int t = 0; t < kNumBins - 1; t++) ba.upper[t] = b.upper[t < 5 ? t : 5];
    for (int t = 0; t <= kNumBins; t++) ba.off[t] = b.off[t];
    ba.list = b.list;
    return ba;
}

int launch_coarsen_stage1(const DevGraph &g, const PhaseState &st, const int32_t *new_id,
                          int64_t k, int64_t n_keep, const int32_t *vg, const int32_t *keep,
                          int32_t *vg_next, i64 *delta_next, CoarsenBufs &cb, Bins &bins,
                          cudaStream_t s, const LaunchCfg &lc)
{
    int launched = 0;
    const int64_t n = g.n;
    k_coarsen_prep<<<grid_for(n, kBlock, lc.max_blocks), kBlock, 0, s>>>(
        n, st.size, st.deg, new_id, vg, keep, cb.csize, delta_next, vg_next);
    launched++;
    launched += exclusive_scan<int32_t>(ArrayIn<int32_t>{cb.csize}, k, cb.moff, cb.scratch32, s);
    cudaMemsetAsync(cb.cursor, 0, sizeof(int32_t) * (size_t)k, s);
    k_coarsen_scatter<<<grid_for(n, kBlock, lc.max_blocks), kBlock, 0, s>>>(
        n, st.C, new_id, vg, keep, cb.moff, g.rp, cb.cursor, cb.members, cb.mrow);
    launched++;
    launched += exclusive_scan<int64_t>(MemberDegIn{cb.members, g.rp}, n_keep, cb.mpre,
                                        cb.scratch64, s);
    cudaMemsetAsync(cb.counts, 0, sizeof(int32_t) * 16, s);
    k_coarsen_bin<false><<<grid_for(k, kBlock, lc.max_blocks), kBlock, 0, s>>>(
        k, cb.moff, cb.mpre, cbin_args(bins), cb.counts);
    launched++;
    return launched;
}

int launch_coarsen_binfill(int64_t k, CoarsenBufs &cb, Bins &bins, cudaStream_t s,
                           const LaunchCfg &lc)
{
    cudaMemsetAsync(cb.counts, 0, sizeof(int32_t) * 16, s);
    k_coarsen_bin<true><<<grid_for(k, kBlock, lc.max_blocks), kBlock, 0, s>>>(
        k, cb.moff, cb.mpre, cbin_args(bins), cb.counts);
    return 1;
}

// shared table bytes: keys + values, plus a claim list when `with_list`
template <typename VT>
inline size_t ctable_bytes(int log2cap, bool with_list = false)
{
    return ((size_t)1 << log2cap) * (sizeof(VT) + (with_list ? 8 : 4));
}

template <typename K>
static int cta_grid(K kernel, int block, size_t smem, int nrows, const LaunchCfg &lc,
                    const char *name)
{
    set_dyn_smem(kernel, smem, name);
    const int per_sm_smem = (int)((227 * 1024) / (smem + 1024));
    const int per_sm_thr = 2048 / block;
    int per_sm = per_sm_smem < per_sm_thr ? per_sm_smem : per_sm_thr;
    if (per_sm < 1) per_sm = 1;
    const int maxg = lc.num_sms * per_sm;
    return nrows < maxg ? nrows : maxg;
}

// cn[v] = new_id[C[v]]: the next-level vertex of every vertex, so that the aggregation
// gathers one label per entry instead of two in a row
__global__ void k_renumbered_labels(int64_t n, const int32_t *C, const int32_t *new_id,
                                    int32_t *cn)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        cn[v] = new_id[C[v]];
}

template <typename WT, typename VT>
static int stage2_impl(const DevGraph &g, const PhaseState &st, const int32_t *new_id, int64_t k,
                       CoarsenBufs &cb, Bins &bins, unsigned *err, cudaStream_t s,
                       const LaunchCfg &lc)
{
    // the phase is over: C_next is free to hold the renumbered labels
    k_renumbered_labels<<<grid_for(g.n, kBlock, lc.max_blocks), kBlock, 0, s>>>(g.n, st.C, new_id,
                                                                              st.Cnext);
    CoarsenArgs<WT> A{g.rp,    g.col,   (const WT *)g.w, st.Cnext,   new_id,   cb.moff,
                      cb.mrow, cb.mpre, cb.ccnt,         cb.tmp_col, cb.tmp_w, err};
    int launched = 1;
    for (int bin = 1; bin < kNumBins; bin++) {
        const BinSpec sp = kBinSpec[bin];
        const int nr = bins.nlist[bin];
        const int32_t *rows = bins.rows(bin);
        if (nr == 0 && sp.kind != BIN_CHUNKED) continue;
        if (sp.kind == BIN_GROUP8) {
            k_coarsen_group<8, 6, WT, VT><<<grid_for(nr, kBlock / 8, lc.max_blocks), kBlock, 0, s>>>(
                A, rows, nr);
            note_launch("k_coarsen_group<8>");
            launched++;
        } else if (sp.kind == BIN_WARP) {
            k_coarsen_group<32, 8, WT, VT><<<grid_for(nr, kBlock / 32, lc.max_blocks), kBlock, 0, s>>>(
                A, rows, nr);
            note_launch("k_coarsen_group<32>");
            launched++;
        } else if (sp.kind == BIN_CTA) {
            const int l2 = cta_log2cap(bins, bin);
            const size_t smem = ctable_bytes<VT>(l2, true);
            if (sp.block == 128) {
                const int grid = cta_grid(k_coarsen_cta<128, WT, VT>, 128, smem, nr, lc, "k_coarsen_cta");
                k_coarsen_cta<128, WT, VT><<<grid, 128, smem, s>>>(A, rows, nr, l2);
            } else if (sp.block == 256) {
                const int grid = cta_grid(k_coarsen_cta<256, WT, VT>, 256, smem, nr, lc, "k_coarsen_cta");
                k_coarsen_cta<256, WT, VT><<<grid, 256, smem, s>>>(A, rows, nr, l2);
            } else {
                const int grid = cta_grid(k_coarsen_cta<1024, WT, VT>, 1024, smem, nr, lc, "k_coarsen_cta");
                k_coarsen_cta<1024, WT, VT><<<grid, 1024, smem, s>>>(A, rows, nr, l2);
            }
            note_launch("k_coarsen_cta");
            launched++;
        } else if (sp.kind == BIN_CHUNKED && bins.nchunks > 0) {
            CBigArgs B{rows,        bins.chunk_b, bins.chunk_first, bins.nch,
                       bins.goff,   bins.glog2,   bins.cpcnt,       bins.cpoff,
                       bins.cpcur,  bins.cpartb,  bins.gslots,      bins.cchm,
                       bins.cpk,    bins.cpv,     bins.chunk,       bins.nchunks,
                       bins.cmem0};
            k_chunk_member0<<<grid_for(bins.nchunks, kBlock, lc.max_blocks), kBlock, 0, s>>>(
                bins.nchunks, bins.chunk_b, bins.chunk_first, rows, cb.moff, cb.mpre, bins.chunk,
                bins.cmem0);
            note_launch("k_chunk_member0");
            launched++;
            const int l2 = 31 - __builtin_clz(2 * bins.chunk);
            const size_t smem = ctable_bytes<VT>(l2, true);
            const int grid = cta_grid(k_coarsen_huge<WT, VT>, kCHugeBlock, smem, bins.nchunks, lc,
                                      "k_coarsen_huge");
            k_coarsen_huge<WT, VT><<<grid, kCHugeBlock, smem, s>>>(A, B);
            note_launch("k_coarsen_huge");
            launched++;
            if (bins.gslots > 0) {  // multi-chunk communities: scatter by partition, merge
                launched += exclusive_scan<int64_t>(I32AsI64In{bins.cpcnt}, bins.gslots, bins.cpoff,
                                                    bins.cpscr, s);
                k_coarsen_huge_scatter<VT><<<grid, kCHugeBlock, 0, s>>>(B, cb.moff, cb.mpre,
                                                                       cb.tmp_col, cb.tmp_w);
                note_launch("k_coarsen_huge_scatter");
                const size_t msmem = ctable_bytes<VT>(kPartTableLog2, true);
                const int64_t mgrid_want = bins.gslots < (int64_t)INT32_MAX ? bins.gslots : INT32_MAX;
                const int mgrid = cta_grid(k_coarsen_huge_merge<WT, VT>, kCHugeBlock, msmem,
                                           (int)mgrid_want, lc, "k_coarsen_huge_merge");
                k_coarsen_huge_merge<WT, VT><<<mgrid, kCHugeBlock, msmem, s>>>(A, B);
                note_launch("k_coarsen_huge_merge");
                launched += 2;
            }
        }
    }
    return launched;
}

int launch_coarsen_stage2(const DevGraph &g, const PhaseState &st, const int32_t *new_id,
                          int64_t k, CoarsenBufs &cb, Bins &bins, bool narrow, unsigned *err,
                          cudaStream_t s, const LaunchCfg &lc)
{
    typedef unsigned int u32;
    if (g.wbytes == 4)
        return narrow ? stage2_impl<int32_t, u32>(g, st, new_id, k, cb, bins, err, s, lc)
                      : stage2_impl<int32_t, u64>(g, st, new_id, k, cb, bins, err, s, lc);
    return narrow ? stage2_impl<i64, u32>(g, st, new_id, k, cb, bins, err, s, lc)
                  : stage2_impl<i64, u64>(g, st, new_id, k, cb, bins, err, s, lc);
}

int launch_coarsen_bigprep(int64_t k, CoarsenBufs &cb, Bins &bins, cudaStream_t s,
                           const LaunchCfg &lc)
{
    const int nb = bins.nlist[kChunkedBin];
    if (nb == 0) return 0;
    k_cbig_prep<<<grid_for(nb, kBlock, lc.max_blocks), kBlock, 0, s>>>(
        nb, bins.rows(kChunkedBin), cb.moff, cb.mpre, k, bins.chunk, bins.nch, bins.gcap,
        bins.glog2);
    int launched = 1;
    launched += exclusive_scan<int32_t>(ArrayIn<int32_t>{bins.nch}, nb, bins.chunk_first,
                                        cb.scratch32, s);
    launched += exclusive_scan<int64_t>(ArrayIn<int64_t>{bins.gcap}, nb, bins.goff, cb.scratch64, s);
    return launched;
}

int launch_coarsen_partfill(Bins &bins, cudaStream_t s, const LaunchCfg &lc)
{
    const int nb = bins.nlist[kChunkedBin];
    if (nb == 0 || bins.gslots == 0) return 0;
    k_cpart_fill<<<grid_for(nb, kBlock / 32, lc.max_blocks), kBlock, 0, s>>>(nb, bins.goff,
                                                                             bins.cpartb);
    return 1;
}

int launch_coarsen_rowptr(int64_t k, CoarsenBufs &cb, int64_t *rp_next, cudaStream_t s)
{
    return exclusive_scan<int64_t>(I32AsI64In{cb.ccnt}, k, rp_next, cb.scratch64, s);
}

template <typename VT>
static void compact_impl(int grid, int64_t k, int64_t nnz_next, const CoarsenBufs &cb,
                         const int64_t *rp_next, int32_t *col_next, void *w_next,
                         int wbytes_next, cudaStream_t s)
{
    const VT *tw = (const VT *)cb.tmp_w;
    if (wbytes_next == 4)
        k_coarsen_compact<int32_t, VT><<<grid, kBlock, 0, s>>>(
            k, nnz_next, cb.moff, cb.mpre, rp_next, cb.tmp_col, tw, col_next, (int32_t *)w_next);
    else
        k_coarsen_compact<i64, VT><<<grid, kBlock, 0, s>>>(
            k, nnz_next, cb.moff, cb.mpre, rp_next, cb.tmp_col, tw, col_next, (i64 *)w_next);
}

int launch_coarsen_compact(int64_t k, int64_t nnz_next, const CoarsenBufs &cb,
                           const int64_t *rp_next, int32_t *col_next, void *w_next,
                           int wbytes_next, bool narrow, cudaStream_t s, const LaunchCfg &lc)
{
    if (k == 0 || nnz_next == 0) return 0;
    const int grid = grid_for((nnz_next + kCompactSlice - 1) / kCompactSlice, kBlock / 32,
                              lc.max_blocks);
    if (narrow)
        compact_impl<unsigned int>(grid, k, nnz_next, cb, rp_next, col_next, w_next, wbytes_next, s);
    else
        compact_impl<u64>(grid, k, nnz_next, cb, rp_next, col_next, w_next, wbytes_next, s);
    return 1;
}

}  // namespace lv
