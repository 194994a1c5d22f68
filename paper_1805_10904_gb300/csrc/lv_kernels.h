// lv_kernels.h -- host-side launchers of the Louvain kernels (internal to the library).
//
// Every launcher enqueues on the given stream and returns the number of kernels it
// launched.  Device pointers only; sizes in elements.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lv_common.cuh"

namespace lv {

// CSR of one level: rows of the symmetric adjacency, int32 columns, int32 or int64
// weights (wbytes = 4 or 8).
struct DevGraph {
    int64_t n = 0;
    int64_t nnz = 0;
    const int64_t *rp = nullptr;
    const int32_t *col = nullptr;
    const void *w = nullptr;
    int wbytes = 4;
};

// State of one phase (indexed by vertex or by community label, both in [0, n)).
struct PhaseState {
    int32_t *C = nullptr;      // current labels
    int32_t *Cnext = nullptr;  // labels proposed by the running sweep
    i64 *deg = nullptr;        // deg_c (Eq. 2)
    int32_t *size = nullptr;   // members of c
    i64 *delta = nullptr;      // weighted degree of each vertex
    // 32-bit copy of deg, read by the sweeps' candidate scans while *deg32_bad is 0 (every
    // community degree below 2^32); the writers of deg keep it and raise the flag
    unsigned *deg32 = nullptr;
    unsigned *deg32_bad = nullptr;
    // colouring variant: only the vertices of colour `cls` decide in this launch
    const int32_t *color = nullptr;
    int32_t cls = 0;
};

// Degree bins of one phase.  Bin b holds the rows (vertices, or communities when coarsening)
// whose entry count d satisfies upper[b-1] < d <= upper[b]; the last bin holds the rest.
enum BinKind { BIN_THREAD, BIN_GROUP8, BIN_WARP, BIN_CTA, BIN_CLUSTER, BIN_CHUNKED };
struct BinSpec {
    BinKind kind;
    int block;    // threads per CTA
    int cluster;  // CTAs per thread-block cluster (distributed shared-memory table)
};
constexpr int kNumBins = 11;
constexpr BinSpec kBinSpec[kNumBins] = {
    {BIN_THREAD, 256, 1},    // 0: one thread per row, registers
    {BIN_GROUP8, 256, 1},    // 1: 8 lanes per row, 64-slot shared table
    {BIN_WARP, 256, 1},      // 2: one warp per row, 256-slot shared table
    {BIN_CTA, 128, 1},       // 3-5: one CTA per row, shared table of >= 4/3 d slots
    {BIN_CTA, 256, 1},
    {BIN_CTA, 1024, 1},
    {BIN_CLUSTER, 1024, 2},  // 6-9: a cluster per row, table spread over the cluster's
    {BIN_CLUSTER, 1024, 4},  //      distributed shared memory (bin-5 table per CTA)
    {BIN_CLUSTER, 1024, 8},
    {BIN_CLUSTER, 1024, 16},
    {BIN_CHUNKED, 512, 1},   // 10: CTA chunks merged in a global-memory table
};
constexpr int kChunkedBin = kNumBins - 1;
// Partitioned aggregation of rows spanning several chunks (table sweeps): a row's distinct
// keys are split by hash over P = 2^plog2 partitions, P the smallest power of two that keeps
// the expected keys per partition at or below the configured part_keys (default kPartKeys,
// P <= 2^kMaxPartLog2); each partition is merged in a shared table of 2^kPartTableLog2
// slots.
constexpr int kPartKeys = 2048;
constexpr int kMaxPartLog2 = 11;
constexpr int kPartTableLog2 = 13;
static_assert(kNumBins <= 16, "per-bin counters of SweepStats hold 16 bins");

struct Bins {
    int64_t upper[kNumBins - 1] = {8, 32, 128, 512, 2048, 12288, 24576, 49152, 98304, 196608};
    int chunk = 4096;               // entries per CTA chunk of a chunked row
    int part_keys = kPartKeys;      // expected distinct keys per partition of a chunked row
    int32_t *list = nullptr;        // rows of bins 1.., grouped by bin
    int64_t off[kNumBins + 1] = {}; // bin b's rows are list[off[b] .. off[b+1])
    int nlist[kNumBins] = {};
    int64_t entries[kNumBins] = {};
    int32_t *counts = nullptr;      // device: [0..15] list sizes / cursors, then int64 entries
    // chunked rows
    int32_t *nch = nullptr;          // chunks per row
    int32_t *chunk_first = nullptr;  // exclusive scan of nch (nb + 1)
    int32_t *chunk_b = nullptr;      // chunked-list index of every chunk
    int nchunks = 0;
    u64 *gloop = nullptr;      // loop weight of every multi-chunk row
    // graph induction: a multi-chunk community merges its chunks' distinct (target, sum)
    // pairs by hash partition of the target: gcap[b] partitions (0 for one chunk), goff
    // their exclusive scan (first partition of each community), glog2 = log2 gcap
    int64_t *gcap = nullptr;
    int64_t *goff = nullptr;
    int32_t *glog2 = nullptr;
    int64_t gslots = 0;        // partitions in all
    int32_t *cpcnt = nullptr;  // pairs per partition
    int64_t *cpoff = nullptr;  // their exclusive scan (gslots + 1)
    int32_t *cpcur = nullptr;  // scatter cursor per partition
    int32_t *cpartb = nullptr; // community (chunked-list index) of every partition
    int32_t *cchm = nullptr;   // distinct pairs of every chunk
    int32_t *cmem0 = nullptr;  // member holding the first entry of every chunk
    int32_t *cpk = nullptr;    // pairs grouped by partition: targets
    void *cpv = nullptr;       //                              sums (u32 or u64)
    int64_t *cpscr = nullptr;  // scan scratch for the partition offsets
    // decision of multi-chunk rows, one work item ("slice") per partition of a row's keys:
    // partial argmax (gain, label, e_{i->C(i)}) and distinct keys of every slice; in the
    // first sweep of a phase one partial per chunk instead, pcnt then holding the chunk's
    // (entries labelled C(i)) << 32 | (other entries)
    void *pgain = nullptr;     // 16 bytes per partial (int64 or int128 gain)
    int32_t *pbest = nullptr;
    i64 *pea = nullptr;
    u64 *pcnt = nullptr;
    int32_t *sdone = nullptr;  // partials finished per row
    int64_t *soff = nullptr;   // row b's slices are soff[b] .. soff[b+1] (nb + 1)
    int32_t *slice_row = nullptr;
    int64_t nslices = 0;
    // partitioned aggregation: chunk q of row b writes its distinct (key, sum) pairs grouped
    // by partition to its region of pkeys / pvals (chunk entries each) and the partitions'
    // offsets to hofs[hoff[b] + q * (P + 1) + p]
    int32_t *plog2 = nullptr;
    int64_t *hoff = nullptr;  // exclusive scan of nch * (P + 1) over multi-chunk rows (nb + 1)
    int32_t *hofs = nullptr;
    int32_t *pkeys = nullptr;
    void *pvals = nullptr;    // u32 or u64 per pair (8 bytes per pair allocated)
    const int32_t *rows(int b) const { return list + off[b]; }
};

// log2 of the shared table of CTA bins (3..5): at least 4/3 of the bin's upper bound, so
// the load factor stays <= 0.75 and there are always more slots than distinct keys.
// Cluster bins use the bin-5 table in each of their CTAs.
inline int cta_log2cap(const Bins &b, int bin)
{
    if (bin > 5) bin = 5;
    const int64_t need = b.upper[bin] + b.upper[bin] / 3;
    int l = 5;
    while (((int64_t)1 << l) < need) l++;
    return l;
}

// Graph context of a batch of graphs stored as one disjoint union (nullptr pointers for a
// single graph): the graph of every vertex, every graph's 2W and phase controller.
// Streams on which the bins of one sweep run side by side (forked from and joined back
// into the sweep's stream with the events).
struct SweepStreams {
    int k = 0;
    cudaStream_t aux[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[4] = {nullptr, nullptr, nullptr, nullptr};
};

struct BatchCtx {
    const int32_t *vg = nullptr;
    const i64 *gtw = nullptr;
    const LevelCtl *gctl = nullptr;
    const SweepStreams *ss = nullptr;  // concurrent bins (nullptr: all on the sweep's stream)
};

struct LaunchCfg {
    int num_sms = 152;
    int max_blocks = 152 * 8;  // persistent grid cap for grid-stride kernels
    bool cluster_ok[4] = {false, false, false, false};  // clusters of 2, 4, 8, 16 resident
};

// Which cluster sizes (2, 4, 8, 16 CTAs of 1024 threads with `smem` bytes of dynamic shared
// memory each) can be resident on the current device.
void probe_cluster_support(size_t smem, bool ok[4]);
// Bytes of a CTA's shared table of 2^log2cap slots with 32-bit (narrow) or 64-bit sums.
size_t shared_table_bytes(int log2cap, bool narrow);

// ---- k_level.cu
int launch_validate_rowptr(const int64_t *rp, int64_t n, unsigned *err, cudaStream_t s,
                           const LaunchCfg &lc);
int launch_fill_ones(int32_t *w, int64_t nnz, cudaStream_t s, const LaunchCfg &lc);
// *out = max_i delta[i] over n vertices (0 when n = 0)
int launch_max_delta(const i64 *delta, int64_t n, u64 *out, cudaStream_t s, const LaunchCfg &lc);
// Columns in [0, n) and weights >= 1 of one graph (w NULL: all 1), *tw += its 2W.
int launch_check_rows(int64_t n, const int64_t *rp, const int32_t *col, const int32_t *w,
                      unsigned *err, u64 *tw, cudaStream_t s, const LaunchCfg &lc);
// Weighted degrees and 2W with column / weight checks, one thread, warp or CTA per row
// according to the row's degree bin (bins must have been filled for g).  With vg set (a
// batch), 2W is summed per graph into tw[vg[i]] and a column must lie in its row's graph
// [gptr[g], gptr[g+1]); otherwise tw[0] gets the total and columns lie in [0, n).
// delta and 2W (per graph in a batch) with the input checks; unsorted[g] (zeroed by the
// caller) is set when a row of graph g does not list strictly increasing columns
int launch_row_sums(const DevGraph &g, const Bins &b, const int32_t *vg, const int64_t *gptr,
                    i64 *delta, u64 *tw, unsigned *unsorted, unsigned *err, cudaStream_t s,
                    const LaunchCfg &lc);
int launch_check_symmetry(const DevGraph &g, unsigned *err, cudaStream_t s, const LaunchCfg &lc);
int launch_init_state(int64_t n, const PhaseState &st, cudaStream_t s, const LaunchCfg &lc);
// Vertex following (degree-one vertices join their neighbour; an isolated pair takes the
// smaller label).  In a batch, only vertices whose graph has vf_on[vg[i]] follow.
int launch_vertex_following(const DevGraph &g, const PhaseState &st, cudaStream_t s,
                            const LaunchCfg &lc, const int32_t *vg = nullptr,
                            const int32_t *vf_on = nullptr);
// Two passes: count rows and entries per bin (then the host reads counts and sets off[]),
// fill the list grouped by bin.  In a batch (vg, gctl given) rows of graphs whose phase has
// stopped are left out of every bin.
// color (optional): only the vertices of colour cls are binned
int launch_bin_count(const DevGraph &g, Bins &b, cudaStream_t s, const LaunchCfg &lc,
                     const int32_t *vg = nullptr, const LevelCtl *gctl = nullptr,
                     const int32_t *color = nullptr, int32_t cls = 0);
int launch_bin_fill(const DevGraph &g, Bins &b, cudaStream_t s, const LaunchCfg &lc,
                    const int32_t *vg = nullptr, const LevelCtl *gctl = nullptr,
                    const int32_t *color = nullptr, int32_t cls = 0);
int launch_big_prep(const DevGraph &g, Bins &b, int64_t *scratch64, int32_t *scratch32,
                    cudaStream_t s, const LaunchCfg &lc);
int launch_big_fill(Bins &b, cudaStream_t s, const LaunchCfg &lc);
// Decision slices of the multi-chunk rows (soff, then slice_row once the host has read the
// total soff[nb] into nslices and sized slice_row).
int launch_huge_slices(Bins &b, int64_t *scratch64, cudaStream_t s);
int launch_huge_slice_fill(Bins &b, cudaStream_t s, const LaunchCfg &lc);
// Phase controllers of G graphs (one thread each): trace entry t of graph g at t * G + g;
// *ndone counts the graphs whose phase has stopped.
int launch_decide(SweepStats *st, LevelCtl *ctl, int G, i64 *tr_moved, i64 *tr_qn,
                  u64 *cand_total, int *ndone, cudaStream_t s);
// ctl nullptr: every proposal is applied (no controller consulted).
int launch_apply(int64_t n, const PhaseState &st, const LevelCtl *ctl, const int32_t *vg,
                 cudaStream_t s, const LaunchCfg &lc);
// Post-phase merge of Sec. 5.1.2 (a vertex whose non-loop neighbours all lie in one other
// community joins it when the move's gain is positive), applied to every vertex of g, then
// the exact Qn of the merged state into ctl[g].qn_final for all G controllers.  stats must
// be zero on entry and are zero on return.
// Colouring variant (one graph).  One Jones-Plassmann round: pick marks every uncoloured
// vertex whose priority is above that of each uncoloured non-loop neighbour, counting the
// uncoloured vertices (counts[0]) and the picks (counts[1]); assign gives every pick the
// smallest colour none of its neighbours has and raises *ncolors to cover it.
int launch_color_pick(const DevGraph &g, const int32_t *color, int32_t *pick, u64 *counts,
                      cudaStream_t s, const LaunchCfg &lc);
int launch_color_assign(const DevGraph &g, int32_t *color, const int32_t *pick, int32_t *ncolors,
                        cudaStream_t s, const LaunchCfg &lc);
// Apply the proposals of the vertices of colour st.cls (deg / size follow), adding the number
// that moved to *moved.
int launch_apply_class(int64_t n, const PhaseState &st, u64 *moved, cudaStream_t s,
                       const LaunchCfg &lc);
// Exact Qn of the current state of one graph into ctl->qn_final (stats must be zero on entry
// and are zero again on return).
int launch_qn_one(const DevGraph &g, const PhaseState &st, SweepStats *stats, LevelCtl *ctl,
                  cudaStream_t s, const LaunchCfg &lc);
int launch_post_merge(const DevGraph &g, const PhaseState &st, const int32_t *vg, const i64 *gtw,
                      i64 tw, bool wide, SweepStats *stats, LevelCtl *ctl, int G, cudaStream_t s,
                      const LaunchCfg &lc);
// State of the device-side sweep loop: sweeps run so far, controllers stopped when it was
// launched, how many more may stop before it returns, and its sweep bound.
struct LoopCtl {
    int iters;
    int nd0;
    int quota;
    int cap;
};
// Sets the while-node condition of the sweep loop after a sweep (one thread).
int launch_loop_ctl(cudaGraphConditionalHandle handle, LoopCtl *lc, const int *ndone, int G,
                    cudaStream_t s);
// new_id[c] = rank of c among used labels (size[c] > 0, and keep[vg[c]] when given).
int launch_renumber(int64_t n, const int32_t *size, const int32_t *vg, const int32_t *keep,
                    int32_t *new_id, int32_t *scratch, cudaStream_t s);
// out[i] = a[idx[i]] for i < cnt (small gathers of per-graph offsets).
int launch_gather64(const int64_t *a, const int64_t *idx, int cnt, int64_t *out, cudaStream_t s);
int launch_gather_ids(const int32_t *a, const int64_t *idx, int cnt, int64_t *out, cudaStream_t s);
// vg[v] = graph of vertex v from the vertex offsets gptr[0..G] of a batch.
int launch_graph_ids(int64_t n, const int64_t *gptr, int G, int32_t *vg, cudaStream_t s,
                     const LaunchCfg &lc);
// Appends a source CSR (int32 weights, NULL = all 1) at (v_base, e_base) of a stacked CSR
// whose weights are wbytes wide; columns are shifted by v_base.  dst_rp[n] is the caller's.
int launch_append_rows(int64_t n_src, int64_t nnz_src, const int64_t *src_rp,
                       const int32_t *src_col, const int32_t *src_w, int64_t v_base,
                       int64_t e_base, int64_t *dst_rp, int32_t *dst_col, void *dst_w, int wbytes,
                       cudaStream_t s, const LaunchCfg &lc);
// Original-vertex maps of M graphs entering at level 0: maps[m][k] = vbase[m] + k for the
// off[m+1] - off[m] vertices of graph m (off, maps, vbase are device arrays).
int launch_map_init(int64_t tot, int M, const int64_t *off, int32_t *const *maps,
                    const int64_t *vbase, cudaStream_t s, const LaunchCfg &lc);
// Labels of the original vertices of M graphs (original vertex o of graph m at
// off[m] <= o < off[m+1], its current vertex maps[m][o - off[m]]): for rec[m],
// out[o] = new_id1[C[v]] - base1[m]; for keep[m], the map moves to new_id2[C[v]].
int launch_compose(int64_t n0, int M, const int64_t *off, int32_t *const *maps,
                   const int32_t *rec, const int32_t *keep, const int32_t *C,
                   const int32_t *new_id1, const int64_t *base1, const int32_t *new_id2,
                   int32_t *out, cudaStream_t s, const LaunchCfg &lc);

// ---- k_edges.cu: symmetric CSR from an undirected edge list (Sec. 5.1.2 neighbour computation)
struct EdgeScratch {
    u64 *keys[2] = {nullptr, nullptr};     // 2m each
    int32_t *vals[2] = {nullptr, nullptr}; // 2m each
    int64_t *pos = nullptr;                // 2m + 1
    u64 *wacc = nullptr;                   // 2m
    int32_t *rowcnt = nullptr;             // n
    int64_t *hist = nullptr;               // 256 * edges_scratch_tiles(m)
    int64_t *offs = nullptr;               // 256 * edges_scratch_tiles(m) + 1
    int64_t *scan64 = nullptr;             // scan_scratch_elems(max(2m, 256 * tiles, n) + 1)
};
int edges_scratch_tiles(int64_t m);
// Entries of non-loop edges in both directions, loops once, equal (row, column) merged by
// adding weights, rows sorted by column.  col_out / w_out need room for 2m entries; the row
// offsets (n + 1) and *nnz_out (device) are written on `s`; bad endpoints, weights or a
// merged weight above 2^31 - 1 set bits of *err.
int launch_edges_to_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                        const int32_t *w, const EdgeScratch &sc, int64_t *rp_out,
                        int32_t *col_out, int32_t *w_out, int64_t *nnz_out, unsigned *err,
                        cudaStream_t s, const LaunchCfg &lc);

// ---- k_move.cu: one synchronous sweep (Algorithm 1 body) over all bins
struct SweepTimers {
    cudaEvent_t ev[2 * kNumBins];  // start/stop pair around each bin's kernel
    bool on = false;
};
// narrow: tables hold 32-bit sums (valid when 2W < 2^32); wide: int128 gains; first: the
// first sweep of a phase on rows without repeated columns (scored without tables).
int launch_sweep(const DevGraph &g, const PhaseState &st, const Bins &b, i64 tw, bool wide,
                 bool narrow, bool first, SweepStats *stats, unsigned *err, cudaStream_t s,
                 const LaunchCfg &lc, SweepTimers *tm, const BatchCtx &bc);

// ---- k_coarsen.cu: graph induction (Sec. 5.1.2), renumbered labels new_id[C[u]]
struct CoarsenBufs {
    int32_t *csize = nullptr;     // k
    int32_t *moff = nullptr;      // k + 1
    int32_t *cursor = nullptr;    // k
    int32_t *members = nullptr;   // n
    int64_t *mrow = nullptr;      // n: row start of every member
    int64_t *mpre = nullptr;      // n + 1
    int32_t *ccnt = nullptr;      // k (distinct neighbours of each community)
    int32_t *tmp_col = nullptr;   // nnz
    void *tmp_w = nullptr;        // nnz sums of the aggregation's width (32 bits when narrow)
    int32_t *counts = nullptr;    // device counters of the community bins
    int64_t *scratch64 = nullptr;
    int32_t *scratch32 = nullptr;
};
// Stage 1: community sizes, next-level delta, member lists, flattened offsets, and the
// count pass of the community bins (by entries; rows of bins 0..2 all go to bin 2).
// Only communities of graphs with keep[vg[c]] (all when vg is nullptr) enter the next
// level; vg_next receives the graph of every next-level vertex (when vg is set), and
// n_keep is the number of vertices of the kept graphs.
int launch_coarsen_stage1(const DevGraph &g, const PhaseState &st, const int32_t *new_id,
                          int64_t k, int64_t n_keep, const int32_t *vg, const int32_t *keep,
                          int32_t *vg_next, i64 *delta_next, CoarsenBufs &cb, Bins &bins,
                          cudaStream_t s, const LaunchCfg &lc);
// Fill pass of the community bins (after the host set bins.off from the counts).
int launch_coarsen_binfill(int64_t k, CoarsenBufs &cb, Bins &bins, cudaStream_t s,
                           const LaunchCfg &lc);
// Chunk counts and global-table sizes of the communities of the chunked bin.
// community of every partition of the multi-chunk communities (bins.cpartb)
int launch_coarsen_partfill(Bins &bins, cudaStream_t s, const LaunchCfg &lc);
int launch_coarsen_bigprep(int64_t k, CoarsenBufs &cb, Bins &bins, cudaStream_t s,
                           const LaunchCfg &lc);
// Stage 2 (after the host read the bin counts): aggregate every community's entries.
int launch_coarsen_stage2(const DevGraph &g, const PhaseState &st, const int32_t *new_id,
                          int64_t k, CoarsenBufs &cb, Bins &bins, bool narrow, unsigned *err,
                          cudaStream_t s, const LaunchCfg &lc);
// Stage 3 (after the host allocated the next graph): row offsets and compaction.
int launch_coarsen_rowptr(int64_t k, CoarsenBufs &cb, int64_t *rp_next, cudaStream_t s);
int launch_coarsen_compact(int64_t k, int64_t nnz_next, const CoarsenBufs &cb,
                           const int64_t *rp_next, int32_t *col_next, void *w_next,
                           int wbytes_next, bool narrow, cudaStream_t s, const LaunchCfg &lc);

}  // namespace lv
