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
};

// Degree bins of one phase.  Bin b holds the vertices (or communities) whose entry count
// d satisfies upper[b-1] < d <= upper[b]; the last bin holds the rest.
//   0: one thread per vertex (dense kernel, no list)   3..5: one CTA per row, shared table
//   1: 8-lane groups, 64-slot tables                   6:    CTA chunks, global table
//   2: one warp, 256-slot tables
constexpr int kNumBins = 7;
constexpr int kCtaBins = 3;                       // bins 3, 4, 5
constexpr int kCtaBlock[kCtaBins] = {128, 256, 1024};

struct Bins {
    int64_t upper[kNumBins - 1] = {8, 32, 128, 512, 2048, 12288};
    int chunk = 4096;   // entries per CTA chunk of a bin-6 row
    int32_t *list[kNumBins] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int nlist[kNumBins] = {0, 0, 0, 0, 0, 0, 0};
    int64_t entries[kNumBins] = {0, 0, 0, 0, 0, 0, 0};
    int32_t *counts = nullptr;  // device: [0..7] list sizes, then 8 int64 entry totals
    // bin-6 rows, split in chunks
    int32_t *nch = nullptr;          // chunks per row
    int32_t *chunk_first = nullptr;  // exclusive scan of nch (nb + 1)
    int32_t *chunk_b = nullptr;      // bin-6 list index of every chunk
    int nchunks = 0;
    // global hash tables of multi-chunk rows
    int64_t *gcap = nullptr;   // slots (0 for single-chunk rows)
    int64_t *goff = nullptr;   // exclusive scan of gcap (nb + 1)
    int32_t *glog2 = nullptr;
    int32_t *gcnt = nullptr;
    int32_t *gdone = nullptr;
    u64 *gloop = nullptr;
    int32_t *gkeys = nullptr;
    void *gvals = nullptr;     // u32 or u64 per slot
    int32_t *glist = nullptr;
    int64_t gslots = 0;
};

// log2 of the shared table of CTA bin b (3..5): at least 4/3 of the bin's upper bound, so
// the load factor stays <= 0.75 and there are always more slots than distinct keys.
inline int cta_log2cap(const Bins &b, int bin)
{
    const int64_t need = b.upper[bin] + b.upper[bin] / 3;
    int l = 5;
    while (((int64_t)1 << l) < need) l++;
    return l;
}

struct LaunchCfg {
    int num_sms = 152;
    int max_blocks = 152 * 8;  // persistent grid cap for grid-stride kernels
};

// ---- k_level.cu
int launch_validate_rowptr(const int64_t *rp, int64_t n, unsigned *err, cudaStream_t s,
                           const LaunchCfg &lc);
int launch_fill_ones(int32_t *w, int64_t nnz, cudaStream_t s, const LaunchCfg &lc);
int launch_row_sums(const DevGraph &g, i64 *delta, u64 *tw, unsigned *err, cudaStream_t s,
                    const LaunchCfg &lc);
int launch_check_symmetry(const DevGraph &g, unsigned *err, cudaStream_t s, const LaunchCfg &lc);
int launch_init_state(int64_t n, const PhaseState &st, cudaStream_t s, const LaunchCfg &lc);
int launch_vertex_following(const DevGraph &g, const PhaseState &st, cudaStream_t s,
                            const LaunchCfg &lc);
int launch_bin(const DevGraph &g, Bins &b, cudaStream_t s, const LaunchCfg &lc);
int launch_big_prep(const DevGraph &g, Bins &b, int64_t *scratch64, int32_t *scratch32,
                    cudaStream_t s, const LaunchCfg &lc);
int launch_big_fill(Bins &b, cudaStream_t s, const LaunchCfg &lc);
int launch_decide(SweepStats *st, LevelCtl *ctl, i64 *tr_moved, i64 *tr_qn, u64 *cand_total,
                  cudaStream_t s);
int launch_apply(int64_t n, const PhaseState &st, const LevelCtl *ctl, cudaStream_t s,
                 const LaunchCfg &lc);
int launch_renumber(int64_t n, const int32_t *size, int32_t *new_id, int32_t *scratch,
                    cudaStream_t s);
int launch_compose(int64_t n0, const int32_t *prev, const int32_t *C, const int32_t *new_id,
                   int32_t *out, cudaStream_t s, const LaunchCfg &lc);

// ---- k_move.cu: one synchronous sweep (Algorithm 1 body) over all bins
struct SweepTimers {
    cudaEvent_t ev[2 * kNumBins];  // start/stop pair around each bin's kernel
    bool on = false;
};
// narrow: tables hold 32-bit sums (valid when 2W < 2^32); wide: int128 gains.
int launch_sweep(const DevGraph &g, const PhaseState &st, const Bins &b, i64 tw, bool wide,
                 bool narrow, SweepStats *stats, unsigned *err, cudaStream_t s,
                 const LaunchCfg &lc, SweepTimers *tm);

// ---- k_coarsen.cu: graph induction (Sec. 5.1.2), renumbered labels new_id[C[u]]
struct CoarsenBufs {
    int32_t *csize = nullptr;     // k
    int32_t *moff = nullptr;      // k + 1
    int32_t *cursor = nullptr;    // k
    int32_t *members = nullptr;   // n
    int64_t *mpre = nullptr;      // n + 1
    int32_t *ccnt = nullptr;      // k (distinct neighbours of each community)
    int32_t *tmp_col = nullptr;   // nnz
    u64 *tmp_w = nullptr;         // nnz
    int32_t *clist = nullptr;     // community lists of bins 2..6 (5 regions of k entries)
    int32_t *counts = nullptr;    // device int32[8]: list sizes of bins 2..6
    int64_t *scratch64 = nullptr;
    int32_t *scratch32 = nullptr;
};
// Stage 1: community sizes, next-level delta, member lists, flattened offsets, bins
// (communities binned by entry count with the thresholds of `bins`, bins 2..6 used).
int launch_coarsen_stage1(const DevGraph &g, const PhaseState &st, const int32_t *new_id,
                          int64_t k, i64 *delta_next, CoarsenBufs &cb, const Bins &bins,
                          cudaStream_t s, const LaunchCfg &lc);
// Chunk counts and global-table sizes of the bin-6 communities (bins.list[6]).
int launch_coarsen_bigprep(int64_t k, CoarsenBufs &cb, Bins &bins, cudaStream_t s,
                           const LaunchCfg &lc);
// Stage 2 (after the host read the bin counts): aggregate every community's entries.
int launch_coarsen_stage2(const DevGraph &g, const PhaseState &st, const int32_t *new_id,
                          int64_t k, CoarsenBufs &cb, Bins &bins, bool narrow, unsigned *err,
                          cudaStream_t s, const LaunchCfg &lc);
// Stage 3 (after the host allocated the next graph): row offsets and compaction.
int launch_coarsen_rowptr(int64_t k, CoarsenBufs &cb, int64_t *rp_next, cudaStream_t s);
int launch_coarsen_compact(int64_t k, const CoarsenBufs &cb, const int64_t *rp_next,
                           int32_t *col_next, void *w_next, int wbytes_next, cudaStream_t s,
                           const LaunchCfg &lc);

}  // namespace lv
