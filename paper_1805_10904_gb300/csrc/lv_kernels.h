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

// Degree bins of one phase.
struct Bins {
    int small_max = 8;  // row length <= small_max: thread per vertex (dense kernel)
    int mid1 = 32;      // <= mid1: 8-lane groups
    int mid2 = 128;     // <= mid2: one warp
    int chunk = 1024;   // CTA chunk of a longer row
    int32_t *list[3] = {nullptr, nullptr, nullptr};  // mid1, mid2, big vertex lists
    int32_t *counts = nullptr;  // device int32[8]: list sizes [0..2], entries per bin [4..7] as int64 pair
    int nlist[3] = {0, 0, 0};
    int64_t entries[4] = {0, 0, 0, 0};  // stored entries in small, mid1, mid2, big rows
    // big rows, split in chunks
    int32_t *nch = nullptr;          // chunks per big row
    int32_t *chunk_first = nullptr;  // exclusive scan of nch (nb + 1)
    int32_t *chunk_b = nullptr;      // big-list index of every chunk
    int nchunks = 0;
    // global hash tables of multi-chunk rows
    int64_t *gcap = nullptr;   // slots (0 for single-chunk rows)
    int64_t *goff = nullptr;   // exclusive scan of gcap (nb + 1)
    int32_t *glog2 = nullptr;
    int32_t *gcnt = nullptr;
    int32_t *gdone = nullptr;
    u64 *gloop = nullptr;
    int32_t *gkeys = nullptr;
    u64 *gvals = nullptr;
    int32_t *glist = nullptr;
    int64_t gslots = 0;
};

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
    cudaEvent_t ev[8];  // start/stop pairs for small, mid1, mid2, big
    bool on = false;
};
int launch_sweep(const DevGraph &g, const PhaseState &st, const Bins &b, i64 tw, bool wide,
                 SweepStats *stats, unsigned *err, cudaStream_t s, const LaunchCfg &lc,
                 SweepTimers *tm);

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
    int32_t *clist = nullptr;     // small communities
    int32_t *blist = nullptr;     // big communities
    int32_t *counts = nullptr;    // device int32[4]
    int64_t *scratch64 = nullptr;
    int32_t *scratch32 = nullptr;
};
// Stage 1: community sizes, next-level delta, member lists, flattened offsets, bins.
int launch_coarsen_stage1(const DevGraph &g, const PhaseState &st, const int32_t *new_id,
                          int64_t k, i64 *delta_next, CoarsenBufs &cb, cudaStream_t s,
                          const LaunchCfg &lc);
// Chunk counts and global-table sizes of the communities in cb.blist (big.nlist[2] of them).
int launch_coarsen_bigprep(int64_t k, CoarsenBufs &cb, Bins &big, cudaStream_t s,
                           const LaunchCfg &lc);
// Stage 2 (after the host read the bin counts): aggregate every community's entries.
int launch_coarsen_stage2(const DevGraph &g, const PhaseState &st, const int32_t *new_id,
                          int64_t k, CoarsenBufs &cb, int nsmall, Bins &big, unsigned *err,
                          cudaStream_t s, const LaunchCfg &lc);
// Stage 3 (after the host allocated the next graph): row offsets and compaction.
int launch_coarsen_rowptr(int64_t k, CoarsenBufs &cb, int64_t *rp_next, cudaStream_t s);
int launch_coarsen_compact(int64_t k, const CoarsenBufs &cb, const int64_t *rp_next,
                           int32_t *col_next, void *w_next, int wbytes_next, cudaStream_t s,
                           const LaunchCfg &lc);

}  // namespace lv
