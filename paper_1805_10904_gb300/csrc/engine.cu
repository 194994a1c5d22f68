// engine.cu -- host orchestration of multi-level synchronous Louvain and the C ABI.
//
// Algorithm 2 of arXiv 1805.10904 around Algorithm 1:
//   level l: init status (delta, singletons; vertex following at level 0), degree bins,
//            sweeps until the phase controller stops (all decisions on device), renumber
//            (prefix-sum compaction), record the level if it merged anything, test the
//            outer threshold, induce the next graph.
// The host only sequences launches, sizes buffers and reads a few scalars per sweep and
// per level; every step of the method runs in the kernels of k_level.cu, k_move.cu and
// k_coarsen.cu.
#include <algorithm>
#include <functional>
#include <array>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/louvain.h"
#include "lv_common.cuh"
#include "lv_kernels.h"
#include "lv_scan.cuh"

using namespace lv;

namespace {

// NVTX range named after the paper's processes (Sec. 5.1.2: neighbour computation, init,
// one level, renumbering, induction); phase() closes the current range and opens the next.
struct ProcRange {
    bool open = false;
    explicit ProcRange(const char *name) { phase(name); }
    void phase(const char *name)
    {
        if (open) nvtxRangePop();
        nvtxRangePushA(name);
        open = true;
    }
    ~ProcRange()
    {
        if (open) nvtxRangePop();
    }
};

struct LvErr {
    int code;
    std::string msg;
};

#define CK(x)                                                                                   \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess)                                                                  \
            throw LvErr{e_ == cudaErrorMemoryAllocation ? LOUVAIN_ERR_OOM : LOUVAIN_ERR_CUDA,   \
                        std::string(#x) + ": " + cudaGetErrorString(e_)};                       \
    } while (0)

// Device memory through the caller's allocator or stream-ordered cudaMallocAsync.
struct DevAlloc {
    louvain_alloc_fn fa = nullptr;
    louvain_free_fn ff = nullptr;
    void *ctx = nullptr;
    cudaStream_t s = nullptr;
    void *get(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        bytes = (bytes + 255) & ~(size_t)255;
        void *p = nullptr;
        if (fa) {
            p = fa(bytes, ctx, (void *)s);
            if (!p) throw LvErr{LOUVAIN_ERR_OOM, "allocator callback returned NULL"};
        } else {
            cudaError_t e = cudaMallocAsync(&p, bytes, s);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                throw LvErr{LOUVAIN_ERR_OOM, "cudaMallocAsync of " + std::to_string(bytes) +
                                                 " bytes failed"};
            }
        }
        return p;
    }
    void put(void *p)
    {
        if (!p) return;
        if (ff) ff(p, ctx, (void *)s);
        else cudaFreeAsync(p, s);
    }
};

template <typename T>
struct DBuf {
    DevAlloc *A = nullptr;
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    void reset(DevAlloc *a, size_t count)
    {
        release();
        A = a;
        n = count;
        p = (T *)A->get(sizeof(T) * (count ? count : 1));
    }
    void release()
    {
        if (p && A) A->put(p);
        p = nullptr;
        n = 0;
    }
    T *take()
    {
        T *q = p;
        p = nullptr;
        n = 0;
        return q;
    }
    void swap(DBuf &o)
    {
        std::swap(A, o.A);
        std::swap(p, o.p);
        std::swap(n, o.n);
    }
    ~DBuf() { release(); }
};

// Scalars shared by host and device during a run (one device block, one pinned mirror).
struct Scalars {
    unsigned err;
    int32_t ndone;  // phase controllers that have stopped
    u64 tw;
    u64 dmax;       // largest weighted degree of the level's graph
    u64 ccounts2[2];  // colouring round: uncoloured vertices, picks
    u64 cmoved;       // colouring variant: vertices moved by the classes of a sweep
    int32_t ncolors;  // colouring variant: colours of the level's graph
    int32_t pad2_;
    SweepStats st;
    LevelCtl ctl;
    int32_t bin_counts[40];
    int32_t ccounts[16];
    u64 cand_total[16];
    LoopCtl loop;
    unsigned unsorted;  // one graph: a row without strictly increasing columns was seen
    unsigned deg32_bad;  // a community degree reached 2^32: the sweeps read the 64-bit deg
    int32_t tail[8];
};

// x * a < y * b for unsigned 128-bit x, y and 64-bit a, b, compared in 192 bits
bool host_less_192(u128 x, u64 a, u128 y, u64 b)
{
    const u128 xl = (u128)(u64)x * a, xh = (u128)(u64)(x >> 64) * a;
    const u128 yl = (u128)(u64)y * b, yh = (u128)(u64)(y >> 64) * b;
    const u128 xmid = (xl >> 64) + (u64)xh, ymid = (yl >> 64) + (u64)yh;
    const u64 x2 = (u64)(xh >> 64) + (u64)(xmid >> 64), y2 = (u64)(yh >> 64) + (u64)(ymid >> 64);
    if (x2 != y2) return x2 < y2;
    if ((u64)xmid != (u64)ymid) return (u64)xmid < (u64)ymid;
    return (u64)xl < (u64)yl;
}

bool host_below_threshold(i128 qn_new, i128 qn_old, i64 tw, i64 num, i64 den)
{
    const i128 diff = qn_new - qn_old;
    if (diff < 0) return true;
    const u128 tw2 = (u128)(u64)tw * (u64)tw;
    return host_less_192((u128)diff, (u64)den, tw2, (u64)num);
}

// relative phase test of Algorithm 1 (reading R14): |qn_new - qn_old| * den < num * |qn_old|;
// qn_old = 0 stops only on an unchanged Qn
bool host_below_threshold_rel(i128 qn_new, i128 qn_old, i64 num, i64 den)
{
    const i128 diff = qn_new - qn_old;
    const u128 ad = (u128)(diff < 0 ? -diff : diff), ao = (u128)(qn_old < 0 ? -qn_old : qn_old);
    if (ao == 0) return ad == 0;
    return host_less_192(ad, (u64)den, ao, (u64)num);
}

i128 limbs_to_i128(const i64 v[2]) { return (i128)(((u128)(u64)v[0] << 64) | (u128)(u64)v[1]); }
void i128_to_limbs(i128 x, int64_t out[2])
{
    out[0] = (int64_t)(x >> 64);
    out[1] = (int64_t)(u64)x;
}

double now_ms()
{
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace

struct LevelRec {
    int64_t ncomm = 0;
    i128 qn = 0, qn_init = 0;
    int32_t iters = 0;
    int64_t n = 0, nnz = 0;
    int32_t hit_cap = 0;
    int32_t *d_labels = nullptr;
    const int32_t *h_labels = nullptr;  // pinned host copy made during the run (host_labels)
};

struct TraceRec {
    int32_t level, iter;
    int64_t moved;
    i128 qn;
};

// Pinned host blocks for labels copied during a run (config.host_labels).  A block goes back
// to the pool when the last result using it is destroyed and is reused by later runs; at most
// kKeep bytes stay cached.  Shared by the handle and the label stores, so it outlives a
// handle whose results are still open.
struct PinnedPool {
    std::mutex mu;
    std::vector<std::pair<size_t, void *>> free_blocks;
    size_t cached = 0;
    static constexpr size_t kKeep = (size_t)16 << 30;
    static constexpr size_t kGrain = (size_t)2 << 20;

    // a block of at least `bytes` (its size in *got), or nullptr when none can be pinned
    void *get(size_t bytes, size_t *got)
    {
        {
            std::lock_guard<std::mutex> lock(mu);
            int best = -1;
            for (int i = 0; i < (int)free_blocks.size(); i++) {
                const size_t b = free_blocks[i].first;
                if (b >= bytes && b <= 2 * bytes + kGrain &&
                    (best < 0 || b < free_blocks[best].first))
                    best = i;
            }
            if (best >= 0) {
                const auto blk = free_blocks[best];
                free_blocks.erase(free_blocks.begin() + best);
                cached -= blk.first;
                *got = blk.first;
                return blk.second;
            }
        }
        const size_t sz = (bytes + kGrain - 1) / kGrain * kGrain;
        void *p = nullptr;
        if (cudaMallocHost(&p, sz) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        *got = sz;
        return p;
    }
    void put(void *p, size_t bytes)
    {
        std::lock_guard<std::mutex> lock(mu);
        if (cached + bytes > kKeep) {
            cudaFreeHost(p);
            return;
        }
        free_blocks.push_back({bytes, p});
        cached += bytes;
    }
    ~PinnedPool()
    {
        for (auto &b : free_blocks) cudaFreeHost(b.second);
    }
};

struct louvain_handle {
    louvain_config cfg;
    std::shared_ptr<PinnedPool> pool = std::make_shared<PinnedPool>();
    int device = 0;
    std::string err;
    LaunchCfg lc;
    Scalars *pinned = nullptr;
    void *server = nullptr;  // the open request loop (louvain_serve_open), if any
    // bin thresholds chosen by the autotuner, per (vertex count, entry count) of a graph
    std::vector<std::pair<std::pair<int64_t, int64_t>, std::array<int32_t, 7>>> tuned;
};

// Label arrays of one engine step (every graph that recorded a level in it has its labels
// there); freed with the last result that refers to it.
struct LabelStore {
    std::vector<void *> arrays;
    louvain_free_fn ff = nullptr;
    void *ctx = nullptr;
    int device = 0;
    // pinned host copy of the labels (host_labels), returned to its pool
    std::shared_ptr<PinnedPool> pool;
    void *pinned = nullptr;
    size_t pinned_bytes = 0;
    ~LabelStore()
    {
        cudaSetDevice(device);
        for (void *p : arrays) {
            if (ff) ff(p, ctx, nullptr);
            else cudaFreeAsync(p, nullptr);
        }
        if (pinned) pool->put(pinned, pinned_bytes);
    }
};

struct louvain_result {
    int64_t n0 = 0;
    int batch_index = -1;  // graph index in its batch, -1 for a plain run
    std::vector<std::shared_ptr<LabelStore>> stores;  // label arrays of its levels
    // graph induced after recorded level l (keep_coarse): input of level l + 1
    struct Coarse {
        int64_t n = 0, nnz = 0;
        int32_t wbytes = 4;
        const int64_t *rp = nullptr;
        const int32_t *col = nullptr;
        const void *w = nullptr;
    };
    std::vector<Coarse> coarse;  // indexed by recorded level; n = -1 when none was induced
    int64_t acc_sweeps = 0, acc_cand = 0, acc_kernels = 0;
    // graph sweeps, host-loop sweeps, steps, captures, autotuning trials, tuned-bins cache hit
    int64_t exec_info[6] = {0, 0, 0, 0, 0, 0};
    double acc_alg_bytes = 0.0, acc_coarsen_ms = 0.0, acc_step_ms = 0.0;
    double acc_coarsen_bytes = 0.0;  // algorithmic bytes of the graph inductions
    int64_t acc_inductions = 0;
    int64_t tw = 0;
    int device = 0;
    std::vector<LevelRec> levels;
    mutable std::vector<std::vector<int32_t>> host_labels;
    std::vector<TraceRec> trace;
    int64_t counters[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double times[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // per degree bin; slots kNumBins + b: bin b in the first sweep of each phase
    double bin_time[2 * kNumBins] = {};
    int64_t bin_launches[2 * kNumBins] = {};
    double bin_bytes[2 * kNumBins] = {};
    int64_t bin_rows[2 * kNumBins] = {};
    int64_t bin_entries[2 * kNumBins] = {};
    louvain_free_fn ff = nullptr;
    void *ctx = nullptr;
};

namespace {

int map_err_bits(unsigned bits, std::string &msg)
{
    if (bits & ERRF_ROWPTR) {
        msg = "row_ptr must start at 0 and never decrease";
        return LOUVAIN_ERR_INDEX_RANGE;
    }
    if (bits & ERRF_INDEX) {
        msg = "a column index is outside [0, n)";
        return LOUVAIN_ERR_INDEX_RANGE;
    }
    if (bits & ERRF_WEIGHT) {
        msg = "a weight is below 1";
        return LOUVAIN_ERR_BAD_WEIGHT;
    }
    if (bits & ERRF_DUP) {
        msg = "a row is unsorted or lists a column twice";
        return LOUVAIN_ERR_DUPLICATE_EDGE;
    }
    if (bits & ERRF_ASYM) {
        msg = "the adjacency is not symmetric (A_ij != A_ji)";
        return LOUVAIN_ERR_NOT_SYMMETRIC;
    }
    if (bits & ERRF_OVERFLOW) {
        msg = "a merged edge weight exceeds 2^31 - 1";
        return LOUVAIN_ERR_TOO_LARGE;
    }
    if (bits & ERRF_HASH_FULL) {
        msg = "internal: a hash table overflowed";
        return LOUVAIN_ERR_INTERNAL;
    }
    msg = "internal device check failed";
    return LOUVAIN_ERR_INTERNAL;
}

// ---------------------------------------------------------------------- step engine
//
// The engine holds a set of resident graphs stacked into one block-diagonal CSR (their
// current levels) and advances all of them by one level per step: Algorithm 1's phase for
// every resident graph at once, then renumbering, recording, Algorithm 2's outer test and
// the induction of the next level for the graphs that go on.  Graphs enter at a step
// boundary (all at once for a batch, one by one as they arrive when serving) and leave when
// their own run ends; every graph keeps its own 2W, controller and outer test, so its result
// does not depend on the graphs it shared steps with.

// A graph in the engine.
struct Member {
    louvain_result *res = nullptr;
    int64_t n0 = 0;          // vertices of the input graph
    i64 tw = 0;              // its 2W
    int level = 0;           // index of the level its next phase computes
    i128 qn_prev = 0;        // Qn of its last recorded level
    int64_t nv = 0, nnz = 0; // vertices and entries in the current stacked graph
    int32_t *map = nullptr;  // device int32[n0]: current-level vertex of each input vertex
    int64_t visits = 0;
    double t0 = 0.0;         // when it was handed to the engine (host ms)
    void *tag = nullptr;     // owner of the member (a served request)
    // its rows list every column at most once: known for an induced graph, checked (strictly
    // increasing columns) for an input graph when it joins
    bool rows_checked = false, distinct_rows = false;
};

// Graphs waiting to enter: one CSR holding K graphs (block-diagonal, global column ids,
// int32 weights).  The arrays belong to the caller and must live until the graphs leave.
struct Source {
    int64_t n = 0, nnz = 0;
    const int64_t *rp = nullptr;
    const int32_t *col = nullptr;
    const int32_t *w = nullptr;  // int32, or int64 when wbytes = 8 (a resumed coarse graph)
    int wbytes = 4;
    std::vector<int64_t> vptr, eptr;  // K + 1 each
    std::vector<Member *> members;    // K
};

struct Engine {
    louvain_handle *h;
    cudaStream_t s;
    DevAlloc &A;
    const louvain_config &cfg;
    const LaunchCfg &lc;
    bool batch;  // batch kernels (any number of graphs) or the one-graph kernels
    Scalars *d_sc = nullptr;
    DBuf<Scalars> sc_buf;
    int64_t kernels = 0;

    std::vector<Member *> mem;  // resident graphs in slot order
    std::vector<Source> pending;
    bool need_row_sums = false;

    // current stacked graph (n = 0: none)
    DevGraph G;
    DBuf<int64_t> g_rp;
    DBuf<int32_t> g_col;
    DBuf<unsigned char> g_w;

    // per-vertex state, sized for the largest stacked graph so far
    DBuf<i64> delta, delta_next, deg;
    DBuf<unsigned> deg32;  // 32-bit copy of deg for the candidate scans
    DBuf<int32_t> C, Cnext, size, new_id, new_id2, lists, vg;
    DBuf<int32_t> colorb, pickb;  // colouring variant: colour of every vertex, round picks
    DBuf<int32_t> b_nch, b_chunk_first, b_plog2, b_glog2;
    DBuf<int64_t> b_hoff, b_gcap, b_goff;
    DBuf<u64> b_gloop;
    DBuf<int32_t> scratch32;
    DBuf<int64_t> scratch64;
    DBuf<int32_t> chunk_b, hp_best, hp_sdone, hp_slice_row;
    // induction of multi-chunk communities: pairs per partition, offsets, cursors, the
    // partition's community, pairs per chunk, the pairs grouped by partition
    DBuf<int32_t> c_pcnt, c_pcur, c_partb, c_chm, c_pk, c_mem0;
    DBuf<int64_t> c_poff, c_pscr;
    DBuf<u64> c_pv;
    DBuf<int64_t> hp_soff;
    DBuf<i64> hp_ea;
    DBuf<u64> hp_cnt;
    DBuf<int32_t> hp_hofs, hp_pkeys;  // partitioned aggregation of multi-chunk rows
    DBuf<u64> hp_pvals;
    DBuf<u128> hp_gain;
    DBuf<int32_t> c_csize, c_moff, c_cursor, c_members, c_ccnt, c_tmp_col;
    DBuf<int64_t> c_mpre, c_mrow;
    DBuf<u64> c_tmp_w;
    // per-slot arrays
    DBuf<int64_t> d_gptr, d_base1, d_gnnz, d_off, d_vbase;
    DBuf<int32_t> d_rec, d_keep, d_vf;
    DBuf<u64> d_tw;
    DBuf<unsigned> d_unsorted;
    DBuf<SweepStats> d_stats;
    DBuf<LevelCtl> d_ctls;
    DBuf<int32_t *> d_maps;
    DBuf<i64> tr_moved, tr_qn;
    std::vector<i64> h_tr_moved, h_tr_qn;

    SweepTimers tm;
    cudaEvent_t coarsen_ev[2] = {nullptr, nullptr};
    cudaStream_t cap = nullptr;  // stream the sweep graphs are captured on (never runs work)
    cudaStream_t lab_s = nullptr;  // host_labels: copies of recorded labels to pinned memory
    cudaEvent_t lab_ev = nullptr;
    SweepStreams ss;             // streams the bins of a sweep run on side by side

    Engine(louvain_handle *h_, cudaStream_t s_, DevAlloc &A_, bool batch_,
           const louvain_config &cfg_)
        : h(h_), s(s_), A(A_), cfg(cfg_), lc(h_->lc), batch(batch_)
    {
        sc_buf.reset(&A, 1);
        d_sc = sc_buf.p;
        CK(cudaMemsetAsync(d_sc, 0, sizeof(Scalars), s));
        G.n = 0;
        G.nnz = 0;
        for (int q = 0; q < cfg.sweep_streams && q < 4; q++) {
            CK(cudaStreamCreateWithFlags(&ss.aux[q], cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&ss.join[q], cudaEventDisableTiming));
            ss.k = q + 1;
        }
        if (ss.k) CK(cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming));
        if (cfg.host_labels) {
            CK(cudaStreamCreateWithFlags(&lab_s, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&lab_ev, cudaEventDisableTiming));
        }
        if (cfg.profile) {
            for (auto &e : tm.ev) CK(cudaEventCreate(&e));
            CK(cudaEventCreate(&coarsen_ev[0]));
            CK(cudaEventCreate(&coarsen_ev[1]));
            tm.on = true;
        }
    }
    ~Engine()
    {
        if (tm.on) {
            for (auto &e : tm.ev) cudaEventDestroy(e);
            cudaEventDestroy(coarsen_ev[0]);
            cudaEventDestroy(coarsen_ev[1]);
        }
        for (Member *m : mem) release_map(m);
        if (cap) cudaStreamDestroy(cap);
        for (int q = 0; q < ss.k; q++) {
            cudaStreamDestroy(ss.aux[q]);
            cudaEventDestroy(ss.join[q]);
        }
        if (ss.fork) cudaEventDestroy(ss.fork);
        if (lab_s) {
            cudaStreamSynchronize(lab_s);  // a failed step may leave a copy in flight
            cudaStreamDestroy(lab_s);
            cudaEventDestroy(lab_ev);
        }
    }
    Engine(const Engine &) = delete;
    Engine &operator=(const Engine &) = delete;

    bool idle() const { return mem.empty() && pending.empty(); }

    void check_launches()
    {
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && launch_site()) e = cudaErrorInvalidValue;
        if (e != cudaSuccess) {
            std::string where = launch_site() ? launch_site() : "a launch";
            launch_site() = nullptr;
            throw LvErr{e == cudaErrorMemoryAllocation ? LOUVAIN_ERR_OOM : LOUVAIN_ERR_CUDA,
                        where + ": " + cudaGetErrorString(e)};
        }
    }

    void sync_scalars()
    {
        check_launches();
        CK(cudaMemcpyAsync(h->pinned, d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (h->pinned->err) {
            std::string msg;
            int code = map_err_bits(h->pinned->err, msg);
            throw LvErr{code, msg};
        }
    }

    template <typename T>
    T read_one(const T *dptr)
    {
        T v;
        CK(cudaMemcpyAsync(&h->pinned->tail[0], dptr, sizeof(T), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        memcpy(&v, &h->pinned->tail[0], sizeof(T));
        return v;
    }

    template <typename T>
    void ensure(DBuf<T> &b, size_t count)
    {
        if (!b.p || b.n < count) b.reset(&A, count);
    }

    template <typename T>
    void upload(DBuf<T> &b, const T *src, size_t count)
    {
        ensure(b, count);
        if (count) CK(cudaMemcpyAsync(b.p, src, sizeof(T) * count, cudaMemcpyHostToDevice, s));
    }

    void release_map(Member *m)
    {
        if (m->map) A.put(m->map);
        m->map = nullptr;
    }

    // Adds the graphs of a source; they enter at the next step.  Empty graphs have no
    // level to compute and are finished at once (returned in `done`).
    void add(Source &&src, std::vector<Member *> &done)
    {
        const size_t K = src.members.size();
        for (size_t k = 0; k < K; k++) {
            Member *m = src.members[k];
            m->n0 = src.vptr[k + 1] - src.vptr[k];
            m->nv = m->n0;
            m->nnz = src.eptr[k + 1] - src.eptr[k];
            m->res->n0 = m->n0;
            if (m->n0 == 0) done.push_back(m);
        }
        if (src.n > 0) pending.push_back(std::move(src));
    }

    Bins make_proto(bool narrow_sums) const;
    Bins make_bins(const DevGraph &gr, const Bins &pr, const int32_t *vgp = nullptr,
                   const LevelCtl *gctl = nullptr, const int32_t *color = nullptr,
                   int32_t cls = 0);
    int color_level(int64_t n);
    void colored_phase(const PhaseState &st, const Bins &proto, i64 TW, bool wide, bool narrow,
                       SweepStats *st_dev, BatchCtx &bc, SweepTimers &tm, int &sweeps,
                       double *t_kernel, int64_t *launches_kernel,
                       const std::function<void(const Bins &, int)> &account);
    void prep_huge(Bins &b, bool coarsen_side, int64_t k_comm, CoarsenBufs *cbp);
    void join();
    void step(std::vector<Member *> &retired);
};

// One phase's sweep loop as a CUDA graph: a while node whose body is the sweep over all
// bins, the controllers, the apply and the loop condition (k_loop_ctl).  Built per bin
// layout (the launch shapes depend on it); any failure to capture or instantiate leaves
// the host loop in charge.
struct SweepGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int per_sweep = 0;

    void reset()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    ~SweepGraph() { reset(); }

    // LOUVAIN_GRAPH_DIAG=1 in the environment reports why a capture fell back
    static bool fail(const char *what, cudaError_t e)
    {
        static const bool diag = getenv("LOUVAIN_GRAPH_DIAG") != nullptr;
        if (diag) fprintf(stderr, "sweep graph: %s failed: %s\n", what, cudaGetErrorString(e));
        cudaGetLastError();
        return false;
    }

    bool build(Engine &E, const DevGraph &G, const PhaseState &st, const Bins &bins, i64 TW,
               bool wide, bool narrow, SweepStats *st_dev, LevelCtl *ctl_dev, int M,
               const BatchCtx &bc, int &out_per_sweep)
    {
        reset();
        // capture on a stream of the engine's own: the caller's stream may be the legacy
        // default stream, which cannot be captured; the graph is launched on the caller's
        cudaError_t e;
        if (!E.cap && (e = cudaStreamCreateWithFlags(&E.cap, cudaStreamNonBlocking)) != cudaSuccess) {
            E.cap = nullptr;
            return fail("stream create", e);
        }
        cudaStream_t s = E.cap;
        cudaGraphConditionalHandle handle;
        cudaGraphNode_t node;
        cudaGraphNodeParams cp = {};
        if ((e = cudaGraphCreate(&graph, 0)) != cudaSuccess) {
            reset();
            return fail("graph create", e);
        }
        if ((e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault)) !=
            cudaSuccess) {
            reset();
            return fail("conditional handle", e);
        }
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if ((e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp)) != cudaSuccess) {
            reset();
            return fail("conditional node", e);
        }
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
            reset();
            return fail("begin capture", e);
        }
        int k = launch_sweep(G, st, bins, TW, wide, narrow, false, st_dev, &E.d_sc->err, s, E.lc,
                             nullptr, bc);
        k += launch_decide(st_dev, ctl_dev, M, E.tr_moved.p, E.tr_qn.p, &E.d_sc->cand_total[0],
                           &E.d_sc->ndone, s);
        k += launch_apply(G.n, st, ctl_dev, bc.vg, s, E.lc);
        k += launch_loop_ctl(handle, &E.d_sc->loop, &E.d_sc->ndone, M, s);
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(s, &captured);
        const char *site = launch_site();
        launch_site() = nullptr;
        if (e != cudaSuccess) {
            reset();
            return fail("end capture", e);
        }
        if (site) {
            reset();
            return fail(site, cudaErrorInvalidValue);
        }
        if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) {
            exec = nullptr;
            reset();
            return fail("instantiate", e);
        }
        per_sweep = k - 1;  // the loop-condition kernel is not a method step
        out_per_sweep = per_sweep;
        return true;
    }
};

Bins Engine::make_proto(bool narrow_sums) const
{
    // bin thresholds: every table must fit shared memory with the chosen sum width; the
    // cluster bins hold rows up to CL times the bin-5 bound (CL CTAs, bin-5 table each);
    // cluster sizes that cannot be resident are left empty.
    Bins pr;
    const int32_t thr[6] = {cfg.bin_small, cfg.bin_mid1, cfg.bin_mid2,
                            cfg.bin_cta1,  cfg.bin_cta2, cfg.bin_cta3};
    for (int t = 0; t < 6; t++) pr.upper[t] = thr[t];
    if (!narrow_sums && pr.upper[5] > 6144) {
        pr.upper[5] = 6144;
        for (int t = 4; t >= 0; t--)
            if (pr.upper[t] > pr.upper[t + 1]) pr.upper[t] = pr.upper[t + 1];
    }
    for (int t = 0; t < 4; t++) {
        const int64_t cl = (int64_t)kBinSpec[6 + t].cluster;
        pr.upper[6 + t] = lc.cluster_ok[t] ? pr.upper[5] * cl : pr.upper[5 + t];
    }
    pr.chunk = cfg.chunk_entries;
    pr.part_keys = cfg.part_keys;
    return pr;
}

// degree bins of graph gr: count, then fill the list grouped by bin (rows of graphs whose
// phase stopped are left out when gctl is given)
Bins Engine::make_bins(const DevGraph &gr, const Bins &pr, const int32_t *vgp,
                       const LevelCtl *gctl, const int32_t *color, int32_t cls)
{
    Bins bins = pr;
    bins.list = lists.p;
    bins.counts = &d_sc->bin_counts[0];
    bins.nch = b_nch.p;
    bins.chunk_first = b_chunk_first.p;
    bins.gloop = b_gloop.p;
    bins.plog2 = b_plog2.p;
    bins.hoff = b_hoff.p;
    kernels += launch_bin_count(gr, bins, s, lc, vgp, gctl, color, cls);
    sync_scalars();
    bins.off[0] = bins.off[1] = 0;
    for (int b = 0; b < kNumBins; b++) {
        bins.nlist[b] = h->pinned->bin_counts[b];
        memcpy(&bins.entries[b], &h->pinned->bin_counts[16 + 2 * b], sizeof(int64_t));
        if (b >= 1) bins.off[b + 1] = bins.off[b] + bins.nlist[b];
    }
    kernels += launch_bin_fill(gr, bins, s, lc, vgp, gctl, color, cls);
    return bins;
}

// Colouring variant: Jones-Plassmann rounds over the level's graph into colorb; returns the
// number of colours.  Every round colours at least the highest-priority uncoloured vertex,
// so n rounds always suffice.
int Engine::color_level(int64_t n)
{
    ensure(colorb, n);
    ensure(pickb, n);
    CK(cudaMemsetAsync(colorb.p, 0xFF, sizeof(int32_t) * (size_t)n, s));  // -1: uncoloured
    CK(cudaMemsetAsync(&d_sc->ncolors, 0, sizeof(int32_t), s));
    for (int64_t round = 0;; round++) {
        kernels += launch_color_pick(G, colorb.p, pickb.p, &d_sc->ccounts2[0], s, lc);
        kernels += launch_color_assign(G, colorb.p, pickb.p, &d_sc->ncolors, s, lc);
        sync_scalars();
        const u64 unc = h->pinned->ccounts2[0], picked = h->pinned->ccounts2[1];
        if (unc == picked) break;
        if (picked == 0 || round > n) throw LvErr{LOUVAIN_ERR_INTERNAL, "colouring did not finish"};
    }
    return h->pinned->ncolors;
}

// Colouring variant of one phase (one graph): every sweep takes the colour classes in
// increasing colour; the class's vertices decide on the current state (the sweep kernels
// over the class's rows), their moves are applied, then the next class.  After each sweep the
// exact Qn of the new state decides the stop as without colouring (nothing moved, the theta
// test, the sweep cap).  The device controller, trace and candidate totals are left as the
// synchronous phase leaves them.
void Engine::colored_phase(const PhaseState &st, const Bins &proto, i64 TW, bool wide,
                           bool narrow, SweepStats *st_dev, BatchCtx &bc, SweepTimers &tm,
                           int &sweeps, double *t_kernel, int64_t *launches_kernel,
                           const std::function<void(const Bins &, int)> &account)
{
    const int64_t n = G.n;
    const int K = color_level(n);
    CK(cudaMemsetAsync(st_dev, 0, sizeof(SweepStats), s));
    kernels += launch_qn_one(G, st, st_dev, &d_sc->ctl, s, lc);
    sync_scalars();
    const i128 qn_init = limbs_to_i128(h->pinned->ctl.qn_final);
    i128 qn_prev = qn_init, qn = qn_init;
    std::vector<i64> tr_m, tr_q;
    u64 cand[16] = {};
    int iters = 0;
    bool cap = false;
    for (;;) {
        CK(cudaMemsetAsync(&d_sc->cmoved, 0, sizeof(u64), s));
        for (int c = 0; c < K; c++) {
            PhaseState sc = st;
            sc.color = colorb.p;
            sc.cls = c;
            Bins cb = make_bins(G, proto, nullptr, nullptr, colorb.p, c);
            prep_huge(cb, false, 0, nullptr);
            kernels += launch_sweep(G, sc, cb, TW, wide, narrow, false, st_dev, &d_sc->err, s,
                                    lc, &tm, bc);
            kernels += launch_apply_class(n, sc, &d_sc->cmoved, s, lc);
            account(cb, 0);
            for (int b = 0; b < kNumBins; b++)
                launches_kernel[b] +=
                    b == 0 ? 1 : (b == kChunkedBin ? cb.nchunks > 0 : cb.nlist[b] > 0);
            if (tm.on) {
                CK(cudaStreamSynchronize(s));
                for (int b = 0; b < kNumBins; b++) {
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, tm.ev[2 * b], tm.ev[2 * b + 1]));
                    t_kernel[b] += ms;
                }
            }
        }
        sync_scalars();
        const u64 moved = h->pinned->cmoved;
        for (int b = 0; b < 16; b++) cand[b] += h->pinned->st.cand[b];
        // exact Qn of the state after the sweep (the sweep kernels' statistics are not used)
        CK(cudaMemsetAsync(st_dev, 0, sizeof(SweepStats), s));
        kernels += launch_qn_one(G, st, st_dev, &d_sc->ctl, s, lc);
        sync_scalars();
        qn = limbs_to_i128(h->pinned->ctl.qn_final);
        iters++;
        sweeps++;
        tr_m.push_back((i64)moved);
        tr_q.push_back((i64)(qn >> 64));
        tr_q.push_back((i64)(u64)qn);
        if (moved == 0) break;
        const bool below = cfg.threshold_mode == 1
                               ? host_below_threshold_rel(qn, qn_prev, cfg.theta_num, cfg.theta_den)
                               : host_below_threshold(qn, qn_prev, TW, cfg.theta_num, cfg.theta_den);
        if (below) break;
        if (iters >= cfg.max_iters) {
            cap = true;
            break;
        }
        qn_prev = qn;
    }
    // leave the controller, trace and candidate totals where the synchronous phase leaves them
    LevelCtl cc = h->pinned->ctl;
    cc.iters = iters;
    cc.sweep = iters;
    cc.hit_cap = cap;
    cc.done = 1;
    cc.qn_init[0] = (i64)(qn_init >> 64);
    cc.qn_init[1] = (i64)(u64)qn_init;
    cc.qn_final[0] = (i64)(qn >> 64);
    cc.qn_final[1] = (i64)(u64)qn;
    cc.qn_prev[0] = (i64)(qn_prev >> 64);
    cc.qn_prev[1] = (i64)(u64)qn_prev;
    h->pinned->ctl = cc;
    CK(cudaMemcpyAsync(&d_sc->ctl, &h->pinned->ctl, sizeof(LevelCtl), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(tr_moved.p, tr_m.data(), sizeof(i64) * tr_m.size(), cudaMemcpyHostToDevice,
                       s));
    CK(cudaMemcpyAsync(tr_qn.p, tr_q.data(), sizeof(i64) * tr_q.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(&d_sc->cand_total[0], cand, sizeof(cand), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
}

// chunk lists and global tables of the chunked bin (after its size is known)
void Engine::prep_huge(Bins &b, bool coarsen_side, int64_t k_comm, CoarsenBufs *cbp)
{
    b.nchunks = 0;
    b.nslices = 0;
    b.gslots = 0;
    const int nb = b.nlist[kChunkedBin];
    if (nb == 0) return;
    if (coarsen_side) kernels += launch_coarsen_bigprep(k_comm, *cbp, b, s, lc);
    else kernels += launch_big_prep(G, b, scratch64.p, scratch32.p, s, lc);
    b.nchunks = read_one(b_chunk_first.p + nb);
    chunk_b.reset(&A, b.nchunks);
    b.chunk_b = chunk_b.p;
    kernels += launch_big_fill(b, s, lc);
    if (coarsen_side) {  // partitioned merge of the multi-chunk communities
        const int64_t np = read_one(b_goff.p + nb);
        b.gslots = np;
        if (np > 0) {
            ensure(c_pcnt, (size_t)np + 1);
            ensure(c_poff, (size_t)np + 1);
            ensure(c_pcur, (size_t)np);
            ensure(c_partb, (size_t)np);
            ensure(c_pscr, (size_t)scan_scratch_elems(np + 1) + 64);
            // a chunk's distinct pairs never outnumber its entries
            ensure(c_pk, (size_t)b.nchunks * b.chunk);
            ensure(c_pv, (size_t)b.nchunks * b.chunk);  // 8 bytes covers both sum widths
            CK(cudaMemsetAsync(c_pcnt.p, 0, sizeof(int32_t) * (np + 1), s));
            CK(cudaMemsetAsync(c_pcur.p, 0, sizeof(int32_t) * np, s));
        }
        ensure(c_chm, (size_t)std::max(b.nchunks, 1));
        ensure(c_mem0, (size_t)std::max(b.nchunks, 1));
        b.cmem0 = c_mem0.p;
        b.cpcnt = c_pcnt.p;
        b.cpoff = c_poff.p;
        b.cpcur = c_pcur.p;
        b.cpartb = c_partb.p;
        b.cchm = c_chm.p;
        b.cpk = c_pk.p;
        b.cpv = c_pv.p;
        b.cpscr = c_pscr.p;
        if (np > 0) kernels += launch_coarsen_partfill(b, s, lc);
        return;
    }
    if (b.nchunks > nb) {  // some rows span several chunks
        ensure(hp_soff, (size_t)nb + 1);
        b.soff = hp_soff.p;
        kernels += launch_huge_slices(b, scratch64.p, s);
        b.nslices = read_one(hp_soff.p + nb);
        ensure(hp_slice_row, b.nslices);
        b.slice_row = hp_slice_row.p;
        kernels += launch_huge_slice_fill(b, s, lc);
        // partials: one per partition (table sweeps), one per chunk (first sweeps)
        const int64_t np = std::max<int64_t>(b.nslices, b.nchunks);
        ensure(hp_gain, np);
        ensure(hp_best, np);
        ensure(hp_ea, np);
        ensure(hp_cnt, np);
        ensure(hp_sdone, nb);
        // each chunk's distinct (key, sum) pairs grouped by partition, with the offsets
        ensure(hp_hofs, std::max<int64_t>(1, read_one(b_hoff.p + nb)));
        ensure(hp_pkeys, (int64_t)b.nchunks * b.chunk);
        ensure(hp_pvals, (int64_t)b.nchunks * b.chunk);
        CK(cudaMemsetAsync(hp_sdone.p, 0, sizeof(int32_t) * nb, s));
    }
    b.pgain = hp_gain.p;
    b.pbest = hp_best.p;
    b.pea = hp_ea.p;
    b.pcnt = hp_cnt.p;
    b.sdone = hp_sdone.p;
    b.hofs = hp_hofs.p;
    b.pkeys = hp_pkeys.p;
    b.pvals = hp_pvals.p;
    CK(cudaMemsetAsync(b_gloop.p, 0, sizeof(u64) * nb, s));
}

// Stacks the waiting graphs after the resident ones: the current graph keeps its rows, each
// source's rows follow with shifted columns; a lone source on an empty engine is used in
// place.  New graphs start at level 0 with their own vertices as their map.
void Engine::join()
{
    const int64_t n_cont = G.n, nnz_cont = G.nnz;
    int64_t n_add = 0, nnz_add = 0;
    for (const Source &src : pending) {
        n_add += src.n;
        nnz_add += src.nnz;
    }
    const int64_t n = n_cont + n_add, nnz = nnz_cont + nnz_add;
    if (n > INT32_MAX) throw LvErr{LOUVAIN_ERR_TOO_LARGE, "stacked vertex count above 2^31 - 1"};
    std::vector<Member *> fresh;
    std::vector<int64_t> vbase;
    for (const Source &src : pending)
        if (src.wbytes != 4 && !(n_cont == 0 && pending.size() == 1))
            throw LvErr{LOUVAIN_ERR_INVALID_ARG, "64-bit weights enter only alone"};
    if (n_cont == 0 && pending.size() == 1) {
        const Source &src = pending[0];
        g_rp.release();
        g_col.release();
        g_w.release();
        G.n = src.n;
        G.nnz = src.nnz;
        G.rp = src.rp;
        G.col = src.col;
        G.w = src.w;
        G.wbytes = src.wbytes;
    } else {
        const int wb = n_cont > 0 ? G.wbytes : 4;
        DBuf<int64_t> j_rp;
        DBuf<int32_t> j_col;
        DBuf<unsigned char> j_w;
        j_rp.reset(&A, (size_t)n + 1);
        j_col.reset(&A, (size_t)nnz);
        j_w.reset(&A, (size_t)nnz * wb);
        if (n_cont > 0) {
            CK(cudaMemcpyAsync(j_rp.p, G.rp, sizeof(int64_t) * n_cont, cudaMemcpyDeviceToDevice, s));
            if (nnz_cont) {
                CK(cudaMemcpyAsync(j_col.p, G.col, sizeof(int32_t) * nnz_cont,
                                   cudaMemcpyDeviceToDevice, s));
                CK(cudaMemcpyAsync(j_w.p, G.w, (size_t)wb * nnz_cont, cudaMemcpyDeviceToDevice, s));
            }
        }
        int64_t v_base = n_cont, e_base = nnz_cont;
        for (const Source &src : pending) {
            kernels += launch_append_rows(src.n, src.nnz, src.rp, src.col, src.w, v_base, e_base,
                                          j_rp.p, j_col.p, j_w.p, wb, s, lc);
            v_base += src.n;
            e_base += src.nnz;
        }
        h->pinned->tail[0] = 0;
        memcpy(&h->pinned->tail[0], &nnz, sizeof(nnz));
        CK(cudaMemcpyAsync(j_rp.p + n, &h->pinned->tail[0], sizeof(int64_t),
                           cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));  // the pinned word is reused below
        g_rp.swap(j_rp);
        g_col.swap(j_col);
        g_w.swap(j_w);
        G.n = n;
        G.nnz = nnz;
        G.rp = g_rp.p;
        G.col = g_col.p;
        G.w = g_w.p;
        G.wbytes = wb;
    }
    int64_t v_base = n_cont;
    for (Source &src : pending) {
        for (size_t k = 0; k < src.members.size(); k++) {
            Member *m = src.members[k];
            if (m->n0 == 0) continue;
            m->map = (int32_t *)A.get(sizeof(int32_t) * (size_t)m->n0);
            fresh.push_back(m);  // at its own level (0, or the level a resumed run starts at)
            vbase.push_back(v_base + src.vptr[k]);
            mem.push_back(m);
        }
        v_base += src.n;
    }
    pending.clear();
    // every input vertex of a new graph is its own level-0 vertex
    const int F = (int)fresh.size();
    std::vector<int64_t> off(F + 1, 0);
    std::vector<int32_t *> maps(F);
    for (int f = 0; f < F; f++) {
        off[f + 1] = off[f] + fresh[f]->n0;
        maps[f] = fresh[f]->map;
    }
    upload(d_off, off.data(), F + 1);
    upload(d_vbase, vbase.data(), F);
    upload(d_maps, maps.data(), F);
    kernels += launch_map_init(off[F], F, d_off.p, d_maps.p, d_vbase.p, s, lc);
    need_row_sums = true;

    // per-vertex buffers for the stacked graph (Theorem 1: later levels never grow)
    ensure(delta, n);
    ensure(delta_next, n);
    ensure(deg, n);
    ensure(C, n);
    ensure(Cnext, n);
    ensure(size, n);
    ensure(new_id, (size_t)n + 1);
    ensure(lists, n);
    ensure(b_nch, n);
    ensure(b_chunk_first, (size_t)n + 1);

    ensure(b_plog2, n);
    ensure(b_glog2, n);
    ensure(b_gcap, n);
    ensure(b_goff, (size_t)n + 1);
    ensure(b_hoff, (size_t)n + 1);
    ensure(b_gloop, n);
    const int64_t scratch_n = scan_scratch_elems(n + 1) + 64;
    ensure(scratch32, scratch_n);
    ensure(scratch64, scratch_n);
    if (batch) {
        ensure(vg, n);
        ensure(new_id2, (size_t)n + 1);
    }
    CK(cudaStreamSynchronize(s));  // host arrays above are uploaded before they go
}

void Engine::step(std::vector<Member *> &retired)
{
    ProcRange proc("init");
    const double wall0 = now_ms();
    const int64_t k_start = kernels;
    if (!pending.empty()) join();
    if (mem.empty()) return;
    const int M = (int)mem.size();
    const int64_t n = G.n;
    if (!batch && M != 1) throw LvErr{LOUVAIN_ERR_INTERNAL, "one-graph engine with several graphs"};

    // slot offsets of the stacked graph
    std::vector<int64_t> h_gptr(M + 1, 0), h_gnnz(M + 1, 0);
    for (int m = 0; m < M; m++) {
        h_gptr[m + 1] = h_gptr[m] + mem[m]->nv;
        h_gnnz[m + 1] = h_gnnz[m] + mem[m]->nnz;
    }
    if (h_gptr[M] != n || h_gnnz[M] != G.nnz)
        throw LvErr{LOUVAIN_ERR_INTERNAL, "graph offsets out of step with the stacked graph"};
    if (batch) {
        upload(d_gptr, h_gptr.data(), M + 1);
        kernels += launch_graph_ids(n, d_gptr.p, M, vg.p, s, lc);
        ensure(d_tw, M);
        ensure(d_stats, M);
        ensure(d_ctls, M);
        ensure(d_base1, M + 1);
        ensure(d_gnnz, M + 1);
        CK(cudaMemsetAsync(d_stats.p, 0, sizeof(SweepStats) * M, s));
    }
    const int32_t *vgp = batch ? vg.p : nullptr;

    // weighted degrees and 2W of every graph (Sec. 2), with the input checks, when graphs
    // joined; otherwise delta comes from the last induction (it is preserved)
    Bins bins0;
    bool have_bins0 = false;
    if (need_row_sums) {
        bins0 = make_bins(G, make_proto(true));
        have_bins0 = true;
        if (batch) {
            ensure(d_unsorted, M);
            CK(cudaMemsetAsync(d_tw.p, 0, sizeof(u64) * M, s));
            CK(cudaMemsetAsync(d_unsorted.p, 0, sizeof(unsigned) * M, s));
        } else {
            CK(cudaMemsetAsync(&d_sc->tw, 0, sizeof(u64), s));
            CK(cudaMemsetAsync(&d_sc->unsorted, 0, sizeof(unsigned), s));
        }
        kernels += launch_row_sums(G, bins0, vgp, batch ? d_gptr.p : nullptr, delta.p,
                                   batch ? d_tw.p : &d_sc->tw,
                                   batch ? d_unsorted.p : &d_sc->unsorted, &d_sc->err, s, lc);
        if (cfg.checks >= 2) kernels += launch_check_symmetry(G, &d_sc->err, s, lc);
        sync_scalars();
        std::vector<u64> tws(M);
        std::vector<unsigned> uns(M);
        if (batch) {
            CK(cudaMemcpyAsync(tws.data(), d_tw.p, sizeof(u64) * M, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(uns.data(), d_unsorted.p, sizeof(unsigned) * M,
                               cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        } else {
            tws[0] = h->pinned->tw;
            uns[0] = h->pinned->unsorted;
        }
        for (int m = 0; m < M; m++) {  // graphs that joined: their rows as given
            if (mem[m]->rows_checked) continue;
            mem[m]->rows_checked = true;
            mem[m]->distinct_rows = uns[m] == 0;
        }
        for (int m = 0; m < M; m++) {
            if (tws[m] > ((u64)1 << 62))
                throw LvErr{LOUVAIN_ERR_TOO_LARGE, "sum of weights above 2^62"};
            mem[m]->tw = (i64)tws[m];
            mem[m]->res->tw = (i64)tws[m];
        }
        need_row_sums = false;
    } else {
        delta.swap(delta_next);
    }
    u64 tw_max = 0;
    std::vector<i64> h_tw(M);
    for (int m = 0; m < M; m++) {
        h_tw[m] = mem[m]->tw;
        if ((u64)h_tw[m] > tw_max) tw_max = (u64)h_tw[m];
    }
    if (batch) upload(d_tw, (const u64 *)h_tw.data(), M);
    // Exact widths of the level's sweeps from its largest weighted degree: a table sum
    // e_{i->c} never exceeds delta_i, so 32-bit sums are exact when every delta_i < 2^32;
    // a gain of vertex i is at most 2W * delta_i in magnitude (both of its products are),
    // so int64 gains are exact when max delta * 2W <= 2^62, else int128.  The induction's
    // widths follow the largest community degree (below).
    kernels += launch_max_delta(delta.p, n, &d_sc->dmax, s, lc);
    const u64 dmax = read_one(&d_sc->dmax);
    const bool wide = cfg.force_int128 || (u128)dmax * tw_max > ((u128)1 << 62);
    const bool narrow = !cfg.wide_sums && dmax < ((u64)1 << 32);
    const i64 TW = h_tw[0];  // one graph: its 2W (a batch reads 2W per graph on the device)

    PhaseState st;
    st.C = C.p;
    st.Cnext = Cnext.p;
    st.deg = deg.p;
    st.size = size.p;
    st.delta = delta.p;
    ensure(deg32, n);
    st.deg32 = deg32.p;
    st.deg32_bad = &d_sc->deg32_bad;
    CK(cudaMemsetAsync(&d_sc->deg32_bad, 0, sizeof(unsigned), s));
    kernels += launch_init_state(n, st, s, lc);
    // vertex following: level 0 of each graph (every level with vf_all_levels)
    if (cfg.vertex_following) {
        if (batch) {
            std::vector<int32_t> vf(M);
            bool any = false;
            for (int m = 0; m < M; m++) {
                vf[m] = mem[m]->level == 0 || cfg.vf_all_levels;
                any = any || vf[m];
            }
            if (any) {
                upload(d_vf, vf.data(), M);
                kernels += launch_vertex_following(G, st, s, lc, vgp, d_vf.p);
            }
        } else if (mem[0]->level == 0 || cfg.vf_all_levels) {
            kernels += launch_vertex_following(G, st, s, lc);
        }
    }

    // degree bins (the row-sum bins are reused when they were made with these thresholds)
    const Bins proto = make_proto(narrow);
    Bins bins;
    if (have_bins0 && narrow) {
        bins = bins0;
    } else {
        bins = make_bins(G, proto);
    }
    prep_huge(bins, false, 0, nullptr);

    // phase controllers
    std::vector<LevelCtl> h_ctl(M);
    for (int m = 0; m < M; m++) {
        LevelCtl &c = h_ctl[m];
        memset(&c, 0, sizeof(c));
        c.tw = h_tw[m];
        c.theta_num = cfg.theta_num;
        c.theta_den = cfg.theta_den;
        c.max_iters = cfg.max_iters;
        c.rel = cfg.threshold_mode == 1;
    }
    LevelCtl *ctl_dev = batch ? d_ctls.p : &d_sc->ctl;
    SweepStats *st_dev = batch ? d_stats.p : &d_sc->st;
    if (batch) {
        CK(cudaMemcpyAsync(d_ctls.p, h_ctl.data(), sizeof(LevelCtl) * M, cudaMemcpyHostToDevice,
                           s));
    } else {
        h->pinned->ctl = h_ctl[0];
        CK(cudaMemcpyAsync(&d_sc->ctl, &h->pinned->ctl, sizeof(LevelCtl), cudaMemcpyHostToDevice,
                           s));
        CK(cudaMemsetAsync(&d_sc->st, 0, sizeof(SweepStats), s));
    }
    h->pinned->ndone = 0;
    CK(cudaMemcpyAsync(&d_sc->ndone, &h->pinned->ndone, sizeof(int32_t), cudaMemcpyHostToDevice,
                       s));
    CK(cudaMemsetAsync(&d_sc->cand_total[0], 0, sizeof(u64) * 16, s));
    const int tcap = cfg.max_iters + 1;
    ensure(tr_moved, (size_t)tcap * M);
    ensure(tr_qn, 2 * (size_t)tcap * M);
    BatchCtx bc;
    bc.ss = ss.k ? &ss : nullptr;
    if (batch) {
        bc.vg = vg.p;
        bc.gtw = (const i64 *)d_tw.p;
        bc.gctl = d_ctls.p;
    }

    proc.phase("onelevel");
    // sweeps (Algorithm 1); one host read of the controllers' count per sweep
    // per bin; slots kNumBins + b: bin b in the first sweep of the phase
    double t_kernel[2 * kNumBins] = {};
    int64_t launches_kernel[2 * kNumBins] = {};
    double bytes_kernel[2 * kNumBins] = {};
    int64_t rows_kernel[2 * kNumBins] = {}, entries_kernel[2 * kNumBins] = {};
    double alg_bytes = 0.0;
    u64 cand_all = 0;
    auto account_sweep = [&](const Bins &bb, int slot0) {  // algorithmic bytes (louvain.h)
        const double per_entry = 8.0 + (double)G.wbytes;
        for (int b = 0; b < kNumBins; b++) {
            double kb = (double)bb.entries[b] * per_entry;
            kb += b == 0 ? (double)n * 16.0 + (double)bb.nlist[0] * 24.0
                         : (double)bb.nlist[b] * 36.0;
            bytes_kernel[slot0 + b] += kb;
            alg_bytes += kb;
            rows_kernel[slot0 + b] += b == 0 ? n : bb.nlist[b];
            entries_kernel[slot0 + b] += bb.entries[b];
        }
    };
    // The first sweep of the phase scores row entries without tables when every graph's
    // rows list each column at most once: the phase starts from singletons (and vertex
    // following), so a row's candidates other than its own community are then distinct.
    bool first = true;
    for (int m = 0; m < M; m++) first = first && mem[m]->distinct_rows;
    bool had_first = false;
    u64 cand_first[kNumBins] = {};
    int sweeps = 0, graph_sweeps = 0, captures = 0;
    int ndone_binned = 0, ndone = 0;
    // the sweeps run either as a CUDA graph whose while node repeats sweep, controllers,
    // apply and loop condition on the device, or (profiling, or no graph support) with one
    // host round trip per sweep
    bool use_graph = cfg.cuda_graphs && !tm.on;
    SweepGraph sg;
    if (cfg.coloring) {
        colored_phase(st, proto, TW, wide, narrow, st_dev, bc, tm, sweeps, t_kernel,
                      launches_kernel, account_sweep);
        ndone = M;
    }
    for (; !cfg.coloring;) {
        int ran = 0, per_sweep = 0;
        const bool fs = first;  // this round is the table-free first sweep
        first = false;
        if (use_graph && !fs && !sg.exec) {
            if (sg.build(*this, G, st, bins, TW, wide, narrow, st_dev, ctl_dev, M, bc, per_sweep))
                captures++;
            else
                use_graph = false;
        }
        if (use_graph && !fs) {
            LoopCtl &lp = h->pinned->loop;
            lp.iters = 0;
            lp.nd0 = ndone;
            lp.quota = batch ? std::max(1, (M - ndone) / 4) : 1;
            lp.cap = cfg.max_iters + 3 - sweeps;
            CK(cudaMemcpyAsync(&d_sc->loop, &lp, sizeof(LoopCtl), cudaMemcpyHostToDevice, s));
            CK(cudaGraphLaunch(sg.exec, s));
            sync_scalars();
            ran = h->pinned->loop.iters;
            per_sweep = sg.per_sweep;
            graph_sweeps += ran;
        } else {
            per_sweep = launch_sweep(G, st, bins, TW, wide, narrow, fs, st_dev, &d_sc->err, s,
                                     lc, &tm, bc);
            per_sweep += launch_decide(st_dev, ctl_dev, M, tr_moved.p, tr_qn.p,
                                       &d_sc->cand_total[0], &d_sc->ndone, s);
            per_sweep += launch_apply(n, st, ctl_dev, bc.vg, s, lc);
            sync_scalars();
            ran = 1;
        }
        kernels += (int64_t)per_sweep * ran;
        sweeps += ran;
        const int slot0 = fs ? kNumBins : 0;
        for (int r = 0; r < ran; r++) account_sweep(bins, slot0);
        for (int b = 0; b < kNumBins; b++) {
            if (tm.on) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, tm.ev[2 * b], tm.ev[2 * b + 1]));
                t_kernel[slot0 + b] += ms;
            }
            launches_kernel[slot0 + b] +=
                ran * (b == 0 ? 1 : (b == kChunkedBin ? bins.nchunks > 0 : bins.nlist[b] > 0));
        }
        if (fs) {  // candidates of the first sweep (the totals were zeroed at phase start)
            had_first = true;
            for (int b = 0; b < kNumBins; b++) cand_first[b] = h->pinned->cand_total[b];
        }
        ndone = h->pinned->ndone;
        if (ndone >= M) break;
        if (sweeps > cfg.max_iters + 2 || ran < 1)
            throw LvErr{LOUVAIN_ERR_INTERNAL, "phase controller did not stop"};
        if (batch && ndone > ndone_binned) {
            // some graphs stopped: bin again without their rows
            bins = make_bins(G, proto, vg.p, d_ctls.p);
            prep_huge(bins, false, 0, nullptr);
            ndone_binned = ndone;
            sg.reset();
        }
    }
    sg.reset();
    if (cfg.post_merge) {  // Sec. 5.1.2: after the phase, before renumbering
        kernels += launch_post_merge(G, st, vgp, batch ? (const i64 *)d_tw.p : nullptr, TW, wide,
                                     st_dev, ctl_dev, M, s, lc);
        sync_scalars();
    }
    if (batch) {
        CK(cudaMemcpyAsync(h_ctl.data(), d_ctls.p, sizeof(LevelCtl) * M, cudaMemcpyDeviceToHost,
                           s));
        CK(cudaStreamSynchronize(s));
    } else {
        h_ctl[0] = h->pinned->ctl;
    }
    for (int b = 0; b < kNumBins; b++) {  // candidate reads, 8 bytes each
        const u64 cb = h->pinned->cand_total[b];
        const u64 cf = had_first ? cand_first[b] : 0;
        bytes_kernel[b] += 8.0 * (double)(cb - cf);
        bytes_kernel[kNumBins + b] += 8.0 * (double)cf;
        alg_bytes += 8.0 * (double)cb;
        cand_all += cb;
    }
    int max_iters_run = 0;
    for (int m = 0; m < M; m++) max_iters_run = std::max(max_iters_run, h_ctl[m].iters);
    if (max_iters_run > 0) {
        const size_t cnt = (size_t)max_iters_run * M;
        h_tr_moved.resize(cnt);
        h_tr_qn.resize(2 * cnt);
        CK(cudaMemcpyAsync(h_tr_moved.data(), tr_moved.p, sizeof(i64) * cnt,
                           cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h_tr_qn.data(), tr_qn.p, sizeof(i64) * 2 * cnt, cudaMemcpyDeviceToHost,
                           s));
        CK(cudaStreamSynchronize(s));
    }
    for (int m = 0; m < M; m++) {
        Member *mb = mem[m];
        const int it = h_ctl[m].iters;
        for (int t = 0; t < it; t++) {
            const size_t e = (size_t)t * M + m;
            mb->res->trace.push_back(
                TraceRec{mb->level, t + 1, h_tr_moved[e], limbs_to_i128(&h_tr_qn[2 * e])});
        }
        mb->visits += (int64_t)it * mb->nnz;
    }

    proc.phase("renumber");
    // renumber (Sec. 5.1.2) -- used labels in increasing order; labels of one graph are
    // contiguous, so the scan also numbers each graph's communities
    kernels += launch_renumber(n, size.p, nullptr, nullptr, new_id.p, scratch32.p, s);
    std::vector<int64_t> h_base1(M + 1, 0);
    if (batch) {
        kernels += launch_gather_ids(new_id.p, d_gptr.p, M + 1, d_base1.p, s);
        CK(cudaMemcpyAsync(h_base1.data(), d_base1.p, sizeof(int64_t) * (M + 1),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } else {
        h_base1[1] = read_one(new_id.p + n);
        upload(d_base1, h_base1.data(), 2);
    }
    // record the level of every graph that merged something (one that merged nothing is
    // finished: no new level), then the outer test of Algorithm 2
    std::vector<int32_t> rec(M, 0), keep(M, 0);
    int nrec = 0, nkeep = 0;
    int64_t k_next = 0, n_keep = 0, nnz_keep = 0, n0_all = 0;
    bool all_kept = true;
    for (int m = 0; m < M; m++) {
        Member *mb = mem[m];
        n0_all += mb->n0;
        const int64_t kg = h_base1[m + 1] - h_base1[m];
        rec[m] = kg < mb->nv;
        if (!rec[m]) {
            all_kept = false;
            continue;
        }
        nrec++;
        const LevelCtl &hc = h_ctl[m];
        LevelRec r;
        r.ncomm = kg;
        r.qn = limbs_to_i128(hc.qn_final);
        r.qn_init = limbs_to_i128(hc.qn_init);
        r.iters = hc.iters;
        r.n = mb->nv;
        r.nnz = mb->nnz;
        r.hit_cap = hc.hit_cap;
        mb->res->levels.push_back(r);
        mb->res->coarse.push_back(louvain_result::Coarse{-1, 0, 4, nullptr, nullptr, nullptr});
        const bool stop = (mb->level >= 1 && host_below_threshold(r.qn, mb->qn_prev, mb->tw,
                                                                  cfg.theta_num, cfg.theta_den)) ||
                          mb->level + 1 >= cfg.max_levels;
        mb->qn_prev = r.qn;
        if (stop) {
            all_kept = false;
        } else {
            keep[m] = 1;
            nkeep++;
            k_next += kg;
            n_keep += mb->nv;
            nnz_keep += mb->nnz;
        }
    }
    // labels of the input vertices of every recorded graph (one array for this step, shared
    // by the results that recorded a level in it)
    const int32_t *nid2 = new_id.p;
    if (nrec > 0) {
        auto store = std::make_shared<LabelStore>();
        store->ff = cfg.free;
        store->ctx = cfg.alloc_ctx;
        store->device = h->device;
        int32_t *out = (int32_t *)A.get(sizeof(int32_t) * (size_t)n0_all);
        store->arrays.push_back(out);
        std::vector<int64_t> off(M + 1, 0);
        std::vector<int32_t *> maps(M);
        for (int m = 0; m < M; m++) {
            off[m + 1] = off[m] + mem[m]->n0;
            maps[m] = mem[m]->map;
            if (rec[m]) {
                mem[m]->res->levels.back().d_labels = out + off[m];
                mem[m]->res->stores.push_back(store);
            }
        }
        upload(d_off, off.data(), M + 1);
        upload(d_maps, maps.data(), M);
        upload(d_rec, rec.data(), M);
        upload(d_keep, keep.data(), M);
        if (batch && nkeep > 0 && !all_kept) {
            // next-level numbering: the kept graphs' communities only
            kernels += launch_renumber(n, size.p, vg.p, d_keep.p, new_id2.p, scratch32.p, s);
            nid2 = new_id2.p;
        }
        kernels += launch_compose(n0_all, M, d_off.p, d_maps.p, d_rec.p, d_keep.p, st.C, new_id.p,
                                  d_base1.p, nid2, out, s, lc);
        if (lab_s) {  // the labels go to pinned host memory while the induction runs
            size_t got = 0;
            void *hb = h->pool->get(sizeof(int32_t) * (size_t)n0_all, &got);
            if (hb) {  // no pinned memory to be had: the labels are copied when asked for
                store->pool = h->pool;
                store->pinned = hb;
                store->pinned_bytes = got;
                CK(cudaEventRecord(lab_ev, s));
                CK(cudaStreamWaitEvent(lab_s, lab_ev, 0));
                CK(cudaMemcpyAsync(hb, out, sizeof(int32_t) * (size_t)n0_all,
                                   cudaMemcpyDeviceToHost, lab_s));
                for (int m = 0; m < M; m++)
                    if (rec[m]) mem[m]->res->levels.back().h_labels = (int32_t *)hb + off[m];
            }
        }
        CK(cudaStreamSynchronize(s));  // host vectors above are uploaded before they go
    }

    proc.phase("induce");
    // ---------------- induce the next graph of the kept graphs (Sec. 5.1.2)
    double t_coarsen = 0.0, coarsen_bytes = 0.0;
    std::vector<int64_t> gptr_next(M + 1, 0), gnnz_next(M + 1, 0);
    if (nkeep > 0) {
        // Exact widths of the induction from the largest community degree: an induced weight
        // A'_ab and every sum of the induction's tables are at most deg_a (Eq. 2), so the
        // tables take 32-bit sums when every deg_a < 2^32 and the next graph keeps int32
        // weights when every deg_a < 2^31.
        kernels += launch_max_delta(deg.p, n, &d_sc->dmax, s, lc);
        const u64 cmax = read_one(&d_sc->dmax);
        const bool narrow_c = !cfg.wide_sums && cmax < ((u64)1 << 32);
        ensure(c_csize, n);
        ensure(c_moff, (size_t)n + 1);
        ensure(c_cursor, n);
        ensure(c_members, n);
        ensure(c_mpre, (size_t)n + 1);
        ensure(c_mrow, n);
        ensure(c_ccnt, n);
        ensure(c_tmp_col, (size_t)G.nnz);
        ensure(c_tmp_w, (size_t)G.nnz);
        CoarsenBufs cb;
        cb.csize = c_csize.p;
        cb.moff = c_moff.p;
        cb.cursor = c_cursor.p;
        cb.members = c_members.p;
        cb.mpre = c_mpre.p;
        cb.mrow = c_mrow.p;
        cb.ccnt = c_ccnt.p;
        cb.tmp_col = c_tmp_col.p;
        cb.tmp_w = c_tmp_w.p;
        cb.counts = &d_sc->ccounts[0];
        cb.scratch32 = scratch32.p;
        cb.scratch64 = scratch64.p;
        if (tm.on) CK(cudaEventRecord(coarsen_ev[0], s));
        Bins cbins = narrow_c == narrow ? proto : make_proto(narrow_c);  // table widths of the induction
        // no cluster bins in the induction (the community binning folds bins 6-9 into 10):
        // communities above the bin-5 bound take the chunked bin's partitioned merge, which
        // is faster there (R-MAT 26: 174.7 -> 163.8 ms of induction per run; the sweeps keep
        // their cluster bins)
        for (int t = 0; t < 4; t++) cbins.upper[6 + t] = cbins.upper[5];
        cbins.nch = b_nch.p;
        cbins.chunk_first = b_chunk_first.p;
        cbins.gloop = b_gloop.p;
        cbins.gcap = b_gcap.p;
        cbins.goff = b_goff.p;
        cbins.glog2 = b_glog2.p;
        cbins.plog2 = b_plog2.p;
        cbins.hoff = b_hoff.p;
        const int64_t k = k_next;
        const bool masked = batch && !all_kept;
        kernels += launch_coarsen_stage1(G, st, nid2, k, masked ? n_keep : n,
                                         masked ? vg.p : nullptr, masked ? d_keep.p : nullptr,
                                         nullptr, delta_next.p, cb, cbins, s, lc);
        sync_scalars();
        cbins.list = lists.p;  // the sweep's lists are free again
        cbins.off[0] = cbins.off[1] = 0;  // bin-0 communities are counted in bin 1
        for (int b = 0; b < kNumBins; b++) {
            cbins.nlist[b] = b < 1 ? 0 : h->pinned->ccounts[b];
            if (b >= 1) cbins.off[b + 1] = cbins.off[b] + cbins.nlist[b];
        }
        kernels += launch_coarsen_binfill(k, cb, cbins, s, lc);
        prep_huge(cbins, true, k, &cb);
        kernels += launch_coarsen_stage2(G, st, nid2, k, cb, cbins, narrow_c, &d_sc->err, s, lc);
        DBuf<int64_t> rp_next;
        rp_next.reset(&A, (size_t)k + 1);
        kernels += launch_coarsen_rowptr(k, cb, rp_next.p, s);
        sync_scalars();
        const int64_t nnz_next = read_one(rp_next.p + k);
        const int wb_next = cmax <= (u64)INT32_MAX ? 4 : 8;
        DBuf<int32_t> col_next;
        DBuf<unsigned char> w_next;
        col_next.reset(&A, (size_t)nnz_next);
        w_next.reset(&A, (size_t)nnz_next * wb_next);
        kernels += launch_coarsen_compact(k, nnz_next, cb, rp_next.p, col_next.p, w_next.p,
                                          wb_next, narrow_c, s, lc);
        // algorithmic bytes of the induction (louvain_result_coarsen_stats)
        coarsen_bytes = (double)nnz_keep * (4 + G.wbytes + 4) + (double)n_keep * (8 + 4) +
                        (double)nnz_next * (4 + wb_next) + (double)(k + 1) * 8;
        if (tm.on) {
            CK(cudaEventRecord(coarsen_ev[1], s));
            CK(cudaEventSynchronize(coarsen_ev[1]));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, coarsen_ev[0], coarsen_ev[1]));
            t_coarsen = ms;
        }
        // vertex and entry offsets of every kept graph in the next graph
        if (batch) {
            kernels += launch_gather_ids(nid2, d_gptr.p, M + 1, d_base1.p, s);
            kernels += launch_gather64(rp_next.p, d_base1.p, M + 1, d_gnnz.p, s);
            CK(cudaMemcpyAsync(gptr_next.data(), d_base1.p, sizeof(int64_t) * (M + 1),
                               cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(gnnz_next.data(), d_gnnz.p, sizeof(int64_t) * (M + 1),
                               cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        } else {
            gptr_next[1] = k;
            gnnz_next[1] = nnz_next;
        }
        if (cfg.keep_coarse && !batch) {  // checkpoint: the next level's input graph
            louvain_result *res0 = mem[0]->res;
            auto store = std::make_shared<LabelStore>();
            store->ff = cfg.free;
            store->ctx = cfg.alloc_ctx;
            store->device = h->device;
            void *crp = A.get(sizeof(int64_t) * (size_t)(k + 1));
            store->arrays.push_back(crp);
            void *ccol = A.get(sizeof(int32_t) * (size_t)nnz_next);
            store->arrays.push_back(ccol);
            void *cw = A.get((size_t)wb_next * (size_t)nnz_next);
            store->arrays.push_back(cw);
            CK(cudaMemcpyAsync(crp, rp_next.p, sizeof(int64_t) * (size_t)(k + 1),
                               cudaMemcpyDeviceToDevice, s));
            if (nnz_next) {
                CK(cudaMemcpyAsync(ccol, col_next.p, sizeof(int32_t) * (size_t)nnz_next,
                                   cudaMemcpyDeviceToDevice, s));
                CK(cudaMemcpyAsync(cw, w_next.p, (size_t)wb_next * (size_t)nnz_next,
                                   cudaMemcpyDeviceToDevice, s));
            }
            res0->coarse.back() = louvain_result::Coarse{k, nnz_next, wb_next, (const int64_t *)crp,
                                                        (const int32_t *)ccol, cw};
            res0->stores.push_back(store);
        }
        g_rp.swap(rp_next);
        g_col.swap(col_next);
        g_w.swap(w_next);
        G.n = k;
        G.nnz = nnz_next;
        G.rp = g_rp.p;
        G.col = g_col.p;
        G.w = g_w.p;
        G.wbytes = wb_next;
    } else {
        g_rp.release();
        g_col.release();
        g_w.release();
        G.n = 0;
        G.nnz = 0;
        G.rp = nullptr;
        G.col = nullptr;
        G.w = nullptr;
    }

    // step totals go to every graph of the step; the kept graphs move on, the rest leave
    const double wall = now_ms() - wall0;
    const int64_t step_kernels = kernels - k_start;
    // this step's label copies (overlapped with its induction) are done before any result
    // leaves the engine
    if (lab_s) CK(cudaStreamSynchronize(lab_s));
    std::vector<Member *> next;
    for (int m = 0; m < M; m++) {
        Member *mb = mem[m];
        louvain_result *r = mb->res;
        r->acc_sweeps += sweeps;
        r->acc_alg_bytes += alg_bytes;
        r->acc_cand += (int64_t)cand_all;
        r->acc_kernels += step_kernels;
        r->acc_coarsen_ms += t_coarsen;
        r->acc_coarsen_bytes += coarsen_bytes;
        r->acc_inductions += nkeep > 0;
        r->acc_step_ms += wall;
        r->exec_info[0] += graph_sweeps;
        r->exec_info[1] += sweeps - graph_sweeps;
        r->exec_info[2] += 1;
        r->exec_info[3] += captures;
        for (int b = 0; b < 2 * kNumBins; b++) {
            r->bin_time[b] += t_kernel[b];
            r->bin_launches[b] += launches_kernel[b];
            r->bin_bytes[b] += bytes_kernel[b];
            r->bin_rows[b] += rows_kernel[b];
            r->bin_entries[b] += entries_kernel[b];
        }
        if (keep[m]) {
            mb->level++;
            mb->distinct_rows = true;  // induced rows merge every column once
            mb->nv = gptr_next[m + 1] - gptr_next[m];
            mb->nnz = gnnz_next[m + 1] - gnnz_next[m];
            next.push_back(mb);
        } else {
            release_map(mb);
            retired.push_back(mb);
        }
    }
    mem.swap(next);
}

// Counters and times of a graph that left the engine (formulas in louvain.h).
void finish_result(Member *m)
{
    louvain_result *r = m->res;
    r->counters[0] = m->visits;
    r->counters[1] = r->acc_sweeps;
    r->counters[2] = (int64_t)r->acc_alg_bytes;
    r->counters[3] = r->acc_cand;
    r->counters[4] = r->acc_kernels;
    int dom = 0;
    for (int b = 1; b < 2 * kNumBins; b++)
        if (r->bin_time[b] > r->bin_time[dom]) dom = b;
    double tot = 0, t_cta = 0;
    for (int b = 0; b < 2 * kNumBins; b++) {
        tot += r->bin_time[b];
        if (b % kNumBins >= 3) t_cta += r->bin_time[b];
    }
    if (tot > 0) {
        r->times[0] = tot;
        r->times[4] = r->bin_time[dom];
        r->times[5] = r->bin_time[0] + r->bin_time[kNumBins];
        r->times[6] = r->bin_time[1] + r->bin_time[2] + r->bin_time[kNumBins + 1] +
                      r->bin_time[kNumBins + 2];
        r->times[7] = t_cta;
        r->counters[5] = r->bin_launches[dom];
        r->counters[6] = (int64_t)r->bin_bytes[dom];
        r->counters[7] = dom;
        r->times[1] = r->acc_coarsen_ms;
    }
    r->times[3] = now_ms() - m->t0;
}

// Runs louvain_run (gvptr null: one graph, one-graph kernels) or louvain_run_batch on the
// engine: the input enters as one source and the engine steps until every graph has left.
// A resumed run (start_level > 0) enters at that level with the previous level's Qn for
// the outer test and may carry int64 weights (wbytes = 8); w_in then points to int64.
void run_engine(louvain_handle *h, const louvain_config &cfg, cudaStream_t s, DevAlloc &A,
                int64_t n0, const int64_t *rp_in,
                const int32_t *col_in, const int32_t *w_in, int kind, int NG,
                const int64_t *gvptr, const int64_t *geptr, std::vector<louvain_result *> &out,
                int start_level = 0, i128 qn_prev_level = 0, int wbytes = 4)
{
    const double t0 = now_ms();
    const bool batch = gvptr != nullptr;
    std::vector<std::unique_ptr<Member>> members(NG);  // outlives the engine
    Engine E(h, s, A, batch, cfg);
    const LaunchCfg &lc = h->lc;

    // ---------------- input graph on the device
    int64_t nnz = 0;
    DBuf<int64_t> rp_own;
    DBuf<int32_t> col_own, w_own;
    const int64_t *d_rp = rp_in;
    const int32_t *d_col = col_in;
    const int32_t *d_w = w_in;
    if (kind == LOUVAIN_PTR_HOST) {
        if (rp_in[0] != 0) throw LvErr{LOUVAIN_ERR_INDEX_RANGE, "row_ptr[0] must be 0"};
        nnz = rp_in[n0];
        if (nnz < 0) throw LvErr{LOUVAIN_ERR_INDEX_RANGE, "row_ptr[n] is negative"};
        if (nnz > 0 && !col_in) throw LvErr{LOUVAIN_ERR_INVALID_ARG, "col_idx is NULL"};
        rp_own.reset(&A, (size_t)n0 + 1);
        CK(cudaMemcpyAsync(rp_own.p, rp_in, sizeof(int64_t) * (size_t)(n0 + 1),
                           cudaMemcpyHostToDevice, s));
        d_rp = rp_own.p;
        col_own.reset(&A, (size_t)nnz);
        if (nnz)
            CK(cudaMemcpyAsync(col_own.p, col_in, sizeof(int32_t) * (size_t)nnz,
                               cudaMemcpyHostToDevice, s));
        d_col = col_own.p;
        if (w_in) {
            w_own.reset(&A, (size_t)nnz * (wbytes / 4));
            if (nnz)
                CK(cudaMemcpyAsync(w_own.p, w_in, (size_t)wbytes * (size_t)nnz,
                                   cudaMemcpyHostToDevice, s));
            d_w = w_own.p;
        }
    } else {
        const int64_t r0 = E.read_one(rp_in);
        nnz = E.read_one(rp_in + n0);
        if (r0 != 0) throw LvErr{LOUVAIN_ERR_INDEX_RANGE, "row_ptr[0] must be 0"};
        if (nnz < 0) throw LvErr{LOUVAIN_ERR_INDEX_RANGE, "row_ptr[n] is negative"};
        if (nnz > 0 && !col_in) throw LvErr{LOUVAIN_ERR_INVALID_ARG, "col_idx is NULL"};
    }
    if (!d_w) {
        wbytes = 4;
        w_own.reset(&A, (size_t)nnz);
        E.kernels += launch_fill_ones(w_own.p, nnz, s, lc);
        d_w = w_own.p;
    }
    Source src;
    src.wbytes = wbytes;
    src.n = n0;
    src.nnz = nnz;
    src.rp = d_rp;
    src.col = d_col;
    src.w = d_w;
    src.vptr.assign(NG + 1, 0);
    src.eptr.assign(NG + 1, 0);
    for (int g = 0; g <= NG; g++) src.vptr[g] = batch ? gvptr[g] : (g ? n0 : 0);
    for (int g = 0; g < NG; g++) {
        members[g].reset(new Member());
        members[g]->res = out[g];
        members[g]->t0 = t0;
        members[g]->level = start_level;
        members[g]->qn_prev = qn_prev_level;
        src.members.push_back(members[g].get());
        out[g]->n0 = src.vptr[g + 1] - src.vptr[g];
        out[g]->batch_index = batch ? g : -1;
    }
    if (n0 > 0) {
        // row offsets must be sane before any row is read
        E.kernels += launch_validate_rowptr(d_rp, n0, &E.d_sc->err, s, lc);
        E.sync_scalars();
        if (batch) {
            DBuf<int64_t> d_v, d_e;
            d_v.reset(&A, NG + 1);
            d_e.reset(&A, NG + 1);
            CK(cudaMemcpyAsync(d_v.p, src.vptr.data(), sizeof(int64_t) * (NG + 1),
                               cudaMemcpyHostToDevice, s));
            E.kernels += launch_gather64(d_rp, d_v.p, NG + 1, d_e.p, s);
            CK(cudaMemcpyAsync(src.eptr.data(), d_e.p, sizeof(int64_t) * (NG + 1),
                               cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (geptr)
                for (int g = 0; g <= NG; g++)
                    if (geptr[g] != src.eptr[g])
                        throw LvErr{LOUVAIN_ERR_INDEX_RANGE, "graph_eptr[" + std::to_string(g) +
                                                                 "] != row_ptr[graph_vptr[g]]"};
        } else {
            src.eptr[1] = nnz;
        }
        std::vector<Member *> left;
        E.add(std::move(src), left);
        while (!E.idle()) E.step(left);
    }
    CK(cudaStreamSynchronize(s));
    for (auto &m : members) finish_result(m.get());
}

// ---------------------------------------------------------------------- serving
//
// A request loop for graphs that arrive over time.  Submitted graphs wait in a FIFO queue
// and are admitted while a slot is free and their estimated device footprint fits the
// budget; an upload thread copies and vets each admitted graph on a stream of its own, and
// the engine thread lets every vetted graph join at its next step boundary, so a graph that
// arrives while others run shares the following steps' launches with them.  A graph leaves
// when its own run ends; its result is then ready for louvain_poll and its slot and budget
// go back to the queue.

enum { kQueued, kUploading, kReady, kResident, kDone };

struct Request {
    uint64_t ticket = 0;
    int64_t n = 0, nnz = 0;
    std::vector<int64_t> rp;
    std::vector<int32_t> col, w;  // w empty: every weight is 1
    uint64_t footprint = 0;
    int state = kQueued;
    int rc = LOUVAIN_OK;
    std::string err;
    louvain_result *res = nullptr;
    double t_submit = 0.0, t_admit = 0.0;
    int64_t *d_rp = nullptr;
    int32_t *d_col = nullptr, *d_w = nullptr;
    Member member;
};

// Device bytes a graph may hold while it is served: its device copy (row offsets, columns,
// weights) and its share of the engine's buffers, about 160 bytes a vertex (state, bins,
// induction and label arrays) and 40 bytes an entry (stacked copy, induction scratch and
// the next level's graph).
uint64_t footprint_estimate(int64_t n, int64_t nnz)
{
    return (uint64_t)(8 * (n + 1) + 8 * nnz) + 160ull * (uint64_t)n + 40ull * (uint64_t)nnz;
}

struct Server {
    louvain_handle *h = nullptr;
    uint64_t budget = 0, in_use = 0;
    int max_slots = 0, slots_used = 0, n_uploading = 0;
    std::mutex mu;
    std::condition_variable cv;  // any change of the queues or of a request's state
    std::deque<Request *> queue;      // submitted, waiting for admission
    std::deque<Request *> to_upload;  // admitted, upload not started
    std::vector<Request *> ready;     // uploaded and vetted, waiting to join
    std::unordered_map<uint64_t, Request *> tickets;
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::thread uploader, worker;
    cudaStream_t compute = nullptr, copy = nullptr;
    DevAlloc A_compute, A_copy;
    unsigned *d_chk = nullptr;  // upload checks: error bits, then 2W (u64) at d_chk + 2

    // FIFO admission under the lock; a graph larger than the whole budget is rejected
    void admit_locked()
    {
        while (!queue.empty()) {
            Request *r = queue.front();
            if (r->footprint > budget) {
                queue.pop_front();
                r->rc = LOUVAIN_ERR_REJECTED;
                r->err = "graph footprint " + std::to_string(r->footprint) +
                         " bytes exceeds the serving budget";
                r->state = kDone;
                continue;
            }
            if (slots_used >= max_slots || in_use + r->footprint > budget) break;
            queue.pop_front();
            slots_used++;
            in_use += r->footprint;
            n_uploading++;
            r->state = kUploading;
            r->t_admit = now_ms();
            to_upload.push_back(r);
        }
        cv.notify_all();
    }

    void release_device(Request *r, DevAlloc &A)
    {
        A.put(r->d_rp);
        A.put(r->d_col);
        A.put(r->d_w);
        r->d_rp = nullptr;
        r->d_col = nullptr;
        r->d_w = nullptr;
    }

    // the request leaves (done or failed): its slot and budget go back to the queue
    void finish_locked(Request *r, int rc, const std::string &msg)
    {
        r->rc = rc;
        r->err = msg;
        r->state = kDone;
        slots_used--;
        in_use -= r->footprint;
        admit_locked();
    }

    void upload_one(Request *r)
    {
        const LaunchCfg &lc = h->lc;
        cudaStream_t s = copy;
        r->d_rp = (int64_t *)A_copy.get(sizeof(int64_t) * (size_t)(r->n + 1));
        r->d_col = (int32_t *)A_copy.get(sizeof(int32_t) * (size_t)r->nnz);
        r->d_w = (int32_t *)A_copy.get(sizeof(int32_t) * (size_t)r->nnz);
        CK(cudaMemcpyAsync(r->d_rp, r->rp.data(), sizeof(int64_t) * (size_t)(r->n + 1),
                           cudaMemcpyHostToDevice, s));
        if (r->nnz) {
            CK(cudaMemcpyAsync(r->d_col, r->col.data(), sizeof(int32_t) * (size_t)r->nnz,
                               cudaMemcpyHostToDevice, s));
            if (!r->w.empty())
                CK(cudaMemcpyAsync(r->d_w, r->w.data(), sizeof(int32_t) * (size_t)r->nnz,
                                   cudaMemcpyHostToDevice, s));
            else
                launch_fill_ones(r->d_w, r->nnz, s, lc);
        }
        // vet the graph alone, so that a bad graph never reaches the others' steps
        CK(cudaMemsetAsync(d_chk, 0, 16, s));
        launch_validate_rowptr(r->d_rp, r->n, d_chk, s, lc);
        unsigned hv[4] = {0, 0, 0, 0};
        CK(cudaMemcpyAsync(hv, d_chk, sizeof(hv), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!hv[0]) {
            launch_check_rows(r->n, r->d_rp, r->d_col, r->d_w, d_chk, (u64 *)(d_chk + 2), s, lc);
            if (h->cfg.checks >= 2) {
                DevGraph g;
                g.n = r->n;
                g.nnz = r->nnz;
                g.rp = r->d_rp;
                g.col = r->d_col;
                g.w = r->d_w;
                g.wbytes = 4;
                launch_check_symmetry(g, d_chk, s, lc);
            }
            CK(cudaMemcpyAsync(hv, d_chk, sizeof(hv), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        }
        CK(cudaGetLastError());
        if (hv[0]) {
            std::string msg;
            const int code = map_err_bits(hv[0], msg);
            throw LvErr{code, msg};
        }
        u64 tw = 0;
        memcpy(&tw, &hv[2], sizeof(tw));
        if (tw > ((u64)1 << 62)) throw LvErr{LOUVAIN_ERR_TOO_LARGE, "sum of weights above 2^62"};
    }

    void upload_loop()
    {
        cudaSetDevice(h->device);
        for (;;) {
            Request *r = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return !to_upload.empty() || (stopping && queue.empty()); });
                if (to_upload.empty()) return;
                r = to_upload.front();
                to_upload.pop_front();
            }
            int rc = LOUVAIN_OK;
            std::string msg;
            try {
                upload_one(r);
            } catch (const LvErr &e) {
                rc = e.code;
                msg = e.msg;
                cudaStreamSynchronize(copy);
                cudaGetLastError();
            } catch (const std::bad_alloc &) {
                rc = LOUVAIN_ERR_OOM;
                msg = "host allocation failed";
            }
            std::vector<int64_t>().swap(r->rp);  // the host copy is no longer needed
            std::vector<int32_t>().swap(r->col);
            std::vector<int32_t>().swap(r->w);
            if (rc != LOUVAIN_OK) release_device(r, A_copy);
            std::lock_guard<std::mutex> lk(mu);
            n_uploading--;
            if (rc == LOUVAIN_OK) {
                r->state = kReady;
                ready.push_back(r);
                cv.notify_all();
            } else {
                finish_locked(r, rc, msg);
            }
        }
    }

    void work_loop()
    {
        cudaSetDevice(h->device);
        std::unique_ptr<Engine> E;
        auto fresh_engine = [&] {
            E.reset();
            E.reset(new Engine(h, compute, A_compute, true, h->cfg));
        };
        try {
            fresh_engine();
        } catch (const LvErr &) {
            cudaGetLastError();
        }
        std::vector<Request *> in_engine;
        for (;;) {
            std::vector<Request *> take;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] {
                    return !ready.empty() || (E && !E->idle()) ||
                           (stopping && queue.empty() && to_upload.empty() && n_uploading == 0);
                });
                take.swap(ready);
                if (take.empty() && (!E || E->idle())) return;  // stopping and drained
            }
            std::vector<Member *> done;
            int rc = LOUVAIN_OK;
            std::string msg;
            try {
                if (!E) throw LvErr{LOUVAIN_ERR_CUDA, "serving engine could not start"};
                for (Request *r : take) {
                    r->state = kResident;
                    r->member = Member();
                    r->member.res = r->res;
                    r->member.t0 = r->t_submit;
                    r->member.tag = r;
                    Source src;
                    src.n = r->n;
                    src.nnz = r->nnz;
                    src.rp = r->d_rp;
                    src.col = r->d_col;
                    src.w = r->d_w;
                    src.vptr = {0, r->n};
                    src.eptr = {0, r->nnz};
                    src.members = {&r->member};
                    in_engine.push_back(r);
                    E->add(std::move(src), done);
                }
                if (!E->idle()) E->step(done);
                CK(cudaStreamSynchronize(compute));
            } catch (const LvErr &e) {
                rc = e.code;
                msg = e.msg;
            } catch (const std::bad_alloc &) {
                rc = LOUVAIN_ERR_OOM;
                msg = "host allocation failed";
            }
            if (rc != LOUVAIN_OK) {
                // the engine state is lost: every graph in it fails with the error
                cudaStreamSynchronize(compute);
                cudaGetLastError();
                done.clear();
                for (Request *r : in_engine) done.push_back(&r->member);
                try {
                    fresh_engine();
                } catch (const LvErr &) {
                    E.reset();
                    cudaGetLastError();
                }
            }
            for (Member *m : done) {
                Request *r = (Request *)m->tag;
                if (rc == LOUVAIN_OK) {
                    finish_result(m);
                    r->res->times[2] = r->t_admit - r->t_submit;
                } else if (m->map) {
                    A_compute.put(m->map);
                    m->map = nullptr;
                }
                release_device(r, A_compute);
                in_engine.erase(std::find(in_engine.begin(), in_engine.end(), r));
                std::lock_guard<std::mutex> lk(mu);
                finish_locked(r, rc, msg);
            }
        }
    }
};

// ---------------------------------------------------------------------- autotuner
//
// Degree-bin thresholds and the chunk length only decide which kernel handles a row, never
// a result, so they can be chosen by measurement: each trial is a whole run with a
// candidate set in the handle's own mode (best of two, CUDA-event time of the run), and a
// coordinate search over the thresholds keeps a change only when it is at least 2%
// faster.  The choice is cached on the handle per (vertex count, entry count).

void get_bins(const louvain_config &c, int32_t b[7])
{
    b[0] = c.bin_small;
    b[1] = c.bin_mid1;
    b[2] = c.bin_mid2;
    b[3] = c.bin_cta1;
    b[4] = c.bin_cta2;
    b[5] = c.bin_cta3;
    b[6] = c.chunk_entries;
}

void set_bins(louvain_config &c, const int32_t b[7])
{
    c.bin_small = b[0];
    c.bin_mid1 = b[1];
    c.bin_mid2 = b[2];
    c.bin_cta1 = b[3];
    c.bin_cta2 = b[4];
    c.bin_cta3 = b[5];
    c.chunk_entries = b[6];
}

bool bins_valid(const int32_t b[7])
{
    return b[0] >= 0 && b[0] <= 8 && b[0] <= b[1] && b[1] <= 32 && b[1] <= b[2] &&
           b[2] <= 128 && b[2] <= b[3] && b[3] <= b[4] && b[4] <= b[5] && b[5] <= 12288 &&
           b[6] >= 32 && b[6] <= 4096 && (b[6] & (b[6] - 1)) == 0;
}

void tuned_bins(louvain_handle *h, cudaStream_t s, DevAlloc &A, int64_t n, const int64_t *rp,
                const int32_t *col, const int32_t *w, int kind, std::array<int32_t, 7> &out,
                int64_t *trials_out, int64_t *hit_out, double *best_ms_out)
{
    int64_t nnz = 0;
    if (kind == LOUVAIN_PTR_HOST) {
        nnz = rp[n];
    } else {
        CK(cudaMemcpyAsync(&h->pinned->tail[0], rp + n, sizeof(int64_t), cudaMemcpyDeviceToHost,
                           s));
        CK(cudaStreamSynchronize(s));
        memcpy(&nnz, &h->pinned->tail[0], sizeof(nnz));
    }
    const std::pair<int64_t, int64_t> key(n, nnz);
    for (const auto &e : h->tuned)
        if (e.first == key) {
            out = e.second;
            *trials_out = 0;
            *hit_out = 1;
            if (best_ms_out) *best_ms_out = -1.0;
            return;
        }
    // trials read the graph from device memory (one copy of a host graph for all of them)
    DBuf<int64_t> rp_d;
    DBuf<int32_t> col_d, w_d;
    if (kind == LOUVAIN_PTR_HOST) {
        rp_d.reset(&A, (size_t)n + 1);
        col_d.reset(&A, (size_t)nnz);
        CK(cudaMemcpyAsync(rp_d.p, rp, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice,
                           s));
        if (nnz) {
            if (!col) throw LvErr{LOUVAIN_ERR_INVALID_ARG, "col_idx is NULL"};
            CK(cudaMemcpyAsync(col_d.p, col, sizeof(int32_t) * (size_t)nnz,
                               cudaMemcpyHostToDevice, s));
        }
        if (w) {
            w_d.reset(&A, (size_t)nnz);
            if (nnz)
                CK(cudaMemcpyAsync(w_d.p, w, sizeof(int32_t) * (size_t)nnz,
                                   cudaMemcpyHostToDevice, s));
        }
        rp = rp_d.p;
        col = col_d.p;
        w = w ? w_d.p : nullptr;
        kind = LOUVAIN_PTR_DEVICE;
    }
    louvain_config base = h->cfg;
    base.profile = 0;  // trials run as the tuned runs will (graphs, concurrent bins)
    base.autotune = 0;
    int64_t trials = 0;
    cudaEvent_t ev[2];
    CK(cudaEventCreate(&ev[0]));
    CK(cudaEventCreate(&ev[1]));
    struct EvFree {
        cudaEvent_t *e;
        ~EvFree()
        {
            cudaEventDestroy(e[0]);
            cudaEventDestroy(e[1]);
        }
    } evf{ev};
    auto trial = [&](const int32_t b[7]) {
        louvain_config t = base;
        set_bins(t, b);
        double best = 1e300;
        for (int rep = 0; rep < 2; rep++) {
            std::unique_ptr<louvain_result> r(new louvain_result());
            r->device = h->device;
            r->ff = h->cfg.free;
            r->ctx = h->cfg.alloc_ctx;
            std::vector<louvain_result *> outs{r.get()};
            CK(cudaEventRecord(ev[0], s));
            run_engine(h, t, s, A, n, rp, col, w, kind, 1, nullptr, nullptr, outs);
            CK(cudaEventRecord(ev[1], s));
            CK(cudaEventSynchronize(ev[1]));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ev[0], ev[1]));
            best = std::min(best, (double)ms);
            trials++;
        }
        return best;
    };
    static const int32_t cand[7][3] = {{0, 4, 8},       {16, 32, 32},       {64, 128, 128},
                                       {256, 512, 1024}, {1024, 2048, 4096}, {4096, 6144, 12288},
                                       {1024, 2048, 4096}};
    int32_t cur[7];
    get_bins(h->cfg, cur);
    double cur_t = trial(cur);
    for (int p = 0; p < 7; p++)
        for (int v = 0; v < 3; v++) {
            int32_t c[7];
            memcpy(c, cur, sizeof(c));
            if (cand[p][v] == cur[p]) continue;
            c[p] = cand[p][v];
            if (!bins_valid(c)) continue;
            const double t = trial(c);
            if (t < 0.98 * cur_t) {
                memcpy(cur, c, sizeof(c));
                cur_t = t;
            }
        }
    for (int k = 0; k < 7; k++) out[k] = cur[k];
    h->tuned.push_back({key, out});
    *trials_out = trials;
    *hit_out = 0;
    if (best_ms_out) *best_ms_out = cur_t;
}

struct RunCtx {
    cudaStream_t s = nullptr;
    DevAlloc A;
};

}  // namespace

// ------------------------------------------------------------ device -> host label copies
// A process-wide pinned staging buffer (two halves) and a stream of its own: a copy into
// ordinary host memory moves each chunk into pinned memory by DMA, then copies it on the host
// while the next chunk is in flight.
struct PinnedStage {
    std::mutex mu;
    int device = -1;
    char *buf = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    static constexpr size_t kHalf = (size_t)8 << 20;

    void release()
    {
        if (ev[0]) cudaEventDestroy(ev[0]);
        if (ev[1]) cudaEventDestroy(ev[1]);
        if (s) cudaStreamDestroy(s);
        if (buf) cudaFreeHost(buf);
        ev[0] = ev[1] = nullptr;
        s = nullptr;
        buf = nullptr;
        device = -1;
    }
    bool ready(int dev)
    {
        if (device == dev && buf) return true;
        release();
        if (cudaMallocHost((void **)&buf, 2 * kHalf) != cudaSuccess) {
            buf = nullptr;
            return false;
        }
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess) {
            release();
            return false;
        }
        device = dev;
        return true;
    }
};

PinnedStage &pinned_stage()
{
    static PinnedStage st;  // lives until the process exits (pinned memory is released then)
    return st;
}

// Host copy of one staged chunk, split over a few threads: the destination is usually fresh
// pageable memory whose first touch (page faults) dominates a single-threaded copy.
void parallel_memcpy(char *to, const char *from, size_t len, int max_threads = 4)
{
    constexpr size_t kMinPart = (size_t)1 << 20;
    int parts = (int)std::min<size_t>((size_t)max_threads, std::max<size_t>(1, len / kMinPart));
    if (parts <= 1) {
        memcpy(to, from, len);
        return;
    }
    const size_t step = (len + parts - 1) / parts;
    std::vector<std::thread> workers;
    for (int t = 1; t < parts; t++) {
        const size_t b = (size_t)t * step, e = std::min(len, b + step);
        if (b >= e) continue;
        try {
            workers.emplace_back([=] { memcpy(to + b, from + b, e - b); });
        } catch (...) {  // no thread to spare: copy this part here
            memcpy(to + b, from + b, e - b);
        }
    }
    memcpy(to, from, std::min(len, step));
    for (auto &w : workers) w.join();
}

bool copy_d2h_staged(int device, void *dst, const void *src, size_t bytes)
{
    PinnedStage &st = pinned_stage();
    std::lock_guard<std::mutex> lock(st.mu);
    struct KeepDevice {  // the caller's current device is restored on return
        int prev = -1;
        KeepDevice()
        {
            if (cudaGetDevice(&prev) != cudaSuccess) {
                cudaGetLastError();
                prev = -1;
            }
        }
        ~KeepDevice()
        {
            if (prev >= 0) cudaSetDevice(prev);
        }
    } keep;
    if (cudaSetDevice(device) != cudaSuccess || !st.ready(device)) return false;
    const char *from = (const char *)src;
    char *to = (char *)dst;
    size_t pend_off[2] = {0, 0}, pend_len[2] = {0, 0};
    bool pend[2] = {false, false};
    int next = 0;
    auto drain = [&](int hb) {
        if (!pend[hb]) return true;
        if (cudaEventSynchronize(st.ev[hb]) != cudaSuccess) return false;
        parallel_memcpy(to + pend_off[hb], st.buf + hb * PinnedStage::kHalf, pend_len[hb]);
        pend[hb] = false;
        return true;
    };
    for (size_t off = 0; off < bytes; off += PinnedStage::kHalf) {
        const size_t len = std::min(PinnedStage::kHalf, bytes - off);
        const int hb = next;
        next ^= 1;
        if (!drain(hb)) return false;
        if (cudaMemcpyAsync(st.buf + hb * PinnedStage::kHalf, from + off, len,
                            cudaMemcpyDeviceToHost, st.s) != cudaSuccess ||
            cudaEventRecord(st.ev[hb], st.s) != cudaSuccess)
            return false;
        pend[hb] = true;
        pend_off[hb] = off;
        pend_len[hb] = len;
    }
    return drain(next) && drain(next ^ 1);  // the older half first
}

// ====================================================================== C ABI

extern "C" {

int louvain_abi_version(void) { return 1; }

int louvain_config_init(louvain_config *cfg)
{
    if (!cfg) return LOUVAIN_ERR_INVALID_ARG;
    memset(cfg, 0, sizeof(*cfg));
    cfg->struct_size = sizeof(louvain_config);
    cfg->theta_num = 1;
    cfg->theta_den = 1000000;
    cfg->max_iters = 1000;
    cfg->max_levels = 64;
    cfg->vertex_following = 1;
    cfg->vf_all_levels = 0;
    cfg->checks = 1;
    cfg->force_int128 = 0;
    cfg->wide_sums = 0;
    cfg->bin_small = 8;
    cfg->bin_mid1 = 32;
    cfg->bin_mid2 = 128;
    cfg->bin_cta1 = 512;
    cfg->bin_cta2 = 2048;
    cfg->bin_cta3 = 12288;
    cfg->chunk_entries = 4096;
    cfg->profile = 0;
    cfg->cuda_graphs = 1;
    cfg->autotune = 0;
    cfg->sweep_streams = 4;
    cfg->part_keys = kPartKeys;
    return LOUVAIN_OK;
}

static int check_config(louvain_config &c, std::string &msg)
{
    if (c.struct_size != sizeof(louvain_config)) {
        msg = "louvain_config.struct_size mismatch (call louvain_config_init)";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (c.theta_den <= 0 || c.theta_num < 0 || c.theta_den > INT32_MAX || c.theta_num > INT32_MAX) {
        msg = "theta must be num/den with 0 <= num, 0 < den, both below 2^31";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (c.max_iters < 1 || c.max_iters > 1000000 || c.max_levels < 1 || c.max_levels > 1024) {
        msg = "max_iters must be in [1, 10^6] and max_levels in [1, 1024]";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (c.checks == 0) c.checks = 1;
    if (c.bin_small == 0 && c.bin_mid1 == 0 && c.bin_mid2 == 0 && c.bin_cta1 == 0 &&
        c.bin_cta2 == 0 && c.bin_cta3 == 0) {
        c.bin_small = 8;
        c.bin_mid1 = 32;
        c.bin_mid2 = 128;
        c.bin_cta1 = 512;
        c.bin_cta2 = 2048;
        c.bin_cta3 = 12288;
    }
    if (c.bin_small < 0 || c.bin_small > 8 || c.bin_mid1 < c.bin_small || c.bin_mid1 > 32 ||
        c.bin_mid2 < c.bin_mid1 || c.bin_mid2 > 128 || c.bin_cta1 < c.bin_mid2 ||
        c.bin_cta2 < c.bin_cta1 || c.bin_cta3 < c.bin_cta2 || c.bin_cta3 > 12288) {
        msg = "bins need 0 <= small <= 8 <= ..., small <= mid1 <= 32, mid1 <= mid2 <= 128, "
              "mid2 <= cta1 <= cta2 <= cta3 <= 12288";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (c.sweep_streams < 0 || c.sweep_streams > 4) {
        msg = "sweep_streams must be in [0, 4]";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (c.keep_coarse != 0 && c.keep_coarse != 1) {
        msg = "keep_coarse must be 0 or 1";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (c.post_merge != 0 && c.post_merge != 1) {
        msg = "post_merge must be 0 or 1";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (c.threshold_mode != 0 && c.threshold_mode != 1) {
        msg = "threshold_mode must be 0 (absolute) or 1 (relative)";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (c.chunk_entries == 0) c.chunk_entries = 4096;
    if (c.chunk_entries < 32 || c.chunk_entries > 4096 ||
        (c.chunk_entries & (c.chunk_entries - 1)) != 0) {
        msg = "chunk_entries must be a power of two in [32, 4096]";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (c.coloring != 0 && c.coloring != 1) {
        msg = "coloring must be 0 or 1";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (c.host_labels != 0 && c.host_labels != 1) {
        msg = "host_labels must be 0 or 1";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (c.part_keys == 0) c.part_keys = kPartKeys;
    if (c.part_keys < 64 || c.part_keys > (1 << 30)) {
        msg = "part_keys must be in [64, 2^30]";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if ((c.alloc == nullptr) != (c.free == nullptr)) {
        msg = "alloc and free callbacks must be given together";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    return LOUVAIN_OK;
}

int louvain_create(const louvain_config *cfg, int device, louvain_handle **out)
{
    if (!out) return LOUVAIN_ERR_INVALID_ARG;
    *out = nullptr;
    louvain_config c;
    if (cfg) c = *cfg;
    else louvain_config_init(&c);
    std::string msg;
    int rc = check_config(c, msg);
    if (rc != LOUVAIN_OK) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return LOUVAIN_ERR_CUDA;
    }
    louvain_handle *h = new (std::nothrow) louvain_handle();
    if (!h) return LOUVAIN_ERR_OOM;
    h->cfg = c;
    h->device = device;
    int sms = 152;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMallocHost((void **)&h->pinned, sizeof(Scalars)) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return LOUVAIN_ERR_CUDA;
    }
    h->lc.num_sms = sms;
    h->lc.max_blocks = sms * 8;
    {
        Bins b;
        b.upper[5] = c.bin_cta3;
        probe_cluster_support(shared_table_bytes(cta_log2cap(b, 5), true), h->lc.cluster_ok);
        cudaGetLastError();
    }
    *out = h;
    return LOUVAIN_OK;
}

void louvain_destroy(louvain_handle *h)
{
    if (!h) return;
    if (h->server) louvain_serve_close(h);
    if (h->pinned) cudaFreeHost(h->pinned);
    delete h;
}

const char *louvain_last_error(const louvain_handle *h) { return h ? h->err.c_str() : ""; }

int louvain_run(louvain_handle *h, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                const int32_t *weights, int ptr_kind, void *stream, louvain_result **out)
{
    if (!h) return LOUVAIN_ERR_INVALID_ARG;
    h->err.clear();
    if (!out) {
        h->err = "out is NULL";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (h->server) {
        h->err = "the handle is serving: use louvain_submit / louvain_poll";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (n < 0 || !row_ptr || (ptr_kind != LOUVAIN_PTR_HOST && ptr_kind != LOUVAIN_PTR_DEVICE)) {
        h->err = "bad n, row_ptr or ptr_kind";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (n > INT32_MAX) {
        h->err = "n above 2^31 - 1";
        return LOUVAIN_ERR_TOO_LARGE;
    }
    louvain_result *res = new (std::nothrow) louvain_result();
    if (!res) return LOUVAIN_ERR_OOM;
    res->device = h->device;
    res->ff = h->cfg.free;
    res->ctx = h->cfg.alloc_ctx;
    RunCtx R;
    R.s = (cudaStream_t)stream;
    R.A.fa = h->cfg.alloc;
    R.A.ff = h->cfg.free;
    R.A.ctx = h->cfg.alloc_ctx;
    R.A.s = R.s;
    int rc = LOUVAIN_OK;
    launch_site() = nullptr;
    try {
        CK(cudaSetDevice(h->device));
        louvain_config cfg = h->cfg;
        int64_t trials = 0, hit = 0;
        if (cfg.autotune && n > 0) {
            std::array<int32_t, 7> b;
            tuned_bins(h, R.s, R.A, n, row_ptr, col_idx, weights, ptr_kind, b, &trials, &hit,
                       nullptr);
            set_bins(cfg, b.data());
        }
        std::vector<louvain_result *> outs{res};
        run_engine(h, cfg, R.s, R.A, n, row_ptr, col_idx, weights, ptr_kind, 1, nullptr, nullptr,
                   outs);
        res->exec_info[4] = trials;
        res->exec_info[5] = hit;
    } catch (const LvErr &e) {
        rc = e.code;
        h->err = e.msg;
    } catch (const std::bad_alloc &) {
        rc = LOUVAIN_ERR_OOM;
        h->err = "host allocation failed";
    }
    if (rc != LOUVAIN_OK) {
        cudaStreamSynchronize(R.s);
        cudaGetLastError();
        louvain_result_free(res);
        return rc;
    }
    *out = res;
    return LOUVAIN_OK;
}

int louvain_autotune(louvain_handle *h, int64_t n, const int64_t *row_ptr,
                     const int32_t *col_idx, const int32_t *weights, int ptr_kind, void *stream,
                     int32_t bins_out[7], double *best_ms, int32_t *trials)
{
    if (!h) return LOUVAIN_ERR_INVALID_ARG;
    h->err.clear();
    if (h->server) {
        h->err = "the handle is serving";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (n < 1 || n > INT32_MAX || !row_ptr || !bins_out ||
        (ptr_kind != LOUVAIN_PTR_HOST && ptr_kind != LOUVAIN_PTR_DEVICE)) {
        h->err = "bad n, row_ptr, bins_out or ptr_kind";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    RunCtx R;
    R.s = (cudaStream_t)stream;
    R.A.fa = h->cfg.alloc;
    R.A.ff = h->cfg.free;
    R.A.ctx = h->cfg.alloc_ctx;
    R.A.s = R.s;
    launch_site() = nullptr;
    try {
        CK(cudaSetDevice(h->device));
        std::array<int32_t, 7> b;
        int64_t tr = 0, hit = 0;
        double ms = 0.0;
        tuned_bins(h, R.s, R.A, n, row_ptr, col_idx, weights, ptr_kind, b, &tr, &hit, &ms);
        for (int k = 0; k < 7; k++) bins_out[k] = b[k];
        if (best_ms) *best_ms = ms;
        if (trials) *trials = (int32_t)tr;
    } catch (const LvErr &e) {
        h->err = e.msg;
        cudaStreamSynchronize(R.s);
        cudaGetLastError();
        return e.code;
    } catch (const std::bad_alloc &) {
        h->err = "host allocation failed";
        return LOUVAIN_ERR_OOM;
    }
    return LOUVAIN_OK;
}

int louvain_resume(louvain_handle *h, int32_t start_level, const int64_t qn_prev[2], int64_t n,
                   const int64_t *row_ptr, const int32_t *col_idx, const void *weights,
                   int32_t weight_bytes, int ptr_kind, void *stream, louvain_result **out)
{
    if (!h) return LOUVAIN_ERR_INVALID_ARG;
    h->err.clear();
    if (!out) return LOUVAIN_ERR_INVALID_ARG;
    *out = nullptr;
    if (h->server) {
        h->err = "the handle is serving";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (start_level < 1 || start_level >= h->cfg.max_levels || !qn_prev || n < 0 || !row_ptr ||
        (weight_bytes != 4 && weight_bytes != 8) ||
        (ptr_kind != LOUVAIN_PTR_HOST && ptr_kind != LOUVAIN_PTR_DEVICE)) {
        h->err = "bad start_level, qn_prev, n, row_ptr, weight_bytes or ptr_kind";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (n > INT32_MAX) {
        h->err = "n above 2^31 - 1";
        return LOUVAIN_ERR_TOO_LARGE;
    }
    louvain_result *res = new (std::nothrow) louvain_result();
    if (!res) return LOUVAIN_ERR_OOM;
    res->device = h->device;
    res->ff = h->cfg.free;
    res->ctx = h->cfg.alloc_ctx;
    RunCtx R;
    R.s = (cudaStream_t)stream;
    R.A.fa = h->cfg.alloc;
    R.A.ff = h->cfg.free;
    R.A.ctx = h->cfg.alloc_ctx;
    R.A.s = R.s;
    int rc = LOUVAIN_OK;
    launch_site() = nullptr;
    try {
        CK(cudaSetDevice(h->device));
        std::vector<louvain_result *> outs{res};
        run_engine(h, h->cfg, R.s, R.A, n, row_ptr, col_idx, (const int32_t *)weights, ptr_kind,
                   1, nullptr, nullptr, outs, start_level,
                   limbs_to_i128((const i64 *)qn_prev), weight_bytes);
    } catch (const LvErr &e) {
        rc = e.code;
        h->err = e.msg;
    } catch (const std::bad_alloc &) {
        rc = LOUVAIN_ERR_OOM;
        h->err = "host allocation failed";
    }
    if (rc != LOUVAIN_OK) {
        cudaStreamSynchronize(R.s);
        cudaGetLastError();
        louvain_result_free(res);
        return rc;
    }
    *out = res;
    return LOUVAIN_OK;
}

int louvain_result_coarse_graph(const louvain_result *r, int level, int64_t *n, int64_t *nnz,
                                int32_t *weight_bytes)
{
    if (!r || level < 0 || level >= (int)r->coarse.size() || r->coarse[level].n < 0)
        return LOUVAIN_ERR_INVALID_ARG;
    const louvain_result::Coarse &c = r->coarse[level];
    if (n) *n = c.n;
    if (nnz) *nnz = c.nnz;
    if (weight_bytes) *weight_bytes = c.wbytes;
    return LOUVAIN_OK;
}

int louvain_result_coarse_copy(const louvain_result *r, int level, int64_t *row_ptr,
                               int32_t *col_idx, void *weights, int ptr_kind)
{
    if (!r || level < 0 || level >= (int)r->coarse.size() || r->coarse[level].n < 0 ||
        (ptr_kind != LOUVAIN_PTR_HOST && ptr_kind != LOUVAIN_PTR_DEVICE))
        return LOUVAIN_ERR_INVALID_ARG;
    const louvain_result::Coarse &c = r->coarse[level];
    const cudaMemcpyKind kind =
        ptr_kind == LOUVAIN_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (cudaSetDevice(r->device) != cudaSuccess ||
        (row_ptr && cudaMemcpy(row_ptr, c.rp, sizeof(int64_t) * (size_t)(c.n + 1), kind) !=
                        cudaSuccess) ||
        (col_idx && c.nnz &&
         cudaMemcpy(col_idx, c.col, sizeof(int32_t) * (size_t)c.nnz, kind) != cudaSuccess) ||
        (weights && c.nnz &&
         cudaMemcpy(weights, c.w, (size_t)c.wbytes * (size_t)c.nnz, kind) != cudaSuccess)) {
        cudaGetLastError();
        return LOUVAIN_ERR_CUDA;
    }
    return LOUVAIN_OK;
}

int louvain_csr_from_edges(louvain_handle *h, int64_t n, int64_t m, const int32_t *src,
                           const int32_t *dst, const int32_t *weights, int ptr_kind, void *stream,
                           int64_t *row_ptr, int32_t *col_idx, int32_t *w_out, int64_t *nnz)
{
    if (!h) return LOUVAIN_ERR_INVALID_ARG;
    h->err.clear();
    if (h->server) {
        h->err = "the handle is serving";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (n < 0 || m < 0 || !row_ptr || !nnz || (m > 0 && (!src || !dst || !col_idx || !w_out)) ||
        (ptr_kind != LOUVAIN_PTR_HOST && ptr_kind != LOUVAIN_PTR_DEVICE) || (n == 0 && m > 0)) {
        h->err = "bad n, m, pointers or ptr_kind";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (n > INT32_MAX || m > ((int64_t)1 << 40)) {
        h->err = "n above 2^31 - 1 or m above 2^40";
        return LOUVAIN_ERR_TOO_LARGE;
    }
    RunCtx R;
    R.s = (cudaStream_t)stream;
    R.A.fa = h->cfg.alloc;
    R.A.ff = h->cfg.free;
    R.A.ctx = h->cfg.alloc_ctx;
    R.A.s = R.s;
    cudaStream_t s = R.s;
    launch_site() = nullptr;
    ProcRange proc("neighbour");
    try {
        CK(cudaSetDevice(h->device));
        DBuf<int32_t> s_own, d_own, w_own;
        if (ptr_kind == LOUVAIN_PTR_HOST && m > 0) {
            s_own.reset(&R.A, m);
            d_own.reset(&R.A, m);
            CK(cudaMemcpyAsync(s_own.p, src, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice,
                               s));
            CK(cudaMemcpyAsync(d_own.p, dst, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice,
                               s));
            src = s_own.p;
            dst = d_own.p;
            if (weights) {
                w_own.reset(&R.A, m);
                CK(cudaMemcpyAsync(w_own.p, weights, sizeof(int32_t) * (size_t)m,
                                   cudaMemcpyHostToDevice, s));
                weights = w_own.p;
            }
        }
        const int64_t len = 2 * m;
        const int64_t tiles = edges_scratch_tiles(m);
        EdgeScratch sc;
        DBuf<u64> k0, k1, wacc;
        DBuf<int32_t> v0, v1, rowcnt;
        DBuf<int64_t> pos, hist, offs, scan64, word;
        k0.reset(&R.A, len);
        k1.reset(&R.A, len);
        v0.reset(&R.A, len);
        v1.reset(&R.A, len);
        pos.reset(&R.A, len + 1);
        wacc.reset(&R.A, len);
        rowcnt.reset(&R.A, n);
        hist.reset(&R.A, 256 * tiles);
        offs.reset(&R.A, 256 * tiles + 1);
        scan64.reset(&R.A, scan_scratch_elems(std::max(std::max(len, 256 * tiles), n) + 1) + 64);
        word.reset(&R.A, 2);  // [0]: error bits, [1]: nnz
        sc.keys[0] = k0.p;
        sc.keys[1] = k1.p;
        sc.vals[0] = v0.p;
        sc.vals[1] = v1.p;
        sc.pos = pos.p;
        sc.wacc = wacc.p;
        sc.rowcnt = rowcnt.p;
        sc.hist = hist.p;
        sc.offs = offs.p;
        sc.scan64 = scan64.p;
        CK(cudaMemsetAsync(word.p, 0, 16, s));
        launch_edges_to_csr(n, m, src, dst, weights, sc, row_ptr, col_idx, w_out, word.p + 1,
                            (unsigned *)word.p, s, h->lc);
        CK(cudaGetLastError());
        if (launch_site()) throw LvErr{LOUVAIN_ERR_CUDA, launch_site()};
        int64_t hw[2] = {0, 0};
        CK(cudaMemcpyAsync(hw, word.p, sizeof(hw), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const unsigned bits = (unsigned)hw[0];
        if (bits) {
            std::string msg;
            const int code = map_err_bits(bits, msg);
            throw LvErr{code, msg};
        }
        *nnz = hw[1];
    } catch (const LvErr &e) {
        h->err = e.msg;
        cudaStreamSynchronize(s);
        cudaGetLastError();
        launch_site() = nullptr;
        return e.code;
    } catch (const std::bad_alloc &) {
        h->err = "host allocation failed";
        return LOUVAIN_ERR_OOM;
    }
    return LOUVAIN_OK;
}

int louvain_run_batch(louvain_handle *h, int32_t num_graphs, const int64_t *graph_vptr,
                      const int64_t *graph_eptr, const int64_t *row_ptr, const int32_t *col_idx,
                      const int32_t *weights, int ptr_kind, void *stream, louvain_result **out)
{
    if (!h) return LOUVAIN_ERR_INVALID_ARG;
    h->err.clear();
    if (!out || num_graphs < 1 || !graph_vptr || !row_ptr ||
        (ptr_kind != LOUVAIN_PTR_HOST && ptr_kind != LOUVAIN_PTR_DEVICE)) {
        h->err = "bad out, num_graphs, graph_vptr, row_ptr or ptr_kind";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    for (int g = 0; g < num_graphs; g++) out[g] = nullptr;
    if (h->server) {
        h->err = "the handle is serving: use louvain_submit / louvain_poll";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (h->cfg.coloring) {
        h->err = "the colouring variant runs one graph at a time (louvain_run)";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (num_graphs > LOUVAIN_MAX_BATCH_GRAPHS) {
        h->err = "more graphs than LOUVAIN_MAX_BATCH_GRAPHS";
        return LOUVAIN_ERR_TOO_LARGE;
    }
    if (graph_vptr[0] != 0) {
        h->err = "graph_vptr[0] must be 0";
        return LOUVAIN_ERR_INDEX_RANGE;
    }
    for (int g = 0; g < num_graphs; g++)
        if (graph_vptr[g + 1] < graph_vptr[g]) {
            h->err = "graph_vptr must not decrease";
            return LOUVAIN_ERR_INDEX_RANGE;
        }
    const int64_t n = graph_vptr[num_graphs];
    if (n > INT32_MAX) {
        h->err = "total vertex count above 2^31 - 1";
        return LOUVAIN_ERR_TOO_LARGE;
    }
    std::vector<louvain_result *> outs(num_graphs, nullptr);
    for (int g = 0; g < num_graphs; g++) {
        outs[g] = new (std::nothrow) louvain_result();
        if (!outs[g]) {
            for (int q = 0; q < g; q++) delete outs[q];
            return LOUVAIN_ERR_OOM;
        }
        outs[g]->device = h->device;
        outs[g]->ff = h->cfg.free;
        outs[g]->ctx = h->cfg.alloc_ctx;
    }
    RunCtx R;
    R.s = (cudaStream_t)stream;
    R.A.fa = h->cfg.alloc;
    R.A.ff = h->cfg.free;
    R.A.ctx = h->cfg.alloc_ctx;
    R.A.s = R.s;
    int rc = LOUVAIN_OK;
    launch_site() = nullptr;
    try {
        CK(cudaSetDevice(h->device));
        run_engine(h, h->cfg, R.s, R.A, n, row_ptr, col_idx, weights, ptr_kind, num_graphs,
                   graph_vptr,
                   graph_eptr, outs);
    } catch (const LvErr &e) {
        rc = e.code;
        h->err = e.msg;
    } catch (const std::bad_alloc &) {
        rc = LOUVAIN_ERR_OOM;
        h->err = "host allocation failed";
    }
    if (rc != LOUVAIN_OK) {
        cudaStreamSynchronize(R.s);
        cudaGetLastError();
        for (louvain_result *r : outs) louvain_result_free(r);
        return rc;
    }
    for (int g = 0; g < num_graphs; g++) out[g] = outs[g];
    return LOUVAIN_OK;
}


// ---------------------------------------------------------------- serving

int louvain_serve_open(louvain_handle *h, uint64_t hbm_budget_bytes, int max_slots)
{
    if (!h) return LOUVAIN_ERR_INVALID_ARG;
    h->err.clear();
    if (h->server) {
        h->err = "serving is already open on this handle";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (max_slots < 1 || hbm_budget_bytes == 0) {
        h->err = "max_slots must be >= 1 and the budget above 0";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (h->cfg.coloring) {
        h->err = "the colouring variant runs one graph at a time (louvain_run)";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    Server *S = new (std::nothrow) Server();
    if (!S) return LOUVAIN_ERR_OOM;
    S->h = h;
    S->budget = hbm_budget_bytes;
    S->max_slots = max_slots;
    if (cudaSetDevice(h->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->compute, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->copy, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        if (S->compute) cudaStreamDestroy(S->compute);
        delete S;
        h->err = "could not create the serving streams";
        return LOUVAIN_ERR_CUDA;
    }
    for (DevAlloc *A : {&S->A_compute, &S->A_copy}) {
        A->fa = h->cfg.alloc;
        A->ff = h->cfg.free;
        A->ctx = h->cfg.alloc_ctx;
    }
    S->A_compute.s = S->compute;
    S->A_copy.s = S->copy;
    try {
        S->d_chk = (unsigned *)S->A_copy.get(16);
        S->uploader = std::thread(&Server::upload_loop, S);
        S->worker = std::thread(&Server::work_loop, S);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stopping = true;
            S->cv.notify_all();
        }
        if (S->uploader.joinable()) S->uploader.join();
        if (S->worker.joinable()) S->worker.join();
        if (S->d_chk) S->A_copy.put(S->d_chk);
        cudaStreamSynchronize(S->copy);
        cudaStreamDestroy(S->compute);
        cudaStreamDestroy(S->copy);
        delete S;
        cudaGetLastError();
        h->err = "could not start serving";
        return LOUVAIN_ERR_OOM;
    }
    h->server = S;
    return LOUVAIN_OK;
}

int louvain_submit(louvain_handle *h, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                   const int32_t *weights, int ptr_kind, uint64_t *ticket)
{
    if (!h) return LOUVAIN_ERR_INVALID_ARG;
    Server *S = (Server *)h->server;
    h->err.clear();
    if (!S || !ticket) {
        h->err = !S ? "serving is not open" : "ticket is NULL";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (ptr_kind != LOUVAIN_PTR_HOST || n < 0 || !row_ptr) {
        h->err = "louvain_submit takes host arrays (ptr_kind LOUVAIN_PTR_HOST) and n >= 0";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    if (n > INT32_MAX) {
        h->err = "n above 2^31 - 1";
        return LOUVAIN_ERR_TOO_LARGE;
    }
    if (row_ptr[0] != 0 || row_ptr[n] < 0) {
        h->err = "row_ptr[0] must be 0 and row_ptr[n] >= 0";
        return LOUVAIN_ERR_INDEX_RANGE;
    }
    const int64_t nnz = row_ptr[n];
    if (nnz > 0 && !col_idx) {
        h->err = "col_idx is NULL";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    Request *r = new (std::nothrow) Request();
    louvain_result *res = new (std::nothrow) louvain_result();
    if (!r || !res) {
        delete r;
        delete res;
        return LOUVAIN_ERR_OOM;
    }
    try {
        r->n = n;
        r->nnz = nnz;
        r->rp.assign(row_ptr, row_ptr + n + 1);
        r->col.assign(col_idx, col_idx + nnz);
        if (weights) r->w.assign(weights, weights + nnz);
    } catch (const std::bad_alloc &) {
        delete r;
        delete res;
        return LOUVAIN_ERR_OOM;
    }
    res->device = h->device;
    res->ff = h->cfg.free;
    res->ctx = h->cfg.alloc_ctx;
    res->n0 = n;
    r->res = res;
    r->footprint = footprint_estimate(n, nnz);
    r->t_submit = now_ms();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) {
        delete r;
        delete res;
        h->err = "serving is closing";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    r->ticket = S->next_ticket++;
    S->tickets[r->ticket] = r;
    S->queue.push_back(r);
    S->admit_locked();
    *ticket = r->ticket;
    return LOUVAIN_OK;
}

int louvain_poll(louvain_handle *h, uint64_t ticket, int wait_ms, louvain_result **out)
{
    if (!h) return LOUVAIN_ERR_INVALID_ARG;
    Server *S = (Server *)h->server;
    if (!S || !out) {
        h->err = !S ? "serving is not open" : "out is NULL";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    *out = nullptr;
    Request *r = nullptr;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->tickets.find(ticket);
        if (it == S->tickets.end()) {
            h->err = "unknown ticket";
            return LOUVAIN_ERR_INVALID_ARG;
        }
        r = it->second;
        auto is_done = [&] { return r->state == kDone; };
        if (wait_ms < 0) S->cv.wait(lk, is_done);
        else if (wait_ms > 0) S->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), is_done);
        if (!is_done()) return LOUVAIN_PENDING;
        S->tickets.erase(it);
    }
    const int rc = r->rc;
    if (rc == LOUVAIN_OK) {
        *out = r->res;
    } else {
        h->err = r->err;
        louvain_result_free(r->res);
    }
    delete r;
    return rc;
}

int louvain_serve_status(const louvain_handle *h, int64_t status[4])
{
    if (!h || !status) return LOUVAIN_ERR_INVALID_ARG;
    Server *S = (Server *)h->server;
    if (!S) return LOUVAIN_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    status[0] = (int64_t)S->in_use;
    status[1] = S->slots_used;
    status[2] = (int64_t)S->queue.size();
    int64_t done = 0;
    for (const auto &kv : S->tickets) done += kv.second->state == kDone;
    status[3] = done;
    return LOUVAIN_OK;
}

int louvain_serve_close(louvain_handle *h)
{
    if (!h) return LOUVAIN_ERR_INVALID_ARG;
    Server *S = (Server *)h->server;
    if (!S) return LOUVAIN_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        S->cv.notify_all();
    }
    S->uploader.join();
    S->worker.join();
    for (auto &kv : S->tickets) {  // finished but never polled
        louvain_result_free(kv.second->res);
        delete kv.second;
    }
    S->A_copy.put(S->d_chk);
    cudaStreamSynchronize(S->copy);
    cudaStreamSynchronize(S->compute);
    cudaStreamDestroy(S->compute);
    cudaStreamDestroy(S->copy);
    delete S;
    h->server = nullptr;
    return LOUVAIN_OK;
}

int louvain_result_num_levels(const louvain_result *r) { return r ? (int)r->levels.size() : 0; }

int64_t louvain_result_num_vertices(const louvain_result *r) { return r ? r->n0 : 0; }

int louvain_result_labels(const louvain_result *r, int level, const int32_t **labels,
                          int64_t *ncomm)
{
    if (!r || level < 0 || level >= (int)r->levels.size() || !labels)
        return LOUVAIN_ERR_INVALID_ARG;
    if (r->levels[level].h_labels) {  // copied during the run (host_labels)
        *labels = r->levels[level].h_labels;
        if (ncomm) *ncomm = r->levels[level].ncomm;
        return LOUVAIN_OK;
    }
    if (r->host_labels.size() != r->levels.size()) r->host_labels.resize(r->levels.size());
    std::vector<int32_t> &hl = r->host_labels[level];
    if (hl.size() != (size_t)r->n0) {
        hl.resize(r->n0);
        if (!copy_d2h_staged(r->device, hl.data(), r->levels[level].d_labels,
                             sizeof(int32_t) * (size_t)r->n0)) {
            cudaGetLastError();
            hl.clear();
            return LOUVAIN_ERR_CUDA;
        }
    }
    *labels = hl.data();
    if (ncomm) *ncomm = r->levels[level].ncomm;
    return LOUVAIN_OK;
}

int louvain_result_labels_into(const louvain_result *r, int level, int32_t *dst)
{
    if (!r || level < 0 || level >= (int)r->levels.size() || (!dst && r->n0 > 0))
        return LOUVAIN_ERR_INVALID_ARG;
    if (r->n0 == 0) return LOUVAIN_OK;
    if (r->levels[level].h_labels) {  // copied during the run (host_labels): a host copy
        parallel_memcpy((char *)dst, (const char *)r->levels[level].h_labels,
                        sizeof(int32_t) * (size_t)r->n0, 8);
        return LOUVAIN_OK;
    }
    if (!copy_d2h_staged(r->device, dst, r->levels[level].d_labels,
                         sizeof(int32_t) * (size_t)r->n0)) {
        cudaGetLastError();
        return LOUVAIN_ERR_CUDA;
    }
    return LOUVAIN_OK;
}

int louvain_result_labels_device(const louvain_result *r, int level, const int32_t **labels)
{
    if (!r || level < 0 || level >= (int)r->levels.size() || !labels)
        return LOUVAIN_ERR_INVALID_ARG;
    *labels = r->levels[level].d_labels;
    return LOUVAIN_OK;
}

int louvain_result_modularity(const louvain_result *r, int level, double *q, int64_t qn[2],
                              int64_t qn_init[2], int64_t *tw)
{
    if (!r || level < 0 || level >= (int)r->levels.size()) return LOUVAIN_ERR_INVALID_ARG;
    const LevelRec &L = r->levels[level];
    if (q) {
        const i128 tw2 = (i128)r->tw * r->tw;
        *q = (double)L.qn / (double)tw2;
    }
    if (qn) i128_to_limbs(L.qn, qn);
    if (qn_init) i128_to_limbs(L.qn_init, qn_init);
    if (tw) *tw = r->tw;
    return LOUVAIN_OK;
}

int louvain_result_level_info(const louvain_result *r, int level, int32_t *iters,
                              int64_t *n_level, int64_t *nnz_level, int64_t *ncomm,
                              int32_t *hit_iter_cap)
{
    if (!r || level < 0 || level >= (int)r->levels.size()) return LOUVAIN_ERR_INVALID_ARG;
    const LevelRec &L = r->levels[level];
    if (iters) *iters = L.iters;
    if (n_level) *n_level = L.n;
    if (nnz_level) *nnz_level = L.nnz;
    if (ncomm) *ncomm = L.ncomm;
    if (hit_iter_cap) *hit_iter_cap = L.hit_cap;
    return LOUVAIN_OK;
}

int louvain_result_trace(const louvain_result *r, int64_t *len, int32_t *level, int32_t *iter,
                         int64_t *moved, int64_t *qn)
{
    if (!r) return LOUVAIN_ERR_INVALID_ARG;
    if (len) *len = (int64_t)r->trace.size();
    for (size_t t = 0; t < r->trace.size(); t++) {
        if (level) level[t] = r->trace[t].level;
        if (iter) iter[t] = r->trace[t].iter;
        if (moved) moved[t] = r->trace[t].moved;
        if (qn) i128_to_limbs(r->trace[t].qn, qn + 2 * t);
    }
    return LOUVAIN_OK;
}

int louvain_result_counters(const louvain_result *r, int64_t counters[8], double times_ms[8])
{
    if (!r) return LOUVAIN_ERR_INVALID_ARG;
    for (int k = 0; k < 8; k++) {
        if (counters) counters[k] = r->counters[k];
        if (times_ms) times_ms[k] = r->times[k];
    }
    return LOUVAIN_OK;
}

int louvain_result_exec_info(const louvain_result *r, int64_t info[6])
{
    if (!r || !info) return LOUVAIN_ERR_INVALID_ARG;
    for (int k = 0; k < 6; k++) info[k] = r->exec_info[k];
    return LOUVAIN_OK;
}

int louvain_num_bins(void) { return kNumBins; }

int louvain_result_bin_stats(const louvain_result *r, int bin, double *time_ms,
                             int64_t *launches, int64_t *alg_bytes, int64_t *rows,
                             int64_t *entries)
{
    if (!r || bin < 0 || bin >= 2 * kNumBins) return LOUVAIN_ERR_INVALID_ARG;
    if (time_ms) *time_ms = r->bin_time[bin];
    if (launches) *launches = r->bin_launches[bin];
    if (alg_bytes) *alg_bytes = (int64_t)r->bin_bytes[bin];
    if (rows) *rows = r->bin_rows[bin];
    if (entries) *entries = r->bin_entries[bin];
    return LOUVAIN_OK;
}

int louvain_result_coarsen_stats(const louvain_result *r, int64_t *inductions,
                                 int64_t *alg_bytes, double *time_ms)
{
    if (!r) return LOUVAIN_ERR_INVALID_ARG;
    if (inductions) *inductions = r->acc_inductions;
    if (alg_bytes) *alg_bytes = (int64_t)r->acc_coarsen_bytes;
    if (time_ms) *time_ms = r->acc_coarsen_ms;
    return LOUVAIN_OK;
}

void louvain_result_free(louvain_result *r)
{
    if (!r) return;
    r->stores.clear();  // label arrays go with the last result that refers to them
    delete r;
}

}  // extern "C"
