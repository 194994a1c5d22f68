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
#include <chrono>
#include <climits>
#include <memory>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/louvain.h"
#include "lv_common.cuh"
#include "lv_kernels.h"
#include "lv_scan.cuh"

using namespace lv;

namespace {

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
    SweepStats st;
    LevelCtl ctl;
    int32_t bin_counts[40];
    int32_t ccounts[16];
    u64 cand_total[16];
    int32_t tail[8];
};

bool host_below_threshold(i128 qn_new, i128 qn_old, i64 tw, i64 num, i64 den)
{
    const i128 diff = qn_new - qn_old;
    if (diff < 0) return true;
    const u128 tw2 = (u128)(u64)tw * (u64)tw;
    const u128 x = (u128)diff;
    const u128 xl = (u128)(u64)x * (u64)den, xh = (u128)(u64)(x >> 64) * (u64)den;
    const u128 yl = (u128)(u64)tw2 * (u64)num, yh = (u128)(u64)(tw2 >> 64) * (u64)num;
    const u128 xmid = (xl >> 64) + (u64)xh, ymid = (yl >> 64) + (u64)yh;
    const u64 x2 = (u64)(xh >> 64) + (u64)(xmid >> 64), y2 = (u64)(yh >> 64) + (u64)(ymid >> 64);
    if (x2 != y2) return x2 < y2;
    if ((u64)xmid != (u64)ymid) return (u64)xmid < (u64)ymid;
    return (u64)xl < (u64)yl;
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
};

struct TraceRec {
    int32_t level, iter;
    int64_t moved;
    i128 qn;
};

struct louvain_handle {
    louvain_config cfg;
    int device = 0;
    std::string err;
    LaunchCfg lc;
    Scalars *pinned = nullptr;
};

// Label arrays of a batch, shared by the results of its graphs; freed with the last one.
struct LabelStore {
    std::vector<int32_t *> arrays;
    louvain_free_fn ff = nullptr;
    void *ctx = nullptr;
    int device = 0;
    ~LabelStore()
    {
        cudaSetDevice(device);
        for (int32_t *p : arrays) {
            if (ff) ff(p, ctx, nullptr);
            else cudaFreeAsync(p, nullptr);
        }
    }
};

struct louvain_result {
    int64_t n0 = 0;
    int batch_index = -1;  // graph index in its batch, -1 for a plain run
    std::shared_ptr<LabelStore> store;  // set for the results of a batch
    int64_t tw = 0;
    int device = 0;
    std::vector<LevelRec> levels;
    mutable std::vector<std::vector<int32_t>> host_labels;
    std::vector<TraceRec> trace;
    int64_t counters[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double times[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double bin_time[kNumBins] = {};
    int64_t bin_launches[kNumBins] = {};
    double bin_bytes[kNumBins] = {};
    int64_t bin_rows[kNumBins] = {};
    int64_t bin_entries[kNumBins] = {};
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
    if (bits & ERRF_HASH_FULL) {
        msg = "internal: a hash table overflowed";
        return LOUVAIN_ERR_INTERNAL;
    }
    msg = "internal device check failed";
    return LOUVAIN_ERR_INTERNAL;
}

struct Runner {
    louvain_handle *h;
    cudaStream_t s;
    DevAlloc A;
    Scalars *d_sc = nullptr;
    DBuf<Scalars> sc_buf;
    int kernels = 0;

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

    // One graph (gvptr null, NG = 1) or a batch of NG graphs stored as one CSR whose graph g
    // owns vertices [gvptr[g], gvptr[g+1]); out holds one result per graph.
    void run(int64_t n0, const int64_t *rp, const int32_t *col, const int32_t *w, int kind,
             int NG, const int64_t *gvptr, const int64_t *geptr,
             std::vector<louvain_result *> &out);
};

void Runner::run(int64_t n0, const int64_t *rp_in, const int32_t *col_in, const int32_t *w_in,
                 int kind, int NG, const int64_t *gvptr, const int64_t *geptr,
                 std::vector<louvain_result *> &out)
{
    const louvain_config &cfg = h->cfg;
    const double wall0 = now_ms();
    const LaunchCfg &lc = h->lc;
    const bool batch = gvptr != nullptr;  // a batch of NG graphs, else one graph (NG = 1)
    sc_buf.reset(&A, 1);
    d_sc = sc_buf.p;
    CK(cudaMemsetAsync(d_sc, 0, sizeof(Scalars), s));

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
            w_own.reset(&A, (size_t)nnz);
            if (nnz)
                CK(cudaMemcpyAsync(w_own.p, w_in, sizeof(int32_t) * (size_t)nnz,
                                   cudaMemcpyHostToDevice, s));
            d_w = w_own.p;
        }
    } else {
        const int64_t r0 = read_one(rp_in);
        nnz = read_one(rp_in + n0);
        if (r0 != 0) throw LvErr{LOUVAIN_ERR_INDEX_RANGE, "row_ptr[0] must be 0"};
        if (nnz < 0) throw LvErr{LOUVAIN_ERR_INDEX_RANGE, "row_ptr[n] is negative"};
        if (nnz > 0 && !col_in) throw LvErr{LOUVAIN_ERR_INVALID_ARG, "col_idx is NULL"};
    }
    if (!d_w) {
        w_own.reset(&A, (size_t)nnz);
        kernels += launch_fill_ones(w_own.p, nnz, s, lc);
        d_w = w_own.p;
    }
    for (int g = 0; g < NG; g++) {
        out[g]->n0 = batch ? gvptr[g + 1] - gvptr[g] : n0;
        out[g]->batch_index = batch ? g : -1;
    }
    if (n0 == 0) {
        CK(cudaStreamSynchronize(s));
        for (int g = 0; g < NG; g++) out[g]->times[3] = now_ms() - wall0;
        return;
    }

    DevGraph G;
    G.n = n0;
    G.nnz = nnz;
    G.rp = d_rp;
    G.col = d_col;
    G.w = d_w;
    G.wbytes = 4;

    // ---------------- validation and weighted degrees (Sec. 2)
    kernels += launch_validate_rowptr(d_rp, n0, &d_sc->err, s, lc);
    sync_scalars();  // row offsets must be sane before any row is read
    // batch bookkeeping: vertex offsets of every graph at the current level, the graph of
    // every vertex (current level and level 0), per-graph 2W, controllers and statistics
    DBuf<int64_t> d_gptr, d_gptr_next, d_base1, d_gnnz;
    DBuf<int32_t> d_vg, d_vg_next, d_vg0, d_rec, d_keep, map0;
    DBuf<u64> d_gtw;
    DBuf<SweepStats> d_stats;
    DBuf<LevelCtl> d_ctls;
    std::vector<int64_t> h_gptr(NG + 1), h_gnnz(NG + 1), h_base1(NG + 1);
    if (batch) {
        for (int g = 0; g <= NG; g++) h_gptr[g] = gvptr[g];
        d_gptr.reset(&A, NG + 1);
        d_gptr_next.reset(&A, NG + 1);
        d_base1.reset(&A, NG + 1);
        d_gnnz.reset(&A, NG + 1);
        CK(cudaMemcpyAsync(d_gptr.p, h_gptr.data(), sizeof(int64_t) * (NG + 1),
                           cudaMemcpyHostToDevice, s));
        kernels += launch_gather64(d_rp, d_gptr.p, NG + 1, d_gnnz.p, s);
        CK(cudaMemcpyAsync(h_gnnz.data(), d_gnnz.p, sizeof(int64_t) * (NG + 1),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (geptr)
            for (int g = 0; g <= NG; g++)
                if (geptr[g] != h_gnnz[g])
                    throw LvErr{LOUVAIN_ERR_INDEX_RANGE,
                                "graph_eptr[" + std::to_string(g) + "] != row_ptr[graph_vptr[g]]"};
        d_vg.reset(&A, n0);
        d_vg_next.reset(&A, n0);
        d_vg0.reset(&A, n0);
        d_rec.reset(&A, NG);
        d_keep.reset(&A, NG);
        map0.reset(&A, n0);
        d_gtw.reset(&A, NG);
        d_stats.reset(&A, NG);
        d_ctls.reset(&A, NG);
        CK(cudaMemsetAsync(d_gtw.p, 0, sizeof(u64) * NG, s));
        CK(cudaMemsetAsync(d_stats.p, 0, sizeof(SweepStats) * NG, s));
        kernels += launch_graph_ids(n0, d_gptr.p, NG, d_vg0.p, s, lc);
        CK(cudaMemcpyAsync(d_vg.p, d_vg0.p, sizeof(int32_t) * n0, cudaMemcpyDeviceToDevice, s));
    } else {
        h_gptr[0] = 0;
        h_gptr[1] = n0;
        h_gnnz[0] = 0;
        h_gnnz[1] = nnz;
    }
    DBuf<i64> delta, delta_next, deg;
    DBuf<int32_t> C, Cnext, size, new_id, new_id2;
    delta.reset(&A, n0);
    delta_next.reset(&A, n0);
    deg.reset(&A, n0);
    C.reset(&A, n0);
    Cnext.reset(&A, n0);
    size.reset(&A, n0);
    new_id.reset(&A, (size_t)n0 + 1);
    DBuf<int32_t> lists;  // rows of bins 1.., grouped by bin
    lists.reset(&A, (size_t)n0);
    // bin thresholds: every table must fit shared memory with the chosen sum width; the
    // cluster bins hold rows up to CL times the bin-5 bound (CL CTAs, bin-5 table each);
    // cluster sizes that cannot be resident are left empty.
    auto make_proto = [&](bool narrow_sums) {
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
        return pr;
    };
    // degree bins of graph G: count, then fill the list grouped by bin
    auto make_bins = [&](const DevGraph &gr, const Bins &pr, const int32_t *vg = nullptr,
                         const LevelCtl *gctl = nullptr) {
        Bins bins = pr;
        bins.list = lists.p;
        bins.counts = &d_sc->bin_counts[0];
        kernels += launch_bin_count(gr, bins, s, lc, vg, gctl);
        sync_scalars();
        bins.off[0] = bins.off[1] = 0;
        for (int b = 0; b < kNumBins; b++) {
            bins.nlist[b] = h->pinned->bin_counts[b];
            memcpy(&bins.entries[b], &h->pinned->bin_counts[16 + 2 * b], sizeof(int64_t));
            if (b >= 1) bins.off[b + 1] = bins.off[b] + bins.nlist[b];
        }
        kernels += launch_bin_fill(gr, bins, s, lc, vg, gctl);
        return bins;
    };
    const Bins proto_narrow = make_proto(true);
    Bins bins0 = make_bins(G, proto_narrow);
    kernels += launch_row_sums(G, bins0, batch ? d_vg.p : nullptr, batch ? d_gptr.p : nullptr,
                               delta.p, batch ? d_gtw.p : &d_sc->tw, &d_sc->err, s, lc);
    if (cfg.checks >= 2) kernels += launch_check_symmetry(G, &d_sc->err, s, lc);
    sync_scalars();
    std::vector<i64> h_tw(NG);
    if (batch) {
        CK(cudaMemcpyAsync(h_tw.data(), d_gtw.p, sizeof(u64) * NG, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } else {
        h_tw[0] = (i64)h->pinned->tw;
    }
    u64 tw_max = 0;
    for (int g = 0; g < NG; g++) {
        const u64 t = (u64)h_tw[g];
        if (t > ((u64)1 << 62)) throw LvErr{LOUVAIN_ERR_TOO_LARGE, "sum of weights above 2^62"};
        if (t > tw_max) tw_max = t;
        out[g]->tw = h_tw[g];
    }
    const i64 TW = h_tw[0];  // one graph: its 2W (a batch reads 2W per graph on the device)
    // gains in int128 when some graph's (2W)^2 leaves int64; 32-bit table sums when every
    // graph's 2W fits (a table sum never exceeds its graph's 2W)
    const bool wide = cfg.force_int128 || (u128)tw_max * tw_max > (u128)INT64_MAX;
    const bool narrow = !cfg.wide_sums && tw_max < ((u64)1 << 32);

    // ---------------- per-run buffers sized by level 0 (Theorem 1: levels never grow)
    const int64_t scratch_n = scan_scratch_elems(n0 + 1) + 64;
    DBuf<int32_t> b_nch, b_chunk_first, b_glog2, b_gcnt, b_gdone;
    DBuf<int64_t> b_gcap, b_goff;
    DBuf<u64> b_gloop;
    b_nch.reset(&A, n0);
    b_chunk_first.reset(&A, (size_t)n0 + 1);
    b_glog2.reset(&A, n0);
    b_gcnt.reset(&A, n0);
    b_gdone.reset(&A, n0);
    b_gcap.reset(&A, n0);
    b_goff.reset(&A, (size_t)n0 + 1);
    b_gloop.reset(&A, n0);
    DBuf<int32_t> scratch32;
    DBuf<int64_t> scratch64;
    scratch32.reset(&A, scratch_n);
    scratch64.reset(&A, scratch_n);
    DBuf<i64> tr_moved, tr_qn;
    const int tcap = cfg.max_iters + 1;
    tr_moved.reset(&A, (size_t)tcap * NG);
    tr_qn.reset(&A, 2 * (size_t)tcap * NG);
    std::vector<i64> h_tr_moved, h_tr_qn;
    // coarsening buffers
    DBuf<int32_t> c_csize, c_moff, c_cursor, c_members, c_ccnt, c_tmp_col;
    DBuf<int64_t> c_mpre;
    DBuf<u64> c_tmp_w;
    // graph buffers of the levels above 0
    DBuf<int64_t> g_rp, g_rp_next;
    DBuf<int32_t> g_col, g_col_next;
    DBuf<unsigned char> g_w, g_w_next;
    DBuf<int32_t> chunk_b;
    DBuf<int32_t> gkeys, glist;
    DBuf<u64> gvals;

    SweepTimers tm;
    double t_kernel[kNumBins] = {};
    int64_t launches_kernel[kNumBins] = {};
    double bytes_kernel[kNumBins] = {};
    cudaEvent_t coarsen_ev[2] = {nullptr, nullptr};
    double t_coarsen = 0.0;
    if (cfg.profile) {
        for (auto &e : tm.ev) CK(cudaEventCreate(&e));
        CK(cudaEventCreate(&coarsen_ev[0]));
        CK(cudaEventCreate(&coarsen_ev[1]));
        tm.on = true;
    }
    struct EvGuard {
        SweepTimers *t;
        cudaEvent_t *ce;
        ~EvGuard()
        {
            if (t->on) {
                for (auto &e : t->ev) cudaEventDestroy(e);
                cudaEventDestroy(ce[0]);
                cudaEventDestroy(ce[1]);
            }
        }
    } evg{&tm, coarsen_ev};

    PhaseState st;
    st.C = C.p;
    st.Cnext = Cnext.p;
    st.deg = deg.p;
    st.size = size.p;
    st.delta = delta.p;

    Bins proto = make_proto(narrow);
    const bool reuse_bins0 = narrow;  // level-0 bins were made with these thresholds
    proto.nch = b_nch.p;
    proto.chunk_first = b_chunk_first.p;
    proto.gcap = b_gcap.p;
    proto.goff = b_goff.p;
    proto.glog2 = b_glog2.p;
    proto.gcnt = b_gcnt.p;
    proto.gdone = b_gdone.p;
    proto.gloop = b_gloop.p;

    // sets up chunk lists and global tables of the chunked bin (after its size is known)
    auto prep_huge = [&](Bins &b, bool coarsen_side, int64_t k_comm, CoarsenBufs *cbp) {
        b.nchunks = 0;
        b.gslots = 0;
        const int nb = b.nlist[kChunkedBin];
        if (nb == 0) return;
        if (coarsen_side) kernels += launch_coarsen_bigprep(k_comm, *cbp, b, s, lc);
        else kernels += launch_big_prep(G, b, scratch64.p, scratch32.p, s, lc);
        b.nchunks = read_one(b_chunk_first.p + nb);
        b.gslots = read_one(b_goff.p + nb);
        chunk_b.reset(&A, b.nchunks);
        b.chunk_b = chunk_b.p;
        kernels += launch_big_fill(b, s, lc);
        if (b.gslots > 0) {
            gkeys.reset(&A, b.gslots);
            gvals.reset(&A, b.gslots);  // 8 bytes per slot covers both sum widths
            glist.reset(&A, b.gslots);
            CK(cudaMemsetAsync(gkeys.p, 0xFF, sizeof(int32_t) * b.gslots, s));
            CK(cudaMemsetAsync(gvals.p, 0, sizeof(u64) * b.gslots, s));
        }
        b.gkeys = gkeys.p;
        b.gvals = gvals.p;
        b.glist = glist.p;
        CK(cudaMemsetAsync(b_gcnt.p, 0, sizeof(int32_t) * nb, s));
        CK(cudaMemsetAsync(b_gdone.p, 0, sizeof(int32_t) * nb, s));
        CK(cudaMemsetAsync(b_gloop.p, 0, sizeof(u64) * nb, s));
    };

    // labels of the original vertices, one array of n0 per level; in a batch, the arrays
    // are shared by the graphs' results (graph g's labels start at gvptr[g])
    std::shared_ptr<LabelStore> store;
    if (batch) {
        store = std::make_shared<LabelStore>();
        store->ff = cfg.free;
        store->ctx = cfg.alloc_ctx;
        store->device = h->device;
        for (int g = 0; g < NG; g++) out[g]->store = store;
    }
    const int32_t *prev_labels = nullptr;
    // per-graph state: in the current level's graph, finished, previous level's Qn
    std::vector<char> active(NG, 1), rec(NG, 0), keep(NG, 0);
    std::vector<i128> qn_prev_level(NG, 0);
    std::vector<int64_t> visits(NG, 0);
    for (int g = 0; g < NG; g++)
        if (h_gptr[g + 1] == h_gptr[g]) active[g] = 0;  // an empty graph has no phase
    std::vector<LevelCtl> h_ctl(NG);
    int64_t edge_visits = 0, sweeps_launched = 0;
    double alg_bytes = 0.0;
    u64 cand_all = 0;
    LevelCtl *ctl_dev = batch ? d_ctls.p : &d_sc->ctl;
    SweepStats *st_dev = batch ? d_stats.p : &d_sc->st;
    BatchCtx bc;
    if (batch) {
        bc.gtw = (const i64 *)d_gtw.p;
        bc.gctl = d_ctls.p;
    }

    for (int level = 0; level < cfg.max_levels; level++) {
        const int64_t n = G.n;
        if (level > 0) {
            delta.swap(delta_next);
            st.delta = delta.p;
        }
        bc.vg = batch ? d_vg.p : nullptr;
        kernels += launch_init_state(n, st, s, lc);
        if (cfg.vertex_following && (level == 0 || cfg.vf_all_levels))
            kernels += launch_vertex_following(G, st, s, lc);

        // degree bins (level 0 reuses the bins made for the row sums)
        Bins bins;
        if (level == 0 && reuse_bins0) {
            bins = proto;
            bins.list = bins0.list;
            bins.counts = bins0.counts;
            for (int b = 0; b <= kNumBins; b++) bins.off[b] = bins0.off[b];
            for (int b = 0; b < kNumBins; b++) {
                bins.nlist[b] = bins0.nlist[b];
                bins.entries[b] = bins0.entries[b];
            }
        } else {
            bins = make_bins(G, proto);
        }
        prep_huge(bins, false, 0, nullptr);

        // phase controllers (graphs without a phase at this level start stopped)
        int ninactive = 0;
        for (int g = 0; g < NG; g++) {
            LevelCtl &c = h_ctl[g];
            memset(&c, 0, sizeof(c));
            c.tw = h_tw[g];
            c.theta_num = cfg.theta_num;
            c.theta_den = cfg.theta_den;
            c.max_iters = cfg.max_iters;
            c.done = active[g] ? 0 : 1;
            ninactive += !active[g];
        }
        if (batch) {
            CK(cudaMemcpyAsync(d_ctls.p, h_ctl.data(), sizeof(LevelCtl) * NG,
                               cudaMemcpyHostToDevice, s));
        } else {
            h->pinned->ctl = h_ctl[0];
            CK(cudaMemcpyAsync(&d_sc->ctl, &h->pinned->ctl, sizeof(LevelCtl),
                               cudaMemcpyHostToDevice, s));
            CK(cudaMemsetAsync(&d_sc->st, 0, sizeof(SweepStats), s));
        }
        h->pinned->ndone = ninactive;
        CK(cudaMemcpyAsync(&d_sc->ndone, &h->pinned->ndone, sizeof(int32_t),
                           cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(&d_sc->cand_total[0], 0, sizeof(u64) * 16, s));

        // sweeps (Algorithm 1); one host read of the controllers' count per sweep
        // algorithmic bytes of one sweep over the current bins (formula in louvain.h)
        auto account_sweep = [&](const Bins &bb) {
            const double per_entry = 8.0 + (double)G.wbytes;
            for (int b = 0; b < kNumBins; b++) {
                double kb = (double)bb.entries[b] * per_entry;
                kb += b == 0 ? (double)n * 16.0 + (double)bb.nlist[0] * 24.0
                             : (double)bb.nlist[b] * 36.0;
                bytes_kernel[b] += kb;
                alg_bytes += kb;
                const int64_t rows = b == 0 ? n : bb.nlist[b];
                for (int g = 0; g < NG; g++) {
                    out[g]->bin_rows[b] += rows;
                    out[g]->bin_entries[b] += bb.entries[b];
                }
            }
        };
        int sweeps = 0;
        int ndone_binned = ninactive;
        for (;;) {
            kernels += launch_sweep(G, st, bins, TW, wide, narrow, st_dev, &d_sc->err, s, lc,
                                    &tm, bc);
            kernels += launch_decide(st_dev, ctl_dev, NG, tr_moved.p, tr_qn.p,
                                     &d_sc->cand_total[0], &d_sc->ndone, s);
            kernels += launch_apply(n, st, ctl_dev, bc.vg, s, lc);
            sweeps++;
            account_sweep(bins);
            sync_scalars();
            for (int b = 0; b < kNumBins; b++) {
                if (tm.on) {
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, tm.ev[2 * b], tm.ev[2 * b + 1]));
                    t_kernel[b] += ms;
                }
                launches_kernel[b] +=
                    b == 0 ? 1 : (b == kChunkedBin ? bins.nchunks > 0 : bins.nlist[b] > 0);
            }
            const int ndone = h->pinned->ndone;
            if (ndone >= NG) break;
            if (sweeps > cfg.max_iters + 2)
                throw LvErr{LOUVAIN_ERR_INTERNAL, "phase controller did not stop"};
            if (batch && ndone > ndone_binned) {
                // some graphs stopped: bin again without their rows
                bins = make_bins(G, proto, d_vg.p, d_ctls.p);
                prep_huge(bins, false, 0, nullptr);
                ndone_binned = ndone;
            }
        }
        sweeps_launched += sweeps;
        if (batch) {
            CK(cudaMemcpyAsync(h_ctl.data(), d_ctls.p, sizeof(LevelCtl) * NG,
                               cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        } else {
            h_ctl[0] = h->pinned->ctl;
        }
        u64 cand_level[kNumBins];
        for (int b = 0; b < kNumBins; b++) cand_level[b] = h->pinned->cand_total[b];
        int max_iters_run = 0;
        for (int g = 0; g < NG; g++)
            if (active[g] && h_ctl[g].iters > max_iters_run) max_iters_run = h_ctl[g].iters;
        if (max_iters_run > 0) {
            const size_t cnt = (size_t)max_iters_run * NG;
            h_tr_moved.resize(cnt);
            h_tr_qn.resize(2 * cnt);
            CK(cudaMemcpyAsync(h_tr_moved.data(), tr_moved.p, sizeof(i64) * cnt,
                               cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(h_tr_qn.data(), tr_qn.p, sizeof(i64) * 2 * cnt,
                               cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        }
        for (int g = 0; g < NG; g++) {
            if (!active[g]) continue;
            const int it = h_ctl[g].iters;
            for (int t = 0; t < it; t++) {
                const size_t e = (size_t)t * NG + g;
                out[g]->trace.push_back(
                    TraceRec{level, t + 1, h_tr_moved[e], limbs_to_i128(&h_tr_qn[2 * e])});
            }
            const int64_t nnz_g = h_gnnz[g + 1] - h_gnnz[g];
            visits[g] += (int64_t)it * nnz_g;
            edge_visits += (int64_t)it * nnz_g;
        }
        // candidate reads (8 bytes each) of the sweeps of this phase
        for (int b = 0; b < kNumBins; b++) {
            bytes_kernel[b] += 8.0 * (double)cand_level[b];
            alg_bytes += 8.0 * (double)cand_level[b];
            cand_all += cand_level[b];
        }

        // renumber (Sec. 5.1.2) -- labels of used communities in increasing order; labels
        // of one graph are contiguous, so the scan also numbers each graph's communities
        kernels += launch_renumber(n, size.p, nullptr, nullptr, new_id.p, scratch32.p, s);
        std::vector<int64_t> kg(NG, 0);
        if (batch) {
            kernels += launch_gather_ids(new_id.p, d_gptr.p, NG + 1, d_base1.p, s);
            CK(cudaMemcpyAsync(h_base1.data(), d_base1.p, sizeof(int64_t) * (NG + 1),
                               cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int g = 0; g < NG; g++) kg[g] = h_base1[g + 1] - h_base1[g];
        } else {
            kg[0] = read_one(new_id.p + n);
        }
        // record the level for every graph that merged something (a graph whose phase
        // merged nothing is finished: no new level), then the outer test of Algorithm 2
        int nrec = 0, nkeep = 0;
        int64_t k_next = 0, n_keep = 0;
        bool all_active_kept = true;
        for (int g = 0; g < NG; g++) {
            const int64_t ng = h_gptr[g + 1] - h_gptr[g];
            rec[g] = active[g] && kg[g] < ng;
            keep[g] = 0;
            if (!rec[g]) {
                if (active[g]) all_active_kept = false;
                active[g] = 0;
                continue;
            }
            nrec++;
            const LevelCtl &hc = h_ctl[g];
            LevelRec r;
            r.ncomm = kg[g];
            r.qn = limbs_to_i128(hc.qn_final);
            r.qn_init = limbs_to_i128(hc.qn_init);
            r.iters = hc.iters;
            r.n = ng;
            r.nnz = h_gnnz[g + 1] - h_gnnz[g];
            r.hit_cap = hc.hit_cap;
            out[g]->levels.push_back(r);
            const bool stop =
                (level >= 1 && host_below_threshold(r.qn, qn_prev_level[g], h_tw[g],
                                                    cfg.theta_num, cfg.theta_den)) ||
                level + 1 >= cfg.max_levels;
            qn_prev_level[g] = r.qn;
            if (stop) {
                all_active_kept = false;
                active[g] = 0;
            } else {
                keep[g] = 1;
                nkeep++;
                k_next += kg[g];
                n_keep += ng;
            }
        }
        if (nrec == 0) break;
        int32_t *d_labels = (int32_t *)A.get(sizeof(int32_t) * (size_t)n0);
        if (batch) {
            store->arrays.push_back(d_labels);
            for (int g = 0; g < NG; g++)
                if (rec[g]) out[g]->levels.back().d_labels = d_labels + gvptr[g];
        } else {
            out[0]->levels.back().d_labels = d_labels;
        }
        // next-level numbering: the kept graphs' communities only
        const int32_t *nid2 = new_id.p;
        if (batch) {
            std::vector<int32_t> hk(NG), hr(NG);
            for (int g = 0; g < NG; g++) {
                hr[g] = rec[g];
                hk[g] = keep[g];
            }
            CK(cudaMemcpyAsync(d_rec.p, hr.data(), sizeof(int32_t) * NG, cudaMemcpyHostToDevice,
                               s));
            CK(cudaMemcpyAsync(d_keep.p, hk.data(), sizeof(int32_t) * NG,
                               cudaMemcpyHostToDevice, s));
            if (nkeep > 0 && !all_active_kept) {
                if (!new_id2.p) new_id2.reset(&A, (size_t)n0 + 1);
                kernels += launch_renumber(n, size.p, d_vg.p, d_keep.p, new_id2.p, scratch32.p, s);
                nid2 = new_id2.p;
            }
            kernels += launch_compose(n0, d_vg0.p, d_rec.p, d_keep.p, level == 0 ? nullptr : map0.p,
                                      map0.p, st.C, new_id.p, d_base1.p, nid2, d_labels, s, lc);
            CK(cudaStreamSynchronize(s));  // host vectors above are copied before they go
        } else {
            kernels += launch_compose(n0, nullptr, nullptr, nullptr, prev_labels, nullptr, st.C,
                                      new_id.p, nullptr, nullptr, d_labels, s, lc);
            prev_labels = d_labels;
        }
        if (nkeep == 0) break;

        // ---------------- induce the next graph (Sec. 5.1.2)
        if (!c_csize.p) {
            c_csize.reset(&A, n0);
            c_moff.reset(&A, (size_t)n0 + 1);
            c_cursor.reset(&A, n0);
            c_members.reset(&A, n0);
            c_mpre.reset(&A, (size_t)n0 + 1);
            c_ccnt.reset(&A, n0);
            c_tmp_col.reset(&A, (size_t)nnz);
            c_tmp_w.reset(&A, (size_t)nnz);
        }
        CoarsenBufs cb;
        cb.csize = c_csize.p;
        cb.moff = c_moff.p;
        cb.cursor = c_cursor.p;
        cb.members = c_members.p;
        cb.mpre = c_mpre.p;
        cb.ccnt = c_ccnt.p;
        cb.tmp_col = c_tmp_col.p;
        cb.tmp_w = c_tmp_w.p;
        cb.counts = &d_sc->ccounts[0];
        cb.scratch32 = scratch32.p;
        cb.scratch64 = scratch64.p;
        if (tm.on) CK(cudaEventRecord(coarsen_ev[0], s));
        Bins cbins = proto;
        const int64_t k = k_next;
        kernels += launch_coarsen_stage1(G, st, nid2, k, batch ? n_keep : n,
                                         batch ? d_vg.p : nullptr, batch ? d_keep.p : nullptr,
                                         batch ? d_vg_next.p : nullptr, delta_next.p, cb, cbins,
                                         s, lc);
        sync_scalars();
        cbins.list = lists.p;  // the sweep's lists are free again
        cbins.off[0] = cbins.off[1] = cbins.off[2] = 0;
        for (int b = 0; b < kNumBins; b++) {
            cbins.nlist[b] = b < 2 ? 0 : h->pinned->ccounts[b];
            if (b >= 2) cbins.off[b + 1] = cbins.off[b] + cbins.nlist[b];
        }
        kernels += launch_coarsen_binfill(k, cb, cbins, s, lc);
        prep_huge(cbins, true, k, &cb);
        kernels += launch_coarsen_stage2(G, st, nid2, k, cb, cbins, narrow, &d_sc->err, s, lc);
        g_rp_next.reset(&A, (size_t)k + 1);
        kernels += launch_coarsen_rowptr(k, cb, g_rp_next.p, s);
        sync_scalars();
        const int64_t nnz_next = read_one(g_rp_next.p + k);
        const int wb_next = tw_max <= (u64)INT32_MAX ? 4 : 8;
        g_col_next.reset(&A, (size_t)nnz_next);
        g_w_next.reset(&A, (size_t)nnz_next * wb_next);
        kernels += launch_coarsen_compact(k, nnz_next, cb, g_rp_next.p, g_col_next.p,
                                          g_w_next.p, wb_next, s, lc);
        if (tm.on) {
            CK(cudaEventRecord(coarsen_ev[1], s));
            CK(cudaEventSynchronize(coarsen_ev[1]));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, coarsen_ev[0], coarsen_ev[1]));
            t_coarsen += ms;
        }
        g_rp.swap(g_rp_next);
        g_col.swap(g_col_next);
        g_w.swap(g_w_next);
        g_rp_next.release();
        g_col_next.release();
        g_w_next.release();
        G.n = k;
        G.nnz = nnz_next;
        G.rp = g_rp.p;
        G.col = g_col.p;
        G.w = g_w.p;
        G.wbytes = wb_next;
        if (batch) {
            // vertex and entry offsets of every graph in the next level's graph
            d_vg.swap(d_vg_next);
            kernels += launch_gather_ids(nid2, d_gptr.p, NG + 1, d_gptr_next.p, s);
            d_gptr.swap(d_gptr_next);
            kernels += launch_gather64(G.rp, d_gptr.p, NG + 1, d_gnnz.p, s);
            CK(cudaMemcpyAsync(h_gptr.data(), d_gptr.p, sizeof(int64_t) * (NG + 1),
                               cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(h_gnnz.data(), d_gnnz.p, sizeof(int64_t) * (NG + 1),
                               cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        } else {
            h_gptr[1] = k;
            h_gnnz[1] = nnz_next;
        }
        if (level == 0) {  // the input copies are no longer needed
            rp_own.release();
            col_own.release();
            w_own.release();
        }
    }
    sync_scalars();
    const double wall = now_ms() - wall0;
    for (int g = 0; g < NG; g++) {
        louvain_result *res = out[g];
        res->counters[0] = batch ? visits[g] : edge_visits;
        res->counters[1] = sweeps_launched;
        res->counters[2] = (int64_t)alg_bytes;
        res->counters[3] = (int64_t)cand_all;
        res->counters[4] = kernels;
        if (tm.on) {
            int dom = 0;
            for (int b = 1; b < kNumBins; b++)
                if (t_kernel[b] > t_kernel[dom]) dom = b;
            double tot = 0;
            for (int b = 0; b < kNumBins; b++) tot += t_kernel[b];
            res->times[0] = tot;
            res->times[4] = t_kernel[dom];
            res->times[5] = t_kernel[0];
            res->times[6] = t_kernel[1] + t_kernel[2];
            res->times[7] = t_kernel[3] + t_kernel[4] + t_kernel[5] + t_kernel[6];
            res->counters[5] = launches_kernel[dom];
            res->counters[6] = (int64_t)bytes_kernel[dom];
            res->counters[7] = dom;
            res->times[1] = t_coarsen;
        }
        for (int b = 0; b < kNumBins; b++) {
            res->bin_time[b] = t_kernel[b];
            res->bin_launches[b] = launches_kernel[b];
            res->bin_bytes[b] = bytes_kernel[b];
        }
        res->times[3] = wall;
    }
}

}  // namespace

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
    if (c.chunk_entries == 0) c.chunk_entries = 4096;
    if (c.chunk_entries < 32 || c.chunk_entries > 4096 ||
        (c.chunk_entries & (c.chunk_entries - 1)) != 0) {
        msg = "chunk_entries must be a power of two in [32, 4096]";
        return LOUVAIN_ERR_INVALID_ARG;
    }
    for (int r : c.reserved)
        if (r != 0) {
            msg = "reserved config fields must be zero";
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
    Runner R;
    R.h = h;
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
        R.run(n, row_ptr, col_idx, weights, ptr_kind, 1, nullptr, nullptr, outs);
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
    Runner R;
    R.h = h;
    R.s = (cudaStream_t)stream;
    R.A.fa = h->cfg.alloc;
    R.A.ff = h->cfg.free;
    R.A.ctx = h->cfg.alloc_ctx;
    R.A.s = R.s;
    int rc = LOUVAIN_OK;
    launch_site() = nullptr;
    try {
        CK(cudaSetDevice(h->device));
        R.run(n, row_ptr, col_idx, weights, ptr_kind, num_graphs, graph_vptr, graph_eptr, outs);
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

int louvain_result_num_levels(const louvain_result *r) { return r ? (int)r->levels.size() : 0; }

int64_t louvain_result_num_vertices(const louvain_result *r) { return r ? r->n0 : 0; }

int louvain_result_labels(const louvain_result *r, int level, const int32_t **labels,
                          int64_t *ncomm)
{
    if (!r || level < 0 || level >= (int)r->levels.size() || !labels)
        return LOUVAIN_ERR_INVALID_ARG;
    if (r->host_labels.size() != r->levels.size()) r->host_labels.resize(r->levels.size());
    std::vector<int32_t> &hl = r->host_labels[level];
    if (hl.size() != (size_t)r->n0) {
        hl.resize(r->n0);
        if (cudaSetDevice(r->device) != cudaSuccess ||
            cudaMemcpy(hl.data(), r->levels[level].d_labels, sizeof(int32_t) * (size_t)r->n0,
                       cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            hl.clear();
            return LOUVAIN_ERR_CUDA;
        }
    }
    *labels = hl.data();
    if (ncomm) *ncomm = r->levels[level].ncomm;
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

int louvain_num_bins(void) { return kNumBins; }

int louvain_result_bin_stats(const louvain_result *r, int bin, double *time_ms,
                             int64_t *launches, int64_t *alg_bytes, int64_t *rows,
                             int64_t *entries)
{
    if (!r || bin < 0 || bin >= kNumBins) return LOUVAIN_ERR_INVALID_ARG;
    if (time_ms) *time_ms = r->bin_time[bin];
    if (launches) *launches = r->bin_launches[bin];
    if (alg_bytes) *alg_bytes = (int64_t)r->bin_bytes[bin];
    if (rows) *rows = r->bin_rows[bin];
    if (entries) *entries = r->bin_entries[bin];
    return LOUVAIN_OK;
}

void louvain_result_free(louvain_result *r)
{
    if (!r) return;
    if (r->store) {  // a batch's label arrays go with the last of its results
        r->store.reset();
        delete r;
        return;
    }
    cudaSetDevice(r->device);
    for (LevelRec &L : r->levels) {
        if (!L.d_labels) continue;
        if (r->ff) r->ff(L.d_labels, r->ctx, nullptr);
        else cudaFreeAsync(L.d_labels, nullptr);
        L.d_labels = nullptr;
    }
    delete r;
}

}  // extern "C"
