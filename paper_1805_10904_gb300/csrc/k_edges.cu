// k_edges.cu -- symmetric CSR from an unsorted undirected edge list (the paper's "neighbor
// computation", Sec. 5.1.2: source-target pairs plus their reverses, sorted by (source,
// target), counted per source and prefix-summed into row offsets).
//
// Every non-loop pair (u, v, w) gives the entries (u, v) and (v, u), a loop (u, u) one entry
// (a loop is stored once, as everywhere in this library); entries with the same (row, column)
// are merged by adding their weights.  The sort is a stable least-significant-digit radix
// sort over keys row * 2^b + column (b = bit length of n), 8-bit digits, written here:
// per pass one histogram kernel (per tile and digit), one prefix sum over the digit-major
// table, and one scatter kernel that ranks each tile's keys stably with warp matching.
#include "lv_common.cuh"
#include "lv_kernels.h"
#include "lv_scan.cuh"

namespace lv {
namespace {

constexpr int kSortBlock = 256;
constexpr int kSortItems = 16;                        // keys per thread
constexpr int kSortTile = kSortBlock * kSortItems;    // 4096 keys per CTA
constexpr int kSortWarps = kSortBlock / 32;
constexpr int kDigits = 256;

// Expands edge e into the key/value slots 2e and 2e+1 (the second stays the sentinel for
// a loop); checks endpoints and weights.
__global__ void __launch_bounds__(kBlock) k_expand_edges(int64_t m, int64_t n, int bits,
                                                         const int32_t *src, const int32_t *dst,
                                                         const int32_t *w, u64 *keys,
                                                         int32_t *vals, unsigned *err)
{
    const u64 sentinel = (bits >= 32) ? ~(u64)0 : (((u64)1 << (2 * bits)) - 1);
    unsigned bad = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[e], v = dst[e];
        const int32_t x = w ? w[e] : 1;
        u64 k0 = sentinel, k1 = sentinel;
        if (u < 0 || v < 0 || (int64_t)u >= n || (int64_t)v >= n) {
            bad |= ERRF_INDEX;
        } else if (x < 1) {
            bad |= ERRF_WEIGHT;
        } else {
            k0 = ((u64)u << bits) | (u64)v;
            if (u != v) k1 = ((u64)v << bits) | (u64)u;
        }
        keys[2 * e] = k0;
        keys[2 * e + 1] = k1;
        vals[2 * e] = x;
        vals[2 * e + 1] = x;
    }
    if (bad) atomicOr(err, bad);
}

__device__ __forceinline__ int digit_of(u64 key, int shift) { return (int)((key >> shift) & 255u); }

// Per tile and digit: number of keys (digit-major table hist[d * ntiles + tile]).
__global__ void __launch_bounds__(kSortBlock) k_radix_hist(const u64 *keys, int64_t len,
                                                           int shift, int64_t ntiles,
                                                           int64_t *hist)
{
    __shared__ int s_cnt[kDigits];
    for (int d = threadIdx.x; d < kDigits; d += kSortBlock) s_cnt[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int j = 0; j < kSortItems; j++) {
        const int64_t i = base + (int64_t)j * kSortBlock + threadIdx.x;
        if (i < len) atomicAdd(&s_cnt[digit_of(keys[i], shift)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kDigits; d += kSortBlock)
        hist[(int64_t)d * ntiles + blockIdx.x] = s_cnt[d];
}

// Stable scatter of one tile: warp w owns the tile's keys [w * 512, (w + 1) * 512), taken in
// rounds of 32 consecutive keys; a key's rank among equal digits before it is the warp's
// running count for that digit plus its rank among matching lanes of the round.  The
// warps' totals are then prefix-summed per digit, so keys keep their order.
__global__ void __launch_bounds__(kSortBlock) k_radix_scatter(const u64 *keys_in,
                                                              const int32_t *vals_in,
                                                              int64_t len, int shift,
                                                              int64_t ntiles,
                                                              const int64_t *offs,
                                                              u64 *keys_out, int32_t *vals_out)
{
    __shared__ int s_cnt[kSortWarps][kDigits];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = lane; d < kDigits; d += 32) s_cnt[warp][d] = 0;
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * (kSortItems * 32);
    u64 k[kSortItems];
    int32_t v[kSortItems];
    int rank[kSortItems];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        const int64_t i = base + (int64_t)r * 32 + lane;
        const bool ok = i < len;
        k[r] = ok ? keys_in[i] : 0;
        v[r] = ok ? vals_in[i] : 0;
        const int d = ok ? digit_of(k[r], shift) : kDigits;  // kDigits: no key
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int before = __popc(peers & lt);
        const int cnt0 = d < kDigits ? s_cnt[warp][d] : 0;
        rank[r] = cnt0 + before;
        __syncwarp();
        if (d < kDigits && before == 0) s_cnt[warp][d] = cnt0 + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over the warps, plus the tile's global offset
    __shared__ int64_t s_base[kDigits];
    for (int d = threadIdx.x; d < kDigits; d += kSortBlock) {
        int run = 0;
        for (int w = 0; w < kSortWarps; w++) {
            const int c = s_cnt[w][d];
            s_cnt[w][d] = run;
            run += c;
        }
        s_base[d] = offs[(int64_t)d * ntiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        const int64_t i = base + (int64_t)r * 32 + lane;
        if (i >= len) continue;
        const int d = digit_of(k[r], shift);
        const int64_t p = s_base[d] + s_cnt[warp][d] + rank[r];
        keys_out[p] = k[r];
        vals_out[p] = v[r];
    }
}

// 1 for the first key of every run of equal keys (sentinels excluded)
struct RunHeadIn {
    const u64 *keys;
    u64 sentinel;
    __device__ __forceinline__ int64_t operator()(int64_t i) const
    {
        const u64 k = keys[i];
        return (k != sentinel && (i == 0 || keys[i - 1] != k)) ? 1 : 0;
    }
};

// Entry i of the sorted keys lands at output pos[i + 1] - 1 (the last run head up to i):
// weights are added there, run heads also write the column and count their row.
__global__ void __launch_bounds__(kBlock) k_merge_runs(int64_t len, int bits, u64 sentinel,
                                                       const u64 *keys, const int32_t *vals,
                                                       const int64_t *pos, int32_t *col_out,
                                                       u64 *wacc, int32_t *rowcnt)
{
    const u64 colmask = ((u64)1 << bits) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        const u64 k = keys[i];
        if (k == sentinel) continue;
        const int64_t o = pos[i + 1] - 1;
        atomicAdd(&wacc[o], (u64)vals[i]);
        if (pos[i + 1] != pos[i]) {  // run head
            col_out[o] = (int32_t)(k & colmask);
            atomicAdd(&rowcnt[k >> bits], 1);
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_weights_out(int64_t nnz, const u64 *wacc,
                                                        int32_t *w_out, unsigned *err)
{
    unsigned bad = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        const u64 x = wacc[p];
        if (x > (u64)INT32_MAX) bad |= ERRF_OVERFLOW;
        w_out[p] = (int32_t)x;
    }
    if (bad) atomicOr(err, bad);
}

}  // namespace

int edges_scratch_tiles(int64_t m) { return (int)((2 * m + kSortTile - 1) / kSortTile); }

int launch_edges_to_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                        const int32_t *w, const EdgeScratch &sc, int64_t *rp_out,
                        int32_t *col_out, int32_t *w_out, int64_t *nnz_out, unsigned *err,
                        cudaStream_t s, const LaunchCfg &lc)
{
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) <= n) bits++;  // n < 2^bits
    const u64 sentinel = ((u64)1 << (2 * bits)) - 1;
    const int64_t len = 2 * m;
    const int64_t ntiles = (len + kSortTile - 1) / kSortTile;
    int launched = 0;
    cudaMemsetAsync(sc.rowcnt, 0, sizeof(int32_t) * (size_t)n, s);
    if (len > 0) {
        k_expand_edges<<<grid_for(m, kBlock, lc.max_blocks), kBlock, 0, s>>>(
            m, n, bits, src, dst, w, sc.keys[0], sc.vals[0], err);
        launched++;
        int cur = 0;
        for (int shift = 0; shift < 2 * bits; shift += 8) {
            k_radix_hist<<<(unsigned)ntiles, kSortBlock, 0, s>>>(sc.keys[cur], len, shift,
                                                                  ntiles, sc.hist);
            launched++;
            launched += exclusive_scan<int64_t>(ArrayIn<int64_t>{sc.hist}, kDigits * ntiles,
                                                sc.offs, sc.scan64, s);
            k_radix_scatter<<<(unsigned)ntiles, kSortBlock, 0, s>>>(
                sc.keys[cur], sc.vals[cur], len, shift, ntiles, sc.offs, sc.keys[1 - cur],
                sc.vals[1 - cur]);
            launched++;
            cur = 1 - cur;
        }
        launched += exclusive_scan<int64_t>(RunHeadIn{sc.keys[cur], sentinel}, len, sc.pos,
                                            sc.scan64, s);
        cudaMemsetAsync(sc.wacc, 0, sizeof(u64) * (size_t)len, s);
        k_merge_runs<<<grid_for(len, kBlock, lc.max_blocks), kBlock, 0, s>>>(
            len, bits, sentinel, sc.keys[cur], sc.vals[cur], sc.pos, col_out, sc.wacc,
            sc.rowcnt);
        k_weights_out<<<grid_for(len, kBlock, lc.max_blocks), kBlock, 0, s>>>(
            len, sc.wacc, w_out, err);  // slots past nnz get 0 (the caller's capacity is 2m)
        launched += 2;
        cudaMemcpyAsync(nnz_out, sc.pos + len, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    } else {
        cudaMemsetAsync(nnz_out, 0, sizeof(int64_t), s);
    }
    launched += exclusive_scan<int64_t>(ArrayIn<int32_t>{sc.rowcnt}, n, rp_out, sc.scan64, s);
    return launched;
}

}  // namespace lv
