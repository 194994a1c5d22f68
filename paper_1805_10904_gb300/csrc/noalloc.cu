// noalloc.cu -- modularity of a given partition without any device allocation.
//
// For callers that cannot allocate device memory while they run: for example a service
// whose GPU memory is entirely reserved up front by another framework's allocator, or code
// that must not trigger the device-wide synchronisation that cudaMalloc / cudaFree imply.
// Everything this entry point needs beyond the caller's inputs lives in one file-scope
// device array.  CUDA loads a library's GPU code lazily by default, so the array is reserved
// on a device when this file's code is first used there -- by the first call on that
// device -- and is held until the process exits.
//
// The computation is the library's exact modularity (Eq. 3 of the method, kept as the
// integer Qn = (2W)^2 * Q): per vertex the weighted degree and the weight of its entries
// whose column shares its label, per community the sum of its members' degrees, then
// Qn = 2W * sum_i e_{i->C(i)} - sum_c deg_c^2.
#include <atomic>
#include <cstring>

#include "../../include/louvain.h"
#include "lv_common.cuh"

namespace lv {
namespace {

// Scratch: per-community degrees for up to LOUVAIN_NOALLOC_MAX_VERTICES labels, then the
// accumulators (internal sum, 2W, sum of squares as two words, error word).
constexpr int64_t kAccWords = 8;
static __device__ __align__(256) u64 g_noalloc_scratch[LOUVAIN_NOALLOC_MAX_VERTICES + kAccWords];

constexpr int kMaxDevices = 64;
// device address of g_noalloc_scratch per device; host threads may race on the first
// lookup, and every one of them stores the same address
static std::atomic<u64 *> g_scratch_ptr[kMaxDevices];

// Sums of weights build up in 64-bit words: with weights below 2^31, fewer than 2^33
// entries cannot wrap them, and larger sums than 2^62 are rejected after the sum.
constexpr int64_t kMaxEntries = (int64_t)1 << 33;

__global__ void k_na_clear(u64 *scratch, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n + kAccWords;
         i += (int64_t)gridDim.x * blockDim.x)
        scratch[i] = 0;
}

__global__ void k_na_rowptr(const int64_t *rp, int64_t n, u64 *acc)
{
    unsigned bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i == 0 && rp[0] != 0) bad |= ERRF_ROWPTR;
        if (rp[i + 1] < rp[i]) bad |= ERRF_ROWPTR;
    }
    if (bad) atomicOr((unsigned *)&acc[4], bad);
}

// One warp per vertex: delta_i, the weight of entries into C(i) (loop included), and
// deg[C(i)] += delta_i.  Columns, labels and weights are checked.
__global__ void __launch_bounds__(kBlock) k_na_rows(int64_t n, const int64_t *rp,
                                                    const int32_t *col, const int32_t *w,
                                                    const int32_t *C, u64 *deg, u64 *acc)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned bad = 0;
    u64 internal = 0, tw = 0;
    for (int64_t i = warp; i < n; i += nwarps) {
        const int32_t a = C[i];
        if ((uint32_t)a >= (uint64_t)n) {
            bad |= ERRF_INDEX;
            continue;
        }
        u64 d = 0, e = 0;
        for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += 32) {
            const int32_t j = col[k];
            const i64 x = w ? (i64)w[k] : 1;
            if ((uint32_t)j >= (uint64_t)n) {
                bad |= ERRF_INDEX;
                continue;
            }
            if (x < 1) bad |= ERRF_WEIGHT;
            d += (u64)x;
            if (C[j] == a) e += (u64)x;
        }
        d = sum_reduce(d, 32);
        e = sum_reduce(e, 32);
        if (lane == 0) {
            if (d) atomicAdd(&deg[a], d);
            internal += e;
            tw += d;
        }
    }
    if (lane == 0) {
        if (internal) atomicAdd(&acc[0], internal);
        if (tw) atomicAdd(&acc[1], tw);
    }
    if (bad) atomicOr((unsigned *)&acc[4], bad);
}

__global__ void __launch_bounds__(kBlock) k_na_squares(int64_t n, const u64 *deg, u64 *acc)
{
    u128 sq = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x)
        sq += (u128)deg[c] * deg[c];
    sq = sum_reduce(sq, 32);
    if ((threadIdx.x & 31) == 0 && sq) atomic_add_u128(&acc[2], &acc[3], sq);
}

}  // namespace
}  // namespace lv

using namespace lv;

extern "C" int louvain_modularity_noalloc(int64_t n, const int64_t *row_ptr,
                                          const int32_t *col_idx, const int32_t *weights,
                                          const int32_t *labels, void *stream, int64_t qn[2],
                                          int64_t *tw_out, double *q)
{
    if (n < 0 || (n > 0 && (!row_ptr || !labels))) return LOUVAIN_ERR_INVALID_ARG;
    if (n > LOUVAIN_NOALLOC_MAX_VERTICES) return LOUVAIN_ERR_TOO_LARGE;
    // an error the caller's earlier work left pending is theirs: report it, do not clear it
    if (cudaPeekAtLastError() != cudaSuccess) return LOUVAIN_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return LOUVAIN_ERR_CUDA;
    }
    // first call on this device: look up the array's device address (host code cannot use
    // the symbol itself as a pointer)
    u64 *deg = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!deg) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return LOUVAIN_ERR_CUDA;
        }
        deg = (u64 *)p;
        g_scratch_ptr[dev].store(deg, std::memory_order_release);
    }
    u64 *acc = deg + LOUVAIN_NOALLOC_MAX_VERTICES;
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = 152 * 4;
    k_na_clear<<<grid, kBlock, 0, s>>>(deg, n);
    // the accumulators sit after the full-size degree area; clear them too
    k_na_clear<<<1, kBlock, 0, s>>>(acc, 0);
    if (n > 0) {
        k_na_rowptr<<<grid, kBlock, 0, s>>>(row_ptr, n, acc);
        u64 host_acc[kAccWords];
        int64_t nnz = 0;
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(host_acc, acc, sizeof(host_acc), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(nnz), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return LOUVAIN_ERR_CUDA;
        }
        if (host_acc[4]) return LOUVAIN_ERR_INDEX_RANGE;  // row offsets unusable: stop here
        if (!col_idx && nnz > 0) return LOUVAIN_ERR_INVALID_ARG;
        if (weights && nnz >= kMaxEntries) return LOUVAIN_ERR_TOO_LARGE;
        k_na_rows<<<grid, kBlock, 0, s>>>(n, row_ptr, col_idx, weights, labels, deg, acc);
        k_na_squares<<<grid, kBlock, 0, s>>>(n, deg, acc);
    }
    u64 host_acc[kAccWords];
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(host_acc, acc, sizeof(host_acc), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return LOUVAIN_ERR_CUDA;
    }
    const unsigned bad = (unsigned)host_acc[4];
    if (bad & (ERRF_ROWPTR | ERRF_INDEX)) return LOUVAIN_ERR_INDEX_RANGE;
    if (bad & ERRF_WEIGHT) return LOUVAIN_ERR_BAD_WEIGHT;
    const u64 tw = host_acc[1];
    if (tw > ((u64)1 << 62)) return LOUVAIN_ERR_TOO_LARGE;
    const u128 sq = ((u128)host_acc[3] << 64) | host_acc[2];
    const i128 value = (i128)tw * (i128)host_acc[0] - (i128)sq;
    if (qn) {
        qn[0] = (int64_t)(value >> 64);
        qn[1] = (int64_t)(u64)value;
    }
    if (tw_out) *tw_out = (int64_t)tw;
    if (q) *q = tw ? (double)value / (double)((i128)tw * (i128)tw) : 0.0;
    return LOUVAIN_OK;
}
