// lv_scan.cuh -- device-wide exclusive prefix sum (reduce, scan of tile sums, rescan).
//
// Used for the prefix-sum compaction of community labels (Sec. 5.1.2 "Renumbering
// nodes"), the row offsets of the induced graph and the work lists of the binned
// move kernels.  The input is a functor f(i) so flags or lengths can be scanned
// without materialising them.
#pragma once

#include "lv_common.cuh"

namespace lv {

constexpr int kScanItems = 8;
constexpr int kScanTile = kBlock * kScanItems;  // 2048 elements per tile

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
    for (int off = 1; off < 32; off <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += u;
    }
    return v;
}

// exclusive block scan of one value per thread; returns the prefix, *total gets the sum
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *total)
{
    __shared__ T s_warp[kBlock / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T incl = warp_incl_scan(v);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T x = lane < kBlock / 32 ? s_warp[lane] : T(0);
        T xi = warp_incl_scan(x);
        if (lane < kBlock / 32) s_warp[lane] = xi - x;
        if (lane == 31) *total = xi;
    }
    __syncthreads();
    T res = s_warp[warp] + incl - v;
    __syncthreads();
    return res;
}

template <typename T, typename F>
__global__ void __launch_bounds__(kBlock) k_scan_reduce(F f, int64_t n, T *tile_sums)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    T s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        int64_t i = base + (int64_t)j * kBlock + threadIdx.x;
        if (i < n) s += f(i);
    }
    __shared__ T s_tot;
    T pre = block_excl_scan(s, &s_tot);
    (void)pre;
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = s_tot;
}

// single CTA: exclusive scan of the tile sums in place; total written to *total
template <typename T>
__global__ void __launch_bounds__(kBlock) k_scan_tiles(T *tile_sums, int64_t ntiles, T *total)
{
    __shared__ T s_carry;
    __shared__ T s_tot;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < ntiles; b += kBlock) {
        int64_t i = b + threadIdx.x;
        T v = i < ntiles ? tile_sums[i] : T(0);
        T pre = block_excl_scan(v, &s_tot);
        T carry = s_carry;
        if (i < ntiles) tile_sums[i] = carry + pre;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + s_tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = s_carry;
}

template <typename T, typename F>
__global__ void __launch_bounds__(kBlock) k_scan_apply(F f, int64_t n, const T *tile_sums, T *out)
{
    __shared__ T s_val[kScanTile];
    __shared__ T s_tot;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        int64_t i = base + (int64_t)j * kBlock + threadIdx.x;
        s_val[j * kBlock + threadIdx.x] = i < n ? f(i) : T(0);
    }
    __syncthreads();
    T local[kScanItems];
    T run = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        local[j] = run;
        run += s_val[threadIdx.x * kScanItems + j];
    }
    T pre = block_excl_scan(run, &s_tot);
    const T off = tile_sums[blockIdx.x] + pre;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) s_val[threadIdx.x * kScanItems + j] = off + local[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        int64_t i = base + (int64_t)j * kBlock + threadIdx.x;
        if (i < n) out[i] = s_val[j * kBlock + threadIdx.x];
    }
}

// Number of T slots of scratch needed by exclusive_scan for n elements.
inline int64_t scan_scratch_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

// out[i] = sum_{j < i} f(j) for i in [0, n), out[n] = total (out has n + 1 slots).
// scratch needs scan_scratch_elems(n) elements.  Launches 3 kernels on `s`; returns the
// number of kernels launched.
template <typename T, typename F>
int exclusive_scan(F f, int64_t n, T *out, T *scratch, cudaStream_t s)
{
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles == 0) {
        cudaMemsetAsync(out, 0, sizeof(T), s);
        return 0;
    }
    k_scan_reduce<T, F><<<(unsigned)ntiles, kBlock, 0, s>>>(f, n, scratch);
    k_scan_tiles<T><<<1, kBlock, 0, s>>>(scratch, ntiles, out + n);
    k_scan_apply<T, F><<<(unsigned)ntiles, kBlock, 0, s>>>(f, n, scratch, out);
    return 3;
}

// ---- common scan inputs
template <typename T>
struct ArrayIn {
    const T *a;
    __device__ __forceinline__ T operator()(int64_t i) const { return a[i]; }
};

template <typename T, typename S>
struct PositiveFlagIn {  // 1 if a[i] > 0
    const S *a;
    __device__ __forceinline__ T operator()(int64_t i) const { return a[i] > 0 ? T(1) : T(0); }
};

}  // namespace lv
