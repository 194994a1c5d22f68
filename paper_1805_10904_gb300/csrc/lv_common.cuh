// lv_common.cuh -- device helpers shared by the kernels of the Louvain library.
//
// Exact integer arithmetic throughout (arXiv 1805.10904, Eq. 3-4 rescaled by (2W)^2):
// sums of weights are int64, products of two of them are int64 when (2W)^2 < 2^63 and
// __int128 otherwise (the GT template parameter of the move kernels).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

namespace lv {

typedef __int128 i128;
typedef unsigned __int128 u128;
typedef unsigned long long u64;
typedef long long i64;

constexpr int kBlock = 256;  // threads per CTA of every kernel unless stated

// error bits raised by device code into a per-run error word
enum : unsigned {
    ERRF_INDEX = 1u,      // column outside [0, n)
    ERRF_WEIGHT = 2u,     // weight < 1
    ERRF_HASH_FULL = 4u,  // open-addressing probe ran through a whole table
    ERRF_ROWPTR = 8u,     // row_ptr[0] != 0 or decreasing
    ERRF_ASYM = 16u,      // A_ij != A_ji (full checks)
    ERRF_DUP = 32u,       // unsorted or duplicate column in a row (full checks)
    ERRF_INTERNAL = 64u,  // consistency check failed
    ERRF_OVERFLOW = 128u, // a merged weight does not fit int32
};

// Per-sweep accumulators, zeroed by the decide kernel after it reads them.
struct SweepStats {
    u64 internal;  // sum_i e_{i->C(i)} including loops (Eq. 3 first term / TW)
    u64 sq_lo;     // sum_c deg_c^2 as a 128-bit value
    u64 sq_hi;
    u64 moved;     // vertices whose proposed label differs from the current one
    u64 cand[16];  // distinct neighbouring communities summed over the vertices of each
                   // degree bin (index = bin, fewer than 16 bins)
};

// Level controller state (one per phase), read and written by the decide kernel.
struct LevelCtl {
    i64 tw;
    i64 theta_num;
    i64 theta_den;
    int max_iters;
    int sweep;     // sweeps applied so far in this phase
    int done;      // 1 once the phase has stopped
    int hit_cap;
    int iters;     // sweeps applied when the phase stopped
    int rel;       // 1: relative phase test |dQ / Q_prev| < theta (Algorithm 1 as printed)
    i64 moved_last;
    i64 qn_init[2];   // {hi, lo}
    i64 qn_prev[2];
    i64 qn_final[2];
    i64 pad1[4];
};

__device__ __forceinline__ i128 i128_from(const i64 v[2])
{
    return (i128)(((u128)(u64)v[0] << 64) | (u128)(u64)v[1]);
}

__device__ __forceinline__ void i128_to(i128 x, i64 v[2])
{
    v[0] = (i64)(x >> 64);
    v[1] = (i64)(u64)x;
}

// ---------------------------------------------------------------- shuffles
__device__ __forceinline__ i64 shfl_xor(i64 v, int m, int width = 32)
{
    return __shfl_xor_sync(0xffffffffu, v, m, width);
}
__device__ __forceinline__ u64 shfl_xor(u64 v, int m, int width = 32)
{
    return __shfl_xor_sync(0xffffffffu, v, m, width);
}
__device__ __forceinline__ int shfl_xor(int v, int m, int width = 32)
{
    return __shfl_xor_sync(0xffffffffu, v, m, width);
}
__device__ __forceinline__ i128 shfl_xor(i128 v, int m, int width = 32)
{
    u64 lo = (u64)v;
    i64 hi = (i64)(v >> 64);
    lo = __shfl_xor_sync(0xffffffffu, lo, m, width);
    hi = __shfl_xor_sync(0xffffffffu, hi, m, width);
    return (i128)(((u128)(u64)hi << 64) | (u128)lo);
}
__device__ __forceinline__ u128 shfl_xor(u128 v, int m, int width = 32)
{
    u64 lo = (u64)v, hi = (u64)(v >> 64);
    lo = __shfl_xor_sync(0xffffffffu, lo, m, width);
    hi = __shfl_xor_sync(0xffffffffu, hi, m, width);
    return ((u128)hi << 64) | (u128)lo;
}

template <typename GT>
__device__ __forceinline__ GT gain_min();
template <>
__device__ __forceinline__ i64 gain_min<i64>()
{
    return (i64)0x8000000000000000ULL;
}
template <>
__device__ __forceinline__ i128 gain_min<i128>()
{
    return (i128)((u128)1 << 127);
}

// Argmax order of Eq. 5 with the Sec. 3.1.2 tie rule: larger gain first, then smaller label.
template <typename GT>
__device__ __forceinline__ bool better(GT g1, int c1, GT g2, int c2)
{
    return g1 > g2 || (g1 == g2 && c1 < c2);
}

// Reduce (gain, label) to the group's argmax over `width` lanes (width a power of two <= 32;
// every lane of the warp must call this).
template <typename GT>
__device__ __forceinline__ void argmax_reduce(GT &g, int &c, int width)
{
    for (int off = width >> 1; off > 0; off >>= 1) {
        GT g2 = shfl_xor(g, off, width);
        int c2 = shfl_xor(c, off, width);
        if (better(g2, c2, g, c)) {
            g = g2;
            c = c2;
        }
    }
}

template <typename T>
__device__ __forceinline__ T sum_reduce(T v, int width)
{
    for (int off = width >> 1; off > 0; off >>= 1) v += shfl_xor(v, off, width);
    return v;
}

// 128-bit unsigned atomic add over two 64-bit words (carry applied per addition).
__device__ __forceinline__ void atomic_add_u128(u64 *lo, u64 *hi, u128 v)
{
    u64 vlo = (u64)v, vhi = (u64)(v >> 64);
    if (vlo) {
        u64 old = atomicAdd(lo, vlo);
        if (old + vlo < old) vhi += 1;
    }
    if (vhi) atomicAdd(hi, vhi);
}

// Block-wide sums of up to four u64 counters and one u128, thread 0 publishes with atomics.
__device__ __forceinline__ void block_flush_stats(SweepStats *st, int slot, u64 internal,
                                                  u64 moved, u64 cand, u128 sq)
{
    __shared__ u64 s_red[32][5];
    internal = sum_reduce(internal, 32);
    moved = sum_reduce(moved, 32);
    cand = sum_reduce(cand, 32);
    u128 sqr = sum_reduce(sq, 32);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_red[warp][0] = internal;
        s_red[warp][1] = moved;
        s_red[warp][2] = cand;
        s_red[warp][3] = (u64)sqr;
        s_red[warp][4] = (u64)(sqr >> 64);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 a = 0, b = 0, c = 0;
        u128 s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            a += s_red[w][0];
            b += s_red[w][1];
            c += s_red[w][2];
            s += ((u128)s_red[w][4] << 64) | (u128)s_red[w][3];
        }
        if (a) atomicAdd(&st->internal, a);
        if (b) atomicAdd(&st->moved, b);
        if (c) atomicAdd(&st->cand[slot], c);
        if (s) atomic_add_u128(&st->sq_lo, &st->sq_hi, s);
    }
}

// ---------------------------------------------------------------- hashing
// Multiplicative (Fibonacci) hashing of a community label into a power-of-two table.
__device__ __forceinline__ unsigned hash_slot(int key, int log2cap)
{
    return log2cap == 0 ? 0u : ((unsigned)key * 2654435761u) >> (32 - log2cap);
}

// Read-once data (a sweep's or an induction's columns and weights): loaded with the
// evict-first hint, so the streamed rows do not push the gathered labels and community
// degrees out of L2.
template <typename T>
__device__ __forceinline__ T ld_stream(const T *p)
{
    return __ldcs(p);
}

// Write-once data that is read back much later (an induction's rows): stored with the
// streaming hint.
template <typename T>
__device__ __forceinline__ void st_stream(T *p, T v)
{
    __stcs(p, v);
}

// Open-addressing insert-or-add of (key, val) into a table of 2^log2cap slots.  `list`
// records the slot of every key the first time it is claimed (count in *cnt), so the table
// can be walked and cleared in O(distinct keys).  A table with more slots than distinct
// keys never fills; if it does anyway the error word is flagged and the value dropped.
// GLOBAL selects L2 reads (tables shared by several CTAs) instead of shared memory.
template <bool GLOBAL>
__device__ __forceinline__ int tbl_key(const int *keys, unsigned h)
{
    if (GLOBAL) return __ldcg(keys + h);
    return ((volatile const int *)keys)[h];
}

template <bool GLOBAL, typename VT>
__device__ __forceinline__ void tbl_insert_at(int *keys, VT *vals, int *list, int *cnt,
                                              int log2cap, unsigned h, int key, VT val,
                                              unsigned *err)
{
    const unsigned mask = (1u << log2cap) - 1u;
#pragma unroll 1
    for (unsigned probe = 0; probe <= mask; probe++) {
        const int k = tbl_key<GLOBAL>(keys, h);
        if (k == key) {
            atomicAdd(&vals[h], val);
            return;
        }
        if (k == -1) {
            const int old = atomicCAS(&keys[h], -1, key);
            if (old == -1) {
                const int p = atomicAdd(cnt, 1);
                list[p] = (int)h;
                atomicAdd(&vals[h], val);
                return;
            }
            if (old == key) {
                atomicAdd(&vals[h], val);
                return;
            }
        }
        h = (h + 1) & mask;
    }
    atomicOr(err, ERRF_HASH_FULL);
}

template <bool GLOBAL, typename VT>
__device__ __forceinline__ void tbl_insert(int *keys, VT *vals, int *list, int *cnt, int log2cap,
                                           int key, VT val, unsigned *err)
{
    tbl_insert_at<GLOBAL, VT>(keys, vals, list, cnt, log2cap, hash_slot(key, log2cap), key, val,
                              err);
}

// Insert-or-add that reports a newly claimed slot instead of appending it to a list, so
// the caller can append claims of a whole warp with one counter update.  Returns true
// (and the slot) only for the call that claimed the slot.
template <typename VT>
__device__ __forceinline__ bool tbl_insert_claim(int *keys, VT *vals, int log2cap, int key, VT val,
                                                 unsigned *err, int &slot)
{
    const unsigned mask = (1u << log2cap) - 1u;
    unsigned h = hash_slot(key, log2cap);
#pragma unroll 1
    for (unsigned probe = 0; probe <= mask; probe++) {
        const int k = ((volatile const int *)keys)[h];
        if (k == key) {
            atomicAdd(&vals[h], val);
            return false;
        }
        if (k == -1) {
            const int old = atomicCAS(&keys[h], -1, key);
            if (old == -1 || old == key) {
                atomicAdd(&vals[h], val);
                slot = (int)h;
                return old == -1;
            }
        }
        h = (h + 1) & mask;
    }
    atomicOr(err, ERRF_HASH_FULL);
    return false;
}

// Append the slots claimed by the lanes of a warp to `list` with one counter update
// (every lane of the warp must call this).
__device__ __forceinline__ void warp_append(bool claimed, int slot, int *list, int *cnt)
{
    const unsigned m = __ballot_sync(0xffffffffu, claimed);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (claimed) list[base + __popc(m & ((1u << lane) - 1u))] = slot;
}

// Insert-or-add of U entries of one thread at once (key < 0: nothing to insert).  The
// claims of all U keys are issued before any result is needed: one CAS per key at its
// home slot (a key already present there returns itself), so a thread has U shared-memory
// round trips in flight instead of one chain per entry; a key whose home slot holds
// another key probes on (tbl_insert_claim).  New slots are appended to `list` once per
// warp (every lane of the warp must call this with the same U), and the sums are added
// with atomics whose results are not used.
template <int U, typename VT>
__device__ __forceinline__ void tbl_insert_batch(int *keys, VT *vals, int *list, int *cnt,
                                                 int log2cap, const int32_t (&key)[U],
                                                 const VT (&val)[U], unsigned *err)
{
    unsigned h[U];
    int old[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        h[u] = key[u] >= 0 ? hash_slot(key[u], log2cap) : 0u;
        old[u] = key[u] >= 0 ? atomicCAS(&keys[h[u]], -1, key[u]) : key[u];
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
        bool claimed = key[u] >= 0 && old[u] == -1;
        int slot = (int)h[u];
        if (key[u] >= 0 && old[u] != -1 && old[u] != key[u]) {  // home slot taken: probe on
            const unsigned mask = (1u << log2cap) - 1u;
            unsigned hh = (h[u] + 1u) & mask;
            bool done = false;
#pragma unroll 1
            for (unsigned probe = 1; probe <= mask && !done; probe++) {
                const int o = atomicCAS(&keys[hh], -1, key[u]);
                if (o == -1 || o == key[u]) {
                    claimed = o == -1;
                    slot = (int)hh;
                    done = true;
                } else {
                    hh = (hh + 1u) & mask;
                }
            }
            if (!done) {
                atomicOr(err, ERRF_HASH_FULL);
                slot = -1;
            }
        }
        warp_append(claimed, slot, list, cnt);
        if (key[u] >= 0 && slot >= 0) atomicAdd(&vals[slot], val[u]);
    }
}

// Mixing hash of a key (multiply, xor-shift, multiply, xor-shift; the constants of
// MurmurHash3's 32-bit finaliser), a bijection of 32-bit values independent of the
// multiplicative hash that indexes the shared tables.  Its top bits choose a key's
// partition, its low bits split a crowded partition into residue classes.
__device__ __forceinline__ unsigned mix_hash(int key)
{
    unsigned x = (unsigned)key * 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x;
}

// Partition of a key among a row's 2^log2p partitions.
__device__ __forceinline__ int part_of(int key, int log2p)
{
    return log2p == 0 ? 0 : (int)(mix_hash(key) >> (32 - log2p));
}

// In-place exclusive prefix sum of a[0..len) in shared memory by a CTA of BLOCK threads;
// a[len] receives the total.  Ends with a barrier.
template <int BLOCK>
__device__ __forceinline__ void cta_excl_scan_smem(int *a, int len)
{
    __shared__ int s_w[BLOCK / 32];
    __shared__ int s_tot;
    const int per = (len + BLOCK - 1) / BLOCK;
    const int lo = threadIdx.x * per;
    int sum = 0;
    for (int t = 0; t < per; t++)
        if (lo + t < len) sum += a[lo + t];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = sum;
    for (int off = 1; off < 32; off <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += u;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int x = lane < BLOCK / 32 ? s_w[lane] : 0;
        int xi = x;
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, xi, off);
            if (lane >= off) xi += u;
        }
        if (lane < BLOCK / 32) s_w[lane] = xi - x;
        if (lane == BLOCK / 32 - 1) s_tot = xi;
    }
    __syncthreads();
    int run = s_w[warp] + incl - sum;
    for (int t = 0; t < per; t++)
        if (lo + t < len) {
            const int v = a[lo + t];
            a[lo + t] = run;
            run += v;
        }
    if (threadIdx.x == 0) a[len] = s_tot;
    __syncthreads();
}

// Merge of the (key, value) pairs of one partition in a shared table of 2^log2cap slots
// (keys -1, values 0 on entry and on return), class by class: class (res, mod) holds the keys
// whose mix_hash is res modulo mod (mod a power of two).  A class whose distinct keys reach
// `thresh` claims is abandoned, its slots cleared, and redone as its two halves (res, 2 mod)
// and (res + mod, 2 mod); inserts stop once the flag is up, so at most thresh + BLOCK slots
// are ever claimed (thresh + BLOCK <= 2^log2cap), and since mix_hash is a bijection a class
// shrinks to one key before mod runs out of bits.  for_pairs(f) calls f(key, value) for
// every pair of the partition, its work spread over the CTA; emit(m) runs on every thread
// for each completed class with m distinct keys in list[0..m) and must clear their slots.
// Every thread of the CTA calls this; it ends with a barrier.
template <int BLOCK, typename VT, typename ForPairs, typename Emit>
__device__ __forceinline__ void merge_partition(int *keys, VT *vals, int *list, int log2cap,
                                                int thresh, unsigned *err, ForPairs for_pairs,
                                                Emit emit)
{
    __shared__ unsigned s_res[34], s_mod[34];
    __shared__ unsigned s_r, s_m;
    __shared__ int s_top, s_cnt, s_over;
    if (threadIdx.x == 0) {
        s_top = 1;
        s_res[0] = 0;
        s_mod[0] = 1;
        s_cnt = 0;
        s_over = 0;
    }
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            if (s_top > 0) {
                --s_top;
                s_r = s_res[s_top];
                s_m = s_mod[s_top];
            } else {
                s_m = 0;
            }
        }
        __syncthreads();
        const unsigned res = s_r, mod = s_m;
        if (mod == 0) break;
        for_pairs([&](int key, VT v) {
            if ((mix_hash(key) & (mod - 1u)) != res || *(volatile int *)&s_over) return;
            tbl_insert<false, VT>(keys, vals, list, &s_cnt, log2cap, key, v, err);
            if (*(volatile int *)&s_cnt >= thresh) s_over = 1;
        });
        __syncthreads();
        const int m = s_cnt;
        if (s_over && mod >= 0x80000000u && threadIdx.x == 0)
            atomicOr(err, ERRF_HASH_FULL);  // unreachable: such a class holds two keys at most
        if (s_over && mod < 0x80000000u) {  // crowded: clear, then its two halves
            for (int r = threadIdx.x; r < m; r += BLOCK) {
                const int s = list[r];
                keys[s] = -1;
                vals[s] = 0;
            }
            if (threadIdx.x == 0) {
                s_res[s_top] = res + mod;
                s_mod[s_top] = 2u * mod;
                s_res[s_top + 1] = res;
                s_mod[s_top + 1] = 2u * mod;
                s_top += 2;
            }
        } else {
            emit(m);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_cnt = 0;
            s_over = 0;
        }
        __syncthreads();
    }
}

// Table spread over the CTAs of a thread-block cluster: one linear-probing table of
// 2^(log2cl + log2cap) slots whose segment r lives in the shared memory of CTA r (virtual
// slot v -> CTA v >> log2cap, local slot v & (cap - 1)).  The key's hash picks the first
// virtual slot, so keys spread over the CTAs, and probing crosses into the next CTA's
// segment instead of overflowing.  `keys`, `vals`, `list`, `cnt` are this CTA's own
// arrays; each segment's list records the local slots claimed in it.
template <typename VT, typename Cluster>
__device__ __forceinline__ void cluster_insert(Cluster &cluster, int *keys, VT *vals, int log2cl,
                                               int log2cap, int key, VT val, unsigned *err,
                                               unsigned start = ~0u)
{
    const unsigned total_mask = (1u << (log2cl + log2cap)) - 1u;
    const unsigned local_mask = (1u << log2cap) - 1u;
    unsigned v = start != ~0u ? start
                              : ((unsigned)key * 2654435761u) >> (32 - (log2cl + log2cap));
    unsigned owner = v >> log2cap;
    int *rk = cluster.map_shared_rank(keys, owner);
#pragma unroll 1
    for (unsigned probe = 0; probe <= total_mask; probe++) {
        const unsigned h = v & local_mask;
        const int k = ((volatile const int *)rk)[h];
        if (k == key) {
            atomicAdd(cluster.map_shared_rank(vals, owner) + h, val);
            return;
        }
        if (k == -1) {
            const int old = atomicCAS(rk + h, -1, key);
            if (old == -1 || old == key) {
                atomicAdd(cluster.map_shared_rank(vals, owner) + h, val);
                return;
            }
        }
        v = (v + 1) & total_mask;
        if ((v & local_mask) == 0) {
            owner = v >> log2cap;
            rk = cluster.map_shared_rank(keys, owner);
        }
    }
    atomicOr(err, ERRF_HASH_FULL);
}

// U entries of one thread into the cluster-wide table at once: one remote CAS per key at
// its home slot issued before any result is needed, probing on only for keys whose home
// slot holds another key, and sums added with atomics whose results are not used.
template <int U, typename VT, typename Cluster>
__device__ __forceinline__ void cluster_insert_batch(Cluster &cluster, int *keys, VT *vals,
                                                     int log2cl, int log2cap,
                                                     const int32_t (&key)[U], const VT (&val)[U],
                                                     unsigned *err)
{
    const unsigned local_mask = (1u << log2cap) - 1u;
    unsigned v[U];
    int old[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        v[u] = key[u] >= 0 ? ((unsigned)key[u] * 2654435761u) >> (32 - (log2cl + log2cap)) : 0u;
        old[u] = key[u] >= 0
                     ? atomicCAS(cluster.map_shared_rank(keys, v[u] >> log2cap) + (v[u] & local_mask),
                                 -1, key[u])
                     : key[u];
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
        if (key[u] < 0) continue;
        if (old[u] == -1 || old[u] == key[u]) {
            atomicAdd(cluster.map_shared_rank(vals, v[u] >> log2cap) + (v[u] & local_mask), val[u]);
        } else {  // home slot taken: probe on from the next virtual slot
            const unsigned total_mask = (1u << (log2cl + log2cap)) - 1u;
            cluster_insert<VT>(cluster, keys, vals, log2cl, log2cap, key[u], val[u], err,
                               (v[u] + 1u) & total_mask);
        }
    }
}

// ---------------------------------------------------------------- launch helpers
// Name of the first launch site that left a CUDA error pending (for error messages).
inline const char *&launch_site()
{
    static thread_local const char *site = nullptr;
    return site;
}
inline void note_launch(const char *name)
{
    if (!launch_site() && cudaPeekAtLastError() != cudaSuccess) launch_site() = name;
}

// Raise a kernel's dynamic shared memory limit; on failure records the kernel's own
// attributes in the launch-site message.
template <typename K>
inline void set_dyn_smem(K kernel, size_t bytes, const char *name)
{
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
        cudaSuccess)
        return;
    if (launch_site()) return;
    static thread_local char msg[256];
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    snprintf(msg, sizeof(msg),
             "%s: dynamic smem %zu rejected (attr query %d: static %zu, max threads %d, regs %d, "
             "max dyn %d)",
             name, bytes, (int)e, a.sharedSizeBytes, a.maxThreadsPerBlock, a.numRegs,
             a.maxDynamicSharedSizeBytes);
    launch_site() = msg;
}

inline int grid_for(int64_t work_items, int per_block, int max_blocks)
{
    int64_t g = (work_items + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

}  // namespace lv
