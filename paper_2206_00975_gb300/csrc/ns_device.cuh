// ns_device.cuh -- device-side helpers shared by the libns kernels (sm_103a).
//
// Random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), key = (seed, 0), counter =
// (index, aux, stream, 0).  Streams: 0 = SRHT signs, 1 = SRHT sample
// permutation, 2 = sparse-sign columns, 3 = Gaussian entries.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/ns.h"

namespace ns {

// ---------------------------------------------------------------- Philox ----
struct u64x4 {
    uint64_t w[4];
};

__device__ __forceinline__ u64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                               uint64_t k1) {
    // multipliers and Weyl increments of the published Philox4x64 definition
    const uint64_t MA = 0xD2E7470EE14C6C93ull, MB = 0xCA5A826395121157ull;
    const uint64_t WA = 0x9E3779B97F4A7C15ull, WB = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t ha = __umul64hi(MA, c0), la = MA * c0;
        const uint64_t hb = __umul64hi(MB, c2), lb = MB * c2;
        const uint64_t n0 = hb ^ c1 ^ k0;
        const uint64_t n2 = ha ^ c3 ^ k1;
        c0 = n0;
        c1 = lb;
        c2 = n2;
        c3 = la;
        k0 += WA;
        k1 += WB;
    }
    u64x4 o;
    o.w[0] = c0;
    o.w[1] = c1;
    o.w[2] = c2;
    o.w[3] = c3;
    return o;
}

__device__ __forceinline__ u64x4 draw(uint64_t seed, uint64_t idx, uint64_t aux, uint64_t stream) {
    return philox4x64_10(idx, aux, stream, 0, seed, 0);
}

// Sample permutation of [0, 2^lg): four Feistel rounds; the low half holds
// lg/2 bits, the high half the rest; even rounds xor the low half with a
// keyed function of the high half, odd rounds the reverse.  A bijection, so
// t -> perm(t), t < s, draws s distinct coordinates in a fixed order.
__device__ __forceinline__ uint32_t sample_perm(uint64_t seed, int lg, uint32_t x) {
    const int nlo = lg >> 1, nhi = lg - nlo;
    const uint64_t mlo = nlo ? ((1ull << nlo) - 1) : 0, mhi = nhi ? ((1ull << nhi) - 1) : 0;
    uint64_t hi = (uint64_t)x >> nlo, lo = (uint64_t)x & mlo;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if ((r & 1) == 0)
            lo ^= draw(seed, hi, (uint64_t)r, 1).w[0] & mlo;
        else
            hi ^= draw(seed, lo, (uint64_t)r, 1).w[0] & mhi;
    }
    return (uint32_t)((hi << nlo) | lo);
}

// Floyd's sampling of zeta distinct rows of [0, s) for column j of S.
__device__ __forceinline__ void sparse_column(uint64_t seed, int64_t s, int zeta, int64_t j, int32_t *rows,
                                              int8_t *signs) {
    uint64_t w[64];
    for (int q = 0; q < (zeta + 3) / 4; ++q) {
        const u64x4 b = draw(seed, (uint64_t)j, (uint64_t)q, 2);
        w[4 * q + 0] = b.w[0];
        w[4 * q + 1] = b.w[1];
        w[4 * q + 2] = b.w[2];
        w[4 * q + 3] = b.w[3];
    }
    for (int i = 0; i < zeta; ++i) {
        const int64_t bound = s - zeta + i;
        int64_t t = (int64_t)__umul64hi(w[i], (uint64_t)(bound + 1));
        for (int u = 0; u < i; ++u)
            if (rows[u] == t) {
                t = bound;
                break;
            }
        rows[i] = (int32_t)t;
        signs[i] = (w[i] & 1ull) ? -1 : 1;
    }
}

// ------------------------------------------------------------ reductions ----
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum of NV values over the whole block; every thread gets the result.
// `scratch` must hold 32*NV doubles; ends with a __syncthreads().
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) scratch[wid * NV + i] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double a = 0.0;
        for (int w = 0; w < nw; ++w) a += scratch[w * NV + i];  // fixed order: deterministic
        v[i] = a;
    }
    __syncthreads();
}

__device__ __forceinline__ double block_max(double v, double *scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double a = scratch[0];
    for (int w = 1; w < nw; ++w) a = fmax(a, scratch[w]);
    __syncthreads();
    return a;
}

// ---------------------------------------------------------- grid barrier ----
// Barrier over all blocks of a cooperative launch on one 32-bit word: each
// block adds 1 with release semantics, except block 0 which adds
// 2^31 - (nblocks - 1), so the word's top bit flips exactly when the last block
// arrives and its low bits return to their previous value.  Every block waits
// (acquire loads) until the top bit differs from the one in the value its own
// add returned.  The host zeroes the word before the launch.  The wait is
// bounded: after `limit` polls (2^24 unless a test hook sets it) the barrier
// records NS_ERR_TIMEOUT in *status and returns false; callers then leave the
// kernel.
struct GridBarrier {
    unsigned int *word;
    int32_t *status;
    long long limit = 1ll << 24;  // polls; a healthy barrier needs a few hundred at most
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned int atom_add_release_u32(unsigned int *p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ bool grid_sync(const GridBarrier &b) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        const unsigned int nblk = gridDim.x * gridDim.y * gridDim.z;
        const bool first = (blockIdx.x | blockIdx.y | blockIdx.z) == 0;
        const unsigned int inc = first ? (0x80000000u - (nblk - 1u)) : 1u;
        const unsigned int old = atom_add_release_u32(b.word, inc);
        int ok = 1;
        long long polls = 0;
        while (((ld_acquire_u32(b.word) ^ old) & 0x80000000u) == 0u) {
            if (++polls > b.limit) {
                atomicMax(b.status, (int32_t)NS_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
        if (*(volatile int32_t *)b.status == NS_ERR_TIMEOUT) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Sum over the block of NV values per thread, valid in thread 0: shuffles down
// to lane 0 of each warp, then warp 0 adds the warp partials.
template <int NV>
__device__ __forceinline__ void block_sum_t0(double (&v)[NV], double *red /* 32 * NV */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) red[i * 32 + wid] = v[i];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double a = lane < nw ? red[i * 32 + lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1)
                if (o < nw) a += __shfl_down_sync(0xffffffffu, a, o);
            v[i] = a;
        }
    }
}

// ------------------------------------------------- clusters (DSMEM) ----
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// address of the same shared-memory location in the CTA of cluster rank `rank`
__device__ __forceinline__ uint32_t peer_addr(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
// barrier over every thread of the cluster (release / acquire at cluster scope)
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t shared_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void set_status(int32_t *status, int32_t code) {
    if (status) atomicMax(status, code);
}

}  // namespace ns
