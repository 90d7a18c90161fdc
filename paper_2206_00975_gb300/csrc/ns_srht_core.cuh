// ns_srht_core.cuh -- the per-block pipeline of the FP64 SRHT (see ns_srht.cu),
// shared by the single-problem chunk kernel and the batched kernel.
#pragma once
#include "ns_device.cuh"
#include "ns_internal.h"

namespace ns {

// Shared-memory swizzle of a 4096-entry int64 block: entry i sits at
// i ^ (((i >> 7) & 15) << 1).  Row-major 16-byte stores of the first layout and
// the strided loads of the second layout are then both bank-conflict free.
__device__ __forceinline__ int swz(int i) { return i ^ (((i >> 7) & 15) << 1); }

// in-register Walsh-Hadamard transform of 64 values (Sylvester order on the
// register index)
__device__ __forceinline__ void fwht64(long long (&z)[64]) {
#pragma unroll
    for (int h = 1; h < 64; h <<= 1) {
#pragma unroll
        for (int k = 0; k < 64; ++k) {
            if ((k & h) == 0) {
                const long long a = z[k], b = z[k + h];
                z[k] = a + b;
                z[k + h] = a - b;
            }
        }
    }
}

// Layout 1: thread t, register k holds element (k & 1) | (t << 1) | ((k >> 1) << 7).
// Layout 2: thread t, register k holds element (t & 1) | (k << 1) | ((t >> 1) << 7).
__device__ __forceinline__ int l2_elem(int t, int k) { return (t & 1) | (k << 1) | ((t >> 1) << 7); }

// One 4096-row block b of a column (64 threads): load, quantise at the running
// exponent Erun (rescaling the accumulator when it grows), H_4096 in two
// register phases around a swizzled shared-memory transpose, and the signed
// gather of the sampled rows into acc[0..s).  Ends with __syncthreads().
__device__ __forceinline__ void srht_f64_block(const double *__restrict__ Acol, int64_t m, int64_t s, int64_t b,
                                               int P, const uint32_t *__restrict__ sign_words,
                                               const int32_t *rows_s, unsigned long long myneed, long long *Zs,
                                               long long *acc, uint32_t *sgn, int *red, int vec_ok, int &Erun,
                                               int &nonfinite) {
    const int t = threadIdx.x;
    const int64_t base = b * kBlock;
    sgn[t] = sign_words[(base >> 5) + t];
    sgn[t + 64] = sign_words[(base >> 5) + 64 + t];
    long long z[64];
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) {
        const int64_t i0 = base + 2 * t + 128 * kk;
        long long a0 = 0, a1 = 0;
        if (vec_ok && i0 + 1 < m) {
            const double2 v = __ldcs((const double2 *)(Acol + i0));
            a0 = __double_as_longlong(v.x);
            a1 = __double_as_longlong(v.y);
        } else {
            if (i0 < m) a0 = __double_as_longlong(__ldcs(Acol + i0));
            if (i0 + 1 < m) a1 = __double_as_longlong(__ldcs(Acol + i0 + 1));
        }
        z[2 * kk] = a0;
        z[2 * kk + 1] = a1;
    }
    int emax = 1;
#pragma unroll
    for (int k = 0; k < 64; ++k) {
        const int e = (int)((unsigned long long)z[k] >> 52) & 0x7FF;
        if (e == 0x7FF) nonfinite = 1;
        else emax = max(emax, e);
    }
    emax = warp_max(emax);
    if ((t & 31) == 0) red[t >> 5] = emax;
    __syncthreads();  // also publishes sgn[]
    emax = max(red[0], red[1]);
    if (emax > Erun) {
        if (Erun > 0) {
            const int d = emax - Erun;
            for (int64_t i = t; i < s; i += 64) acc[i] = (d >= 63) ? (acc[i] >> 63) : (acc[i] >> d);
        }
        Erun = emax;
    }
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) {
        const uint32_t sw = sgn[4 * kk + (t >> 4)] >> (2 * (t & 15));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const unsigned long long raw = (unsigned long long)z[2 * kk + h];
            const int e = (int)(raw >> 52) & 0x7FF;
            const unsigned long long frac = raw & 0x000FFFFFFFFFFFFFull;
            const unsigned long long mant = e ? (frac | 0x0010000000000000ull) : frac;
            const int sh = Erun - (e ? e : 1) + 53 - P;
            unsigned long long q = (sh >= 64 || e == 0x7FF) ? 0ull : ((mant + (1ull << (sh - 1))) >> sh);
            const unsigned long long neg = ((raw >> 63) ^ ((sw >> h) & 1u)) & 1u;
            const unsigned long long msk = 0ull - neg;
            z[2 * kk + h] = (long long)((q ^ msk) + neg);
        }
    }
    fwht64(z);
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) {
        const int i = 2 * t + 128 * kk;
        longlong2 v;
        v.x = z[2 * kk];
        v.y = z[2 * kk + 1];
        *(longlong2 *)(Zs + swz(i)) = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 64; ++k) z[k] = Zs[swz(l2_elem(t, k))];
    __syncthreads();
    fwht64(z);
#pragma unroll
    for (int k = 0; k < 64; ++k)
        if ((myneed >> k) & 1ull) Zs[swz(l2_elem(t, k))] = z[k];
    __syncthreads();
    for (int64_t i = t; i < s; i += 64) {
        const int r = rows_s[i];
        const long long v = Zs[swz(r & (kBlock - 1))];
        const int neg = __popcll((unsigned long long)(r >> kBlockLog) & (unsigned long long)b) & 1;
        acc[i] += neg ? -v : v;
    }
    __syncthreads();
}

// layout-2 registers that hold a sampled row (the same for every block): one
// 64-bit mask per thread, built in need[64] from rows_s[0..s)
__device__ __forceinline__ unsigned long long srht_need_mask(const int32_t *rows_s, int64_t s,
                                                             unsigned long long *need) {
    const int t = threadIdx.x;
    need[t] = 0ull;
    __syncthreads();
    for (int64_t i = t; i < s; i += 64) {
        const int lo = rows_s[i] & (kBlock - 1);
        atomicOr(&need[(lo & 1) | ((lo >> 7) << 1)], 1ull << ((lo >> 1) & 63));
    }
    __syncthreads();
    return need[t];
}

}  // namespace ns
