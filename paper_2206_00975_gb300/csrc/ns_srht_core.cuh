// ns_srht_core.cuh -- the per-block pipelines of the FP64 SRHT (see ns_srht.cu)
// and their shared quantiser (srht_quant2): the 64-thread form (srht_f64_block,
// used by the batched kernel), the 128-thread form (srht_block128_core +
// srht_f64_block128, used by the row-window chunk kernel) and the 256-thread
// form (srht_block256_core, used by the whole-column chunk kernel and by pass 1
// of the H-RHT).  All three give the same bits for the same blocks.
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

// Quantisation of two entries of a block (the raw IEEE words in a, b, the
// signs of D in bits 0 and 1 of sw) onto the block's fixed-point grid
// 2^(Erun - 1022 - P): the magnitude truncated toward zero, then the sign of
// the entry times d_i in two's complement.  A magnitude stays below 2^P.
// While Erun >= P no subnormal can reach the grid, so every entry takes the
// hidden bit and the 64-bit shift runs on 32-bit words (an entry 64 or more
// binades below the grid shifts to 0); below that, subnormals are handled
// exactly (exponent 1, no hidden bit).  Erun and P are uniform over the block,
// so the branch is too.
__device__ __forceinline__ void srht_quant2(long long &a, long long &b, uint32_t sw, int Erun, int P) {
    if (Erun >= P) {
        const int C = Erun + 53 - P;  // shift = C - e
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const unsigned long long raw = (unsigned long long)(h ? b : a);
            const uint32_t whi = (uint32_t)(raw >> 32), wlo = (uint32_t)raw;
            const uint32_t sh = (uint32_t)(C - (int)((whi >> 20) & 0x7FFu));
            const uint32_t mhi = (whi & 0x000FFFFFu) | 0x00100000u;
            uint32_t qhi, qmid, qlo;
            asm("shr.b32 %0, %1, %2;" : "=r"(qhi) : "r"(mhi), "r"(sh));  // 0 for sh >= 32
            asm("shf.r.clamp.b32 %0, %1, %2, %3;" : "=r"(qmid) : "r"(wlo), "r"(mhi), "r"(sh));
            const uint32_t sh2 = (uint32_t)max((int)sh - 32, 0);
            asm("shr.b32 %0, %1, %2;" : "=r"(qlo) : "r"(qmid), "r"(sh2));
            const long long msk = (long long)((int)(whi ^ (sw << (31 - h))) >> 31);
            const long long q = (long long)(((unsigned long long)qhi << 32) | qlo);
            (h ? b : a) = (q ^ msk) - msk;
        }
    } else {
        const int sh1b = Erun + 53 - P;  // shift = sh1b - max(e, 1)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const unsigned long long raw = (unsigned long long)(h ? b : a);
            const uint32_t hi = (uint32_t)(raw >> 32);
            const int e = (int)((hi >> 20) & 0x7FF), e1 = max(e, 1);
            const uint32_t sh = (uint32_t)(sh1b - e1);
            const uint32_t mhi = (hi & 0x000FFFFFu) | ((uint32_t)(1 - (e1 - e)) << 20);
            const unsigned long long mant = ((unsigned long long)mhi << 32) | (uint32_t)raw;
            unsigned long long q;
            asm("shr.b64 %0, %1, %2;" : "=l"(q) : "l"(mant), "r"(sh));  // clamps shifts >= 64 to 0
            const long long msk = (long long)((int)(hi ^ (sw << (31 - h))) >> 31);
            (h ? b : a) = ((long long)q ^ msk) - msk;
        }
    }
}

// Layout 1: thread t, register k holds element (k & 1) | (t << 1) | ((k >> 1) << 7).
// Layout 2: thread t, register k holds element (t & 1) | (k << 1) | ((t >> 1) << 7).
__device__ __forceinline__ int l2_elem(int t, int k) { return (t & 1) | (k << 1) | ((t >> 1) << 7); }

// One 4096-row block b of a column (64 threads): load, quantise at the running
// exponent Erun (rescaling the accumulator when it grows), H_4096 in two
// register phases around a swizzled shared-memory transpose, and the signed
// gather of the sampled rows (rows_s packed by srht_pack_row) into acc[0..s).
// Ends with __syncthreads().
__device__ __forceinline__ void srht_f64_block(const double *__restrict__ Acol, int64_t m, int64_t s, int64_t b,
                                               int P, const uint32_t *__restrict__ sign_words,
                                               const int32_t *rows_s, long long *Zs,
                                               long long *acc, uint32_t *sgn, int *red, int vec_ok, int &Erun,
                                               int &nonfinite, bool prefetch_next) {
    const int t = threadIdx.x;
    const int64_t base = b * kBlock;
    sgn[t] = sign_words[(base >> 5) + t];
    sgn[t + 64] = sign_words[(base >> 5) + 64 + t];
    if (t == 0 && prefetch_next && vec_ok && base + 2 * kBlock <= m)  // the next block, into L2 (one bulk copy)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(Acol + base + kBlock),
                     "r"((uint32_t)(kBlock * 8))
                     : "memory");
    long long z[64];
    if (vec_ok && base + kBlock <= m) {  // whole block, 16-byte aligned: no bounds tests
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) {
            const double2 v = __ldcs((const double2 *)(Acol + base + 2 * t + 128 * kk));
            z[2 * kk] = __double_as_longlong(v.x);
            z[2 * kk + 1] = __double_as_longlong(v.y);
        }
    } else {
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) {
            const int64_t i0 = base + 2 * t + 128 * kk;
            z[2 * kk] = (i0 < m) ? __double_as_longlong(__ldcs(Acol + i0)) : 0;
            z[2 * kk + 1] = (i0 + 1 < m) ? __double_as_longlong(__ldcs(Acol + i0 + 1)) : 0;
        }
    }
    // largest biased exponent (an Inf or NaN shows up as 0x7FF and is flagged)
    unsigned int hmax = 0x00100000u;  // biased exponent 1
#pragma unroll
    for (int k = 0; k < 64; ++k) hmax = max(hmax, (unsigned int)((unsigned long long)z[k] >> 32) & 0x7FF00000u);
    hmax = warp_max(hmax);
    if ((t & 31) == 0) red[t >> 5] = (int)(hmax >> 20);
    __syncthreads();  // also publishes sgn[]
    const int emax = max(red[0], red[1]);
    if (emax == 0x7FF) nonfinite = 1;
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
        srht_quant2(z[2 * kk], z[2 * kk + 1], sw, Erun, P);
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
    fwht64(z);
#pragma unroll
    for (int k = 0; k < 64; ++k) Zs[swz(l2_elem(t, k))] = z[k];  // in place; all of them: cheaper than testing
    __syncthreads();
    for (int64_t i = t; i < s; i += 64) {
        const uint32_t pr = (uint32_t)rows_s[i];  // srht_pack_row: (hi(r) << 12) | swz(lo(r))
        const long long v = Zs[pr & (kBlock - 1)];
        const long long msk = -(long long)(__popc(pr >> kBlockLog & (uint32_t)b) & 1);
        acc[i] += (v ^ msk) - msk;
    }
    __syncthreads();
}

// in-register Walsh-Hadamard transform of 32 values (Sylvester order on the
// register index)
__device__ __forceinline__ void fwht32(long long (&z)[32]) {
#pragma unroll
    for (int h = 1; h < 32; h <<= 1) {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            if ((k & h) == 0) {
                const long long a = z[k], b = z[k + h];
                z[k] = a + b;
                z[k + h] = a - b;
            }
        }
    }
}

// The same block pipeline with 128 threads of 32 values (twice the warps per
// SM of the 64-thread form, for the same shared memory), H in three register
// phases around two swizzled transposes:
//   layout A: thread t, register k holds element (k & 1) | (t << 1) | ((k >> 1) << 8)
//     (H over index bits 0, 8..11);
//   layout B: (t & 1) | (k << 1) | ((t >> 1) << 6)  (bits 1..5);
//   layout C: (t & 63) | (k << 6) | ((t >> 6) << 11)  (bits 6, 7: the first
//     two register bits only; bits 8..10 are done).
// The lanes of a warp reading one register of layout B (C) differ in index
// bits 0, 6..9 (0..4), which swz spreads over all banks.  The quantisation
// is the 64-thread form's (srht_quant2) and the adds are exact integer adds:
// for the same blocks and exponent the result is that form's, bit for bit.
//
// srht_block128_core runs the load, the quantisation at Erun (rescaling
// acc[0..s) when Erun grows) and all 12 levels, and returns Z_b in registers
// in layout C.  Each thread reads a layout-B or layout-C register set from
// entries that only it rewrites (the transposes are in place), so no barrier
// separates a thread's reads of a layout from its stores back to it; a caller
// that stores Z_b elsewhere must synchronise before reusing Zs.
//
// Row window: the column holds global rows [lo, m) of the padded column and
// Acol points at global row lo (lo = 0 for a whole column); rows outside the
// window read as zero, and b is the global block index (the signs of D and
// the row parities of H follow it).  A row block of A sketched this way gives
// its partial sum S[:, lo:m] A[lo:m, :] of the whole sketch.
__device__ __forceinline__ int layout_c(int t, int k) { return (t & 63) | (k << 6) | ((t >> 6) << 11); }

__device__ __forceinline__ void srht_block128_core(const double *__restrict__ Acol, int64_t m, int64_t s, int64_t b,
                                                   int P, const uint32_t *__restrict__ sign_words, long long *Zs,
                                                   long long *acc, uint32_t *sgn, int *red, int vec_ok, int &Erun,
                                                   int &nonfinite, bool prefetch_next, long long (&z)[32],
                                                   int64_t lo = 0) {
    const int t = threadIdx.x, lane = t & 31;
    const int64_t base = b * kBlock;
    const double *Ab = Acol + (base - lo);  // global row base (not dereferenced below lo)
    sgn[t] = sign_words[(base >> 5) + t];
    if (t == 0 && prefetch_next && vec_ok && base >= lo && base + 2 * kBlock <= m)  // the next block, into L2
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(Ab + kBlock), "r"((uint32_t)(kBlock * 8))
                     : "memory");
    if (vec_ok && base >= lo && base + kBlock <= m) {
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const double2 v = __ldcs((const double2 *)(Ab + 2 * t + 256 * kk));
            z[2 * kk] = __double_as_longlong(v.x);
            z[2 * kk + 1] = __double_as_longlong(v.y);
        }
    } else {
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const int64_t i0 = base + 2 * t + 256 * kk;
            z[2 * kk] = (i0 >= lo && i0 < m) ? __double_as_longlong(__ldcs(Acol + (i0 - lo))) : 0;
            z[2 * kk + 1] = (i0 + 1 >= lo && i0 + 1 < m) ? __double_as_longlong(__ldcs(Acol + (i0 + 1 - lo))) : 0;
        }
    }
    unsigned int hmax = 0x00100000u;  // biased exponent 1
#pragma unroll
    for (int k = 0; k < 32; ++k) hmax = max(hmax, (unsigned int)((unsigned long long)z[k] >> 32) & 0x7FF00000u);
    hmax = warp_max(hmax);
    if (lane == 0) red[t >> 5] = (int)(hmax >> 20);
    __syncthreads();  // also publishes sgn[]
    const int emax = max(max(red[0], red[1]), max(red[2], red[3]));
    if (emax == 0x7FF) nonfinite = 1;
    if (emax > Erun) {
        if (Erun > 0) {
            const int d = emax - Erun;
            for (int64_t i = t; i < s; i += 128) acc[i] = (d >= 63) ? (acc[i] >> 63) : (acc[i] >> d);
        }
        Erun = emax;
    }
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
        const uint32_t sw = sgn[8 * kk + (t >> 4)] >> (2 * (t & 15));
        srht_quant2(z[2 * kk], z[2 * kk + 1], sw, Erun, P);
    }
    fwht32(z);  // index bits 0, 8..11
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
        const int i = 2 * t + 256 * kk;
        longlong2 v;
        v.x = z[2 * kk];
        v.y = z[2 * kk + 1];
        *(longlong2 *)(Zs + swz(i)) = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 32; ++k) z[k] = Zs[swz((t & 1) | (k << 1) | ((t >> 1) << 6))];
    fwht32(z);  // index bits 1..5 (stored back in place: each thread rewrites the entries it read)
#pragma unroll
    for (int k = 0; k < 32; ++k) Zs[swz((t & 1) | (k << 1) | ((t >> 1) << 6))] = z[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 32; ++k) z[k] = Zs[swz((t & 63) | (k << 6) | ((t >> 6) << 11))];
#pragma unroll
    for (int h = 1; h <= 2; h <<= 1) {  // index bits 6, 7
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            if ((k & h) == 0) {
                const long long a = z[k], c = z[k + h];
                z[k] = a + c;
                z[k + h] = a - c;
            }
        }
    }
}

// One 4096-row block of the SRHT with 128 threads: srht_block128_core, then
// the signed gather of the sampled rows (rows_s packed by srht_pack_row) into
// acc[0..s).  Ends with __syncthreads().
__device__ __forceinline__ void srht_f64_block128(const double *__restrict__ Acol, int64_t m, int64_t s, int64_t b,
                                                  int P, const uint32_t *__restrict__ sign_words,
                                                  const int32_t *rows_s, long long *Zs, long long *acc,
                                                  uint32_t *sgn, int *red, int vec_ok, int &Erun, int &nonfinite,
                                                  bool prefetch_next, int64_t lo = 0) {
    const int t = threadIdx.x;
    long long z[32];
    srht_block128_core(Acol, m, s, b, P, sign_words, Zs, acc, sgn, red, vec_ok, Erun, nonfinite, prefetch_next, z,
                       lo);
#pragma unroll
    for (int k = 0; k < 32; ++k) Zs[swz(layout_c(t, k))] = z[k];
    __syncthreads();
    for (int64_t i = t; i < s; i += 128) {
        const uint32_t pr = (uint32_t)rows_s[i];  // srht_pack_row: (hi(r) << 12) | swz(lo(r))
        const long long v = Zs[pr & (kBlock - 1)];
        const long long msk = -(long long)(__popc(pr >> kBlockLog & (uint32_t)b) & 1);
        acc[i] += (v ^ msk) - msk;
    }
    __syncthreads();
}

// The block pipeline with 256 threads of 16 values: four CTAs of eight warps
// share an SM (twice the warps of the 128-thread form, for the same shared
// memory), which hides the shared-memory and dependent-add latencies that bind
// the 128-thread form.  H runs in three register phases of four levels around
// two transposes:
//   layout A: register k holds element (k & 1) | (t << 1) | ((k >> 1) << 9)  (index bits 0, 9..11)
//   layout B: (t & 1) | (k << 1) | ((t >> 1) << 5)                           (bits 1..4)
//   layout C: (t & 31) | (k << 5) | ((t >> 5) << 9)                          (bits 5..8)
// Entry i sits at swz5(i) = i ^ (((i >> 5) & 15) << 1) in shared memory.  The
// 16-byte stores of layout A cover 256 consecutive bytes per half warp; the
// lanes reading one register of layout B differ in index bits 0 and 5..8,
// which swz5 spreads over all banks; a register of layout C is 32 consecutive
// entries.  A thread's layout-A addresses are one base plus a constant per
// register pair; its layout-B and layout-C addresses one base XOR a constant
// per register.
// A thread writes each layout back to the entries it read it from, so only
// the A -> B and B -> C hand-overs need barriers.  The quantisation
// (srht_quant2) and the adds are the 128-thread form's, so the result is that
// form's, bit for bit.
__device__ __forceinline__ int swz5(int i) { return i ^ (((i >> 5) & 15) << 1); }

__device__ __forceinline__ void fwht16(long long (&z)[16]) {
#pragma unroll
    for (int h = 1; h < 16; h <<= 1) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if ((k & h) == 0) {
                const long long a = z[k], c = z[k + h];
                z[k] = a + c;
                z[k + h] = a - c;
            }
        }
    }
}

// srht_block256_core: block b of the column Acol (rows >= m read as zero):
// the load (and, with prefetch_next, a bulk L2 prefetch of block b + 1), the
// largest exponent (a barrier that also publishes the sign words and orders
// the caller's previous use of Zs), the quantisation at Erun (rescaling
// acc[0..s) when Erun grows), all 12 levels; Z_b is returned in registers in
// layout C, read from entries of Zs that only this thread rewrites.  Zs holds
// 4096 int64, sgn 128 words, red 8 ints.
__device__ __forceinline__ void srht_block256_core(const double *__restrict__ Acol, int64_t m, int64_t s, int64_t b,
                                                   int P, const uint32_t *__restrict__ sign_words, long long *Zs,
                                                   long long *acc, uint32_t *sgn, int *red, int vec_ok, int &Erun,
                                                   int &nonfinite, bool prefetch_next, long long (&z)[16]) {
    const int t = threadIdx.x;
    const int64_t base = b * kBlock;
    // shared addresses: layout A stores (plus 4096 kk), layout B (XOR 16 k), layout C (XOR 272 k)
    const uint32_t zs = (uint32_t)__cvta_generic_to_shared(Zs);
    const uint32_t offA = 8u * (uint32_t)swz5(2 * t);
    const uint32_t offB = 8u * (uint32_t)swz5((t & 1) | ((t >> 1) << 5));
    const uint32_t offC = 8u * (uint32_t)((t & 31) | ((t >> 5) << 9));
    if (t < 128) sgn[t] = sign_words[(base >> 5) + t];
    if (t == 0 && prefetch_next && vec_ok && base + 2 * kBlock <= m)  // the next block, into L2
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(Acol + base + kBlock),
                     "r"((uint32_t)(kBlock * 8))
                     : "memory");
    if (vec_ok && base + kBlock <= m) {
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const double2 v = __ldcs((const double2 *)(Acol + base + 2 * t + 512 * kk));
            z[2 * kk] = __double_as_longlong(v.x);
            z[2 * kk + 1] = __double_as_longlong(v.y);
        }
    } else {
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const int64_t i0 = base + 2 * t + 512 * kk;
            z[2 * kk] = (i0 < m) ? __double_as_longlong(__ldcs(Acol + i0)) : 0;
            z[2 * kk + 1] = (i0 + 1 < m) ? __double_as_longlong(__ldcs(Acol + i0 + 1)) : 0;
        }
    }
    unsigned int hmax = 0x00100000u;  // biased exponent 1
#pragma unroll
    for (int k = 0; k < 16; ++k) hmax = max(hmax, (unsigned int)((unsigned long long)z[k] >> 32) & 0x7FF00000u);
    hmax = warp_max(hmax);
    if ((t & 31) == 0) red[t >> 5] = (int)(hmax >> 20);
    __syncthreads();
    int emax = red[0];
#pragma unroll
    for (int q = 1; q < 8; ++q) emax = max(emax, red[q]);
    if (emax == 0x7FF) nonfinite = 1;
    if (emax > Erun) {
        if (Erun > 0) {
            const int d = emax - Erun;
            for (int64_t i = t; i < s; i += 256) acc[i] = (d >= 63) ? (acc[i] >> 63) : (acc[i] >> d);
        }
        Erun = emax;
    }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const uint32_t sw = sgn[16 * kk + (t >> 4)] >> (2 * (t & 15));
        srht_quant2(z[2 * kk], z[2 * kk + 1], sw, Erun, P);
    }
    fwht16(z);  // index bits 0, 9..11
#pragma unroll
    for (int kk = 0; kk < 8; ++kk)
        asm volatile("st.shared.v2.s64 [%0], {%1, %2};" ::"r"(zs + offA + 4096u * kk), "l"(z[2 * kk]),
                     "l"(z[2 * kk + 1])
                     : "memory");
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) asm volatile("ld.shared.s64 %0, [%1];" : "=l"(z[k]) : "r"(zs + (offB ^ (16u * k))) : "memory");
    fwht16(z);  // index bits 1..4, stored back in place
#pragma unroll
    for (int k = 0; k < 16; ++k) asm volatile("st.shared.s64 [%0], %1;" ::"r"(zs + (offB ^ (16u * k))), "l"(z[k]) : "memory");
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) asm volatile("ld.shared.s64 %0, [%1];" : "=l"(z[k]) : "r"(zs + (offC ^ (272u * k))) : "memory");
    fwht16(z);  // index bits 5..8
}

// in-register Walsh-Hadamard transform of 64 FP32 values (Sylvester order on
// the register index)
__device__ __forceinline__ void fwht64_f32(float (&z)[64]) {
#pragma unroll
    for (int h = 1; h < 64; h <<= 1) {
#pragma unroll
        for (int k = 0; k < 64; ++k) {
            if ((k & h) == 0) {
                const float a = z[k], b = z[k + h];
                z[k] = a + b;
                z[k + h] = a - b;
            }
        }
    }
}

// One 4096-row block b of an FP32 column with 64 threads (the FP32-stream
// precision mode): load, exact sign flip by D, H_4096 in FP32 in two register
// phases around the swizzled transpose (the layouts of srht_f64_block), and the
// signed gather of the sampled rows (rows_s packed by srht_pack_row) into the
// FP32 accumulator acc[0..s).  Zs holds 4096 floats.  Ends with __syncthreads().
__device__ __forceinline__ void srht_f32_block(const float *__restrict__ Acol, int64_t m, int64_t s, int64_t b,
                                               const uint32_t *__restrict__ sign_words, const int32_t *rows_s,
                                               float *Zs, float *acc, uint32_t *sgn, int vec_ok, int &nonfinite) {
    const int t = threadIdx.x;
    const int64_t base = b * kBlock;
    sgn[t] = sign_words[(base >> 5) + t];
    sgn[t + 64] = sign_words[(base >> 5) + 64 + t];
    float z[64];
    if (vec_ok && base + kBlock <= m) {
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) {
            const float2 v = __ldcs((const float2 *)(Acol + base + 2 * t + 128 * kk));
            z[2 * kk] = v.x;
            z[2 * kk + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) {
            const int64_t i0 = base + 2 * t + 128 * kk;
            z[2 * kk] = (i0 < m) ? __ldcs(Acol + i0) : 0.0f;
            z[2 * kk + 1] = (i0 + 1 < m) ? __ldcs(Acol + i0 + 1) : 0.0f;
        }
    }
    __syncthreads();  // publishes sgn[]
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) {
        const uint32_t sw = sgn[4 * kk + (t >> 4)] >> (2 * (t & 15));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t bits = __float_as_uint(z[2 * kk + h]);
            if ((bits & 0x7F800000u) == 0x7F800000u) nonfinite = 1;
            bits ^= ((sw >> h) & 1u) << 31;
            z[2 * kk + h] = __uint_as_float(bits);
        }
    }
    fwht64_f32(z);
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) {
        const int i = 2 * t + 128 * kk;
        *(float2 *)(Zs + swz(i)) = make_float2(z[2 * kk], z[2 * kk + 1]);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 64; ++k) z[k] = Zs[swz(l2_elem(t, k))];
    __syncthreads();
    fwht64_f32(z);
#pragma unroll
    for (int k = 0; k < 64; ++k) Zs[swz(l2_elem(t, k))] = z[k];
    __syncthreads();
    for (int64_t i = t; i < s; i += 64) {
        const uint32_t pr = (uint32_t)rows_s[i];
        const float v = Zs[pr & (kBlock - 1)];
        acc[i] += (__popc(pr >> kBlockLog & (uint32_t)b) & 1) ? -v : v;
    }
    __syncthreads();
}

// sample row r as the gather uses it: (hi(r) << 12) | swz(lo(r)) (r < 2^31)
__device__ __forceinline__ int32_t srht_pack_row(int32_t r) {
    return (int32_t)(((uint32_t)r >> kBlockLog << kBlockLog) | (uint32_t)swz(r & (kBlock - 1)));
}

}  // namespace ns
