// ns_hrht.cu -- H-RHT sketch SA = S_h (1/sqrt m') H D [A; 0] (Section 2, after
// Theorem 2.2: the SRFT with its restriction R replaced by a random 1-hashing
// matrix S_h, whose column i holds one sign sg_i in row h(i)), FP64 input.
//
// Unlike the SRHT, every one of the m' transformed coordinates reaches the
// sketch, so the transform cannot be pruned to s rows.  With the Kronecker
// split H_{m'} = H_B (x) H_4096 (B = m'/4096 blocks):
//   pass 1 (hrht_block_kernel): Z_b = H_4096 (D a)_b for every (column, block)
//     by the exact fixed-point pipeline of the SRHT (quantised at the block's
//     own largest exponent), written to workspace as int64 with the block's
//     quantum exponent and the exponent just above its largest |Z|;
//   pass 2 (hrht_cross_kernel): for a slab of W = 4096/B consecutive lo and
//     all B blocks (staged into shared memory by cp.async, the next slab's
//     copies in flight while this one is transformed), each Z_b[lo] is
//     rounded once onto the column's common
//     quantum (so that the column's largest |Z| sits at 2^P2), H_B runs across
//     the blocks in 4-bit register phases around a shared-memory transpose,
//     and each result y[(hi << 12) | lo] is added with its sign into the
//     accumulator of row h(i): three 21-bit limbs in 32-bit words while a
//     bucket takes at most 2^11 values of a segment, else one int64;
//   the segment partials go to FP64 and are summed in segment order.
// All adds after the two roundings (input quantisation, alignment) are exact
// integer adds, so the result does not depend on the order of the atomics.
// Headroom: P2 = 62 - log2(B) - cb, with cb = ceil(log2(largest number of
// rows any segment sends to one bucket)), counted by the meta kernel.
#include <climits>
#include <cmath>
#include "ns_device.cuh"
#include "ns_internal.h"
#include "ns_srht_core.cuh"

namespace ns {

constexpr int kHrhtP1 = 63 - kBlockLog - 1;  // pass-1 magnitude bits (one block per accumulator)

HrhtGeom hrht_geom(int64_t m, int64_t n) {
    HrhtGeom g;
    g.lg = ceil_log2(m);
    g.mp = (int64_t)1 << g.lg;
    g.B = g.mp > kBlock ? g.mp / kBlock : 1;
    g.LB = ceil_log2(g.B);
    g.lw = kBlockLog - g.LB;
    int64_t want = (2048 + n - 1) / n;
    if (want < 16) want = 16;
    int64_t nseg = 1;
    while (nseg < want && nseg < 64) nseg *= 2;
    if (nseg > g.B) nseg = g.B;
    g.nseg = (int)nseg;
    g.sps = g.B / nseg;
    g.sign_words = (g.mp > kBlock ? g.mp : kBlock) / 32;
    return g;
}

HrhtWork hrht_carve(Carver &c, int64_t m, int64_t n, int64_t s) {
    const HrhtGeom g = hrht_geom(m, n);
    HrhtWork w;
    w.sign_words = c.take<uint32_t>((size_t)g.sign_words);
    w.hash = c.take<uint32_t>((size_t)(g.mp > kBlock ? g.mp : kBlock));  // the staged tiles read whole slabs
    w.cmax = c.take<unsigned int>(1);
    w.blk = c.take<int2>((size_t)(n * g.B));
    w.Z = c.take<long long>((size_t)(n * g.B * kBlock));
    w.partial = c.take<double>((size_t)(g.nseg * n * s));
    return w;
}

// ------------------------------------------------------------------- meta ----
// hash[i] = h(i) | (sg_i < 0) << 31 for i < m', from word (i mod 4) of
// stream-4 block i/4: h(i) = floor(s (w mod 2^32) / 2^32), sg_i = -1 when bit
// 63 of w is set.  CTA g covers segment g (lo in [g L, (g+1) L), all blocks)
// and raises *cmax to its largest bucket count.
__global__ void __launch_bounds__(256) hrht_meta_kernel(uint64_t seed, int64_t s, int64_t mp, int64_t B, int L,
                                                        uint32_t *__restrict__ hash, unsigned int *cmax) {
    extern __shared__ unsigned int hist[];  // s
    const int t = threadIdx.x;
    for (int64_t r = t; r < s; r += 256) hist[r] = 0;
    __syncthreads();
    const int64_t lo_base = (int64_t)blockIdx.x * L;
    const int64_t quads = B * (L / 4);
    for (int64_t q = t; q < quads; q += 256) {
        const int64_t hi = q / (L / 4);
        const int64_t i0 = (hi << kBlockLog) | (lo_base + 4 * (q - hi * (L / 4)));
        if (i0 >= mp) continue;
        const u64x4 w = draw(seed, (uint64_t)(i0 >> 2), 0, 4);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (i0 + u < mp) {
                const uint64_t word = w.w[u];
                const uint32_t bucket = (uint32_t)(((word & 0xFFFFFFFFull) * (uint64_t)s) >> 32);
                hash[i0 + u] = bucket | ((uint32_t)(word >> 63) << 31);
                atomicAdd(&hist[bucket], 1u);
            }
        }
    }
    __syncthreads();
    unsigned int mx = 0;
    for (int64_t r = t; r < s; r += 256) mx = max(mx, hist[r]);
    mx = warp_max(mx);
    if ((t & 31) == 0 && mx) atomicMax(cmax, mx);
}

// ----------------------------------------------------------------- pass 1 ----
// One (column, block) per CTA of 256 threads (srht_block256_core): Z_b in int64
// at quantum 2^(E_b - 1022 - P1), E_b the block's largest biased exponent.  blk
// gets (quantum exponent, exponent above the largest |Z|; INT_MIN for Z_b = 0).
__global__ void __launch_bounds__(256, 4) hrht_block_kernel(const double *__restrict__ A, int64_t m, int64_t lda,
                                                            int64_t B, const uint32_t *__restrict__ sign_words,
                                                            long long *__restrict__ Z, int2 *__restrict__ blk,
                                                            int32_t *status, int vec_ok) {
    __shared__ __align__(16) long long Zs[kBlock];
    __shared__ uint32_t sgn[128];
    __shared__ int red[8];
    const int t = threadIdx.x;
    const int64_t item = blockIdx.x;
    const int64_t c = item / B, b = item - c * B;
    int Erun = 0, nonfinite = 0;
    long long z[16];
    srht_block256_core(A + c * lda, m, 0, b, kHrhtP1, sign_words, Zs, nullptr, sgn, red, vec_ok, Erun, nonfinite,
                       false, z);
    unsigned long long mx = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const unsigned long long a = (unsigned long long)(z[k] < 0 ? -z[k] : z[k]);
        mx = mx > a ? mx : a;
    }
    int bl = mx ? 64 - __clzll((long long)mx) : 0;
    bl = warp_max(bl);
    if ((t & 31) == 0) red[t >> 5] = bl;  // the core's later barriers ordered every read of the exponents
    long long *out = Z + (item << kBlockLog);
#pragma unroll
    for (int k = 0; k < 16; ++k) out[(t & 31) | (k << 5) | ((t >> 5) << 9)] = z[k];  // layout C
    __syncthreads();
    if (t == 0) {
        int bmax = red[0];
#pragma unroll
        for (int q = 1; q < 8; ++q) bmax = max(bmax, red[q]);
        const int qx = Erun - 1022 - kHrhtP1;
        blk[item] = make_int2(qx, bmax ? qx + bmax : INT_MIN);
    }
    if (nonfinite) set_status(status, NS_ERR_NONFINITE);
}

// ----------------------------------------------------------------- pass 2 ----
// Register j of thread t in phase p (b bits [4p, 4p + nb)) holds tile element
// (b, w): j's low nb bits are the phase bits; the other bits of j sit above
// t's 8 bits, so consecutive lanes take consecutive w (coalesced loads).
__device__ __forceinline__ void hrht_coord(int t, int j, int p, int nb, int lw, int &b, int &w) {
    const int pb = j & ((1 << nb) - 1);
    const int rest = t | ((j >> nb) << 8);
    w = rest & ((1 << lw) - 1);
    const int bo = rest >> lw;
    const int lowmask = (1 << (4 * p)) - 1;
    b = (bo & lowmask) | (pb << (4 * p)) | ((bo >> (4 * p)) << (4 * p + nb));
}

__device__ __forceinline__ void fwht16_bits(long long (&z)[16], int nb) {
#pragma unroll
    for (int h = 1; h < 16; h <<= 1) {
        if (h < (1 << nb)) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                if ((j & h) == 0) {
                    const long long a = z[j], c = z[j + h];
                    z[j] = a + c;
                    z[j + h] = a - c;
                }
            }
        }
    }
}

// q rounded (half up) from its block's quantum onto the column's, given the
// block's shift sh packed by hrht_pack_shift: an exact left shift by -sh when
// sh <= 0 (the bound on the block's top exponent keeps the result within
// 2^P2), else ((q >> (sh - 1)) + 1) >> 1, with shr.s64 clamping shifts past 63
// (a block far below the column's top rounds to 0).
__device__ __forceinline__ uint32_t hrht_pack_shift(int sh) {
    const int ls = sh < 0 ? (sh < -62 ? 62 : -sh) : 0;
    const int rs = sh > 0 ? (sh > 64 ? 64 : sh) : 0;
    return (uint32_t)ls | ((uint32_t)(rs > 0 ? rs - 1 : 0) << 8) | ((uint32_t)(rs > 0) << 16);
}
__device__ __forceinline__ long long hrht_align(long long q, uint32_t pk) {
    const long long v = (long long)((unsigned long long)q << (pk & 0xFF));
    long long r;
    asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"((pk >> 8) & 0xFF));
    return (pk >> 16) ? (r + 1) >> 1 : r;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Stage the slab at lo0 of a column: the B x W tile of Z (element (b, w) at
// index (b << lw) | w) and the matching B x W tile of hash words (rows
// (b << 12) | (lo0 + w)).  16-byte copies where a row of the tile allows.
__device__ __forceinline__ void hrht_stage(long long *zt, uint32_t *ht, const long long *Zc,
                                           const uint32_t *__restrict__ hash, int lw, int64_t lo0) {
    const int t = threadIdx.x;
    if (lw >= 1) {
        for (int q = t; q < kBlock / 2; q += 256) {
            const int e = 2 * q, b = e >> lw, w = e & ((1 << lw) - 1);
            cp_async16(zt + e, Zc + ((int64_t)b << kBlockLog) + lo0 + w);
        }
    } else {
        for (int e = t; e < kBlock; e += 256) cp_async8(zt + e, Zc + ((int64_t)e << kBlockLog) + lo0);
    }
    if (lw >= 2) {
        for (int q = t; q < kBlock / 4; q += 256) {
            const int e = 4 * q, b = e >> lw, w = e & ((1 << lw) - 1);
            cp_async16(ht + e, hash + ((int64_t)b << kBlockLog) + lo0 + w);
        }
    } else {
        for (int e = t; e < kBlock; e += 256) {
            const int b = e >> lw, w = e & ((1 << lw) - 1);
            cp_async4(ht + e, hash + ((int64_t)b << kBlockLog) + lo0 + w);
        }
    }
    cp_async_commit();
}

// LB = log2 B is a template parameter, so every tile coordinate below folds to
// a per-thread base plus a constant.  nst = 2: the copies of slab k + 1 run
// while slab k is transformed; nst = 1 where shared memory is short.
template <int LB>
__global__ void __launch_bounds__(256) hrht_cross_kernel(const long long *__restrict__ Z,
                                                         const int2 *__restrict__ blk, int64_t n, int nst,
                                                         int limbs_ok, int nseg, int64_t sps, int64_t mp, int64_t s,
                                                         const uint32_t *__restrict__ hash,
                                                         const unsigned int *cmax, double *__restrict__ partial) {
    constexpr int lw = kBlockLog - LB;
    constexpr int nph = LB > 0 ? (LB + 3) / 4 : 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    long long *zst = (long long *)smem_raw;                       // nst x 4096
    uint32_t *hst = (uint32_t *)(zst + nst * kBlock);             // nst x 4096
    long long *acc = (long long *)(hst + nst * kBlock);           // s int64, or 3 x s uint32 limbs
    uint32_t *shb = (uint32_t *)((uint32_t *)acc + (limbs_ok ? 3 : 2) * s);  // B
    __shared__ int red[8];
    const int t = threadIdx.x;
    const int64_t B = (int64_t)1 << LB;
    const int64_t c = blockIdx.x / nseg, g = blockIdx.x - c * nseg;
    const int2 *bc = blk + c * B;
    const long long *Zc = Z + ((c * B) << kBlockLog);
    const int64_t slab0 = g * sps, slab1 = (g + 1) * sps;
    hrht_stage(zst, hst, Zc, hash, lw, slab0 << lw);

    // the column's top exponent and each block's alignment shift
    int top = INT_MIN;
    for (int64_t b = t; b < B; b += 256) top = max(top, bc[b].y);
    top = warp_max(top);
    if ((t & 31) == 0) red[t >> 5] = top;
    uint32_t *acc32 = (uint32_t *)acc;
    for (int64_t r = t; r < (limbs_ok ? 3 : 2) * s; r += 256) acc32[r] = 0;
    __syncthreads();
    top = red[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) top = max(top, red[k]);
    const unsigned int cm = *cmax;
    const int cb = cm > 1 ? 32 - __clz(cm - 1) : 0;
    const int P2 = 62 - LB - cb;
    // Bucket sums on three 21-bit limbs in 32-bit words (32-bit shared atomics
    // run several times faster than 64-bit ones): exact while a bucket takes
    // at most 2^11 values, since |value| <= 2^(62 - cb).
    const bool limbs = limbs_ok && cb <= 11;
    const int qx2 = (top == INT_MIN) ? 0 : top - P2;
    for (int64_t b = t; b < B; b += 256) {
        const int2 e = bc[b];
        shb[b] = hrht_pack_shift((e.y == INT_MIN || top == INT_MIN) ? 64 : qx2 - e.x);
    }

    for (int64_t slab = slab0; slab < slab1; ++slab) {
        const int cur = nst == 2 ? (int)((slab - slab0) & 1) : 0;
        if (nst == 2) {
            if (slab + 1 < slab1) {
                hrht_stage(zst + (cur ^ 1) * kBlock, hst + (cur ^ 1) * kBlock, Zc, hash, lw, (slab + 1) << lw);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
        } else {
            if (slab > slab0) hrht_stage(zst, hst, Zc, hash, lw, slab << lw);  // the single stage is free again
            cp_async_wait<0>();
        }
        __syncthreads();  // slab's tiles (and shb) visible to all
        long long *tile = zst + cur * kBlock;
        const uint32_t *htile = hst + cur * kBlock;
        const int64_t lo0 = slab << lw;
        long long z[16];
        int nb = LB < 4 ? LB : 4;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            int b, w;
            hrht_coord(t, j, 0, nb, lw, b, w);
            z[j] = hrht_align(tile[(b << lw) | w], shb[b]);
        }
        fwht16_bits(z, nb);
        int p = 0;
#pragma unroll
        for (int pn = 1; pn < nph; ++pn) {
            // in place: each element is read and written by its owner only
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                int b, w;
                hrht_coord(t, j, p, nb, lw, b, w);
                tile[(b << lw) | w] = z[j];
            }
            __syncthreads();
            p = pn;
            nb = LB - 4 * p < 4 ? LB - 4 * p : 4;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                int b, w;
                hrht_coord(t, j, p, nb, lw, b, w);
                z[j] = tile[(b << lw) | w];
            }
            fwht16_bits(z, nb);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            int b, w;
            hrht_coord(t, j, p, nb, lw, b, w);
            if ((((int64_t)b << kBlockLog) | (lo0 + w)) < mp) {
                const uint32_t hv = htile[(b << lw) | w];
                const long long v = (hv >> 31) ? -z[j] : z[j];
                const uint32_t bk = hv & 0x7FFFFFFFu;
                if (limbs) {
                    atomicAdd(&acc32[bk], (uint32_t)v & 0x1FFFFFu);
                    atomicAdd(&acc32[s + bk], (uint32_t)(v >> 21) & 0x1FFFFFu);
                    atomicAdd(&acc32[2 * s + bk], (uint32_t)(int32_t)(v >> 42));
                } else {
                    atomicAdd((unsigned long long *)&acc[bk], (unsigned long long)v);
                }
            }
        }
        __syncthreads();  // this stage is refilled two slabs on
    }
    double *out = partial + (g * n + c) * s;
    for (int64_t r = t; r < s; r += 256) {
        const long long a = limbs ? (long long)acc32[r] + ((long long)acc32[s + r] << 21) +
                                        ((long long)(int32_t)acc32[2 * s + r] << 42)
                                  : acc[r];
        out[r] = ldexp((double)a, qx2);
    }
}

template <int LB>
static void launch_cross(const HrhtGeom &g, const HrhtWork &w, int64_t n, int64_t s, int nst, int limbs_ok,
                         size_t smem, cudaStream_t st, cudaError_t *e) {
    *e = cudaFuncSetAttribute(hrht_cross_kernel<LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (*e != cudaSuccess) return;
    hrht_cross_kernel<LB><<<(unsigned)(n * g.nseg), 256, smem, st>>>(w.Z, w.blk, n, nst, limbs_ok, g.nseg, g.sps,
                                                                      g.mp, s, w.hash, w.cmax, w.partial);
    *e = cudaGetLastError();
}

static size_t hrht_cross_smem(const HrhtGeom &g, int64_t s, int stages, int limbs) {
    return (size_t)stages * kBlock * (8 + 4) + (size_t)s * (limbs ? 12 : 8) + (size_t)g.B * 4;
}

cudaError_t launch_hrht_f64(uint64_t seed, const double *A, int64_t m, int64_t n, int64_t lda, int64_t s,
                            const HrhtWork &w, double *SA, int32_t *status, cudaStream_t st) {
    const HrhtGeom g = hrht_geom(m, n);
    cudaError_t e = cudaMemsetAsync(w.cmax, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    e = launch_srht_meta(seed, g.lg, g.sign_words, 0, w.sign_words, nullptr, st);
    if (e != cudaSuccess) return e;
    const size_t msmem = (size_t)s * 4;
    e = cudaFuncSetAttribute(hrht_meta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem);
    if (e != cudaSuccess) return e;
    hrht_meta_kernel<<<(unsigned)g.nseg, 256, msmem, st>>>(seed, s, g.mp, g.B, (int)(kBlock / g.nseg), w.hash,
                                                           w.cmax);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int vec_ok = ((((uintptr_t)A) & 15) == 0 && (lda & 1) == 0) ? 1 : 0;
    hrht_block_kernel<<<(unsigned)(n * g.B), 256, 0, st>>>(A, m, lda, g.B, w.sign_words, w.Z, w.blk, status, vec_ok);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // two stages where shared memory allows (s up to ~9000 with B = 4096)
    const size_t cap = (size_t)200 * 1024;
    const bool two = hrht_cross_smem(g, s, 2, 0) <= cap;
    const int nst = two ? 2 : 1;
    const int limbs_ok = hrht_cross_smem(g, s, nst, 1) <= cap ? 1 : 0;
    const size_t csmem = hrht_cross_smem(g, s, nst, limbs_ok);
    switch (g.LB) {
        case 0: launch_cross<0>(g, w, n, s, nst, limbs_ok, csmem, st, &e); break;
        case 1: launch_cross<1>(g, w, n, s, nst, limbs_ok, csmem, st, &e); break;
        case 2: launch_cross<2>(g, w, n, s, nst, limbs_ok, csmem, st, &e); break;
        case 3: launch_cross<3>(g, w, n, s, nst, limbs_ok, csmem, st, &e); break;
        case 4: launch_cross<4>(g, w, n, s, nst, limbs_ok, csmem, st, &e); break;
        case 5: launch_cross<5>(g, w, n, s, nst, limbs_ok, csmem, st, &e); break;
        case 6: launch_cross<6>(g, w, n, s, nst, limbs_ok, csmem, st, &e); break;
        case 7: launch_cross<7>(g, w, n, s, nst, limbs_ok, csmem, st, &e); break;
        case 8: launch_cross<8>(g, w, n, s, nst, limbs_ok, csmem, st, &e); break;
        case 9: launch_cross<9>(g, w, n, s, nst, limbs_ok, csmem, st, &e); break;
        case 10: launch_cross<10>(g, w, n, s, nst, limbs_ok, csmem, st, &e); break;
        case 11: launch_cross<11>(g, w, n, s, nst, limbs_ok, csmem, st, &e); break;
        case 12: launch_cross<12>(g, w, n, s, nst, limbs_ok, csmem, st, &e); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return launch_srht_reduce(w.partial, n, s, g.nseg, 1.0 / std::sqrt((double)g.mp), SA, st);
}

}  // namespace ns
