// ns_srht.cu -- SRHT sketch SA = (1/sqrt s) R H D [A; 0] (the SRFT of Section 2
// with the Sylvester Walsh-Hadamard matrix H for F), FP64 input.
//
// Arithmetic.  FP64 throughput on this part is ~1/64 of INT32, so the
// streaming pass never touches the FP64 pipe.  Each 4096-row block of a column
// is mapped exactly onto 64-bit fixed point (integer bit manipulation of the
// IEEE words, the magnitude truncated toward zero: srht_quant2), at a scale set
// by the largest exponent seen so far in the chunk, with P = 63 - 12 -
// log2(chunk) magnitude bits: a truncated magnitude stays below 2^P, so the
// 2^(12 + log2 chunk) terms of a chunk sum to less than 2^63.  The signs of D
// make the truncation error zero-mean in every output, and, uniform on one
// quantum, it has the spread of rounding to nearest at P - 1 bits.  The +-1
// butterflies of H are exact integer adds, so the transform and the pruned sum
// over blocks carry no rounding at all; the only rounding is the input
// quantisation (relative 2^-P of the chunk's largest entry) and one conversion
// per output.
//
// Structure (Kronecker split H_{m'} = H_{m'/4096} (x) H_{4096}):
//   y[r] = sum_b (-1)^popcount(hi(r) & b) Z_b[lo(r)],   Z_b = H_4096 (D a)_b,
// with hi(r) = r >> 12, lo(r) = r & 4095.  A CTA holds a block in registers,
// takes the 12 butterfly levels in three register phases around two swizzled
// shared-memory transposes, and adds the s sampled values Z_b[lo(r_t)] into its
// accumulator: 256 threads of 16 values for whole columns
// (srht_f64_chunk256_kernel), 128 threads of 32 values for row windows
// (srht_f64_chunk128_kernel over srht_block128_core in ns_srht_core.cuh).  The
// two forms agree bit for bit on the same chunks.  For m' <= 4096 the column is
// one zero-padded block: H's entries depend only on popcount(i & j), so padding
// to 4096 leaves the sampled rows unchanged.
#include <cmath>
#include "ns_device.cuh"
#include "ns_internal.h"
#include "ns_srht_core.cuh"

namespace ns {

SrhtGeom srht_geom(int64_t m, int64_t n) {
    SrhtGeom g;
    g.lg = ceil_log2(m);
    const int64_t mp = (int64_t)1 << g.lg;
    g.nblk = mp > kBlock ? mp / kBlock : 1;
    // about 2048 (column, chunk) work items; chunk is a power of two <= 16
    int64_t want = (g.nblk * n) / 2048;
    int chunk = 1;
    while (chunk * 2 <= want && chunk * 2 <= kMaxChunkBlocks) chunk *= 2;
    while (chunk > g.nblk) chunk /= 2;
    g.chunk = chunk;
    g.nchunk = g.nblk / chunk;
    g.fx_bits = 63 - kBlockLog - ceil_log2(chunk);
    g.sign_words = (mp > kBlock ? mp : kBlock) / 32;
    return g;
}

size_t srht_work_bytes(int64_t m, int64_t n, int64_t s) {
    Carver c(nullptr);
    srht_carve(c, m, n, s);
    return c.used;
}

SrhtWork srht_carve(Carver &c, int64_t m, int64_t n, int64_t s) {
    SrhtGeom g = srht_geom(m, n);
    SrhtWork w;
    w.sign_words = c.take<uint32_t>((size_t)g.sign_words);
    w.rows = c.take<int32_t>((size_t)s);
    w.partial = c.take<double>((size_t)(g.nchunk * n * s));
    return w;
}

// ------------------------------------------------------------------- meta ----
// sign word j holds bits 32j..32j+31 of the sign vector; bit i comes from bit
// (i mod 64) of 64-bit word ((i mod 256)/64) of stream-0 block i/256.
__global__ void srht_meta_kernel(uint64_t seed, int lg, int64_t nwords, int64_t s, uint32_t *sign_words,
                                 int32_t *rows) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (sign_words && idx < nwords) {
        const u64x4 w = draw(seed, (uint64_t)(idx >> 3), 0, 0);
        const uint64_t word = w.w[(idx & 7) >> 1];
        sign_words[idx] = (idx & 1) ? (uint32_t)(word >> 32) : (uint32_t)word;
    }
    if (rows && idx < s) rows[idx] = (int32_t)sample_perm(seed, lg, (uint32_t)idx);
}

cudaError_t launch_srht_meta(uint64_t seed, int lg, int64_t nsign_words, int64_t s, uint32_t *sign_words,
                             int32_t *rows, cudaStream_t st) {
    const int64_t total = nsign_words > s ? nsign_words : s;
    const int threads = 256;
    const int64_t blocks = (total + threads - 1) / threads;
    srht_meta_kernel<<<(unsigned)blocks, threads, 0, st>>>(seed, lg, nsign_words, s, sign_words, rows);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(128, 4) srht_f64_chunk128_kernel(const double *__restrict__ A, int64_t m, int64_t n,
                                                            int64_t lda, int64_t s, int chunk, int64_t nchunk,
                                                            int P, const uint32_t *__restrict__ sign_words,
                                                            const int32_t *__restrict__ rows,
                                                            double *__restrict__ partial, int32_t *status,
                                                            int vec_ok, int64_t lo, int64_t b0, int64_t b_end) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    long long *Zs = (long long *)smem_raw;                       // 4096
    long long *acc = Zs + kBlock;                                // s
    uint32_t *sgn = (uint32_t *)(acc + s);                       // 128
    int *red = (int *)(sgn + 128);                               // 4
    int32_t *rows_s = (int32_t *)(red + 4);                      // s

    const int t = threadIdx.x;
    const int64_t item = blockIdx.x;
    const int64_t c = item / nchunk, ch = item - c * nchunk;
    const double *Acol = A + c * lda;

    for (int64_t i = t; i < s; i += 128) {
        rows_s[i] = srht_pack_row(rows[i]);
        acc[i] = 0;
    }
    __syncthreads();

    int Erun = 0;  // running biased exponent of the chunk (0: none yet)
    int nonfinite = 0;
    // blocks b0 + ch * chunk + bl of the column (global block indices), up to b_end
    for (int bl = 0; bl < chunk; ++bl) {
        const int64_t b = b0 + ch * chunk + bl;
        if (b >= b_end) break;
        srht_f64_block128(Acol, m, s, b, P, sign_words, rows_s, Zs, acc, sgn, red, vec_ok, Erun, nonfinite,
                          bl + 1 < chunk && b + 1 < b_end, lo);
    }
    // chunk partial in FP64: value = acc * 2^(E - 1022 - P)
    const double scale = ldexp(1.0, Erun - 1022 - P);
    double *out = partial + (ch * n + c) * s;
    for (int64_t i = t; i < s; i += 128) out[i] = (double)acc[i] * scale;
    if (nonfinite) set_status(status, NS_ERR_NONFINITE);
}

// SA[t, c] = (1/sqrt s) * sum over chunks, in chunk order (deterministic)
__global__ void srht_reduce_kernel(const double *__restrict__ partial, int64_t n, int64_t s, int64_t nchunk,
                                   double scale, double *__restrict__ SA) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * s) return;
    const int64_t c = idx / s, t = idx - c * s;
    double a = 0.0;
    for (int64_t ch = 0; ch < nchunk; ++ch) a += partial[(ch * n + c) * s + t];
    SA[t + c * s] = a * scale;
}

cudaError_t launch_srht_reduce(const double *partial, int64_t n, int64_t s, int64_t nchunk, double scale, double *SA,
                               cudaStream_t st) {
    const int threads = 256;
    const int64_t blocks = (n * s + threads - 1) / threads;
    srht_reduce_kernel<<<(unsigned)blocks, threads, 0, st>>>(partial, n, s, nchunk, scale, SA);
    return cudaGetLastError();
}

// --------------------------------------------------------- FP32 stream ----
// Precision variant: A stored in FP32 is streamed through the same blocked
// transform in FP32 arithmetic.  The signs of D are applied exactly (sign-bit
// flip); the +-1 butterflies and the sum over a chunk's blocks round in FP32;
// chunk partials are summed in FP64.  Same layouts as the FP64 kernel.
__device__ __forceinline__ void fwht64f(float (&z)[64]) {
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

__global__ void __launch_bounds__(64) srht_f32_chunk_kernel(const float *__restrict__ A, int64_t m, int64_t n,
                                                            int64_t lda, int64_t s, int chunk, int64_t nchunk,
                                                            const uint32_t *__restrict__ sign_words,
                                                            const int32_t *__restrict__ rows,
                                                            double *__restrict__ partial, int32_t *status,
                                                            int vec_ok) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *Zs = (float *)smem_raw;                                 // 4096
    float *acc = Zs + kBlock;                                      // s
    unsigned long long *need = (unsigned long long *)(acc + ((s + 1) & ~1ll));  // 64
    uint32_t *sgn = (uint32_t *)(need + 64);                       // 128
    int32_t *rows_s = (int32_t *)(sgn + 128);                      // s

    const int t = threadIdx.x;
    const int64_t item = blockIdx.x;
    const int64_t c = item / nchunk, ch = item - c * nchunk;
    const float *Acol = A + c * lda;
    for (int64_t i = t; i < s; i += 64) {
        rows_s[i] = rows[i];
        acc[i] = 0.0f;
    }
    need[t] = 0ull;
    __syncthreads();
    for (int64_t i = t; i < s; i += 64) {
        const int lo = rows_s[i] & (kBlock - 1);
        atomicOr(&need[(lo & 1) | ((lo >> 7) << 1)], 1ull << ((lo >> 1) & 63));
    }
    __syncthreads();
    const unsigned long long myneed = need[t];
    int nonfinite = 0;
    float z[64];
    for (int bl = 0; bl < chunk; ++bl) {
        const int64_t b = ch * chunk + bl;
        const int64_t base = b * kBlock;
        sgn[t] = sign_words[(base >> 5) + t];
        sgn[t + 64] = sign_words[(base >> 5) + 64 + t];
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) {
            const int64_t i0 = base + 2 * t + 128 * kk;
            float a0 = 0.0f, a1 = 0.0f;
            if (vec_ok && i0 + 1 < m) {
                const float2 v = __ldcs((const float2 *)(Acol + i0));
                a0 = v.x;
                a1 = v.y;
            } else {
                if (i0 < m) a0 = __ldcs(Acol + i0);
                if (i0 + 1 < m) a1 = __ldcs(Acol + i0 + 1);
            }
            z[2 * kk] = a0;
            z[2 * kk + 1] = a1;
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
        fwht64f(z);
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) {
            const int i = 2 * t + 128 * kk;
            const int p = i ^ (((i >> 7) & 15) << 1);
            *(float2 *)(Zs + p) = make_float2(z[2 * kk], z[2 * kk + 1]);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 64; ++k) z[k] = Zs[swz(l2_elem(t, k))];
        __syncthreads();
        fwht64f(z);
#pragma unroll
        for (int k = 0; k < 64; ++k)
            if ((myneed >> k) & 1ull) Zs[swz(l2_elem(t, k))] = z[k];
        __syncthreads();
        for (int64_t i = t; i < s; i += 64) {
            const int r = rows_s[i];
            const float v = Zs[swz(r & (kBlock - 1))];
            const int neg = __popcll((unsigned long long)(r >> kBlockLog) & (unsigned long long)b) & 1;
            acc[i] += neg ? -v : v;
        }
        __syncthreads();
    }
    double *out = partial + (ch * n + c) * s;
    for (int64_t i = t; i < s; i += 64) out[i] = (double)acc[i];
    if (nonfinite) set_status(status, NS_ERR_NONFINITE);
}

// Same transform with the sampled rows' sums in registers (s <= 64 RPT): each
// thread owns the rows t + 64 q, so the per-block gather is one shared-memory
// load and one add per owned row, in the same order as the kernel above (the
// results are identical).  The next block is prefetched into L2 with one bulk
// copy while the current one is transformed.
template <int RPT>
__global__ void __launch_bounds__(64) srht_f32_chunk_reg_kernel(const float *__restrict__ A, int64_t m, int64_t n,
                                                                int64_t lda, int64_t s, int chunk, int64_t nchunk,
                                                                const uint32_t *__restrict__ sign_words,
                                                                const int32_t *__restrict__ rows,
                                                                double *__restrict__ partial, int32_t *status,
                                                                int vec_ok) {
    __shared__ __align__(16) float Zs[kBlock];
    __shared__ unsigned long long need[64];
    __shared__ uint32_t sgn[128];
    const int t = threadIdx.x;
    const int64_t item = blockIdx.x;
    const int64_t c = item / nchunk, ch = item - c * nchunk;
    const float *Acol = A + c * lda;
    int32_t pr[RPT];
    float acc[RPT];
    need[t] = 0ull;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int64_t i = t + 64 * q;
        acc[q] = 0.0f;
        pr[q] = -1;
        if (i < s) {
            const int32_t r = rows[i];
            pr[q] = srht_pack_row(r);
            const int lo = r & (kBlock - 1);
            atomicOr(&need[(lo & 1) | ((lo >> 7) << 1)], 1ull << ((lo >> 1) & 63));
        }
    }
    __syncthreads();
    const unsigned long long myneed = need[t];
    int nonfinite = 0;
    float z[64];
    for (int bl = 0; bl < chunk; ++bl) {
        const int64_t b = ch * chunk + bl;
        const int64_t base = b * kBlock;
        sgn[t] = sign_words[(base >> 5) + t];
        sgn[t + 64] = sign_words[(base >> 5) + 64 + t];
        if (t == 0 && bl + 1 < chunk && vec_ok && base + 2 * kBlock <= m)  // the next block, into L2
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(Acol + base + kBlock),
                         "r"((uint32_t)(kBlock * 4))
                         : "memory");
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
        fwht64f(z);
#pragma unroll
        for (int kk = 0; kk < 32; ++kk) {
            const int i = 2 * t + 128 * kk;
            const int p = i ^ (((i >> 7) & 15) << 1);
            *(float2 *)(Zs + p) = make_float2(z[2 * kk], z[2 * kk + 1]);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 64; ++k) z[k] = Zs[swz(l2_elem(t, k))];
        __syncthreads();
        fwht64f(z);
#pragma unroll
        for (int k = 0; k < 64; ++k)
            if ((myneed >> k) & 1ull) Zs[swz(l2_elem(t, k))] = z[k];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            if (pr[q] >= 0) {
                const float v = Zs[pr[q] & (kBlock - 1)];
                const int neg = __popc((uint32_t)(pr[q] >> kBlockLog) & (uint32_t)b) & 1;
                acc[q] += neg ? -v : v;
            }
        }
        __syncthreads();
    }
    double *out = partial + (ch * n + c) * s;
#pragma unroll
    for (int q = 0; q < RPT; ++q)
        if (t + 64 * q < s) out[t + 64 * q] = (double)acc[q];
    if (nonfinite) set_status(status, NS_ERR_NONFINITE);
}

size_t srht_f32_smem(int64_t s) {
    return (size_t)kBlock * 4 + (size_t)((s + 1) & ~1ll) * 4 + 64 * 8 + 128 * 4 + (size_t)s * 4;
}

cudaError_t launch_srht_f32(const float *A, int64_t m, int64_t n, int64_t lda, int64_t s, const SrhtWork &w,
                            double *SA, int32_t *status, cudaStream_t st) {
    const SrhtGeom g = srht_geom(m, n);
    cudaError_t e = cudaSuccess;
    const int vec_ok = ((((uintptr_t)A) & 7) == 0 && (lda & 1) == 0) ? 1 : 0;
    const unsigned grid = (unsigned)(n * g.nchunk);
    if (s <= 64 * 32) {  // sampled rows in registers
        // the bulk L2 prefetch wants 16-byte aligned blocks
        const int vec16 = (vec_ok && (((uintptr_t)A) & 15) == 0 && (lda & 3) == 0) ? 1 : 0;
        if (s <= 64 * 8)
            srht_f32_chunk_reg_kernel<8><<<grid, 64, 0, st>>>(A, m, n, lda, s, g.chunk, g.nchunk, w.sign_words,
                                                               w.rows, w.partial, status, vec16);
        else if (s <= 64 * 16)
            srht_f32_chunk_reg_kernel<16><<<grid, 64, 0, st>>>(A, m, n, lda, s, g.chunk, g.nchunk, w.sign_words,
                                                                w.rows, w.partial, status, vec16);
        else
            srht_f32_chunk_reg_kernel<32><<<grid, 64, 0, st>>>(A, m, n, lda, s, g.chunk, g.nchunk, w.sign_words,
                                                                w.rows, w.partial, status, vec16);
    } else {
        const size_t smem = srht_f32_smem(s);
        e = cudaFuncSetAttribute(srht_f32_chunk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        srht_f32_chunk_kernel<<<grid, 64, smem, st>>>(A, m, n, lda, s, g.chunk, g.nchunk, w.sign_words, w.rows,
                                                      w.partial, status, vec_ok);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    srht_reduce_kernel<<<(unsigned)((n * s + 255) / 256), 256, 0, st>>>(w.partial, n, s, g.nchunk,
                                                                        1.0 / std::sqrt((double)s), SA);
    return cudaGetLastError();
}

// ------------------------------------------------------ 256-thread form ----
// Whole columns with the 256-thread block pipeline (srht_block256_core in
// ns_srht_core.cuh): per block the core, the in-place publication of layout C,
// and the signed gather of the sampled rows (packed with swz5) into acc.
__global__ void __launch_bounds__(256, 4) srht_f64_chunk256_kernel(const double *__restrict__ A, int64_t m,
                                                                    int64_t n, int64_t lda, int64_t s, int chunk,
                                                                    int64_t nchunk, int P,
                                                                    const uint32_t *__restrict__ sign_words,
                                                                    const int32_t *__restrict__ rows,
                                                                    double *__restrict__ partial, int32_t *status,
                                                                    int vec_ok) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    long long *Zs = (long long *)smem_raw;   // 4096
    long long *acc = Zs + kBlock;            // s
    uint32_t *sgn = (uint32_t *)(acc + s);   // 128
    int *red = (int *)(sgn + 128);           // 8
    int32_t *rows_s = (int32_t *)(red + 8);  // s

    const int t = threadIdx.x;
    const int64_t item = blockIdx.x;
    const int64_t c = item / nchunk, ch = item - c * nchunk;
    const double *Acol = A + c * lda;
    for (int64_t i = t; i < s; i += 256) {
        const uint32_t r = (uint32_t)rows[i];
        rows_s[i] = (int32_t)((r >> kBlockLog << kBlockLog) | (uint32_t)swz5((int)(r & (kBlock - 1))));
        acc[i] = 0;
    }
    const uint32_t zs = (uint32_t)__cvta_generic_to_shared(Zs);
    const uint32_t offC = 8u * (uint32_t)((t & 31) | ((t >> 5) << 9));
    __syncthreads();

    int Erun = 0, nonfinite = 0;
    for (int bl = 0; bl < chunk; ++bl) {
        const int64_t b = ch * chunk + bl;
        long long z[16];
        srht_block256_core(Acol, m, s, b, P, sign_words, Zs, acc, sgn, red, vec_ok, Erun, nonfinite, bl + 1 < chunk,
                           z);
#pragma unroll
        for (int k = 0; k < 16; ++k)  // publication, in place (layout C entries this thread read)
            asm volatile("st.shared.s64 [%0], %1;" ::"r"(zs + (offC ^ (272u * k))), "l"(z[k]) : "memory");
        __syncthreads();
        for (int64_t i = t; i < s; i += 256) {
            const uint32_t pr = (uint32_t)rows_s[i];  // (hi(r) << 12) | swz5(lo(r))
            const long long v = Zs[pr & (kBlock - 1)];
            const long long msk = -(long long)(__popc(pr >> kBlockLog & (uint32_t)b) & 1);
            acc[i] += (v ^ msk) - msk;
        }
        // the next block's first barrier orders this gather before Zs is reused
    }
    __syncthreads();
    const double scale = ldexp(1.0, Erun - 1022 - P);
    double *out = partial + (ch * n + c) * s;
    for (int64_t i = t; i < s; i += 256) out[i] = (double)acc[i] * scale;
    if (nonfinite) set_status(status, NS_ERR_NONFINITE);
}

static size_t srht_f64_smem256(int64_t s) { return (size_t)kBlock * 8 + (size_t)s * 8 + 128 * 4 + 8 * 4 + (size_t)s * 4; }

size_t srht_f64_smem(int64_t s) { return (size_t)kBlock * 8 + (size_t)s * 8 + 64 * 8 + 128 * 4 + 16 + (size_t)s * 4; }

cudaError_t launch_srht_f64(const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, const SrhtWork &w,
                            double *SA, int32_t *status, cudaStream_t st) {
    const SrhtGeom g = srht_geom(m, n);
    const size_t smem = srht_f64_smem256(s);
    cudaError_t e = cudaFuncSetAttribute(srht_f64_chunk256_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int vec_ok = ((((uintptr_t)A) & 15) == 0 && (lda & 1) == 0) ? 1 : 0;
    const int64_t items = n * g.nchunk;
    srht_f64_chunk256_kernel<<<(unsigned)items, 256, smem, st>>>(A, m, n, lda, s, g.chunk, g.nchunk, g.fx_bits,
                                                                 w.sign_words, w.rows, w.partial, status, vec_ok);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const int64_t blocks = (n * s + threads - 1) / threads;
    srht_reduce_kernel<<<(unsigned)blocks, threads, 0, st>>>(w.partial, n, s, g.nchunk, 1.0 / std::sqrt((double)s),
                                                            SA);
    return cudaGetLastError();
}

// ------------------------------------------------------------- row window ----
// The partial sketch of rows [lo, hi) of A (A_p points at row lo): the blocks
// that overlap the window, with global block indices (so the signs of D and
// the row parities of H are the whole sketch's), grouped into chunks as for a
// whole column; rows outside the window count as zero.  Summing the partials of
// windows that cover [0, m) gives the whole sketch up to the FP64 rounding of
// the chunk sums (exactly, on integer data).
SrhtRowsGeom srht_rows_geom(int64_t m_total, int64_t lo, int64_t hi, int64_t n) {
    SrhtRowsGeom g;
    g.lg = ceil_log2(m_total);
    const int64_t mp = (int64_t)1 << g.lg;
    g.b0 = lo / kBlock;
    g.b_end = mp > kBlock ? (hi + kBlock - 1) / kBlock : 1;
    const int64_t nb = g.b_end - g.b0;
    int64_t want = (nb * n) / 2048;
    int chunk = 1;
    while (chunk * 2 <= want && chunk * 2 <= kMaxChunkBlocks) chunk *= 2;
    while (chunk > 1 && chunk > nb) chunk /= 2;
    g.chunk = chunk;
    g.nchunk = (nb + chunk - 1) / chunk;
    g.fx_bits = 63 - kBlockLog - ceil_log2(chunk);
    g.sign_words = (mp > kBlock ? mp : kBlock) / 32;
    return g;
}

SrhtWork srht_rows_carve(Carver &c, int64_t m_total, int64_t lo, int64_t hi, int64_t n, int64_t s) {
    const SrhtRowsGeom g = srht_rows_geom(m_total, lo, hi, n);
    SrhtWork w;
    w.sign_words = c.take<uint32_t>((size_t)g.sign_words);
    w.rows = c.take<int32_t>((size_t)s);
    w.partial = c.take<double>((size_t)(g.nchunk * n * s));
    return w;
}

cudaError_t launch_srht_f64_rows(const double *A_p, int64_t m_total, int64_t lo, int64_t hi, int64_t n, int64_t lda,
                                 int64_t s, const SrhtWork &w, double *SA_p, int32_t *status, cudaStream_t st) {
    const SrhtRowsGeom g = srht_rows_geom(m_total, lo, hi, n);
    const size_t smem = srht_f64_smem(s);
    cudaError_t e = cudaFuncSetAttribute(srht_f64_chunk128_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    // whole blocks are loaded with 16-byte loads when global row lo sits on a
    // 16-byte boundary of the row block's storage
    const int vec_ok = ((((uintptr_t)A_p) & 15) == 0 && (lda & 1) == 0 && (lo & 1) == 0) ? 1 : 0;
    const int64_t items = n * g.nchunk;
    srht_f64_chunk128_kernel<<<(unsigned)items, 128, smem, st>>>(A_p, hi, n, lda, s, g.chunk, g.nchunk, g.fx_bits,
                                                                 w.sign_words, w.rows, w.partial, status, vec_ok, lo,
                                                                 g.b0, g.b_end);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    srht_reduce_kernel<<<(unsigned)((n * s + 255) / 256), 256, 0, st>>>(w.partial, n, s, g.nchunk,
                                                                        1.0 / std::sqrt((double)s), SA_p);
    return cudaGetLastError();
}

}  // namespace ns
