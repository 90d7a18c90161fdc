// ns_gauss.cu -- Gaussian sketch SA = G A / sqrt(s) (Theorem 2.1; G standard
// Gaussian, s x m) on the 5th-generation tensor cores (tcgen05.mma, TMEM
// accumulators), precision mode NS_PREC_BF16X3 with A stored in FP32.
//
// Split products: each operand x is split as hi = bf16(x), lo = bf16(x - hi),
// and G A ~ Gh Ah + Gh Al + Gl Ah (the lo*lo term, ~2^-18 relative, dropped),
// accumulated in FP32 in TMEM; the per-split FP32 partials are summed in FP64
// in a fixed order.
//
// G is never stored: entry (r, j) is generated where it is used, from Philox
// stream 3, block (r, j/8) (word (j mod 8)/2: u_a, u_b from its 32-bit halves;
// Box-Muller sqrt(-2 ln u_a) cos/sin(2 pi u_b) for even/odd j), in FP32 with
// CUDA's __logf, sqrtf and __sincosf.  One block gives the 8 consecutive K
// values of one row, i.e. one 16-byte row of an 8x8 core matrix of the operand.
//
// CTA tile: 128 rows of G (= rows of SA) x all n <= 512 columns of A (two
// accumulators of up to 256 columns in TMEM), over a slice of K = m (split-K
// across CTAs).  Per K chunk of 32: the 512 threads write Gh, Gl (128 x 32) and
// Ah, Al (n x 32) into shared memory in the canonical K-major no-swizzle layout
// (8x8 core matrices, 128 bytes apart along K, 512 bytes apart along M/N), then
// one thread issues 2 K-steps x 2 N-halves x 3 products of
// tcgen05.mma.cta_group::1.kind::f16 (M = 128, N <= 256, K = 16) and commits
// to an mbarrier; two buffers let the generation of chunk i+1 overlap the
// MMAs of chunk i.  All mbarrier waits are bounded.
#include <cmath>
#include <cuda_bf16.h>
#include "ns_device.cuh"
#include "ns_internal.h"

namespace ns {

constexpr int kGM = 128;        // rows of G per CTA (MMA M)
constexpr int kGK = 32;         // K per pipeline stage
constexpr int kGThreads = 512;
constexpr int kGMaxN = 512;
constexpr int kGSbo = (kGK / 8) * 128;  // bytes between 8-row groups (512)
constexpr int kGStageG = kGM * kGK * 2;  // bytes of one bf16 G tile (8 KB)

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: start address, leading (K) and
// stride (M/N) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major
__device__ __forceinline__ uint32_t umma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit) {
    uint32_t done = 0;
    long long polls = 0;
    while (!done) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity));
        if (!done && ++polls > limit) return false;
    }
    return true;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *(const uint32_t *)&v;
}

// split 8 values into hi and lo bf16 rows of a core matrix
__device__ __forceinline__ void split8(const float (&z)[8], uint4 &hi, uint4 &lo) {
    float h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        h[i] = __bfloat162float(__float2bfloat16_rn(z[i]));
        l[i] = z[i] - h[i];
    }
    hi = make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]), pack_bf16x2(h[4], h[5]), pack_bf16x2(h[6], h[7]));
    lo = make_uint4(pack_bf16x2(l[0], l[1]), pack_bf16x2(l[2], l[3]), pack_bf16x2(l[4], l[5]), pack_bf16x2(l[6], l[7]));
}

__global__ void __launch_bounds__(kGThreads, 1) gauss_bf16x3_kernel(const float *__restrict__ A, int64_t m, int64_t n,
                                                                   int64_t lda, int64_t s, int NP, int64_t kper,
                                                                   uint64_t seed, float *__restrict__ partial,
                                                                   int32_t *status) {
    extern __shared__ __align__(1024) unsigned char gsm[];
    // stage b: Gh | Gl | Ah | Al
    const int stage_bytes = 2 * kGStageG + 2 * NP * kGK * 2;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int timed_out;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t mtile = blockIdx.x, split = blockIdx.y;
    const int64_t row0 = mtile * kGM;
    const int64_t kbeg = split * kper, kend = (kbeg + kper < m) ? kbeg + kper : m;
    const int ncols_alloc = NP <= 32 ? 32 : (NP <= 64 ? 64 : (NP <= 128 ? 128 : (NP <= 256 ? 256 : 512)));
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        timed_out = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(ncols_alloc));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const int nstages = (int)((kend - kbeg + kGK - 1) / kGK);
    const int nhalf = NP > 256 ? 2 : 1;
    const long long kLimit = 1ll << 26;
    for (int it = 0; it < nstages; ++it) {
        const int b = it & 1;
        if (it >= 2) {
            if (!mbar_wait(smem_addr(&mbar[b]), (uint32_t)(((it - 2) >> 1) & 1), kLimit)) timed_out = 1;
        }
        __syncthreads();
        if (timed_out) break;
        unsigned char *st = gsm + (size_t)b * stage_bytes;
        unsigned char *sGh = st, *sGl = st + kGStageG, *sAh = st + 2 * kGStageG, *sAl = sAh + NP * kGK * 2;
        const int64_t k0 = kbeg + (int64_t)it * kGK;
        // ---- A: NP columns x 4 octets of K, loads issued first so that the
        // generation of G below hides their latency
        constexpr int kAItems = kGMaxN * (kGK / 8) / kGThreads;  // items per thread (8)
        float za[kAItems][8];
#pragma unroll
        for (int q = 0; q < kAItems; ++q) {
            const int id = tid + q * kGThreads;
            const int c = id >> 2, o = id & 3;
            const int64_t j0 = k0 + 8 * o;
            if (c < NP && c < n && j0 + 8 <= kend && (((uintptr_t)(A + j0 + c * lda)) & 15) == 0) {
                const float4 v0 = __ldcs((const float4 *)(A + j0 + c * lda));
                const float4 v1 = __ldcs((const float4 *)(A + j0 + c * lda) + 1);
                za[q][0] = v0.x; za[q][1] = v0.y; za[q][2] = v0.z; za[q][3] = v0.w;
                za[q][4] = v1.x; za[q][5] = v1.y; za[q][6] = v1.z; za[q][7] = v1.w;
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    za[q][u] = (c < NP && c < n && j0 + u < kend) ? A[j0 + u + c * lda] : 0.0f;
            }
        }
        // ---- G: 128 rows x 4 octets of K, one Philox block per (row, octet)
        for (int id = tid; id < kGM * (kGK / 8); id += kGThreads) {
            const int r = id >> 2, o = id & 3;
            const int64_t gr = row0 + r;
            float z[8];
            if (gr < s && k0 + 8 * o < kend) {
                const u64x4 w = draw(seed, (uint64_t)gr, (uint64_t)((k0 >> 3) + o), 3);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float ua = ((float)(uint32_t)w.w[q] + 0.5f) * 2.3283064365386963e-10f;
                    const float ub = ((float)(uint32_t)(w.w[q] >> 32) + 0.5f) * 2.3283064365386963e-10f;
                    const float rad = sqrtf(-2.0f * __logf(ua));
                    float sn, cs;
                    __sincosf(6.283185307179586f * (ub - 0.5f), &sn, &cs);  // angle 2 pi u_b - pi
                    z[2 * q] = -rad * cs;
                    z[2 * q + 1] = -rad * sn;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) z[q] = 0.0f;
            }
            uint4 hi, lo;
            split8(z, hi, lo);
            const int off = (r >> 3) * kGSbo + o * 128 + (r & 7) * 16;
            *(uint4 *)(sGh + off) = hi;
            *(uint4 *)(sGl + off) = lo;
        }
        // ---- A: split into bf16 hi / lo core-matrix rows
#pragma unroll
        for (int q = 0; q < kAItems; ++q) {
            const int id = tid + q * kGThreads;
            const int c = id >> 2, o = id & 3;
            if (c < NP) {
                uint4 hi, lo;
                split8(za[q], hi, lo);
                const int off = (c >> 3) * kGSbo + o * 128 + (c & 7) * 16;
                *(uint4 *)(sAh + off) = hi;
                *(uint4 *)(sAl + off) = lo;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t aGh = smem_addr(sGh), aGl = smem_addr(sGl), aAh = smem_addr(sAh), aAl = smem_addr(sAl);
#pragma unroll
            for (int kk = 0; kk < kGK / 16; ++kk) {
                for (int h = 0; h < nhalf; ++h) {
                    const int nh = (h == 0) ? (NP < 256 ? NP : 256) : NP - 256;
                    const uint32_t idesc = umma_idesc(kGM, nh);
                    const uint32_t dcol = tmem + 256 * h;
                    const uint32_t koff = kk * 256, noff = h * 256 * (kGSbo / 8);
                    const uint64_t gh = umma_desc(aGh + koff, 128, kGSbo), gl = umma_desc(aGl + koff, 128, kGSbo);
                    const uint64_t ah = umma_desc(aAh + noff + koff, 128, kGSbo);
                    const uint64_t al = umma_desc(aAl + noff + koff, 128, kGSbo);
                    const uint32_t first = (it == 0 && kk == 0) ? 0u : 1u;
                    umma_bf16(dcol, gh, ah, idesc, first);
                    umma_bf16(dcol, gh, al, idesc, 1u);
                    umma_bf16(dcol, gl, ah, idesc, 1u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&mbar[b])));
        }
    }
    // ---- wait for the last commit (it covers every MMA this thread issued)
    if (nstages > 0) {
        const int last = nstages - 1;
        if (!mbar_wait(smem_addr(&mbar[last & 1]), (uint32_t)((last >> 1) & 1), kLimit)) timed_out = 1;
    }
    __syncthreads();
    if (timed_out) {
        // give MMAs in flight a second bounded chance before the memory is released
        if (nstages > 0) mbar_wait(smem_addr(&mbar[(nstages - 1) & 1]), (uint32_t)(((nstages - 1) >> 1) & 1), kLimit);
        if (tid == 0) set_status(status, NS_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!timed_out && nstages > 0) {
        // TMEM lanes 32 (warp % 4) .. +31 = rows; warp group warp / 4 takes a
        // quarter of the columns (16-column granules)
        const int granules = NP / 16, g4 = warp >> 2;
        const int c0 = 16 * ((granules * g4) / 4), c1 = 16 * ((granules * (g4 + 1)) / 4);
        const int64_t r = row0 + 32 * (warp & 3) + lane;
        for (int cb = c0; cb < c1; cb += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)cb;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int64_t c = cb + q;
                if (r < s && c < n) partial[(split * n + c) * s + r] = __uint_as_float(v[q]);
            }
        }
    } else if (nstages == 0) {
        for (int64_t idx = tid; idx < (int64_t)kGM * n; idx += kGThreads) {
            const int64_t r = row0 + idx % kGM, c = idx / kGM;
            if (r < s) partial[(split * n + c) * s + r] = 0.0f;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols_alloc));
}

__global__ void gauss_reduce_kernel(const float *__restrict__ partial, int64_t n, int64_t s, int64_t nsplit,
                                    double scale, double *__restrict__ SA) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * s) return;
    const int64_t c = idx / s, r = idx - c * s;
    double a = 0.0;
    for (int64_t sp = 0; sp < nsplit; ++sp) a += (double)partial[(sp * n + c) * s + r];
    SA[r + c * s] = a * scale;
}

GaussGeom gauss_geom(int64_t m, int64_t n, int64_t s) {
    GaussGeom g;
    g.mtiles = (s + kGM - 1) / kGM;
    g.NP = (int)(((n + 15) / 16) * 16);
    const int sms = device_sm_count();
    int64_t nsplit = sms / (g.mtiles > 0 ? g.mtiles : 1);
    if (nsplit < 1) nsplit = 1;
    const int64_t kchunks = (m + kGK - 1) / kGK;
    if (nsplit > kchunks) nsplit = kchunks;
    g.kper = ((kchunks + nsplit - 1) / nsplit) * kGK;
    g.nsplit = (m + g.kper - 1) / g.kper;
    return g;
}

size_t gauss_work_bytes(int64_t m, int64_t n, int64_t s) {
    const GaussGeom g = gauss_geom(m, n, s);
    return align256(sizeof(float) * (size_t)(g.nsplit * n * s));
}

cudaError_t launch_gauss_bf16x3(uint64_t seed, const float *A, int64_t m, int64_t n, int64_t lda, int64_t s,
                                float *partial, double *SA, int32_t *status, cudaStream_t st) {
    const GaussGeom g = gauss_geom(m, n, s);
    const size_t smem = (size_t)2 * (2 * kGStageG + 2 * (size_t)g.NP * kGK * 2);
    cudaError_t e = cudaFuncSetAttribute(gauss_bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)g.mtiles, (unsigned)g.nsplit);
    gauss_bf16x3_kernel<<<grid, kGThreads, smem, st>>>(A, m, n, lda, s, g.NP, g.kper, seed, partial, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    gauss_reduce_kernel<<<(unsigned)((n * s + 255) / 256), 256, 0, st>>>(partial, n, s, g.nsplit,
                                                                        1.0 / std::sqrt((double)s), SA);
    return cudaGetLastError();
}

}  // namespace ns
