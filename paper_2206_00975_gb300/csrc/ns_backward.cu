// ns_backward.cu -- adjoint of Algorithm 1 (ns_solve with the SRHT) for a
// loss L that depends on the returned W = V(:, n-k+1:n) only through W W^T.
//
// With M = SA^T SA = V Sigma^2 V^T (SA and R share V and Sigma), T the k
// trailing indices and N the others, perturbation theory of the eigenvectors
// of M gives
//   dL/dM  = sum_{i in T, j in N} c_ji (v_j v_i^T + v_i v_j^T),
//   c_ji   = (v_j . g_i) / (2 (sigma_i^2 - sigma_j^2)),   g_i = dL/dw_i,
// i.e. dL/dM = Y W^T + W Y^T with Y = V_N C (n x k);
//   dL/dSA = 2 SA dL/dM = 2 (SA Y) W^T + 2 (SA W) Y^T     (rank 2k);
//   dL/dA  = S^T dL/dSA = (1/sqrt s) D H R^T dL/dSA,
// truncated to the first m rows.  S^T is applied without storing anything of
// the forward transform: D and R are regenerated from the seed.
//
// The last step writes m x n FP64 and is HBM-write bound.  Each column of
// G = dL/dSA / sqrt(s) is mapped exactly to 64-bit fixed point (one scale per
// column, P = min(52, 62 - ceil(log2 s)) bits), so the scatter R^T, the signs
// of the Kronecker split H = H_{m'/4096} (x) H_4096 and the 4096-point
// transforms are exact integer arithmetic; the only roundings are that input
// quantisation and the final conversion to FP64 (done with integer
// instructions, round to nearest even).
#include <cmath>
#include "ns_device.cuh"
#include "ns_internal.h"

namespace ns {

size_t backward_work_bytes(int64_t m, int64_t n, int64_t s, int32_t k) {
    Carver c(nullptr);
    backward_carve(c, m, n, s, k);
    return c.used;
}

BackwardWork backward_carve(Carver &c, int64_t m, int64_t n, int64_t s, int32_t k) {
    const SrhtGeom g = srht_geom(m, n);
    BackwardWork w;
    w.sign_words = c.take<uint32_t>((size_t)g.sign_words);
    w.rows = c.take<int32_t>((size_t)s);
    w.rank = c.take<int32_t>((size_t)n);
    w.Y = c.take<double>((size_t)(n * k));
    w.P = c.take<double>((size_t)(s * 2 * k));
    w.q = c.take<long long>((size_t)(s * n));
    w.colexp = c.take<int32_t>((size_t)n);
    return w;
}

// rank of each singular value in non-increasing order (ties: lower index first)
__global__ void bw_rank_kernel(const double *__restrict__ sigma, int64_t n, int32_t *__restrict__ rank) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double si = sigma[i];
    int64_t r = 0;
    for (int64_t j = 0; j < n; ++j) {
        const double sj = sigma[j];
        r += (sj > si || (sj == si && j < i)) ? 1 : 0;
    }
    rank[i] = (int32_t)r;
}

// Y(:, i) = sum_{j in N} v_j c_ji, one CTA per returned column i: thread j
// forms c_ji = (v_j . g_i) / (2 (sigma_i^2 - sigma_j^2)) (zero for j in T), then
// thread r forms row r of Y.  Four partial sums break the FP64 dependency chains.
__global__ void __launch_bounds__(256) bw_y_kernel(const double *__restrict__ V, const double *__restrict__ sigma,
                                                   const int32_t *__restrict__ rank, const double *__restrict__ dVk,
                                                   int64_t n, int32_t k, double *__restrict__ Y) {
    extern __shared__ double sh[];   // g_i (n), then c (n)
    double *g = sh, *cj = sh + n;
    __shared__ double si_sh;
    const int64_t i = blockIdx.x;
    const int tid = threadIdx.x;
    for (int64_t r = tid; r < n; r += blockDim.x) {
        g[r] = dVk[r + i * n];
        if (rank[r] == (n - k) + i) si_sh = sigma[r];
    }
    __syncthreads();
    const double si = si_sh;
    for (int64_t j = tid; j < n; j += blockDim.x) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        const double *v = V + j * n;
        int64_t r = 0;
        for (; r + 4 <= n; r += 4) {
            a0 = fma(v[r], g[r], a0);
            a1 = fma(v[r + 1], g[r + 1], a1);
            a2 = fma(v[r + 2], g[r + 2], a2);
            a3 = fma(v[r + 3], g[r + 3], a3);
        }
        for (; r < n; ++r) a0 = fma(v[r], g[r], a0);
        const double dot = (a0 + a1) + (a2 + a3);
        const double sj = sigma[j];
        cj[j] = (rank[j] < n - k) ? 0.5 * dot / ((si - sj) * (si + sj)) : 0.0;
    }
    __syncthreads();
    for (int64_t r = tid; r < n; r += blockDim.x) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int64_t j = 0;
        for (; j + 4 <= n; j += 4) {
            a0 = fma(V[r + j * n], cj[j], a0);
            a1 = fma(V[r + (j + 1) * n], cj[j + 1], a1);
            a2 = fma(V[r + (j + 2) * n], cj[j + 2], a2);
            a3 = fma(V[r + (j + 3) * n], cj[j + 3], a3);
        }
        for (; j < n; ++j) a0 = fma(V[r + j * n], cj[j], a0);
        Y[r + i * n] = (a0 + a1) + (a2 + a3);
    }
}

// P(:, 0:k) = SA Y, P(:, k:2k) = SA W   (s x 2k), one thread per (row, column)
__global__ void bw_p_kernel(const double *__restrict__ SA, const double *__restrict__ Y,
                            const double *__restrict__ Vk, int64_t s, int64_t n, int32_t k, double *__restrict__ P) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= s * 2 * k) return;
    const int64_t t = idx % s, c = idx / s;
    const double *B = (c < k) ? (Y + c * n) : (Vk + (c - k) * n);
    double a = 0.0;
    for (int64_t j = 0; j < n; ++j) a = fma(SA[t + j * s], B[j], a);
    P[t + c * s] = a;
}

// G(:, col) = (2/sqrt s) (P_Y W^T + P_W Y^T)(:, col), quantised to 64-bit fixed
// point with one scale per column: q = round(G 2^F), |q| < 2^P.  One CTA per
// column; colexp[col] = F.
__global__ void __launch_bounds__(256) bw_quant_kernel(const double *__restrict__ P, const double *__restrict__ Y,
                                                       const double *__restrict__ Vk, int64_t s, int64_t n, int32_t k,
                                                       double scale, int Pbits, long long *__restrict__ q,
                                                       int32_t *__restrict__ colexp) {
    extern __shared__ double gcol[];  // s
    __shared__ int red[32];
    const int64_t col = blockIdx.x;
    const int tid = threadIdx.x;
    int emax = 0;
    for (int64_t t = tid; t < s; t += blockDim.x) {
        double a = 0.0;
        for (int32_t i = 0; i < k; ++i) {
            a = fma(P[t + i * s], Vk[col + i * n], a);
            a = fma(P[t + (k + i) * s], Y[col + i * n], a);
        }
        a *= scale;
        gcol[t] = a;
        emax = max(emax, (int)((unsigned long long)__double_as_longlong(a) >> 52) & 0x7FF);
    }
    emax = warp_max(emax);
    if ((tid & 31) == 0) red[tid >> 5] = emax;
    __syncthreads();
    int E = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) E = max(E, red[w]);
    if (E < 1) E = 1;
    // F = P + 1022 - E: |a| < 2^(E - 1022) maps below 2^P
    for (int64_t t = tid; t < s; t += blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(gcol[t]);
        const int e = (int)(b >> 52) & 0x7FF;
        const unsigned long long frac = b & 0x000FFFFFFFFFFFFFull;
        const unsigned long long mant = e ? (frac | 0x0010000000000000ull) : frac;
        const int sh = E - (e ? e : 1) + 53 - Pbits;
        unsigned long long v;
        if (sh >= 64) v = 0ull;
        else if (sh <= 0) v = mant << (-sh);
        else v = (mant + (1ull << (sh - 1))) >> sh;
        q[t + col * s] = (b >> 63) ? -(long long)v : (long long)v;
    }
    if (tid == 0) colexp[col] = Pbits + 1022 - E;
}

// exact int64 -> double of v * 2^(-F), round to nearest even, sign flipped if neg
__device__ __forceinline__ double fixed_to_double(long long v, int F, int neg) {
    if (v == 0) return 0.0;
    unsigned long long sgn = (v < 0) ? 1ull : 0ull;
    unsigned long long mag = (v < 0) ? (unsigned long long)(-v) : (unsigned long long)v;
    const int lz = __clzll(mag);
    const unsigned long long norm = mag << lz;      // top bit set
    unsigned long long m53 = norm >> 11;
    const unsigned long long rem = norm & 0x7FFull;
    int ex = 63 - lz - F;                            // unbiased exponent of the leading bit
    if (rem > 0x400ull || (rem == 0x400ull && (m53 & 1ull))) {
        ++m53;
        if (m53 == (1ull << 53)) {
            m53 >>= 1;
            ++ex;
        }
    }
    sgn ^= (unsigned long long)neg;
    const unsigned long long bits = (sgn << 63) | ((unsigned long long)(ex + 1023) << 52) | (m53 & 0x000FFFFFFFFFFFFFull);
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ int swz_b(int i) { return i ^ (((i >> 7) & 15) << 1); }

__device__ __forceinline__ void fwht64i(long long (&z)[64]) {
#pragma unroll
    for (int h = 1; h < 64; h <<= 1) {
#pragma unroll
        for (int kk = 0; kk < 64; ++kk) {
            if ((kk & h) == 0) {
                const long long a = z[kk], b = z[kk + h];
                z[kk] = a + b;
                z[kk + h] = a - b;
            }
        }
    }
}

// dA(:, col) rows of block b: scatter q_t (sign of hi(r_t) & b) to lo(r_t),
// 4096-point integer transform, D's signs, FP64 out.  64 threads, 64 values each.
__global__ void __launch_bounds__(64) bw_transform_kernel(const long long *__restrict__ q,
                                                          const int32_t *__restrict__ colexp,
                                                          const int32_t *__restrict__ rows,
                                                          const uint32_t *__restrict__ sign_words, int64_t m,
                                                          int64_t s, int64_t nblk, double *__restrict__ dA,
                                                          int64_t ldd) {
    __shared__ __align__(16) long long u[kBlock];
    __shared__ uint32_t sgn[128];
    const int t = threadIdx.x;
    const int64_t col = blockIdx.x / nblk, b = blockIdx.x % nblk;
    const int64_t base = b * kBlock;
    if (base >= m) return;
    for (int i = t; i < kBlock; i += 64) u[i] = 0;
    sgn[t] = sign_words[(base >> 5) + t];
    sgn[t + 64] = sign_words[(base >> 5) + 64 + t];
    __syncthreads();
    const long long *qc = q + col * s;
    for (int64_t i = t; i < s; i += 64) {
        const int r = rows[i];
        const long long v = qc[i];
        const int neg = __popcll((unsigned long long)(r >> kBlockLog) & (unsigned long long)b) & 1;
        atomicAdd((unsigned long long *)&u[swz_b(r & (kBlock - 1))], (unsigned long long)(neg ? -v : v));
    }
    __syncthreads();
    long long z[64];
    // layout 2: thread t, register k holds element (t & 1) | (k << 1) | ((t >> 1) << 7)
#pragma unroll
    for (int kk = 0; kk < 64; ++kk) z[kk] = u[swz_b((t & 1) | (kk << 1) | ((t >> 1) << 7))];
    fwht64i(z);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 64; ++kk) u[swz_b((t & 1) | (kk << 1) | ((t >> 1) << 7))] = z[kk];
    __syncthreads();
    // layout 1: thread t, register k holds element (k & 1) | (t << 1) | ((k >> 1) << 7)
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) {
        const longlong2 v = *(const longlong2 *)(u + swz_b(2 * t + 128 * kk));
        z[2 * kk] = v.x;
        z[2 * kk + 1] = v.y;
    }
    fwht64i(z);
    const int F = colexp[col];
    double *out = dA + col * ldd;
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) {
        const int64_t i0 = base + 2 * t + 128 * kk;
        const uint32_t sw = sgn[4 * kk + (t >> 4)] >> (2 * (t & 15));
        const double d0 = fixed_to_double(z[2 * kk], F, (int)(sw & 1u));
        const double d1 = fixed_to_double(z[2 * kk + 1], F, (int)((sw >> 1) & 1u));
        if (i0 + 1 < m && ((ldd & 1) == 0)) {
            __stcs((double2 *)(out + i0), make_double2(d0, d1));
        } else {
            if (i0 < m) out[i0] = d0;
            if (i0 + 1 < m) out[i0 + 1] = d1;
        }
    }
}

cudaError_t launch_backward(uint64_t seed, int64_t m, int64_t n, int32_t k, int64_t s, const double *save,
                            const double *Vk, const double *dVk, double *dA, int64_t ldd, const BackwardWork &w,
                            cudaStream_t st) {
    const SrhtGeom g = srht_geom(m, n);
    const double *SA = save, *V = save + s * n, *sigma = save + s * n + n * n;
    cudaError_t e = launch_srht_meta(seed, g.lg, g.sign_words, s, w.sign_words, w.rows, st);
    if (e != cudaSuccess) return e;
    bw_rank_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(sigma, n, w.rank);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t ysmem = sizeof(double) * (size_t)(2 * n);
    e = cudaFuncSetAttribute(bw_y_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ysmem);
    if (e != cudaSuccess) return e;
    bw_y_kernel<<<(unsigned)k, 256, ysmem, st>>>(V, sigma, w.rank, dVk, n, k, w.Y);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    bw_p_kernel<<<(unsigned)((s * 2 * k + 127) / 128), 128, 0, st>>>(SA, w.Y, Vk, s, n, k, w.P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int lgs = ceil_log2(s);
    int Pbits = 62 - lgs;
    if (Pbits > 52) Pbits = 52;
    const size_t qsmem = sizeof(double) * (size_t)s;
    e = cudaFuncSetAttribute(bw_quant_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsmem);
    if (e != cudaSuccess) return e;
    bw_quant_kernel<<<(unsigned)n, 256, qsmem, st>>>(w.P, w.Y, Vk, s, n, k, 2.0 / std::sqrt((double)s), Pbits, w.q,
                                                    w.colexp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t nblk = (m + kBlock - 1) / kBlock;
    bw_transform_kernel<<<(unsigned)(n * nblk), 64, 0, st>>>(w.q, w.colexp, w.rows, w.sign_words, m, s, nblk, dA,
                                                            ldd);
    return cudaGetLastError();
}

}  // namespace ns
