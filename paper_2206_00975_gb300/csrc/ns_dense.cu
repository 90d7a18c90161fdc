// ns_dense.cu -- Algorithm 1 lines 3-4 on the GPU in FP64: the SVD of SA
// (s x n) through Householder QR and a one-sided Jacobi SVD of the n x n
// triangular factor (SA and R share singular values and right singular
// vectors, proof of Theorem 3.2), then the k trailing right singular vectors.
//
// Preconditioned one-sided Jacobi (Drmac & Veselic, SIAM J. Matrix Anal.
// Appl. 29 (2008)):
//   1. SA P = Q1 R          Householder QR with column pivoting;
//   2. R^T  = Q2 R2         Householder QR of the transpose (no pivoting);
//   3. X = R2^T,  X Vx = U Sigma   one-sided Jacobi (Hestenes) on the columns;
//   4. V = P Q2 Vx          right singular vectors of SA.
// R = R2^T Q2^T, so SA P = Q1 X Q2^T and the right singular vectors of SA P are
// Q2 Vx; Vx comes from accumulated rotations and Q2 from reflectors, both
// orthogonal to working precision.  The pivoted, twice-factored X has nearly
// orthogonal graded columns, so the Jacobi iteration needs about a third of
// the sweeps it needs on R itself.
//
// FP64 runs at ~2 FMA/clock/SM on this part: the kernels spread the work over
// the whole GPU (cooperative launches, one CTA per SM, columns owned
// round-robin, a bounded grid barrier per Householder or Jacobi step) and keep
// scalar FP64 chains (norms, reflector and rotation parameters) to one thread.
//
// Jacobi rule: a pair (p, q) is rotated when gamma^2 > tol^2 alpha beta with
// alpha = |x_p|^2, beta = |x_q|^2, gamma = x_p . x_q, tol = n 2^-53; the
// rotation (zeta = (beta - alpha)/(2 gamma), t = sign(zeta)/(|zeta| +
// sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = c t) makes the pair orthogonal.
// t needs only modest accuracy (it sets the angle; an inexact angle leaves a
// small residual cosine for the next sweep), so it is formed in FP32 from
// power-of-two-scaled alpha, beta, gamma; c is then computed from that t to full
// FP64 accuracy (FP32 reciprocal-square-root seed and two Newton steps), so
// every applied rotation is orthogonal to working precision.  Pairs follow the
// round-robin (circle) ordering, n'/2 disjoint pairs per step, n'-1 steps per
// sweep.  The iteration stops when a sweep makes no rotation.  When a sweep
// made few rotations, the next one first runs a barrier-free check of all
// pairs on the current columns; if no pair needs a rotation the iteration has
// converged without a full barrier-separated sweep.  30 sweeps without
// convergence report NS_ERR_NOCONV.
#include <cmath>
#include "ns_device.cuh"
#include "ns_internal.h"

namespace ns {

constexpr int kDenseThreads = 256;
constexpr int kMaxSweeps = 30;
constexpr int kCheckBelow = 4096;        // run the barrier-free check after a sweep with fewer rotations
constexpr int kBarWords = 64 + 2 * 64 + 32;  // barrier word (padded), rotation counts, check flags, stats,
                                             // FP32-phase control (bar[196..212])
// words of bar from kJ32Ctl: 1 if the FP32 phase ran, its sweeps, its rotations,
// the completions' verdict (2: start the FP64 iteration with the convergence
// check), then 6 words per completion (see ns_jacobi32.cu)
constexpr int kJ32Ctl = 196;
static_assert(kJ32Ctl + 17 <= kBarWords, "FP32-phase control words");

size_t dense_work_bytes(int64_t s, int64_t n) {
    Carver c(nullptr);
    dense_carve(c, s, n);
    return c.used;
}

DenseWork dense_carve(Carver &c, int64_t s, int64_t n) {
    DenseWork w;
    w.W = c.take<double>((size_t)(s * n));
    w.tau = c.take<double>((size_t)(4 * n));   // per reflector: u0 and coefficient, both QRs
    w.X = c.take<double>((size_t)(n * n));
    w.V = c.take<double>((size_t)(n * n));
    w.sigma = c.take<double>((size_t)n);
    w.L = c.take<double>((size_t)(2 * n * n));
    w.R2 = c.take<double>((size_t)(2 * n * n));
    w.U = c.take<double>((size_t)(s * n));
    w.perm = c.take<int32_t>((size_t)n);
    w.pivslot = c.take<unsigned long long>((size_t)n + 1);
    w.bar = c.take<unsigned int>(kBarWords);
    w.colver = c.take<unsigned int>((size_t)n + 32);
    return w;
}

// |x| as an ordered integer key (the bit pattern of a non-negative double
// orders like the value); integer max keeps the FP64 pipe free.
__device__ __forceinline__ long long abs_key(double x) { return __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll; }

// 2^-e with e the exponent of the largest |x| over the block: multiplying by it
// is exact and brings the largest entry into [1, 2).  Returns the scale in every
// thread (0 if all entries are zero).
__device__ double block_pow2_scale(long long key, long long *redk) {
    key = warp_max(key);
    if ((threadIdx.x & 31) == 0) redk[threadIdx.x >> 5] = key;
    __syncthreads();
    long long k = redk[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) k = max(k, redk[w]);
    __syncthreads();
    if (k == 0) return 0.0;
    const int e = (int)((unsigned long long)k >> 52);  // biased exponent of max |x|
    int se = 2046 - e;                                  // 2^(1023 - e), biased
    if (se < 1) se = 1;
    if (se > 2045) se = 2045;                           // keeps 1/scale representable
    return __longlong_as_double((long long)se << 52);
}

// ------------------------------------------------------------------- QR ----
// Cooperative Householder QR of W (rows x cols, ld = rows) with optional
// column pivoting.  Logical column j is physical column perm[j].  With x the
// pivot column's rows j..rows-1, beta = -sign(x_0) |x| and u = [x_0 - beta;
// x_1; ...], reflector j is H = I - coef u u^T with coef = 1/(beta (beta - x_0))
// (= 2/|u|^2).  The rows below the diagonal keep x itself (u below the first
// entry); u0[j] = x_0 - beta and cf[j] = coef are kept aside and W[j, perm[j]]
// receives beta = R[j, j].  Each step needs one square root and one
// reciprocal, and one block reduction that also yields u . y for the CTA's
// owned columns.  The R factor (logical column order) is written to Rout.
// Every CTA forms reflector j from the final pivot column, so a step needs a
// single grid barrier.
template <int NB>
__global__ void __launch_bounds__(kDenseThreads) hqr_coop_kernel(double *W, int64_t rows, int64_t cols, int pivot,
                                                                double *u0, double *cf, int32_t *perm,
                                                                unsigned long long *pivslot, double *Rout,
                                                                GridBarrier bar) {
    extern __shared__ double sh[];
    double *vsh = sh;                                   // rows
    double *nrm = sh + rows;                            // owned columns: current |.|^2 (-1: done)
    double *nref = nrm + (cols + gridDim.x - 1) / gridDim.x;  // value at the last recomputation
    __shared__ double red[32 * (NB + 1)];
    __shared__ long long redk[32];
    __shared__ double par[3];                           // coef, beta, u0
    __shared__ double fsh[NB];
    const int64_t G = gridDim.x, me = blockIdx.x;
    const int tid = threadIdx.x;
    const int64_t nown = (cols - me + G - 1) / G;       // owned physical columns me, me+G, ...
    const int64_t steps = rows < cols ? rows : cols;

    auto key_of = [&](double n2, int64_t l) -> unsigned long long {
        return ((unsigned long long)__double_as_longlong(n2) & ~0x1FFFull) | (unsigned long long)(8191 - l);
    };
    if (pivot) {  // initial squared norms of the owned columns, first pivot candidate
        unsigned long long best = 0;
        for (int64_t o = 0; o < nown; ++o) {
            const int64_t l = me + o * G;
            double v[1] = {0.0};
            for (int64_t i = tid; i < rows; i += blockDim.x) v[0] = fma(W[i + l * rows], W[i + l * rows], v[0]);
            block_sum_t0<1>(v, red);
            if (tid == 0) {
                nrm[o] = v[0];
                nref[o] = v[0];
                const unsigned long long kk = key_of(v[0], l);
                best = kk > best ? kk : best;
            }
            __syncthreads();
        }
        if (tid == 0 && nown > 0) atomicMax(pivslot, best);
    }
    for (int64_t j = 0; j < steps; ++j) {
        if (!grid_sync(bar)) return;
        const int64_t p = pivot ? 8191 - (int64_t)(__ldcg(pivslot + j) & 0x1FFFull) : j;
        const int64_t len = rows - j;
        const double *xp = W + j + p * rows;
        long long key = 0;
        for (int64_t i = tid; i < len; i += blockDim.x) {
            const double a = __ldcg(xp + i);
            vsh[i] = a;
            key = max(key, abs_key(a));
        }
        if (pivot && p % G == me && tid == 0) nrm[(p - me) / G] = -1.0;  // the pivot column is done
        const double sc = block_pow2_scale(key, redk);  // includes __syncthreads
        const double isc = (sc == 0.0) ? 0.0 : __longlong_as_double((2046ll << 52) - __double_as_longlong(sc));
        const double alpha = vsh[0];
        for (int64_t o0 = 0; o0 < nown || o0 == 0; o0 += NB) {
            int64_t cl[NB];
            int nb = 0;
            for (int64_t o = o0; o < nown && nb < NB; ++o, ++nb) {
                const int64_t l = me + o * G;
                cl[nb] = (pivot ? (nrm[o] >= 0.0) : (l > j)) ? l : -1;
            }
            double acc[NB + 1];
#pragma unroll
            for (int b = 0; b <= NB; ++b) acc[b] = 0.0;
            for (int64_t i = 1 + tid; i < len; i += blockDim.x) {
                const double a = vsh[i];
                if (o0 == 0) {
                    const double as = a * sc;
                    acc[0] = fma(as, as, acc[0]);
                }
#pragma unroll
                for (int b = 0; b < NB; ++b)
                    if (b < nb && cl[b] >= 0) acc[b + 1] = fma(a, W[j + i + cl[b] * rows], acc[b + 1]);
            }
            block_sum_t0<NB + 1>(acc, red);
            if (tid == 0) {
                if (o0 == 0) {
                    if (sc == 0.0 || acc[0] == 0.0) {
                        par[0] = 0.0;  // x[1:] = 0: H = I, R[j, j] = x_0
                        par[1] = alpha;
                        par[2] = 0.0;
                    } else {
                        const double as = alpha * sc;
                        const double r = sqrt(fma(as, as, acc[0])) * isc;  // |x|
                        const double beta = alpha >= 0.0 ? -r : r;
                        par[0] = 1.0 / (beta * (beta - alpha));
                        par[1] = beta;
                        par[2] = alpha - beta;
                    }
                }
                for (int b = 0; b < nb; ++b) {
                    if (cl[b] < 0) continue;
                    const double y0 = W[j + cl[b] * rows];
                    fsh[b] = par[0] * fma(par[2], y0, acc[b + 1]);   // coef * (u . y)
                }
            }
            __syncthreads();
            const double coef = par[0], ua = par[2];
            if (coef != 0.0) {
                for (int b = 0; b < nb; ++b) {
                    if (cl[b] < 0) continue;
                    double *y = W + j + cl[b] * rows;
                    const double f = fsh[b];
                    for (int64_t i = tid; i < len; i += blockDim.x) y[i] = fma(-f, i == 0 ? ua : vsh[i], y[i]);
                }
            }
            __syncthreads();
            if (o0 + NB >= nown) break;
        }
        if (p % G == me && tid == 0) {  // owner: R's diagonal entry, reflector scalars, permutation
            W[j + p * rows] = par[1];
            cf[j] = par[0];
            u0[j] = par[2];
            perm[j] = (int32_t)p;
        }
        if (pivot) {  // downdate the owned norms; next pivot candidate
            unsigned long long best = 0;
            for (int64_t o = 0; o < nown; ++o) {
                const int64_t l = me + o * G;
                __syncthreads();
                const bool skip = nrm[o] < 0.0;
                __syncthreads();
                if (skip) continue;
                const double *y = W + j + l * rows;
                if (tid == 0) {
                    const double r = y[0];
                    const double n2 = nrm[o] - r * r;
                    nrm[o] = (n2 > 1e-8 * nref[o]) ? n2 : -2.0;  // -2: recompute below
                }
                __syncthreads();
                if (nrm[o] == -2.0) {
                    double v[1] = {0.0};
                    for (int64_t i = 1 + tid; i < len; i += blockDim.x) v[0] = fma(y[i], y[i], v[0]);
                    block_sum_t0<1>(v, red);
                    if (tid == 0) {
                        nrm[o] = v[0];
                        nref[o] = v[0];
                    }
                    __syncthreads();
                }
                if (tid == 0) {
                    const unsigned long long kk = key_of(nrm[o], l);
                    best = kk > best ? kk : best;
                }
            }
            if (tid == 0 && best) atomicMax(pivslot + j + 1, best);
        }
    }
    if (!grid_sync(bar)) return;
    for (int64_t j = me; j < steps; j += G) {  // R in logical column order
        const int64_t pj = __ldcg(perm + j);
        for (int64_t i = tid; i < cols; i += blockDim.x)
            Rout[i + j * cols] = (i <= j) ? __ldcg(W + i + pj * rows) : 0.0;
    }
}

// FP32 image of x * 2^-shift from the IEEE fields (integer work, mantissa
// truncated; zero, subnormal and below-range values give 0).
__device__ __forceinline__ float f32_image(double x, int shift) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF), fe = e - shift - 1023 + 127;
    if (e == 0 || fe <= 0) return 0.0f;
    const unsigned int f = ((unsigned int)(b >> 32) & 0x80000000u) | ((unsigned int)min(fe, 254) << 23) |
                           (unsigned int)((b >> 29) & 0x7FFFFFu);
    return __uint_as_float(f);
}
// exact FP64 value of a normal or zero FP32 number (integer work)
__device__ __forceinline__ double f64_of(float f) {
    const unsigned int u = __float_as_uint(f);
    const unsigned int e = (u >> 23) & 0xFF;
    if (e == 0) return 0.0;
    const unsigned long long b = ((unsigned long long)(u >> 31) << 63) |
                                 ((unsigned long long)(e - 127 + 1023) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
}

// biased exponent field of an IEEE double
__device__ __forceinline__ uint32_t exp_field(double x) {
    return (uint32_t)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFu;
}

// ------------------------------------------------------- pipelined QR ----
// Householder QR without pivoting, pipelined instead of barrier-separated.
// CTA me owns columns me, me + G, ... and keeps them in shared memory.
// Reflector j (same form and storage as hqr_coop_kernel: tail in W below the
// diagonal, u0[j], cf[j], R[j, j] = beta) is formed by the owner of column j
// as soon as reflectors 0..j-1 have reached that column, written to global
// memory and announced by flag[j], which carries the coefficient itself (the
// bits of cf[j]; all ones = not yet formed).  The reflectors go to U (same
// layout as W: tail below the diagonal, u0[j] on it, |u[j+1:]|^2 in the slot
// above it), which starts filled with all-ones words: the owner of column
// j + 1, the only consumer on the critical path, polls its rows of U[:, j]
// directly instead of the flag and then the data; every other CTA takes the
// flag (acquire) and then reads U.  The owner of column j + 1 applies
// reflector j to that column before its other columns (look-ahead), so the
// chain from one reflector to the next runs through one CTA and one flag;
// every other CTA only waits for the flags of the reflectors it applies.
constexpr int kPipeThreads = 256;

constexpr unsigned long long kPipeEmpty = ~0ull;  // flag and U words of a reflector not formed yet

// publish one FP64 word of a reflector (never the all-ones pattern)
__device__ __forceinline__ void st_pub(double *p, double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    if (b == kPipeEmpty) b = 0x7FF8000000000000ull;
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(b) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const double *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_flag(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Sum over the CTA, result in every thread (fixed order).  The tree adds only
// in the lanes whose sums survive: FP64 issue is scarce, idle lanes are not.
__device__ __forceinline__ double lane0_sum(double v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_down_sync(0xffffffffu, v, o);
        if (lane < o) v += w;
    }
    return v;  // valid in lane 0
}
__device__ __forceinline__ double pipe_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = lane0_sum(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double a = lane < kPipeThreads / 32 ? red[lane] : 0.0;
#pragma unroll
        for (int o = kPipeThreads / 64; o > 0; o >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, a, o);
            if (lane < o) a += w;
        }
        if (lane == 0) red[2 * (kPipeThreads / 32)] = a;
    }
    __syncthreads();
    return red[2 * (kPipeThreads / 32)];
}

// Sums of two values over the CTA (fixed order), valid in thread 0 only.
// Lanes 0-15 carry a and lanes 16-31 b after the first exchange, so every
// warp level costs one FP64 add for both; red needs 2 * warps entries.
__device__ __forceinline__ void pipe_sum2_t0(double &a, double &b, double *red) {
    constexpr int kW = kPipeThreads / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool hi = lane >= 16;
    double v = (hi ? b : a) + __shfl_xor_sync(0xffffffffu, hi ? a : b, 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        const double w = __shfl_down_sync(0xffffffffu, v, o);
        if ((lane & 15) < o) v += w;
    }
    if ((lane & 15) == 0) red[(hi ? kW : 0) + wid] = v;
    __syncthreads();
    if (wid == 0) {
        double x = (lane & 15) < kW ? red[(lane >= 16 ? kW : 0) + (lane & 15)] : 0.0;
#pragma unroll
        for (int o = kW / 2; o > 0; o >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, x, o);
            if ((lane & 15) < o) x += w;
        }
        const double bb = __shfl_sync(0xffffffffu, x, 16);
        if (lane == 0) {
            a = x;
            b = bb;
        }
    }
}

// x 2^k for a positive normal x and a normal result (integer work)
__device__ __forceinline__ double exp_shift(double x, int k) {
    return __longlong_as_double(__double_as_longlong(x) + ((long long)k << 52));
}

// Reflector parameters for head x0 and tail norm^2 nrm2 > 0 when
// t = x0^2 + nrm2 needs no rescaling: r = sqrt(t), beta = -sign(x0) r,
// ua = x0 - beta and coef = 1 / (beta (beta - x0)) = 1 / (r (r + |x0|)).
// FP64 square root and division are long serial chains on this part, so r and
// coef come from FP32 seeds (exponent-shifted images) refined by one
// third-order step of the binomial series each: y <- y (1 + e/2 + 3e^2/8),
// e = 1 - t y^2, for t^(-1/2), and z <- z (1 + e + e^2), e = 1 - s z, for
// 1/s.  The seeds' relative error (< 2^-21) becomes < 2^-60.  Returns false
// (nothing written) when t is not a normal number.
__device__ __forceinline__ bool pipe_reflector(double x0, double nrm2, double *beta, double *ua, double *coef) {
    const double t = fma(x0, x0, nrm2);
    const uint32_t eb = exp_field(t);
    if (eb < 64 || eb > 2046 - 64) return false;
    const int sh = ((int)eb - 1023) & ~1;  // even: the image of t lies in [1, 4)
    double y = exp_shift(f64_of(rsqrtf(f32_image(t, sh))), -(sh / 2));
    const double ty = t * y, e = fma(-ty, y, 1.0);
    y = fma(y, e * fma(e, 0.375, 0.5), y);
    const double r = t * y, sv = r + fabs(x0);
    const int es = (int)exp_field(sv) - 1023;
    double z = exp_shift(f64_of(__frcp_rn(f32_image(sv, es))), -es);
    const double e2 = fma(-sv, z, 1.0);
    z = fma(z, fma(e2, e2, e2), z);
    *beta = x0 >= 0.0 ? -r : r;
    *ua = x0 - *beta;
    *coef = y * z;  // y = 1/r to within a few units of the last place
    return true;
}

// Form reflector j from the owned column x (shared memory, rows entries):
// publishes the tail, u0, cf and the flag; leaves u (u0 at index j) in ush,
// the coefficient in *coef_sh and returns beta (every thread).  The scalar
// chain (square root, reciprocal) runs in thread 0 only: FP64 is scarce.
// The tail norm^2 |u[j+1:]|^2 goes to *unrm_sh and, for j >= 1, to the slot
// U[j-1, j] for the consumers (NaN when the column was rescaled).
__device__ double pipe_form(double *U, int64_t rows, int64_t j, const double *x, double *ush, double *u0, double *cf,
                            unsigned long long *flag, double *red, double *coef_sh, double *unrm_sh) {
    __shared__ double s_par[2];
    const int tid = threadIdx.x;
    double ss = 0.0;
    for (int64_t i = j + 1 + tid; i < rows; i += kPipeThreads) ss = fma(x[i], x[i], ss);
    double nrm2 = pipe_sum(ss, red);
    double sc = 1.0;
    if (nrm2 != 0.0 && (nrm2 < 1e-280 || nrm2 > 1e280)) {
        // rescale by a power of two from the largest entry (rare)
        long long key = 0;
        for (int64_t i = j + tid; i < rows; i += kPipeThreads) key = max(key, abs_key(x[i]));
        __shared__ long long redk[32];
        sc = block_pow2_scale(key, redk);
        ss = 0.0;
        for (int64_t i = j + 1 + tid; i < rows; i += kPipeThreads) {
            const double a = x[i] * sc;
            ss = fma(a, a, ss);
        }
        nrm2 = pipe_sum(ss, red);
    }
    for (int64_t i = j + 1 + tid; i < rows; i += kPipeThreads) {
        const double v = x[i];
        ush[i] = v;
        st_pub(U + i + j * rows, v);
    }
    if (tid == 0) {
        const double x0 = x[j];
        double beta, ua, coef;
        if (nrm2 == 0.0) {  // H = I
            beta = x0;
            ua = 0.0;
            coef = 0.0;
        } else if (sc != 1.0 || !pipe_reflector(x0, nrm2, &beta, &ua, &coef)) {
            const double xs = x0 * sc;
            double r = sqrt(fma(xs, xs, nrm2));
            if (sc != 1.0) r /= sc;  // rescaled column (rare): an exact power of two
            beta = x0 >= 0.0 ? -r : r;
            ua = x0 - beta;
            coef = 1.0 / (beta * (beta - x0));
        }
        const double tn = (sc == 1.0) ? nrm2 : __longlong_as_double(0x7FF8000000000000ll);
        *unrm_sh = tn;
        if (j >= 1) st_pub(U + j - 1 + j * rows, tn);
        ush[j] = ua;
        u0[j] = ua;
        st_pub(U + j + j * rows, ua);
        cf[j] = coef;
        *coef_sh = coef;
        s_par[0] = beta;
    }
    __syncthreads();  // orders every thread's stores before thread 0's release
    if (tid == 0) {
        unsigned long long fw = (unsigned long long)__double_as_longlong(*coef_sh);
        if (fw == kPipeEmpty) fw = 0x7FF8000000000000ull;  // a NaN coefficient keeps a NaN flag word
        asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(flag + j), "l"(fw) : "memory");
    }
    return s_par[0];
}

// The owner of the next column polls its rows i0, i0 + kPipeThreads, ... of a
// published reflector (Ucol = U[:, j]) into ush: four loads in flight at a
// time, then the ones still empty polled again (one L2 round trip per group
// of four instead of one per row).  Returns true if a wait ran out.
__device__ __forceinline__ bool pipe_poll_rows(const double *Ucol, int64_t i0, int64_t rows, double *ush, long long t0) {
    for (int64_t base = i0; base < rows; base += 4 * kPipeThreads) {
        unsigned long long b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t i = base + q * kPipeThreads;
            b[q] = i < rows ? ld_relaxed_u64(Ucol + i) : 0ull;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t i = base + q * kPipeThreads;
            if (i >= rows) continue;
            while (b[q] == kPipeEmpty) {
                if (clock64() - t0 > (1ll << 32)) return true;  // ~2 s; a healthy pipeline waits microseconds
                b[q] = ld_relaxed_u64(Ucol + i);
            }
            ush[i] = __longlong_as_double((long long)b[q]);
        }
    }
    return false;
}

// y <- H_j y on rows j.. (u in ush, coefficient coef)
__device__ __forceinline__ void pipe_apply(int64_t rows, int64_t j, const double *ush, double coef, double *y,
                                           double *red) {
    const int tid = threadIdx.x;
    double d = 0.0;
    for (int64_t i = j + tid; i < rows; i += kPipeThreads) d = fma(ush[i], y[i], d);
    const double f = coef * pipe_sum(d, red);
    for (int64_t i = j + tid; i < rows; i += kPipeThreads) y[i] = fma(-f, ush[i], y[i]);
    __syncthreads();
}

// The owner of column j + 1 (j >= 1): y <- H_j y, then reflector j + 1 from
// the updated column, with one CTA reduction for both.  The tail norm of the
// updated column follows from sums over the old one (norm downdating):
//   |y'_T|^2 = S_yy - 2 f S_uy + f^2 S_uu,   f = coef (u . y),   T = rows j+2..,
// with S_uu = |u[j+1:]|^2 - u_{j+1}^2 (published with reflector j) and
// S_uy = u . y - u_j y_j - u_{j+1} y_{j+1}.  Where the result is below 1/16 of
// the magnitudes it was formed from (the rounding of the cancellations is
// bounded by u times those) or the norm would need rescaling, the norm is
// recomputed from the updated column (pipe_form).
//
// Reflector j's head u_j and its scalars come out of its producer's scalar
// chain, after the tail rows u[j+1:] are already published.  So the sums
// run over the tail first (u . y without its head term, S_yy), and only then
// does thread 0 wait for flag j (acquire; the coefficient), read u_j and the
// tail-norm slot U[j-1, j], and add u_j y_j: the CTA reduction overlaps the
// producer's chain instead of following it.  ush[j] and *coef_now receive
// u_j and the coefficient for the caller.  A wait that runs out sets status
// and *ok_sh = 0 (every thread returns 0.0 then).
__device__ double pipe_apply_form(double *U, int64_t rows, int64_t j, double *ush, double *y, double *ushn,
                                  double *u0, double *cf, unsigned long long *flag, double *red, double *coef_sh,
                                  double *unrm_sh, double *coef_now, int *ok_sh, int32_t *status) {
    __shared__ double s_f, s_beta;
    __shared__ int s_redo;
    const int tid = threadIdx.x;
    const int64_t jn = j + 1;
    double d = 0.0, syy = 0.0;
    for (int64_t i = jn + tid; i < rows; i += kPipeThreads) {
        const double yi = y[i];
        d = fma(ush[i], yi, d);
        if (i > jn) syy = fma(yi, yi, syy);
    }
    double yj = 0.0, yn = 0.0, uj = 0.0, un = 0.0, coef = 0.0, unrm2 = 0.0;  // head entries, before the update
    if (tid == 0) {
        yj = y[j];
        yn = y[jn];
        un = ush[jn];
    }
    pipe_sum2_t0(d, syy, red);
    if (tid == 0) {
        const long long t0 = clock64();
        unsigned long long fw;
        bool late = false;
        while ((fw = ld_acquire_flag(flag + j)) == kPipeEmpty)
            if (clock64() - t0 > (1ll << 32)) {  // ~2 s; a healthy pipeline waits microseconds
                late = true;
                break;
            }
        if (late) {
            set_status(status, NS_ERR_TIMEOUT);
            *ok_sh = 0;
        } else {
            coef = __longlong_as_double((long long)fw);
            uj = __longlong_as_double((long long)ld_relaxed_u64(U + j + j * rows));  // written before the flag
            unrm2 = __longlong_as_double((long long)ld_relaxed_u64(U + j - 1 + j * rows));
            ush[j] = uj;
            *coef_now = coef;
            d = fma(uj, yj, d);
        }
        s_f = coef * d;
    }
    __syncthreads();
    if (!*ok_sh) return 0.0;
    const double f = s_f;
    for (int64_t i = j + tid; i < rows; i += kPipeThreads) {
        const double v = fma(-f, ush[i], y[i]);
        y[i] = v;
        if (i > jn) {
            ushn[i] = v;
            st_pub(U + i + jn * rows, v);
        }
    }
    if (tid == 0) {
        const double x0 = fma(-f, un, yn);  // y'_{j+1}, as the update computes it
        const double p1 = uj * yj, p2 = un * yn, u2 = un * un;
        const double suy = (d - p1) - p2, suu = unrm2 - u2;
        // With no rows below j + 1 the tail norm is exactly 0 (H = I).  Otherwise
        // S_uy and S_uu come from cancellations whose rounding is bounded by u
        // times the magnitudes they were formed from, so those set the guard.
        const bool notail = jn + 1 >= rows;
        const double n2 = notail ? 0.0 : fma(f, fma(f, suu, -2.0 * suy), syy);
        const double af = fabs(f);
        const double mag = syy + af * fma(af, unrm2 + u2, 2.0 * (fabs(d) + fabs(p1) + fabs(p2)));
        bool ok = notail || (n2 >= 0.0625 * mag && mag <= 1e280 && (n2 == 0.0 || n2 >= 1e-280));
        double beta = x0, ua = 0.0, cfn = 0.0;  // n2 == 0: H = I
        if (ok && n2 != 0.0) ok = pipe_reflector(x0, n2, &beta, &ua, &cfn);
        if (ok) {
            ushn[jn] = ua;
            u0[jn] = ua;
            st_pub(U + jn + jn * rows, ua);
            st_pub(U + j + jn * rows, n2);  // the tail-norm slot of reflector j + 1
            cf[jn] = cfn;
            *coef_sh = cfn;
            *unrm_sh = n2;
            s_beta = beta;
        }
        s_redo = ok ? 0 : 1;
    }
    __syncthreads();  // the update, the tail and the parameters are in place
    if (s_redo) return pipe_form(U, rows, jn, y, ushn, u0, cf, flag, red, coef_sh, unrm_sh);
    if (tid == 0) {
        unsigned long long fw = (unsigned long long)__double_as_longlong(*coef_sh);
        if (fw == kPipeEmpty) fw = 0x7FF8000000000000ull;
        asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(flag + jn), "l"(fw) : "memory");
    }
    return s_beta;
}

__device__ __forceinline__ void red_release_add(unsigned int *p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One CTA's part of the pipelined QR: CTA `me` of a group of G CTAs.  With Lg
// non-null (the fused two-QR kernel) it also publishes each finished entry of
// R as an entry of L = R^T (Lg, column-major, leading dimension ldl: column j
// of L is row j of R) and adds the number it published for row j to rowcnt[j]
// (release): row j is complete when rowcnt[j] = cols - j.
__device__ void pipe_qr_cta(const double *W, double *U, int64_t rows, int64_t cols, int64_t nown_max, double *u0,
                            double *cf, unsigned long long *flag, double *Rout, int32_t *status, int me, int G,
                            double *Lg, int64_t ldl, unsigned int *rowcnt) {
    extern __shared__ double sm[];
    double *own = sm;                          // nown_max * rows: owned columns
    double *ubuf = sm + nown_max * rows;       // 2 * rows: reflectors j (even/odd)
    double *beta = ubuf + 2 * rows;            // nown_max: R's diagonal of owned columns
    __shared__ double red[2 * (kPipeThreads / 32) + 1];
    __shared__ double s_coef[2], s_unrm[2];  // coefficient and tail norm^2 of reflectors j (by parity)
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    const int64_t nown = (cols - me + G - 1) / G;
    const int64_t steps = rows < cols ? rows : cols;
    for (int64_t o = 0; o < nown; ++o)
        for (int64_t i = tid; i < rows; i += kPipeThreads) own[o * rows + i] = W[i + (me + o * G) * rows];
    if (tid == 0) s_ok = 1;
    __syncthreads();
    if (me == 0 && steps > 0) {
        const double b0 = pipe_form(U, rows, 0, own, ubuf, u0, cf, flag, red, &s_coef[0], &s_unrm[0]);
        if (tid == 0) beta[0] = b0;
        if (Lg && tid == 0) {
            Lg[0] = b0;  // R[0, 0]
            red_release_add(rowcnt, 1u);
        }
        __syncthreads();
    }
    int jm = 0;                                // j mod G: the CTA that formed reflector j
    int64_t o_first = (me > 0) ? 0 : 1;        // first owned column (index into own) after column j
    for (int64_t j = 0; j < steps; ++j) {
        double *ush = ubuf + (j & 1) * rows;
        const int jn_owner = (jm + 1 == G) ? 0 : jm + 1;
        const bool mine = (j + 1 < steps) && jn_owner == me;  // this CTA forms reflector j + 1
        if (jm != me) {
            const long long t0 = clock64();
            if (mine) {  // poll this thread's rows of U[:, j] (and the scalars) directly
                bool late = false;
                // from j = 1 on only the tail: pipe_apply_form takes the head and
                // the scalars once its sums over the tail are done
                late = pipe_poll_rows(U + j * rows, (j >= 1 ? j + 1 : j) + tid, rows, ush, t0);
                if (tid == 0 && !late && j == 0) {
                    unsigned long long fw, nw = 0;
                    while ((fw = ld_acquire_flag(flag + j)) == kPipeEmpty)
                        if (clock64() - t0 > (1ll << 32)) {
                            late = true;
                            break;
                        }
                    while (!late && j >= 1 && (nw = ld_relaxed_u64(U + j - 1 + j * rows)) == kPipeEmpty)
                        if (clock64() - t0 > (1ll << 32)) late = true;
                    s_coef[j & 1] = __longlong_as_double((long long)fw);
                    s_unrm[j & 1] = __longlong_as_double((long long)nw);
                }
                if (late) {
                    set_status(status, NS_ERR_TIMEOUT);
                    s_ok = 0;
                }
                __syncthreads();
                if (!s_ok) return;
            } else {  // wait for flag j (acquire), then read U[:, j]
                if (tid == 0) {
                    unsigned long long fw;
                    while ((fw = ld_acquire_flag(flag + j)) == kPipeEmpty) {
                        if (clock64() - t0 > (1ll << 32)) {
                            set_status(status, NS_ERR_TIMEOUT);
                            s_ok = 0;
                            break;
                        }
                    }
                    s_coef[j & 1] = __longlong_as_double((long long)fw);
                }
                __syncthreads();
                if (!s_ok) return;
                for (int64_t i = j + tid; i < rows; i += kPipeThreads) ush[i] = __ldcg(U + i + j * rows);
                __syncthreads();
            }
        }
        double coef = s_coef[j & 1];  // (the owner of column j + 1 learns it in pipe_apply_form)
        // the owner of column j + 1 takes it first and forms reflector j + 1
        // right away (look-ahead), then applies reflector j to its other columns
        if (mine) {
            double *y = own + o_first * rows;
            double *ushn = ubuf + ((j + 1) & 1) * rows;
            double bj;
            if (j >= 1) {
                bj = pipe_apply_form(U, rows, j, ush, y, ushn, u0, cf, flag, red, &s_coef[(j + 1) & 1],
                                     &s_unrm[(j + 1) & 1], &s_coef[j & 1], &s_ok, status);
                if (!s_ok) return;
            } else {
                if (coef != 0.0) pipe_apply(rows, j, ush, coef, y, red);
                bj = pipe_form(U, rows, j + 1, y, ushn, u0, cf, flag, red, &s_coef[(j + 1) & 1],
                               &s_unrm[(j + 1) & 1]);
            }
            if (tid == 0) beta[o_first] = bj;
            if (Lg && tid == 0) {
                Lg[(j + 1) + (j + 1) * ldl] = bj;  // R[j + 1, j + 1]
                red_release_add(rowcnt + j + 1, 1u);
            }
        }
        coef = s_coef[j & 1];
        if (coef != 0.0)
            for (int64_t o = o_first + (mine ? 1 : 0); o < nown; ++o) pipe_apply(rows, j, ush, coef, own + o * rows, red);
        if (jn_owner == me) ++o_first;
        __syncthreads();
        if (Lg && tid == 0) {  // row j of R is final in every owned column past j
            unsigned int cnt = 0;
            for (int64_t o = 0; o < nown; ++o) {
                const int64_t c = me + o * G;
                if (c > j) {
                    Lg[c + j * ldl] = own[o * rows + j];
                    ++cnt;
                }
            }
            if (cnt) red_release_add(rowcnt + j, cnt);
        }
        if (++jm == G) jm = 0;
    }
    // R: rows 0..steps-1 of every column (column order as stored in W),
    // leading dimension steps; for cols > rows the columns past the last
    // reflector come out as Q^T times their input
    if (!Rout) return;
    for (int64_t o = 0; o < nown; ++o) {
        const int64_t c = me + o * G;
        for (int64_t i = tid; i < steps; i += kPipeThreads) {
            double r = 0.0;
            if (i < c) r = own[o * rows + i];
            else if (i == c) r = beta[o];
            Rout[i + c * steps] = r;
        }
    }
}

__global__ void __launch_bounds__(kPipeThreads) hqr_pipe_kernel(const double *W, double *U, int64_t rows,
                                                               int64_t cols, int64_t nown_max, double *u0, double *cf,
                                                               unsigned long long *flag, double *Rout,
                                                               int32_t *status) {
    pipe_qr_cta(W, U, rows, cols, nown_max, u0, cf, flag, Rout, status, (int)blockIdx.x, (int)gridDim.x, nullptr, 0,
                nullptr);
}

// ------------------------------------------------- fused two-QR pipeline ----
// The second QR (of L = [R^T | I], n x 2n) needs column c of L, row c of R,
// which is final once the first QR has applied reflector c to every column.
// In one cooperative launch CTAs [0, G1) run the first QR's pipeline and
// publish each row of R as it becomes final (pipe_qr_cta with Lg); CTAs
// [G1, G) run the second QR's pipeline on L.  They hold the identity columns
// from the start and load each column of R^T when its row of R is complete,
// then bring it up to date with the second QR's reflectors published so far
// (one warp per column, the reflectors read from U through registers).  The
// second QR then trails the first by the catch-up of its newest column
// instead of starting after it.  The arithmetic of each reflector and of its
// application is that of pipe_form / pipe_apply_form / pipe_apply, so R2 and
// Q2 equal those of the two separate launches up to the order of the sums in
// the catch-up and in the warp-level applications.
constexpr int kQ2MaxOwn = 32;  // owned columns per second-QR CTA
constexpr int kQ2Lane = 8;     // rows per lane in a warp-level application (n <= 256 = 4 blocks of 64)

// The inner product u . y of a second-QR reflector with a column (n <= 256)
// in one fixed order, whichever path applies it: lane l forms
// q_b = u[64b+32+l] y[64b+32+l] + u[64b+l] y[64b+l] (one FMA after a product)
// for the four blocks b, adds (q_0 + q_1) + (q_2 + q_3), and the warp sums the
// lanes with the butterfly of warp_sum.  So a column gets the same bits
// whether a reflector reaches it in the step loop or in a catch-up.
__device__ __forceinline__ double q2_block_term(const double *u, const double *y, int64_t rows, int64_t k, int b) {
    const int lane = threadIdx.x & 31;
    const int64_t i0 = 64 * b + lane, i1 = i0 + 32;
    const bool a0 = i0 >= k && i0 < rows, a1 = i1 >= k && i1 < rows;
    return fma(a1 ? u[i1] : 0.0, a1 ? y[i1] : 0.0, (a0 ? u[i0] : 0.0) * (a0 ? y[i0] : 0.0));
}

// y <- H_{to-1} ... H_from y with the published reflectors (u_i = U[i + k rows]
// for i >= k, u_k = U[k, k]; coefficient cf[k]).  Warps 0-3 of the CTA, one
// per SM sub-partition (FP64 issue is scarce per sub-partition): warp w forms
// q_w for every lane from its rows 64 w + l, 64 w + 32 + l; the four q's meet
// in shared memory (two slots by parity, a named barrier of the four warps)
// and every warp finishes the sum in the order above.  The next reflector
// is loaded while the current one is applied.
__device__ void q2_catch_up4(double *y, int64_t rows, int64_t from, int64_t to, const double *U, const double *cf,
                             double (*qbuf)[4][32]) {
    if (from >= to) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i0 = 64 * w + lane, i1 = i0 + 32;
    auto ld = [&](int64_t k, double &a, double &b, double &c) {
        a = (i0 >= k && i0 < rows) ? __ldcg(U + i0 + k * rows) : 0.0;
        b = (i1 >= k && i1 < rows) ? __ldcg(U + i1 + k * rows) : 0.0;
        c = __ldcg(cf + k);
    };
    double u0, u1, c;
    ld(from, u0, u1, c);
    for (int64_t k = from; k < to; ++k) {
        double v0 = 0.0, v1 = 0.0, cn = 0.0;
        if (k + 1 < to) ld(k + 1, v0, v1, cn);
        const bool a0 = i0 >= k && i0 < rows, a1 = i1 >= k && i1 < rows;
        const double y0 = a0 ? y[i0] : 0.0, y1 = a1 ? y[i1] : 0.0;
        qbuf[k & 1][w][lane] = fma(u1, y1, u0 * y0);
        asm volatile("bar.sync 1, 128;" ::: "memory");
        const double p = (qbuf[k & 1][0][lane] + qbuf[k & 1][1][lane]) + (qbuf[k & 1][2][lane] + qbuf[k & 1][3][lane]);
        const double f = c * warp_sum(p);
        if (a0) y[i0] = fma(-f, u0, y0);
        if (a1) y[i1] = fma(-f, u1, y1);
        u0 = v0;
        u1 = v1;
        c = cn;
    }
}

// Column o of this CTA (column c of L, c < n) from Lg once row c of R is
// complete: blocking (bounded wait) or a single probe.  Returns false if the
// probe found the row incomplete or the wait timed out (then status is set).
__device__ bool q2_load(const double *Lg, int64_t ldl, const unsigned int *rowcnt, int64_t n, int64_t c, double *y,
                        bool block, int32_t *status, int *s_flag) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        const unsigned int want = (unsigned int)(n - c);
        int ok = ld_acquire_u32(rowcnt + c) >= want ? 1 : 0;
        if (!ok && block) {
            const long long t0 = clock64();
            while (!ok) {
                ok = ld_acquire_u32(rowcnt + c) >= want ? 1 : 0;
                if (!ok && clock64() - t0 > (1ll << 32)) {  // ~2 s; rows arrive microseconds apart
                    set_status(status, NS_ERR_TIMEOUT);
                    ok = -1;
                }
            }
        }
        *s_flag = ok;
    }
    __syncthreads();
    const int ok = *s_flag;
    if (ok != 1) return false;
    for (int64_t i = tid; i < n; i += kPipeThreads) y[i] = (i < c) ? 0.0 : __ldcg(Lg + i + c * ldl);
    __syncthreads();
    return true;
}

// One CTA of the second QR in the fused kernel: CTA me of G, columns me,
// me + G, ... of L = [R^T | I] (n x 2n).
__device__ void pipe_qr2_cta(const double *Lg, int64_t ldl, const unsigned int *rowcnt, double *U, int64_t n,
                             int64_t nown_max, double *u0, double *cf, unsigned long long *flag, double *Rout,
                             int32_t *status, int me, int G) {
    extern __shared__ double sm[];
    const int64_t rows = n, cols = 2 * n, steps = n;
    double *own = sm;                     // nown_max * rows: owned columns
    double *ubuf = sm + nown_max * rows;  // 2 * rows: reflectors j (even/odd)
    double *beta = ubuf + 2 * rows;       // nown_max: R2's diagonal of owned columns
    __shared__ double red[2 * (kPipeThreads / 32) + 1];
    __shared__ double s_coef[2], s_unrm[2];
    __shared__ int s_ok, s_flag;
    __shared__ int s_app[kQ2MaxOwn];  // reflectors applied to owned column o; -1: not loaded yet
    __shared__ double qbuf[2][4][32];  // catch-up: the four warps' lane terms by parity
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t nown = (cols - me + G - 1) / G;
    for (int64_t o = 0; o < nown; ++o) {
        const int64_t c = me + o * G;
        if (c >= n)
            for (int64_t i = tid; i < rows; i += kPipeThreads) own[o * rows + i] = (i == c - n) ? 1.0 : 0.0;
        if (tid == 0) s_app[o] = (c >= n) ? 0 : -1;
    }
    if (tid == 0) s_ok = 1;
    __syncthreads();
    if (me == 0) {  // column 0 of L: row 0 of R, then reflector 0
        if (!q2_load(Lg, ldl, rowcnt, n, 0, own, true, status, &s_flag)) return;
        const double b0 = pipe_form(U, rows, 0, own, ubuf, u0, cf, flag, red, &s_coef[0], &s_unrm[0]);
        if (tid == 0) {
            beta[0] = b0;
            s_app[0] = 1;
        }
        __syncthreads();
    }
    int jm = 0;                          // j mod G: the CTA that formed reflector j
    int64_t o_first = (me > 0) ? 0 : 1;  // first owned column after column j
    for (int64_t j = 0; j < steps; ++j) {
        double *ush = ubuf + (j & 1) * rows;
        const int jn_owner = (jm + 1 == G) ? 0 : jm + 1;
        const bool mine = (j + 1 < steps) && jn_owner == me;  // this CTA forms reflector j + 1
        if (mine) {  // column j + 1 loaded and brought up to reflector j - 1
            double *y = own + o_first * rows;
            if (s_app[o_first] < 0) {
                if (!q2_load(Lg, ldl, rowcnt, n, j + 1, y, true, status, &s_flag)) return;
                if (tid == 0) s_app[o_first] = 0;
                __syncthreads();
            }
            if (s_app[o_first] < j) {
                if (warp < 4) q2_catch_up4(y, rows, s_app[o_first], j, U, cf, qbuf);
                __syncthreads();
                if (tid == 0) s_app[o_first] = (int)j;
                __syncthreads();
            }
        }
        if (jm != me) {  // reflector j from its owner (as in pipe_qr_cta)
            const long long t0 = clock64();
            if (mine) {  // as in pipe_qr_cta: from j = 1 on only the tail
                bool late = false;
                late = pipe_poll_rows(U + j * rows, (j >= 1 ? j + 1 : j) + tid, rows, ush, t0);
                if (tid == 0 && !late && j == 0) {
                    unsigned long long fw, nw = 0;
                    while ((fw = ld_acquire_flag(flag + j)) == kPipeEmpty)
                        if (clock64() - t0 > (1ll << 32)) {
                            late = true;
                            break;
                        }
                    while (!late && j >= 1 && (nw = ld_relaxed_u64(U + j - 1 + j * rows)) == kPipeEmpty)
                        if (clock64() - t0 > (1ll << 32)) late = true;
                    s_coef[j & 1] = __longlong_as_double((long long)fw);
                    s_unrm[j & 1] = __longlong_as_double((long long)nw);
                }
                if (late) {
                    set_status(status, NS_ERR_TIMEOUT);
                    s_ok = 0;
                }
                __syncthreads();
                if (!s_ok) return;
            } else {
                if (tid == 0) {
                    unsigned long long fw;
                    while ((fw = ld_acquire_flag(flag + j)) == kPipeEmpty) {
                        if (clock64() - t0 > (1ll << 32)) {
                            set_status(status, NS_ERR_TIMEOUT);
                            s_ok = 0;
                            break;
                        }
                    }
                    s_coef[j & 1] = __longlong_as_double((long long)fw);
                }
                __syncthreads();
                if (!s_ok) return;
                for (int64_t i = j + tid; i < rows; i += kPipeThreads) ush[i] = __ldcg(U + i + j * rows);
                __syncthreads();
            }
        }
        double coef = s_coef[j & 1];  // (the owner of column j + 1 learns it in pipe_apply_form)
        if (mine) {  // look-ahead: column j + 1 first, then reflector j + 1
            double *y = own + o_first * rows;
            double *ushn = ubuf + ((j + 1) & 1) * rows;
            double bj;
            if (j >= 1) {
                bj = pipe_apply_form(U, rows, j, ush, y, ushn, u0, cf, flag, red, &s_coef[(j + 1) & 1],
                                     &s_unrm[(j + 1) & 1], &s_coef[j & 1], &s_ok, status);
                if (!s_ok) return;
            } else {
                if (coef != 0.0) pipe_apply(rows, j, ush, coef, y, red);
                bj = pipe_form(U, rows, j + 1, y, ushn, u0, cf, flag, red, &s_coef[(j + 1) & 1],
                               &s_unrm[(j + 1) & 1]);
            }
            if (tid == 0) {
                beta[o_first] = bj;
                s_app[o_first] = (int)(j + 2);  // reflectors 0..j applied, j + 1 formed from it
            }
        }
        coef = s_coef[j & 1];
        // reflector j to the other loaded columns past j, one warp per column
        {
            int rank = 0;
            for (int64_t o = o_first + (mine ? 1 : 0); o < nown; ++o) {
                if (s_app[o] != (int)j) continue;
                if ((rank & 7) == warp) {
                    if (coef != 0.0) {
                        double *y = own + o * rows;
                        const int lane = tid & 31;
                        const double p = (q2_block_term(ush, y, rows, j, 0) + q2_block_term(ush, y, rows, j, 1)) +
                                         (q2_block_term(ush, y, rows, j, 2) + q2_block_term(ush, y, rows, j, 3));
                        const double f = coef * warp_sum(p);
#pragma unroll
                        for (int m = 0; m < kQ2Lane; ++m) {
                            const int64_t i = lane + 32 * m;
                            if (i >= j && i < rows) y[i] = fma(-f, ush[i], y[i]);
                        }
                    }
                }
                ++rank;
            }
        }
        __syncthreads();
        if (tid == 0)
            for (int64_t o = o_first + (mine ? 1 : 0); o < nown; ++o)
                if (s_app[o] == (int)j) s_app[o] = (int)(j + 1);
        if (jn_owner == me) ++o_first;
        __syncthreads();
        // the next own column (the one this CTA forms a reflector from next):
        // once its row of R is complete, load it and bring it up to reflector
        // j, off the critical path when the row completed early enough
        // (columns further on wait: their catch-up would delay this CTA's
        // next turn on the critical path)
        if (o_first < nown && me + o_first * G < n && s_app[o_first] < 0 &&
            q2_load(Lg, ldl, rowcnt, n, me + o_first * G, own + o_first * rows, false, status, &s_flag)) {
            if (warp < 4) q2_catch_up4(own + o_first * rows, rows, 0, j + 1, U, cf, qbuf);
            __syncthreads();
            if (tid == 0) s_app[o_first] = (int)(j + 1);
            __syncthreads();
        }
        if (++jm == G) jm = 0;
    }
    for (int64_t o = 0; o < nown; ++o) {  // [R2 | Q2^T], leading dimension n
        const int64_t c = me + o * G;
        for (int64_t i = tid; i < steps; i += kPipeThreads) {
            double r = 0.0;
            if (i < c) r = own[o * rows + i];
            else if (i == c) r = beta[o];
            Rout[i + c * steps] = r;
        }
    }
}

// At most 80 registers a thread (no spills), so three CTAs fit on an SM: the
// fused QRs of solves in flight on other streams, and a QR beside the FP32
// Jacobi phase's cluster, can then be resident together (two per SM made
// concurrent solves wait for one another's QR or FP32 phase to drain).
__global__ void __launch_bounds__(kPipeThreads, 3) hqr_fused_kernel(const double *W, double *U1, int64_t s, int64_t n,
                                                                int64_t nown1, double *u0a, double *cfa,
                                                                unsigned long long *flag1, double *Lg,
                                                                unsigned int *rowcnt, double *U2, int64_t nown2,
                                                                double *u0b, double *cfb, unsigned long long *flag2,
                                                                double *Rout2, int G1, int32_t *status) {
    if ((int)blockIdx.x < G1)
        pipe_qr_cta(W, U1, s, n, nown1, u0a, cfa, flag1, nullptr, status, (int)blockIdx.x, G1, Lg, n, rowcnt);
    else
        pipe_qr2_cta(Lg, n, rowcnt, U2, n, nown2, u0b, cfb, flag2, Rout2, status, (int)blockIdx.x - G1,
                     (int)gridDim.x - G1);
}

// ------------------------------------------------- static column order ----
// The pipelined QR does not pivot.  For the relative accuracy of the
// preconditioned Jacobi on column-graded inputs the rows of R must be graded,
// which column pivoting achieves; ordering the columns once by decreasing norm
// before the QR achieves it for column-scaled matrices (row i of R is bounded
// by the norm of column i).  perm[j] = the column of SA placed at position j.
__global__ void __launch_bounds__(256) colnorm_kernel(const double *__restrict__ SA, int64_t s, int64_t n,
                                                      double *__restrict__ key) {
    __shared__ double red[32];
    __shared__ long long redk[32];
    for (int64_t c = blockIdx.x; c < n; c += gridDim.x) {
        const double *a = SA + c * s;
        long long mx = 0;
        for (int64_t i = threadIdx.x; i < s; i += blockDim.x) mx = max(mx, abs_key(a[i]));
        const double sc = block_pow2_scale(mx, redk);  // largest entry scaled into [1, 2)
        double v[1] = {0.0};
        for (int64_t i = threadIdx.x; i < s; i += blockDim.x) {
            const double x = a[i] * sc;
            v[0] = fma(x, x, v[0]);
        }
        block_sum_t0<1>(v, red);
        if (threadIdx.x == 0) {
            // log2 |a|^2 = log2(scaled |a|^2) - 2 log2(sc); -inf-like for a zero column
            const int esc = (int)((__double_as_longlong(sc) >> 52) & 0x7FF) - 1023;
            key[c] = (sc == 0.0 || v[0] == 0.0) ? -1e300 : log2(v[0]) - 2.0 * (double)esc;
        }
        __syncthreads();
    }
}

// one CTA: perm = the columns by decreasing key, ties to the lower index
// (bitonic sort of np2 >= n entries in dynamic shared memory, n <= 4096)
__global__ void __launch_bounds__(1024) sort_perm_kernel(const double *__restrict__ key, int64_t n, int64_t np2,
                                                         int32_t *__restrict__ perm) {
    extern __shared__ double sk[];                // np2 keys
    int32_t *si = (int32_t *)(sk + np2);          // np2 indices
    for (int64_t i = threadIdx.x; i < np2; i += blockDim.x) {
        sk[i] = i < n ? key[i] : -2e300;
        si[i] = (int32_t)i;
    }
    __syncthreads();
    for (int64_t k = 2; k <= np2; k <<= 1) {
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            for (int64_t i = threadIdx.x; i < np2; i += blockDim.x) {
                const int64_t l = i ^ j;
                if (l > i) {
                    // "x before y": larger key, then smaller index
                    const bool l_before_i = sk[l] > sk[i] || (sk[l] == sk[i] && si[l] < si[i]);
                    const bool up = (i & k) == 0;
                    if (up ? l_before_i : !l_before_i) {
                        const double tk = sk[i];
                        const int32_t ti = si[i];
                        sk[i] = sk[l];
                        si[i] = si[l];
                        sk[l] = tk;
                        si[l] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) perm[i] = si[i];
}

// W[:, j] = SA[:, perm[j]]
__global__ void permute_cols_kernel(const double *__restrict__ SA, int64_t s, int64_t n,
                                    const int32_t *__restrict__ perm, double *__restrict__ W) {
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        const double *a = SA + (int64_t)perm[j] * s;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s; i += (int64_t)gridDim.x * blockDim.x)
            W[i + j * s] = a[i];
    }
}

// ------------------------------------------------------------ transpose ----
__global__ void transpose_kernel(const double *__restrict__ A, int64_t n, double *__restrict__ B) {
    __shared__ double tile[32][33];
    const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = bx + threadIdx.x, j = by + r;
        if (i < n && j < n) tile[r][threadIdx.x] = A[i + j * n];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = by + threadIdx.x, j = bx + r;
        if (i < n && j < n) B[i + j * n] = tile[threadIdx.x][r];
    }
}

// X = R2^T from the QR of L (upper triangle of the output of hqr, in place)
__global__ void r2t_kernel(const double *__restrict__ R2, int64_t n, double *__restrict__ X) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int64_t i = idx % n, j = idx / n;
    X[i + j * n] = (i >= j) ? R2[j + i * n] : 0.0;
}

// B (n x n) = I
__global__ void identity_kernel(double *__restrict__ B, int64_t n) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n * n) B[idx] = (idx % n == idx / n) ? 1.0 : 0.0;
}

// rows of V to the input column order: W[perm[i], c] = V[i, c]
__global__ void permute_rows_kernel(const double *__restrict__ V, int64_t n, const int32_t *__restrict__ perm,
                                    double *__restrict__ W) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int64_t i = idx % n, c = idx / n;
    W[perm[i] + c * n] = V[idx];
}

// --------------------------------------------------------------- Jacobi ----
__device__ __forceinline__ int64_t rr_player(int64_t pos, int64_t step, int64_t n2) {
    return pos == 0 ? 0 : 1 + (pos - 1 + step) % (n2 - 1);
}

// The FP32 images of a pair's sums (a, b the squared norms, g the inner
// product, all scaled alike) cannot resolve the angle when the norms agree to
// about their rounding and the inner product is small as well: there
// tan(2 theta) = 2 g / (a - b) is decided by a difference the images lost, an
// angle taken from them leaves the inner product at the images' noise level,
// and the pair would stall (clustered singular values).  Those pairs take the
// angle from FP64 sums.
__device__ __forceinline__ bool ring_unresolved(float a, float b, float g) {
    const float mx = fmaxf(a, b);
    return fabsf(b - a) <= 0x1p-12f * mx && fabsf(g) <= 0x1p-10f * mx;
}

// tan(theta) = sign(z) / (|z| + (1 + z^2)^(1/2)), z = num / den, in FP64;
// `fallback` when z is not a finite number
__device__ __forceinline__ double exact_tan(double num, double den, double fallback) {
    const double z = num / den;
    if (!isfinite(z)) return fallback;
    const double az = fabs(z);
    return (az > 1e150) ? 0.5 / z : copysign(1.0, z) / (az + sqrt(fma(z, z, 1.0)));
}

// Rotation for (alpha, beta, gamma): returns false if the pair is already
// orthogonal to the tolerance.  One thread.
__device__ __forceinline__ bool rotation(double alpha, double beta, double gamma, double tol2, double *c_out,
                                         double *s_out) {
    const double gg = gamma * gamma, ab = alpha * beta;
    if (gamma == 0.0 || !(gg > tol2 * ab)) return false;
    // FP32 images of alpha, beta, gamma scaled by the same power of two (the
    // larger of alpha, beta lands in [1, 2)); integer work on the exponent
    const double mx = fmax(alpha, beta);
    const int e = (int)(((unsigned long long)__double_as_longlong(mx) >> 52) & 0x7FF);
    int se = 2046 - e;
    se = se < 1 ? 1 : (se > 2046 ? 2046 : se);
    const double sc = __longlong_as_double((long long)se << 52);
    const float a32 = (float)(alpha * sc), b32 = (float)(beta * sc), g32 = (float)(gamma * sc);
    double t;
    if (ring_unresolved(a32, b32, g32)) {
        // nearly equal norms and a small inner product: the FP32 images cannot
        // resolve beta - alpha, which then decides the angle
        t = exact_tan(beta - alpha, 2.0 * gamma, 1.0);
    } else if (fabsf(g32) >= 1e-30f) {
        const float z = (b32 - a32) / (2.0f * g32);
        t = (double)((fabsf(z) > 1e18f) ? 0.5f / z : copysignf(1.0f, z) / (fabsf(z) + sqrtf(1.0f + z * z)));
    } else {
        // tiny angle: t ~ gamma / (beta - alpha), from the mantissas and the
        // exponents separately (the scaled FP32 image of gamma underflows)
        const double d = beta - alpha;
        if (d == 0.0) {
            t = gamma > 0.0 ? 1.0 : -1.0;  // alpha = beta: the 45-degree rotation
        } else {
            const long long gb = __double_as_longlong(gamma), db = __double_as_longlong(d);
            const int eg = (int)((gb >> 52) & 0x7FF), ed = (int)((db >> 52) & 0x7FF), k = eg - ed + 1023;
            if (eg == 0 || ed == 0 || k < 1 || k > 2046) {
                t = gamma / d;  // subnormal operands or an extreme ratio (rare)
            } else {
                const float gm = (float)__longlong_as_double((gb & 0x800FFFFFFFFFFFFFll) | (1023ll << 52));
                const float dm = (float)__longlong_as_double((db & 0x800FFFFFFFFFFFFFll) | (1023ll << 52));
                t = (double)(gm / dm) * __longlong_as_double((long long)k << 52);
            }
        }
    }
    const double tt = fma(t, t, 1.0);
    double y = (double)rsqrtf((float)tt);
    const double h = -0.5 * tt;
    y = y * fma(h, y * y, 1.5);
    y = y * fma(h, y * y, 1.5);
    *c_out = y;
    *s_out = y * t;
    return true;
}

// Barrier-free convergence check over all n(n-1)/2 pairs of the columns of X
// (all CTAs of the grid; nrm: n doubles of scratch).  Returns 1 if the check
// ran and no pair needs a rotation, 0 if some pair does, -1 if a grid barrier
// timed out.
__device__ int jacobi_check_pass(const double *X, int64_t n, double tol2, GridBarrier bar, unsigned int *flag,
                                 double *nrm) {
    // column norms once (one warp per column, into nrm), then one warp per
    // pair for the inner product only; pairs are indexed p-major and found by
    // an integer binary search
    if (!grid_sync(bar)) return -1;
    const int lane = threadIdx.x & 31;
    const int64_t nw = blockDim.x >> 5, gw = (int64_t)blockIdx.x * nw + (threadIdx.x >> 5), Wn = gridDim.x * nw;
    for (int64_t c = gw; c < n; c += Wn) {
        double a = 0.0;
        for (int64_t i = lane; i < n; i += 32) {
            const double x = __ldcg(X + i + c * n);
            a = fma(x, x, a);
        }
        a = warp_sum(a);
        if (lane == 0) nrm[c] = a;
    }
    if (!grid_sync(bar)) return -1;
    const int64_t total = n * (n - 1) / 2;
    int any = 0;
    for (int64_t pi = gw; pi < total && !any; pi += Wn) {
        int64_t lo = 0, hi = n - 1;  // pairs before row p: p (2n - p - 1) / 2
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (mid * (2 * n - mid - 1) / 2 <= pi) lo = mid;
            else hi = mid;
        }
        const int64_t p = lo, q = pi - p * (2 * n - p - 1) / 2 + p + 1;
        double g = 0.0;
        for (int64_t i = lane; i < n; i += 32) g = fma(__ldcg(X + i + p * n), __ldcg(X + i + q * n), g);
        g = warp_sum(g);
        if (g != 0.0 && g * g > tol2 * __ldcg(nrm + p) * __ldcg(nrm + q)) any = 1;
    }
    if (any && lane == 0) atomicAdd(flag, 1u);
    if (!grid_sync(bar)) return -1;
    return (*(volatile unsigned int *)flag == 0u) ? 1 : 0;
}

// sigma_l = |x_l| for the columns of X (power-of-two scaled, CTAs round-robin)
__device__ void jacobi_sigma(const double *X, int64_t n, double *sigma) {
    __shared__ double red[32];
    __shared__ long long redk[32];
    const int64_t G = gridDim.x, me = blockIdx.x;
    const int tid = threadIdx.x;
    for (int64_t l = me; l < n; l += G) {
        long long key = 0;
        for (int64_t i = tid; i < n; i += blockDim.x) key = max(key, abs_key(__ldcg(X + i + l * n)));
        const double sc = block_pow2_scale(key, redk);
        double v[1] = {0.0};
        if (sc != 0.0)
            for (int64_t i = tid; i < n; i += blockDim.x) {
                const double a = __ldcg(X + i + l * n) * sc;
                v[0] = fma(a, a, v[0]);
            }
        block_sum_t0<1>(v, red);
        if (tid == 0) sigma[l] = (sc == 0.0) ? 0.0 : sqrt(v[0]) / sc;
        __syncthreads();
    }
}

// statistics of the iteration: full sweeps, rotations, barrier-free checks,
// and which kernel ran (the cluster-ring size C, or 0: barrier-separated)
__device__ __forceinline__ void jacobi_record_stats(unsigned int *rotcount, int full_sweeps, int check_passes,
                                                    int ring) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned int rots = 0;
        for (int sw = 0; sw < kMaxSweeps; ++sw) rots += *(volatile unsigned int *)(rotcount + sw);
        rotcount[128] = (unsigned int)full_sweeps;
        rotcount[129] = rots;
        rotcount[130] = (unsigned int)check_passes;
        rotcount[131] = (unsigned int)ring;
    }
}

template <int RPT>
__global__ void __launch_bounds__(kDenseThreads) jacobi_coop_kernel(double *X, double *V, int64_t n, double tol,
                                                                   GridBarrier bar, unsigned int *rotcount,
                                                                   unsigned int *checkflag, double *sigma,
                                                                   int32_t *status, int vinit, int max_sweeps) {
    __shared__ double red[32 * 3];
    __shared__ double par[3];
    const int64_t G = gridDim.x, me = blockIdx.x;
    const int tid = threadIdx.x;
    const double tol2 = tol * tol;
    if (!vinit)  // V = I, else V arrives holding Q2
        for (int64_t l = me; l < n; l += G)
            for (int64_t i = tid; i < n; i += blockDim.x) V[i + l * n] = (i == l) ? 1.0 : 0.0;
    const int64_t n2 = n + (n & 1), npairs = n2 / 2, steps = n2 - 1;
    bool converged = (n < 2);
    unsigned int prev_rot = 0xFFFFFFFFu;
    int full_sweeps = 0, check_passes = 0;
    for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
        if (prev_rot < (unsigned int)kCheckBelow) {
            ++check_passes;
            const int c = jacobi_check_pass(X, n, tol2, bar, checkflag + sweep, sigma);
            if (c < 0) return;
            if (c == 1) {
                converged = true;
                break;
            }
        }
        unsigned int local = 0;
        ++full_sweeps;
        for (int64_t step = 0; step < steps; ++step) {
            if (!grid_sync(bar)) return;
            for (int64_t pi = me; pi < npairs; pi += G) {
                int64_t p = rr_player(pi, step, n2), q = rr_player(n2 - 1 - pi, step, n2);
                if (p > q) {
                    const int64_t tmp = p;
                    p = q;
                    q = tmp;
                }
                if (q >= n) continue;  // phantom column of an odd n
                double *xp = X + p * n, *xq = X + q * n;
                double ra[RPT], rb[RPT];
                double a3[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const int64_t i = tid + (int64_t)r * kDenseThreads;
                    ra[r] = (i < n) ? __ldcg(xp + i) : 0.0;
                    rb[r] = (i < n) ? __ldcg(xq + i) : 0.0;
                    a3[0] = fma(ra[r], ra[r], a3[0]);
                    a3[1] = fma(rb[r], rb[r], a3[1]);
                    a3[2] = fma(ra[r], rb[r], a3[2]);
                }
                block_sum_t0<3>(a3, red);
                if (tid == 0) {
                    double c = 1.0, s = 0.0;
                    const bool rot = rotation(a3[0], a3[1], a3[2], tol2, &c, &s);
                    par[0] = rot ? 1.0 : 0.0;
                    par[1] = c;
                    par[2] = s;
                }
                __syncthreads();
                if (par[0] == 0.0) {
                    __syncthreads();
                    continue;
                }
                const double cs = par[1], sn = par[2];
                double *vp = V + p * n, *vq = V + q * n;
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const int64_t i = tid + (int64_t)r * kDenseThreads;
                    if (i < n) {
                        xp[i] = fma(cs, ra[r], -sn * rb[r]);
                        xq[i] = fma(sn, ra[r], cs * rb[r]);
                        const double c0 = __ldcg(vp + i), d0 = __ldcg(vq + i);
                        vp[i] = fma(cs, c0, -sn * d0);
                        vq[i] = fma(sn, c0, cs * d0);
                    }
                }
                ++local;
                __syncthreads();
            }
        }
        if (tid == 0 && local) atomicAdd(rotcount + sweep, local);
        if (!grid_sync(bar)) return;
        prev_rot = *(volatile unsigned int *)(rotcount + sweep);
        converged = (prev_rot == 0u);
    }
    if (!converged && me == 0 && tid == 0) set_status(status, NS_ERR_NOCONV);
    jacobi_record_stats(rotcount, full_sweeps, check_passes, 0);
    if (!grid_sync(bar)) return;
    jacobi_sigma(X, n, sigma);
}

// ------------------------------------------------- Jacobi, cluster ring ----
// The same iteration as jacobi_coop_kernel (same rotation rule, threshold and
// stopping test, every pair visited once per sweep), in an order that lets
// most parallel steps run without a grid barrier.  For n <= 2 G kRingC the
// n' = 2 G kRingC columns (columns >= n are zero and never rotate) form 2G
// blocks of kRingC columns.  A sweep visits the block pairs round-robin: 2G - 1
// outer steps with G disjoint block pairs each, cluster g (kRingC CTAs) taking
// block pair g.  Within an outer step CTA i keeps column i of block P in
// registers while the columns of block Q travel around the cluster: in round j
// CTA i rotates the pair (P[i], Q[(i + j) mod kRingC]) and hands its Q column
// to CTA i - 1 with st.async into that CTA's shared memory, the bytes counted
// on the receiver's mbarrier.  A round thus waits only for one neighbour's
// column.  The pairs inside each block are visited at the first outer step of
// a sweep (kRingC - 1 round-robin rounds through global memory, one grid
// barrier each).  Blocks move between clusters through global memory: each
// CTA publishes the two columns it stores with a release of their version
// and the next outer step's reader acquires exactly those versions, so only a
// sweep's end (rotation count) takes a grid barrier.  kRingT threads with kRingR rows each: four
// warps keep all four FP64 units of the SM busy while the reduction tree stays
// short (FP64 runs at 2 operations per clock per SM here, so every add of a
// reduction counts).
// The cluster size C (CTAs per cluster = columns per block) is a template
// parameter: 8 (portable), or 16 for n > 240, where 16 clusters of 8 would
// not all find SMs of their own (the one that shares SMs paces every other).
constexpr int kRingT = 128;    // threads per CTA
constexpr int kRingR = 2;      // rows per thread: n <= kRingT * kRingR
constexpr int kRingN = kRingT * kRingR;

// Warp sums of three values with six additions per lane: two butterfly levels
// that halve a 4-vector (the fourth entry is zero), then three levels on the
// remaining value.  Afterwards lanes 0-7 hold the total of v0, lanes 8-15 of
// v1, lanes 16-23 of v2.  The order of the additions is fixed.
__device__ __forceinline__ double warp_sum3(double v0, double v1, double v2) {
    const int lane = threadIdx.x & 31;
    const bool hi4 = (lane & 16) != 0, hi3 = (lane & 8) != 0;
    const double s0 = hi4 ? v0 : v2, s1 = hi4 ? v1 : 0.0;
    double k0 = hi4 ? v2 : v0, k1 = hi4 ? 0.0 : v1;
    k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    const double s2 = hi3 ? k0 : k1;
    double k = hi3 ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, s2, 8);
    k += __shfl_xor_sync(0xffffffffu, k, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    return k;
}


// Waiting threads are suspended in hardware until the phase completes (or the
// hint elapses) instead of re-polling: a polling loop of whole warps keeps the
// shared-memory pipe busy and delays the scalar warp's loads.
constexpr uint32_t kRingSuspendNs = 1000000;

// bounded wait for phase `parity` of a local mbarrier that peers complete
// (limit in clock cycles: ~2 s by default; a healthy ring waits microseconds)
__device__ __forceinline__ bool ring_wait(uint32_t mbar, uint32_t parity, long long limit = 1ll << 32) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity), "r"(kRingSuspendNs)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// CTA layout (kRingCta threads): warp 0 is the scalar warp (the angle of
// each pair, the column scales, the hand-over of the scales), warps 1-4 hold
// rows of the X columns, warps 5-8 the same rows of the V columns.  The row
// warps never wait on the scalar chain of the previous round, and the V
// update of one round overlaps the X work of the next.
constexpr int kRingCta = 32 + 2 * kRingT;
constexpr int kRingBar = 32 + kRingT;  // scalar warp + X row warps (named barrier 1)
constexpr int kRingXV = kRingCta;      // X rows arrive, V rows and the scalar warp wait (named barrier 2)

__device__ __forceinline__ void xbar() { asm volatile("bar.sync 1, %0;" ::"n"(kRingBar) : "memory"); }

// bounded wait for phase `parity` of a local mbarrier completed inside the CTA
__device__ __forceinline__ bool ring_wait_cta(uint32_t mbar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity), "r"(kRingSuspendNs)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1ll << 32)) return false;
    }
}

// FP32 value in [1, 2) of the leading 23 fraction bits of an IEEE double
__device__ __forceinline__ float lead_mant(unsigned long long k) {
    return __uint_as_float(0x3F800000u | (unsigned int)((k >> 29) & 0x7FFFFFu));
}
// 2^k as an FP32 number (0 below the normal range; k <= 127)
__device__ __forceinline__ float pow2f(int k) { return k < -126 ? 0.0f : __uint_as_float((unsigned int)(127 + k) << 23); }

// The ring kernel's sums of a pair.  The squared norms need only modest
// accuracy (no cancellation; they set the angle and the threshold test), so
// they are FP32 sums of FP32 images: alpha = fa 4^(Ea - 1023) with Ea the
// largest biased exponent of the column's entries, likewise beta.  The inner
// product can cancel and stays FP64.
struct RingSums {
    float fa, fb;
    int Ea, Eb;
    double g;
};

// unbiased exponent of alpha = fa 4^(E - 1023) (fa > 0 normal)
__device__ __forceinline__ int ring_lexp(float f, int E) { return (int)((__float_as_uint(f) >> 23) & 0xFF) - 127 + 2 * (E - 1023); }

// The threshold test g^2 > tol2 alpha beta on the exponents and the leading 23
// fraction bits: no FP64 instruction, no overflow or underflow of the
// products, and no branch (it runs beside the angle on the scalar warp's
// critical path).  It can differ from the exact comparison only within a
// relative 2^-20 of the threshold (plus the FP32 rounding of the norms).  A
// zero or subnormal gamma, or a column whose entries are all zero or
// subnormal, is below the threshold; an infinite gamma is above it.
__device__ __forceinline__ bool ring_above(const RingSums &r, double tol2) {
    const unsigned long long kg = (unsigned long long)__double_as_longlong(r.g) & 0x7FFFFFFFFFFFFFFFull;
    const unsigned long long kt = (unsigned long long)__double_as_longlong(tol2);
    const int eg = (int)(kg >> 52), et = (int)(kt >> 52);
    const uint32_t ua = __float_as_uint(r.fa), ub = __float_as_uint(r.fb);
    const bool special = eg == 0 || eg == 0x7FF || ((ua >> 23) & 0xFF) == 0 || ((ub >> 23) & 0xFF) == 0;
    // gamma^2 / (tol2 alpha beta) = 2^k mg^2 / (mt ma mb), mg^2 in [1, 4), mt ma mb in [1, 8)
    const int k = 2 * (eg - 1023) - ring_lexp(r.fa, r.Ea) - ring_lexp(r.fb, r.Eb) - (et - 1023);
    const float mg = lead_mant(kg), ma = __uint_as_float(0x3F800000u | (ua & 0x7FFFFFu)),
                mb = __uint_as_float(0x3F800000u | (ub & 0x7FFFFFu));
    const bool cmp = k >= 3 || (k > -2 && (mg * mg) * pow2f(min(k, 2)) > (lead_mant(kt) * ma) * mb);
    return special ? kg == 0x7FF0000000000000ull : cmp;
}

// Jacobi angle of a pair held as scaled columns x = d x~ (ring kernel): the
// sums are those of x~_p, x~_q; dp2, dq2, dpq the squares and product of the
// scales (FP32).  The threshold test does not depend on the scales.
// t = tan(theta) needs only modest accuracy (the applied rotation is
// orthogonal whatever t is), so it comes from FP32 images of the scaled sums;
// it is evaluated unconditionally, beside the threshold test.
__device__ __forceinline__ bool ring_angle(const RingSums &r, double tol2, float dp2, float dq2, float dpq, double dp,
                                           double dq, double *t_out, bool *exact) {
    const bool above = ring_above(r, tol2);
    const int la = ring_lexp(r.fa, r.Ea), lb = ring_lexp(r.fb, r.Eb), shift = max(la, lb);
    const float a32 = r.fa * pow2f(2 * (r.Ea - 1023) - shift) * dp2;
    const float b32 = r.fb * pow2f(2 * (r.Eb - 1023) - shift) * dq2;
    const float g32 = f32_image(r.g, shift) * dpq;
    const float z = __fdividef(b32 - a32, 2.0f * g32), az = fabsf(z);
    const float w = fmaf(z, z, 1.0f);
    const float tb = (az > 1e18f) ? __fdividef(0.5f, z) : copysignf(__fdividef(1.0f, az + w * rsqrtf(w)), z);
    *exact = above && ring_unresolved(a32, b32, g32);
    if (!above) return false;
    if (fabsf(g32) >= 1e-30f) {
        *t_out = f64_of(tb);
        return true;
    }
    // tiny angle: t ~ gamma / (beta - alpha) with the true (scaled) sums (rare)
    const double a = ldexp(f64_of(r.fa), 2 * (r.Ea - 1023)), b = ldexp(f64_of(r.fb), 2 * (r.Eb - 1023));
    const double al = a * dp * dp, be = b * dq * dq, ga = r.g * dp * dq, d = be - al;
    *t_out = (d == 0.0) ? (ga > 0.0 ? 1.0 : -1.0) : ga / d;
    return true;
}

// Combines the X row warps' partial sums (red[v * 4 + w]: value v of row
// warp w) in lanes 0-2 of the scalar warp and returns them in every lane.
__device__ __forceinline__ void ring_combine(const double *red, double *al, double *be, double *ga) {
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    if (lane < 3) v = (red[lane * 4 + 0] + red[lane * 4 + 1]) + (red[lane * 4 + 2] + red[lane * 4 + 3]);
    *al = __shfl_sync(0xffffffffu, v, 0);
    *be = __shfl_sync(0xffffffffu, v, 1);
    *ga = __shfl_sync(0xffffffffu, v, 2);
}

// The X row warps' share of a pair's sums: warp sums in red[v * 4 + w].
__device__ __forceinline__ void ring_partials(double a, double b, double g, int t, double *red) {
    const double k = warp_sum3(a, b, g);
    if ((t & 7) == 0 && (t & 31) < 24) red[((t & 31) >> 3) * 4 + (t >> 5)] = k;
}

// one pair of columns through global memory (CTA-uniform p, q), all threads
// of the CTA; plain (unscaled) rotation.  Returns 1 in thread 0 if rotated.
__device__ unsigned int jacobi_pair_global(double *X, double *V, int64_t n, int64_t p, int64_t q, double tol2,
                                           double *red, double *par) {
    if (p >= n || q >= n) return 0u;
    const int tid = threadIdx.x;
    const bool scalar = tid < 32, isx = tid >= 32 && tid < 32 + kRingT;
    const int t = isx ? tid - 32 : tid - 32 - kRingT;
    double *M = isx ? X : V;
    double ya[kRingR] = {0.0, 0.0}, yb[kRingR] = {0.0, 0.0};
    if (!scalar) {
#pragma unroll
        for (int r = 0; r < kRingR; ++r) {
            const int64_t i = t + r * kRingT;
            ya[r] = (i < n) ? __ldcg(M + i + p * n) : 0.0;
            yb[r] = (i < n) ? __ldcg(M + i + q * n) : 0.0;
        }
    }
    if (isx) ring_partials(fma(ya[1], ya[1], ya[0] * ya[0]), fma(yb[1], yb[1], yb[0] * yb[0]),
                           fma(ya[1], yb[1], ya[0] * yb[0]), t, red);
    if (scalar || isx) xbar();
    if (scalar) {
        double al, be, ga;
        ring_combine(red, &al, &be, &ga);
        if (tid == 0) {
            double c = 1.0, s = 0.0;
            par[0] = rotation(al, be, ga, tol2, &c, &s) ? 1.0 : 0.0;
            par[1] = c;
            par[2] = s;
        }
    }
    __syncthreads();
    const bool rot = par[0] != 0.0;
    if (rot && !scalar) {
        const double cs = par[1], sn = par[2];
#pragma unroll
        for (int r = 0; r < kRingR; ++r) {
            const int64_t i = t + r * kRingT;
            if (i < n) {
                M[i + p * n] = fma(cs, ya[r], -sn * yb[r]);
                M[i + q * n] = fma(sn, ya[r], cs * yb[r]);
            }
        }
    }
    __syncthreads();  // par and red are rewritten by the next pair
    return rot ? 1u : 0u;
}

__device__ __forceinline__ void mbar_arm(unsigned long long *mb, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(shared_addr(mb)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void send_pair(uint32_t dst, double a, double b, uint32_t mb) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(dst),
                 "d"(a), "d"(b), "r"(mb)
                 : "memory");
}

template <int kRingC>
__global__ void __cluster_dims__(kRingC, 1, 1) __launch_bounds__(kRingCta, 2)
    jacobi_ring_kernel(double *X, double *V, int64_t n, int64_t G, double tol, GridBarrier bar,
                       unsigned int *rotcount, unsigned int *checkflag, double *sigma, unsigned int *colver,
                       int32_t *status, int vinit, int max_sweeps, const unsigned int *fp32_ran) {
    // Slot j receives the Q column of round j: rows t and t + kRingT of X in
    // xbuf[j][t] and of V in vbuf[j][t], and its scale pair in sbuf[j], each
    // completed on its own mbarrier (mbx, mbv, mbs).  Columns are held scaled,
    // x = d x~, so a rotation costs one FMA per entry:
    //   x~_p <- x~_p - mu x~_q,  x~_q <- x~_q + nu x~_p,  mu = t d_q / d_p,
    //   nu = t d_p / d_q,  d_p, d_q <- c d_p, c d_q  (c = cos, t = tan of the angle),
    // the same first-order rounding as the plain rotation; the scales stay in
    // [2^-kRingC/2, 1] within an outer step (at most kRingC rotations per column) and are
    // folded back into the columns when they are stored.  par[j] = (rotated,
    // mu, nu) of round j, announced to the V warps by mbr[j]; mbf announces
    // the final scales of the outer step to the row warps.
    static_assert(kRingR == 2, "one double2 per thread and slot");
    extern __shared__ __align__(16) double2 ring_dyn[];  // 2 kRingC kRingT double2 (ring_smem)
    double2(*xbuf)[kRingT] = reinterpret_cast<double2(*)[kRingT]>(ring_dyn);
    double2(*vbuf)[kRingT] = reinterpret_cast<double2(*)[kRingT]>(ring_dyn + kRingC * kRingT);
    __shared__ __align__(16) double2 sbuf[kRingC];
    __shared__ __align__(8) unsigned long long mbx[kRingC], mbv[kRingC], mbs[kRingC], mbr[kRingC], mbf;
    __shared__ double red[16];
    __shared__ double rg[4];          // per X row warp: x~_p . x~_q
    __shared__ float2 rab[4];         // per X row warp: FP32 images of |x~_p|^2, |x~_q|^2
    __shared__ uint32_t rexp[4];      // per X row warp: (E_p << 16) | E_q, the images' exponents
    __shared__ double2 rn[4];         // per X row warp: FP64 |x~_p|^2, |x~_q|^2 (unresolved pairs only)
    __shared__ double par[kRingC][3];
    __shared__ double s_fin[2];
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x;
    {
        // The ring needs the launch geometry it was built for: kRingC CTAs per
        // cluster and G clusters.  A launch that did not honour the cluster
        // dimension (a tool that re-issues the launch, say) leaves without
        // touching distributed shared memory and reports NS_ERR_CUDA.
        uint32_t ncta, ncl;
        asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
        asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(ncl));
        if (ncta != (uint32_t)kRingC || (int64_t)ncl != G || (int64_t)gridDim.x != G * kRingC ||
            blockDim.x != (unsigned)kRingCta) {
            if (tid == 0) set_status(status, NS_ERR_CUDA);
            return;
        }
    }
    const bool scalar = tid < 32, isx = tid >= 32 && tid < 32 + kRingT;
    const int t = isx ? tid - 32 : tid - 32 - kRingT;  // row thread index (unused in the scalar warp)
    const uint32_t ci = cluster_rank();
    const int64_t g = blockIdx.x / kRingC;
    const int64_t nblk = 2 * G, nouter = nblk - 1;
    const double tol2 = tol * tol;
    if (tid == 0) {
        for (int j = 0; j < kRingC; ++j) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(shared_addr(&mbx[j])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(shared_addr(&mbv[j])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(shared_addr(&mbs[j])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(shared_addr(&mbr[j])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(shared_addr(&mbf)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (!vinit)  // V = I, else V arrives holding Q2
        for (int64_t l = blockIdx.x; l < n; l += gridDim.x)
            for (int64_t i = tid; i < n; i += blockDim.x) V[i + l * n] = (i == l) ? 1.0 : 0.0;
    cluster_sync_all();  // every mbarrier of the cluster is initialised before the first st.async
    const uint32_t peer = (ci + kRingC - 1) % kRingC;
    const uint32_t xb_peer = peer_addr(shared_addr(&xbuf[0][0]), peer);
    const uint32_t vb_peer = peer_addr(shared_addr(&vbuf[0][0]), peer);
    const uint32_t sb_peer = peer_addr(shared_addr(&sbuf[0]), peer);
    const uint32_t mx_peer = peer_addr(shared_addr(&mbx[0]), peer);
    const uint32_t mv_peer = peer_addr(shared_addr(&mbv[0]), peer);
    const uint32_t ms_peer = peer_addr(shared_addr(&mbs[0]), peer);
    double *M = isx ? X : V;
    const int64_t i0 = t, i1 = t + kRingT;
    const bool r0 = !scalar && i0 < n, r1 = !scalar && i1 < n;

    bool converged = (n < 2), ok = true;
    unsigned int prev_rot = 0xFFFFFFFFu;
    int full_sweeps = 0, check_passes = 0;
    uint32_t ostep = 0;  // outer steps so far: phase parity of the slot mbarriers
    // After the FP32 phase and its first-order completions the columns start
    // nearly orthogonal: the barrier-free check runs from the third sweep on
    // whatever the rotation count was.  When the last completion left no pair
    // out and only tiny rotations (verdict 2), the convergence test has
    // already run on the Gram matrix of X (the FP64 rule of the check pass,
    // on G = X^T X), and with no pair above the tolerance (word 16 still 0)
    // there is nothing left to do but the singular values.
    const unsigned int ran = fp32_ran ? *(volatile const unsigned int *)fp32_ran : 0u;
    const bool gram_checked = ran && *(volatile const unsigned int *)(fp32_ran + 3) == 2u;
    if (gram_checked && *(volatile const unsigned int *)(fp32_ran + 16) == 0u) {
        converged = true;
        check_passes = 1;
    }
    const int check_from = ran ? 2 : max_sweeps + 1;
    for (int sweep = 0; sweep < max_sweeps && !converged && ok; ++sweep) {
        if (prev_rot < (unsigned int)kCheckBelow || sweep >= check_from) {
            ++check_passes;
            const int c = jacobi_check_pass(X, n, tol2, bar, checkflag + sweep, sigma);
            if (c < 0) {
                ok = false;
                break;
            }
            if (c == 1) {
                converged = true;
                break;
            }
        }
        ++full_sweeps;
        unsigned int local = 0;
        if (!grid_sync(bar)) {
            ok = false;
            break;
        }
        for (int64_t ot = 0; ot < nouter; ++ot) {
            const int64_t P = rr_player(g, ot, nblk), Q = rr_player(nblk - 1 - g, ot, nblk);
            if (ot == 0) {  // pairs inside blocks P and Q
                // Both blocks belong to this cluster alone at the first outer step
                // (the grid barrier at the start of the sweep ordered their last
                // writes), so a cluster barrier (release/acquire at cluster scope)
                // separates the rounds.
                const int half = kRingC / 2;
                const int64_t B = ((int)ci < half) ? P : Q;
                const int k = (int)ci % half;
                for (int j = 0; j < kRingC - 1; ++j) {
                    const int64_t a = B * kRingC + rr_player(k, j, kRingC);
                    const int64_t b = B * kRingC + rr_player(kRingC - 1 - k, j, kRingC);
                    local += jacobi_pair_global(X, V, n, a, b, tol2, red, &par[0][0]);
                    cluster_sync_all();
                }
            }
            if (ot > 0) {
                // the two columns this CTA loads were stored at the previous outer
                // step by CTAs of other clusters: wait for their versions
                __shared__ int s_late;
                if (tid == 0) {
                    const int64_t a = P * kRingC + ci, b = Q * kRingC + ci;
                    const long long t0 = clock64();
                    int late = 0;
                    while (ld_acquire_u32(colver + a) < ostep || ld_acquire_u32(colver + b) < ostep) {
                        if (s_abort || clock64() - t0 > (1ll << 32)) {
                            late = 1;
                            break;
                        }
                    }
                    s_late = late;
                }
                __syncthreads();
                if (s_late && !s_abort) {
                    s_abort = 1;
                    set_status(status, NS_ERR_TIMEOUT);
                }
            }
            if (tid == 0)
                for (int j = 1; j < kRingC; ++j) {
                    mbar_arm(&mbx[j], (uint32_t)(kRingT * sizeof(double2)));
                    mbar_arm(&mbv[j], (uint32_t)(kRingT * sizeof(double2)));
                    mbar_arm(&mbs[j], (uint32_t)sizeof(double2));
                }
            const uint32_t parity = ostep & 1u;
            const int64_t cp = P * kRingC + ci, cq0 = Q * kRingC + ci;
            const int64_t cq = Q * kRingC + (ci + kRingC - 1) % kRingC;  // Q column held after the last round
            const bool lp = cp < n, lq = cq0 < n;
            double p0 = (r0 && lp) ? __ldcg(M + i0 + cp * n) : 0.0, p1 = (r1 && lp) ? __ldcg(M + i1 + cp * n) : 0.0;
            double q0 = (r0 && lq) ? __ldcg(M + i0 + cq0 * n) : 0.0, q1 = (r1 && lq) ? __ldcg(M + i1 + cq0 * n) : 0.0;
            if (scalar) {
                // The scales of the held columns, one per lane (x = d x~, e = 1/d):
                // lane 0 d_P, lane 1 d_Q, lane 2 e_P, lane 3 e_Q.  A warp
                // instruction costs the FP64 pipe the same for one lane as for
                // four, so independent scalar steps share instructions.  The Q
                // column's scales arrive after its entries, on their own mbarrier.
                const int lane = tid;
                double sv = 1.0;
                for (int j = 0; j < kRingC; ++j) {
                    if (j > 0) {
                        if (!s_abort && !ring_wait(shared_addr(&mbs[j]), parity) && lane == 0) {
                            s_abort = 1;
                            set_status(status, NS_ERR_TIMEOUT);
                        }
                        const double2 sc = sbuf[j];
                        if (lane == 1) sv = sc.x;
                        if (lane == 3) sv = sc.y;
                    }
                    // before the sums arrive: d_Q e_P (lane 0, for mu), d_P e_Q
                    // (lane 1, for nu) and the FP32 images of the scales
                    double dP = __shfl_sync(0xffffffffu, sv, 0), dQ = __shfl_sync(0xffffffffu, sv, 1);
                    const double ee = __shfl_sync(0xffffffffu, sv, lane == 0 ? 2 : 3);
                    double rr = (lane == 0 ? dQ : dP) * ee;
                    float fP = f32_image(dP, 0), fQ = f32_image(dQ, 0);
                    // computed here, before the barrier, not after it on the critical path
                    asm volatile("" : "+d"(rr), "+d"(dP), "+d"(dQ), "+f"(fP), "+f"(fQ));
                    xbar();  // the row warps' sums of round j are in rg, rab, rexp
                    // lanes 0-3 hold row warp w = lane; sums in the order (w0 + w1) + (w2 + w3)
                    RingSums rs;
                    {
                        const bool lw = lane < 4;
                        const double gw = lw ? rg[lane] : 0.0;
                        const float2 abw = lw ? rab[lane] : make_float2(0.0f, 0.0f);
                        const uint32_t ew = lw ? rexp[lane] : 0u;
                        uint32_t em = __vmaxu2(ew, __shfl_xor_sync(0xffffffffu, ew, 1));
                        em = __vmaxu2(em, __shfl_xor_sync(0xffffffffu, em, 2));
                        const int Ea = (int)(em >> 16), Eb = (int)(em & 0xFFFFu);
                        float fa = abw.x * pow2f(2 * ((int)(ew >> 16) - Ea));
                        float fb = abw.y * pow2f(2 * ((int)(ew & 0xFFFFu) - Eb));
                        double gs = gw + __shfl_xor_sync(0xffffffffu, gw, 1);
                        fa += __shfl_xor_sync(0xffffffffu, fa, 1);
                        fb += __shfl_xor_sync(0xffffffffu, fb, 1);
                        gs += __shfl_xor_sync(0xffffffffu, gs, 2);
                        fa += __shfl_xor_sync(0xffffffffu, fa, 2);
                        fb += __shfl_xor_sync(0xffffffffu, fb, 2);
                        rs.g = __shfl_sync(0xffffffffu, gs, 0);
                        rs.fa = __shfl_sync(0xffffffffu, fa, 0);
                        rs.fb = __shfl_sync(0xffffffffu, fb, 0);
                        rs.Ea = __shfl_sync(0xffffffffu, Ea, 0);
                        rs.Eb = __shfl_sync(0xffffffffu, Eb, 0);
                    }
                    double tn = 0.0;
                    bool exact = false;
                    const bool rot = ring_angle(rs, tol2, fP * fP, fQ * fQ, fP * fQ, dP, dQ, &tn, &exact);
                    if (exact) {  // (rare; uniform over the warp) the angle from FP64 norms
                        if (lane == 0) par[j][0] = 2.0;  // the request to the X row warps
                        __syncwarp();
                        xbar();  // the request is visible
                        xbar();  // their FP64 squared norms are in rn
                        const double at = (rn[0].x + rn[1].x) + (rn[2].x + rn[3].x);
                        const double bt = (rn[0].y + rn[1].y) + (rn[2].y + rn[3].y);
                        tn = exact_tan((dQ * dQ) * bt - (dP * dP) * at, 2.0 * (dP * dQ) * rs.g, tn);
                    }
                    const double mn = tn * rr;  // lane 0: mu (x~_p -= mu x~_q), lane 1: nu (x~_q += nu x~_p)
                    if (lane < 2) par[j][1 + lane] = rot ? mn : 0.0;
                    if (lane == 0) par[j][0] = rot ? 1.0 : 0.0;
                    __syncwarp();
                    if (lane == 0)
                        asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(shared_addr(&mbr[j]))
                                     : "memory");
                    xbar();  // par[j] is visible to the X row warps
                    // the scale update waits for the X rows' sends, like the V warps
                    asm volatile("bar.sync 2, %0;" ::"n"(kRingXV) : "memory");
                    if (rot) {  // new scales: d <- c d, e <- e / c, c = (1 + t^2)^(-1/2)
                        ++local;
                        const double u = tn * tn;
                        double m;
                        if (u < 0x1p-12) {
                            // binomial series to u^4 (the next term is below 2^-62):
                            // (1 + u)^(-1/2) in lanes 0-1, (1 + u)^(1/2) in lanes 2-3
                            const bool cl = lane < 2;
                            double q = cl ? 35.0 / 128.0 : -5.0 / 128.0;
                            q = fma(u, q, cl ? -5.0 / 16.0 : 1.0 / 16.0);
                            q = fma(u, q, cl ? 3.0 / 8.0 : -1.0 / 8.0);
                            q = fma(u, q, cl ? -0.5 : 0.5);
                            m = fma(u, q, 1.0);
                        } else {  // FP32 seed and two Newton steps for the inverse square root
                            const double tt = 1.0 + u, h = -0.5 * tt;
                            double c = f64_of(rsqrtf(f32_image(tt, 0)));
                            c = c * fma(h, c * c, 1.5);
                            c = c * fma(h, c * c, 1.5);
                            m = (lane < 2) ? c : tt * c;
                        }
                        sv *= m;
                    }
                    if (j < kRingC - 1) {
                        const double sQ = __shfl_sync(0xffffffffu, sv, 1), eQ = __shfl_sync(0xffffffffu, sv, 3);
                        if (lane == 0)
                            send_pair(sb_peer + (uint32_t)((j + 1) * sizeof(double2)), sQ, eQ,
                                      ms_peer + (uint32_t)((j + 1) * 8));
                    }
                }
                const double fPs = __shfl_sync(0xffffffffu, sv, 0), fQs = __shfl_sync(0xffffffffu, sv, 1);
                if (lane == 0) {  // final scales of the held columns
                    s_fin[0] = fPs;
                    s_fin[1] = fQs;
                    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(shared_addr(&mbf))
                                 : "memory");
                }
            } else {
                for (int j = 0; j < kRingC; ++j) {
                    if (isx) {
                        if (j > 0) {
                            if (!s_abort && !ring_wait(shared_addr(&mbx[j]), parity)) {
                                s_abort = 1;
                                set_status(status, NS_ERR_TIMEOUT);
                            }
                            const double2 in = xbuf[j][t];
                            q0 = in.x;
                            q1 = in.y;
                        }
                        // FP32 images at the warp's largest exponent of each column (the
                        // largest entry lands in [1, 2)), FP64 inner product
                        uint32_t e2 = (max(exp_field(p0), exp_field(p1)) << 16) | max(exp_field(q0), exp_field(q1));
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) e2 = __vmaxu2(e2, __shfl_xor_sync(0xffffffffu, e2, o));
                        const int sp = (int)(e2 >> 16) - 1023, sq = (int)(e2 & 0xFFFFu) - 1023;
                        const float a0 = f32_image(p0, sp), a1 = f32_image(p1, sp);
                        const float b0 = f32_image(q0, sq), b1 = f32_image(q1, sq);
                        float fa = fmaf(a1, a1, a0 * a0), fb = fmaf(b1, b1, b0 * b0);
                        double gg = fma(p1, q1, p0 * q0);
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {  // every lane ends with the same sums
                            gg += __shfl_xor_sync(0xffffffffu, gg, o);
                            fa += __shfl_xor_sync(0xffffffffu, fa, o);
                            fb += __shfl_xor_sync(0xffffffffu, fb, o);
                        }
                        if ((t & 31) == 0) {
                            rg[t >> 5] = gg;
                            rab[t >> 5] = make_float2(fa, fb);
                            rexp[t >> 5] = e2;
                        }
                        xbar();  // sums to the scalar warp
                        xbar();  // par[j] from the scalar warp, or its request for FP64 norms
                        if (par[j][0] == 2.0) {
                            double a2 = fma(p1, p1, p0 * p0), b2 = fma(q1, q1, q0 * q0);
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) {
                                a2 += __shfl_xor_sync(0xffffffffu, a2, o);
                                b2 += __shfl_xor_sync(0xffffffffu, b2, o);
                            }
                            if ((t & 31) == 0) rn[t >> 5] = make_double2(a2, b2);
                            xbar();  // norms to the scalar warp
                            xbar();  // the final par[j]
                        }
                    } else {
                        if (!s_abort && !ring_wait_cta(shared_addr(&mbr[j]), parity)) {
                            s_abort = 1;
                            set_status(status, NS_ERR_TIMEOUT);
                        }
                        if (j > 0) {
                            if (!s_abort && !ring_wait(shared_addr(&mbv[j]), parity)) {
                                s_abort = 1;
                                set_status(status, NS_ERR_TIMEOUT);
                            }
                            const double2 in = vbuf[j][t];
                            q0 = in.x;
                            q1 = in.y;
                        }
                    }
                    // the Q half first: it is what the neighbour waits for.  The V
                    // warps start after the X warps have sent their Q rows, so the
                    // X updates, on the critical path, do not queue behind the V
                    // updates for the shared FP64 pipe.
                    const bool rj = par[j][0] != 0.0;
                    const double mu = par[j][1], nu = par[j][2];
                    const double oq0 = q0, oq1 = q1;
                    if (!isx) asm volatile("bar.sync 2, %0;" ::"n"(kRingXV) : "memory");
                    if (rj) {
                        q0 = fma(nu, p0, q0);
                        q1 = fma(nu, p1, q1);
                    }
                    if (j < kRingC - 1) {
                        const uint32_t off = (uint32_t)(((j + 1) * kRingT + t) * sizeof(double2));
                        if (isx) send_pair(xb_peer + off, q0, q1, mx_peer + (uint32_t)((j + 1) * 8));
                        else send_pair(vb_peer + off, q0, q1, mv_peer + (uint32_t)((j + 1) * 8));
                    }
                    if (isx) asm volatile("bar.arrive 2, %0;" ::"n"(kRingXV) : "memory");
                    if (rj) {
                        p0 = fma(-mu, oq0, p0);
                        p1 = fma(-mu, oq1, p1);
                    }
                }
                if (!s_abort && !ring_wait_cta(shared_addr(&mbf), parity)) {
                    s_abort = 1;
                    set_status(status, NS_ERR_TIMEOUT);
                }
                // unscale and store the held columns (P and the last Q)
                const double fP = s_fin[0], fQ = s_fin[1];
                if (lp) {
                    if (r0) M[i0 + cp * n] = p0 * fP;
                    if (r1) M[i1 + cp * n] = p1 * fP;
                }
                if (cq < n) {
                    if (r0) M[i0 + cq * n] = q0 * fQ;
                    if (r1) M[i1 + cq * n] = q1 * fQ;
                }
            }
            ++ostep;
            if (ot < nouter - 1) {
                // publish this CTA's two stored columns (version = outer steps done)
                __syncthreads();
                if (tid == 0) {
                    const int64_t a = P * kRingC + ci, b = Q * kRingC + (ci + kRingC - 1) % kRingC;
                    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(colver + a), "r"(ostep) : "memory");
                    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(colver + b), "r"(ostep) : "memory");
                }
            } else {
                if (tid == 0 && local) atomicAdd(rotcount + sweep, local);
                if (!grid_sync(bar)) {  // end of the sweep: rotation count, every column stored
                    ok = false;
                    break;
                }
            }
        }
        if (!ok) break;
        prev_rot = *(volatile unsigned int *)(rotcount + sweep);
        converged = (prev_rot == 0u);
    }
    if (ok) {
        if (!converged && blockIdx.x == 0 && tid == 0) set_status(status, NS_ERR_NOCONV);
        jacobi_record_stats(rotcount, full_sweeps, check_passes, kRingC);
        if (grid_sync(bar)) jacobi_sigma(X, n, sigma);
    }
    cluster_sync_all();  // no CTA leaves while a peer may still address its shared memory
}

// --------------------------------------------- V = P Q2 Vx (no barriers) ----
// Q2 = H_0 H_1 ... H_{n-1} (reflectors of the QR of L = R^T: u = [u0[j];
// L[j+1:n, j]], coefficient cf[j]); column c of Q2 Vx is H_0 (... (H_{n-1} vx_c)).
// Row i of that product is row perm[i] of V.
__global__ void __launch_bounds__(kDenseThreads) apply_q2_kernel(const double *__restrict__ Lq,
                                                                 const double *__restrict__ u0,
                                                                 const double *__restrict__ cf,
                                                                 const int32_t *__restrict__ perm,
                                                                 const double *__restrict__ Vx, int64_t n,
                                                                 double *__restrict__ V) {
    extern __shared__ double col[];  // n
    __shared__ double red[32];
    __shared__ double fsh;
    const int tid = threadIdx.x;
    for (int64_t c = blockIdx.x; c < n; c += gridDim.x) {
        for (int64_t i = tid; i < n; i += blockDim.x) col[i] = Vx[i + c * n];
        __syncthreads();
        for (int64_t j = n - 1; j >= 0; --j) {
            const double coef = cf[j];
            if (coef == 0.0) continue;
            const double *v = Lq + j * n;
            const double ua = u0[j];
            double w[1] = {0.0};
            for (int64_t i = j + tid; i < n; i += blockDim.x) w[0] = fma(i == j ? ua : v[i], col[i], w[0]);
            block_sum_t0<1>(w, red);
            if (tid == 0) fsh = coef * w[0];
            __syncthreads();
            const double f = fsh;
            for (int64_t i = j + tid; i < n; i += blockDim.x) col[i] = fma(-f, i == j ? ua : v[i], col[i]);
            __syncthreads();
        }
        for (int64_t i = tid; i < n; i += blockDim.x) V[perm[i] + c * n] = col[i];
        __syncthreads();
    }
}

// ----------------------------------------------------------- extraction ----
// Order by non-increasing sigma (ties: lower index first); W = the last k
// columns; each returned column is signed so its entry of largest magnitude
// (lowest index on ties) is positive.  One CTA per returned column.
__global__ void __launch_bounds__(kDenseThreads) extract_kernel(const double *V, const double *sigma, int64_t n,
                                                               int32_t k, double *Vk, double *sigk) {
    extern __shared__ long long skey[];  // n: sigma as ordered integer keys
    __shared__ int src_sh;
    __shared__ long long bestk[32];
    __shared__ int besti[32];
    const int tid = threadIdx.x;
    const int64_t col = blockIdx.x;  // output column
    const int64_t want = (n - k) + col;  // rank of the wanted singular value
    if (tid == 0) src_sh = -1;
    // sigma >= 0 orders like its bit pattern (NaN above every number), so the
    // ranks are integer compares
    for (int64_t i = tid; i < n; i += blockDim.x) skey[i] = __double_as_longlong(sigma[i]);
    __syncthreads();
    for (int64_t i = tid; i < n; i += blockDim.x) {
        const long long si = skey[i];
        int64_t r = 0;
        for (int64_t j = 0; j < n; ++j) {
            const long long sj = skey[j];
            r += (sj > si || (sj == si && j < i)) ? 1 : 0;
        }
        if (r == want) src_sh = (int)i;
    }
    __syncthreads();
    const int64_t src = src_sh;
    const double *v = V + src * n;
    long long bk = -1;
    int bi = 0;
    for (int64_t i = tid; i < n; i += blockDim.x) {
        const long long kk = abs_key(v[i]);
        if (kk > bk) {
            bk = kk;
            bi = (int)i;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ok > bk || (ok == bk && oi < bi)) {
            bk = ok;
            bi = oi;
        }
    }
    if ((tid & 31) == 0) {
        bestk[tid >> 5] = bk;
        besti[tid >> 5] = bi;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (bestk[w] > bestk[0] || (bestk[w] == bestk[0] && besti[w] < besti[0])) {
                bestk[0] = bestk[w];
                besti[0] = besti[w];
            }
    }
    __syncthreads();
    const double sg = (v[besti[0]] < 0.0) ? -1.0 : 1.0;
    for (int64_t i = tid; i < n; i += blockDim.x) Vk[i + col * n] = sg * v[i];
    if (tid == 0) sigk[col] = sigma[src];
}

// The tolerance version of Algorithm 1 (Section 2, after Algorithm 1): W =
// the right singular vectors whose singular values are below eps.  Vs, ss
// hold all n extracted columns (extract_kernel with k = n: non-increasing
// sigma, signed), so those are the last k = #{sigma < eps}; they go to
// columns 0..k-1 of Vk in the same order, and k to *dev_k.
__global__ void __launch_bounds__(kDenseThreads) eps_select_kernel(const double *__restrict__ Vs,
                                                                  const double *__restrict__ ss, int64_t n,
                                                                  double eps, double *__restrict__ Vk,
                                                                  double *__restrict__ sigk, int32_t *dev_k) {
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    int c = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) c += (ss[i] < eps) ? 1 : 0;
    atomicAdd(&s_cnt, c);  // an integer count: the order of the adds does not matter
    __syncthreads();
    const int64_t k = s_cnt;
    if (blockIdx.x == 0 && threadIdx.x == 0) *dev_k = (int32_t)k;
    for (int64_t col = blockIdx.x; col < k; col += gridDim.x) {
        const int64_t src = n - k + col;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) Vk[i + col * n] = Vs[i + src * n];
        if (threadIdx.x == 0) sigk[col] = ss[src];
    }
}


__global__ void copy_kernel(const double *__restrict__ a, int64_t len, double *__restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

static int sm_count() { return device_sm_count(); }

// ------------------------------------------- failure-detection test hook ----
// Runs one of the library's bounded waits on something nothing completes, so
// the wait runs out: the kernel writes NS_ERR_TIMEOUT and returns, and the
// stream stays usable.  Used by the tests only (ns_test_bounded_wait).
//
// Grid barrier: two CTAs; CTA 1 leaves without arriving, CTA 0 polls the
// barrier word `limit` times.
__global__ void test_grid_wait_kernel(GridBarrier bar) {
    if (blockIdx.x != 0) return;
    grid_sync(bar);
}

// Cluster-peer wait: a cluster of two CTAs; CTA 0 waits for phase 0 of a local
// mbarrier that only CTA 1 could complete (as a ring neighbour completes a
// slot), for `limit` clock cycles.  Both CTAs then meet at the final cluster
// barrier, as the ring kernel's CTAs do after an abandoned wait.
__global__ void __cluster_dims__(2, 1, 1) test_cluster_wait_kernel(int32_t *status, long long limit) {
    __shared__ __align__(8) unsigned long long mb;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(shared_addr(&mb)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster_sync_all();
    if (cluster_rank() == 0 && threadIdx.x == 0) {
        if (!ring_wait(shared_addr(&mb), 0u, limit)) set_status(status, NS_ERR_TIMEOUT);
    }
    __syncwarp();
    cluster_sync_all();
}

cudaError_t launch_test_wait(int which, long long limit, int32_t *status, unsigned int *word, cudaStream_t st) {
    if (which == 0) {
        cudaError_t e = cudaMemsetAsync(word, 0, sizeof(unsigned int), st);
        if (e != cudaSuccess) return e;
        GridBarrier bar{word, status, limit};
        test_grid_wait_kernel<<<2, 32, 0, st>>>(bar);
        return cudaGetLastError();
    }
    test_cluster_wait_kernel<<<2, 32, 0, st>>>(status, limit);
    return cudaGetLastError();
}

cudaError_t launch_dense_select_eps(const DenseWork &w, int64_t n, double eps, double *Vk, double *sigk,
                                    int32_t *dev_k, cudaStream_t st) {
    // all n columns in order into X (free after the iteration), their sigma into L
    extract_kernel<<<(unsigned)n, kDenseThreads, sizeof(long long) * (size_t)n, st>>>(w.W, w.sigma, n, (int32_t)n, w.X,
                                                                                      w.L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t blocks = n < sm_count() * 4 ? n : sm_count() * 4;
    eps_select_kernel<<<(unsigned)blocks, kDenseThreads, 0, st>>>(w.X, w.L, n, eps, Vk, sigk, dev_k);
    return cudaGetLastError();
}

template <int RPT>
static cudaError_t launch_jacobi(const DenseWork &w, int64_t n, GridBarrier bar, int32_t *status, int vinit,
                                 int max_sweeps, cudaStream_t st) {
    const int64_t npairs = (n + (n & 1)) / 2;
    int64_t G = npairs < sm_count() ? npairs : sm_count();
    if (G < 1) G = 1;
    double *X = w.X, *V = w.V, *sigma = w.sigma;
    int64_t n_ = n;
    double tol = (double)n * std::ldexp(1.0, -53);
    unsigned int *rot = w.bar + 64, *chk = w.bar + 64 + 64;
    int32_t *status_ = status;
    int vinit_ = vinit, ms_ = max_sweeps;
    void *args[] = {&X, &V, &n_, &tol, &bar, &rot, &chk, &sigma, &status_, &vinit_, &ms_};
    return cudaLaunchCooperativeKernel((const void *)jacobi_coop_kernel<RPT>, (int)G, kDenseThreads, args, 0, st);
}

// The ring Jacobi (cluster size C fixed at compile time) needs its G clusters,
// 2 G C >= n columns, resident at once: a cooperative launch.  Returns without
// launching (*used = false) when the device cannot hold them or rejects the
// launch.
static size_t ring_smem(int C) { return (size_t)2 * C * kRingT * sizeof(double2); }

template <int C>
static cudaError_t launch_ring_c(const DenseWork &w, int64_t n, GridBarrier bar, int32_t *status, int vinit,
                                 int max_sweeps, const unsigned int *fp32_ran, cudaStream_t st, bool *used) {
    static int state[64] = {0};  // per device: 0 unknown, 1 usable, -1 not usable
    *used = false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaSuccess;
    if (state[dev] < 0) return cudaSuccess;
    int64_t G = (n + 2 * C - 1) / (2 * C);
    if (G < 1) G = 1;
    const size_t dyn = ring_smem(C);
    if ((C > 8 && cudaFuncSetAttribute(jacobi_ring_kernel<C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                      cudaSuccess) ||
        cudaFuncSetAttribute(jacobi_ring_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) !=
            cudaSuccess) {
        cudaGetLastError();
        state[dev] = -1;
        return cudaSuccess;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(G * C), 1, 1);
    cfg.blockDim = dim3(kRingCta, 1, 1);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 0;
    int maxc = 0;
    if (cudaOccupancyMaxActiveClusters(&maxc, (void *)jacobi_ring_kernel<C>, &cfg) != cudaSuccess || maxc < G) {
        cudaGetLastError();
        return cudaSuccess;
    }
    cfg.numAttrs = 1;
    double *X = w.X, *V = w.V, *sigma = w.sigma;
    unsigned int *rot = w.bar + 64, *chk = w.bar + 64 + 64;
    const double tol = (double)n * std::ldexp(1.0, -53);
    unsigned int *colver = w.colver;
    cudaError_t e = cudaMemsetAsync(colver, 0, sizeof(unsigned int) * (size_t)(n + 32), st);
    if (e != cudaSuccess) return e;
    e = cudaLaunchKernelEx(&cfg, jacobi_ring_kernel<C>, X, V, n, G, tol, bar, rot, chk, sigma, colver, status,
                           vinit, max_sweeps, fp32_ran);
    if (e != cudaSuccess) {
        cudaGetLastError();
        state[dev] = -1;
        return cudaSuccess;
    }
    state[dev] = 1;
    *used = true;
    return cudaSuccess;
}

static cudaError_t launch_jacobi_ring(const DenseWork &w, int64_t n, GridBarrier bar, int32_t *status, int vinit,
                                      int max_sweeps, const unsigned int *fp32_ran, cudaStream_t st, bool *used) {
    if (n > 2 * 15 * 8) {  // 16 clusters of 8 would share SMs: try clusters of 16
        const cudaError_t e = launch_ring_c<16>(w, n, bar, status, vinit, max_sweeps, fp32_ran, st, used);
        if (e != cudaSuccess || *used) return e;
    }
    return launch_ring_c<8>(w, n, bar, status, vinit, max_sweeps, fp32_ran, st, used);
}

template <int NB>
static cudaError_t launch_hqr_nb(double *W, int64_t rows, int64_t cols, int pivot, double *u0, double *cf,
                                 int32_t *perm, unsigned long long *pivslot, double *Rout, GridBarrier bar, int64_t G,
                                 cudaStream_t st) {
    const int64_t nown = (cols + G - 1) / G;
    const size_t smem = sizeof(double) * (size_t)(rows + 2 * nown);
    cudaError_t e =
        cudaFuncSetAttribute(hqr_coop_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {&W, &rows, &cols, &pivot, &u0, &cf, &perm, &pivslot, &Rout, &bar};
    return cudaLaunchCooperativeKernel((const void *)hqr_coop_kernel<NB>, (int)G, kDenseThreads, args, smem, st);
}

// Pipelined QR (no pivoting) when the owned columns fit in shared memory;
// returns false (nothing launched) otherwise.
static size_t pipe_smem(int64_t rows, int64_t cols) {
    int64_t G = cols < sm_count() ? cols : sm_count();
    if (G < 1) G = 1;
    const int64_t nown = (cols + G - 1) / G;
    return sizeof(double) * (size_t)(nown * rows + 2 * rows + nown);
}
static bool pipe_fits(int64_t rows, int64_t cols) { return pipe_smem(rows, cols) <= 200 * 1024 && cols <= 4096; }

static bool launch_hqr_pipe(const double *W, double *U, int64_t rows, int64_t cols, double *u0, double *cf,
                            unsigned long long *flags, double *Rout, int32_t *status, cudaStream_t st,
                            cudaError_t *err) {
    int64_t G = cols < sm_count() ? cols : sm_count();
    if (G < 1) G = 1;
    const int64_t nown = (cols + G - 1) / G;
    const size_t smem = pipe_smem(rows, cols);
    if (!pipe_fits(rows, cols)) return false;
    *err = cudaMemsetAsync(flags, 0xFF, sizeof(unsigned long long) * (size_t)cols, st);  // kPipeEmpty
    if (*err != cudaSuccess) return true;
    const int64_t steps = rows < cols ? rows : cols;
    *err = cudaMemsetAsync(U, 0xFF, sizeof(double) * (size_t)(rows * steps), st);  // kPipeEmpty
    if (*err != cudaSuccess) return true;
    *err = cudaFuncSetAttribute(hqr_pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (*err != cudaSuccess) return true;
    int64_t nown_ = nown;
    void *args[] = {&W, &U, &rows, &cols, &nown_, &u0, &cf, &flags, &Rout, &status};
    *err = cudaLaunchCooperativeKernel((const void *)hqr_pipe_kernel, (int)G, kPipeThreads, args, smem, st);
    return true;
}

// The fused two-QR launch (hqr_fused_kernel): both QRs on the pipelined path,
// n <= 256 (the warp-level applications hold 8 rows per lane).  The CTAs are
// split in proportion to the two QRs' work per reflector (s n against 2 n^2).
struct FusedGeom {
    int G1, G2;
    int64_t nown1, nown2;
    size_t smem;
};
static bool fused_geom(int64_t s, int64_t n, FusedGeom *g) {
    if (n < 2 || n > 32 * kQ2Lane || s < n || !pipe_fits(s, n) || !pipe_fits(n, 2 * n)) return false;
    const int64_t G = sm_count();
    // columns per first-QR CTA for a split in proportion to the work per
    // reflector (s n against 2 n^2), then the fewest CTAs with that many: the
    // second QR, whose CTAs also catch columns up, gets the rest
    const int64_t per1 = (n * (s + 2 * n) + G * s - 1) / (G * s);
    int64_t G1 = (n + per1 - 1) / per1;
    const int64_t g2min = (2 * n + kQ2MaxOwn - 1) / kQ2MaxOwn;
    if (G1 > n) G1 = n;
    if (G1 > G - g2min) G1 = G - g2min;
    if (G1 < 1) return false;
    int64_t G2 = G - G1;
    if (G2 > 2 * n) G2 = 2 * n;
    g->G1 = (int)G1;
    g->G2 = (int)G2;
    g->nown1 = (n + G1 - 1) / G1;
    g->nown2 = (2 * n + G2 - 1) / G2;
    if (g->nown2 > kQ2MaxOwn) return false;
    const int64_t d1 = g->nown1 * s + 2 * s + g->nown1, d2 = g->nown2 * n + 2 * n + g->nown2;
    g->smem = sizeof(double) * (size_t)(d1 > d2 ? d1 : d2);
    return g->smem <= 200 * 1024;
}

// Both QRs of the dense stage in one launch: W (s x n, ordered) -> R2 and Q2^T
// in Rout2 = [R2 | Q2^T] (n x 2n).  Scratch: U1 (s x n), flag1 (n), Lg (n x n),
// rowcnt (n words), U2 (n x n), flag2 (n).
static cudaError_t launch_hqr_fused(const FusedGeom &g, const double *W, double *U1, int64_t s, int64_t n,
                                    double *u0a, double *cfa, unsigned long long *flag1, double *Lg,
                                    unsigned int *rowcnt, double *U2, double *u0b, double *cfb,
                                    unsigned long long *flag2, double *Rout2, int32_t *status, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(flag1, 0xFF, sizeof(unsigned long long) * (size_t)n, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(U1, 0xFF, sizeof(double) * (size_t)(s * n), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(flag2, 0xFF, sizeof(unsigned long long) * (size_t)n, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(U2, 0xFF, sizeof(double) * (size_t)(n * n), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(rowcnt, 0, sizeof(unsigned int) * (size_t)n, st)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(hqr_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem)) !=
        cudaSuccess)
        return e;
    int64_t s_ = s, n_ = n, nown1 = g.nown1, nown2 = g.nown2;
    int G1 = g.G1;
    void *args[] = {&W,  &U1,     &s_, &n_,    &nown1, &u0a, &cfa,   &flag1, &Lg,    &rowcnt,
                    &U2, &nown2,  &u0b, &cfb,  &flag2, &Rout2, &G1, &status};
    return cudaLaunchCooperativeKernel((const void *)hqr_fused_kernel, g.G1 + g.G2, kPipeThreads, args, g.smem, st);
}

static cudaError_t launch_hqr(double *W, int64_t rows, int64_t cols, int pivot, double *u0, double *cf,
                              int32_t *perm, unsigned long long *pivslot, double *Rout, GridBarrier bar,
                              cudaStream_t st) {
    int64_t G = cols < sm_count() ? cols : sm_count();
    if (G < 1) G = 1;
    cudaError_t e = cudaMemsetAsync(pivslot, 0, sizeof(unsigned long long) * (size_t)(cols + 1), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(bar.word, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const int64_t nown = (cols + G - 1) / G;
    if (nown <= 1) return launch_hqr_nb<1>(W, rows, cols, pivot, u0, cf, perm, pivslot, Rout, bar, G, st);
    if (nown <= 2) return launch_hqr_nb<2>(W, rows, cols, pivot, u0, cf, perm, pivslot, Rout, bar, G, st);
    if (nown <= 4) return launch_hqr_nb<4>(W, rows, cols, pivot, u0, cf, perm, pivslot, Rout, bar, G, st);
    return launch_hqr_nb<8>(W, rows, cols, pivot, u0, cf, perm, pivslot, Rout, bar, G, st);
}

__global__ void dense_stats_kernel(const unsigned int *bar, int64_t *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        out[0] = bar[64 + 128];
        out[1] = bar[64 + 129];
        out[2] = bar[64 + 130];
        out[3] = bar[64 + 131];
        out[4] = bar[kJ32Ctl] ? bar[kJ32Ctl + 1] : 0;  // FP32-phase sweeps (0: the phase did not run)
        out[5] = bar[kJ32Ctl] ? bar[kJ32Ctl + 2] : 0;  // FP32-phase rotations
        // completions that formed the K^4 and K^6 terms; convergence test ran on the Gram matrix
        out[6] = bar[kJ32Ctl] ? (int64_t)bar[kJ32Ctl + 5] + (int64_t)bar[kJ32Ctl + 11] : 0;
        out[7] = (bar[kJ32Ctl] && bar[kJ32Ctl + 3] == 2u) ? 1 : 0;
    }
}

cudaError_t launch_dense_stats(const DenseWork &w, int64_t *out, cudaStream_t st) {
    dense_stats_kernel<<<1, 32, 0, st>>>(w.bar, out);
    return cudaGetLastError();
}

cudaError_t launch_dense_solve(const double *SA, int64_t s, int64_t n, int32_t k, const DenseWork &w, double *Vk,
                               double *sigk, double *save_V, double *save_sigma, int32_t *status, cudaStream_t st,
                               int max_sweeps, bool fp32_phase, cudaEvent_t after_qr) {
    cudaError_t e = cudaSuccess;
    if (max_sweeps <= 0 || max_sweeps > kMaxSweeps) max_sweeps = kMaxSweeps;
    GridBarrier bar{w.bar, status};
    double *u0a = w.tau, *cfa = w.tau + n, *u0b = w.tau + 2 * n, *cfb = w.tau + 3 * n;
    // 1. SA P = Q1 R; R (n x n) lands in X.  Pipelined after a static ordering
    // of the columns by decreasing norm when it fits, else barrier-separated
    // with column pivoting.
    unsigned long long *flags = w.pivslot;  // n + 1 words >= n flags
    bool fused = false;
    if (pipe_fits(s, n)) {
        double *key = w.X;  // n doubles; X is free until the QR writes R
        colnorm_kernel<<<(unsigned)(n < 1024 ? n : 1024), 256, 0, st>>>(SA, s, n, key);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        int64_t np2 = 1;
        while (np2 < n) np2 <<= 1;
        const size_t sort_smem = (size_t)np2 * (sizeof(double) + sizeof(int32_t));
        e = cudaFuncSetAttribute(sort_perm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem);
        if (e != cudaSuccess) return e;
        sort_perm_kernel<<<1, 1024, sort_smem, st>>>(key, n, np2, w.perm);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        dim3 grid((unsigned)((s + 255) / 256 < 8 ? (s + 255) / 256 : 8), (unsigned)(n < 1024 ? n : 1024));
        permute_cols_kernel<<<grid, 256, 0, st>>>(SA, s, n, w.perm, w.W);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        FusedGeom fg;
        if (fused_geom(s, n, &fg)) {
            // both QRs in one launch: [R2 | Q2^T] lands in R2 (Lg in L, U2 in X,
            // the second QR's flags in sigma, row counts in colver)
            e = launch_hqr_fused(fg, w.W, w.U, s, n, u0a, cfa, flags, w.L, w.colver, w.X, u0b, cfb,
                                 reinterpret_cast<unsigned long long *>(w.sigma), w.R2, status, st);
            fused = (e == cudaSuccess);
            if (e != cudaSuccess) return e;
        } else {
            launch_hqr_pipe(w.W, w.U, s, n, u0a, cfa, flags, w.X, status, st, &e);
        }
    } else {
        e = cudaMemcpyAsync(w.W, SA, sizeof(double) * (size_t)(s * n), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        e = launch_hqr(w.W, s, n, 1, u0a, cfa, w.perm, w.pivslot, w.X, bar, st);
    }
    if (e != cudaSuccess) return e;
    // 2. QR of L = R^T without pivoting.  On the pipelined path L carries the
    // identity as n more columns, [R^T | I]: the reflectors applied to them
    // give Q2^T beside R2, so V starts as Q2 and the Jacobi rotations
    // accumulate Q2 Vx directly.  Otherwise (barrier-separated QR) Q2 is
    // applied to Vx afterwards.
    const dim3 ttb(32, 8), tgrid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
    const unsigned nn_blocks = (unsigned)((n * n + 255) / 256);
    if (!fused) {
        transpose_kernel<<<tgrid, ttb, 0, st>>>(w.X, n, w.L);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const bool q2_in_v = fused || pipe_fits(n, 2 * n);
    const double *Lq = w.L;  // reflectors of the second QR (barrier-separated path)
    if (q2_in_v) {
        if (!fused) {
            identity_kernel<<<nn_blocks, 256, 0, st>>>(w.L + n * n, n);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            launch_hqr_pipe(w.L, w.U, n, 2 * n, u0b, cfb, flags, w.R2, status, st, &e);
            if (e != cudaSuccess) return e;
        }
        // 3. X = R2^T, V = (Q2^T)^T
        r2t_kernel<<<nn_blocks, 256, 0, st>>>(w.R2, n, w.X);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        transpose_kernel<<<tgrid, ttb, 0, st>>>(w.R2 + n * n, n, w.V);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
        int32_t *perm2 = (int32_t *)w.sigma;  // identity permutation of the unpivoted QR (unused)
        e = launch_hqr(w.L, n, n, 0, u0b, cfb, perm2, w.pivslot, w.V, bar, st);
        if (e != cudaSuccess) return e;
        // 3. X = R2^T (R2 landed in V)
        r2t_kernel<<<nn_blocks, 256, 0, st>>>(w.V, n, w.X);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // Jacobi on X; V receives Q2 Vx (pipelined path) or Vx
    e = cudaMemsetAsync(w.bar, 0, sizeof(unsigned int) * kBarWords, st);
    if (e != cudaSuccess) return e;
    const int vinit = q2_in_v ? 1 : 0;
    if (after_qr && (e = cudaEventRecord(after_qr, st)) != cudaSuccess) return e;
    bool ring = false;
    unsigned int *fp32_ran = nullptr;
    if (q2_in_v && n <= kRingN && jacobi32_applicable(n) && fp32_phase) {
        // the linear phase of the Jacobi iteration in FP32 (X = X0 V0, V = Q2 V0)
        fp32_ran = w.bar + kJ32Ctl;
        e = launch_jacobi32_precondition(w, n, fp32_ran, st);
        if (e != cudaSuccess) return e;
    }
    if (n <= kRingN) {
        e = launch_jacobi_ring(w, n, bar, status, vinit, max_sweeps, fp32_ran, st, &ring);
        if (e != cudaSuccess) return e;
    }
    if (ring) e = cudaSuccess;
    else if (n <= 256) e = launch_jacobi<1>(w, n, bar, status, vinit, max_sweeps, st);
    else if (n <= 1024) e = launch_jacobi<4>(w, n, bar, status, vinit, max_sweeps, st);
    else e = launch_jacobi<16>(w, n, bar, status, vinit, max_sweeps, st);
    if (e != cudaSuccess) return e;
    // 4. V = P Q2 Vx into w.W (reused as n x n)
    if (q2_in_v) {
        permute_rows_kernel<<<nn_blocks, 256, 0, st>>>(w.V, n, w.perm, w.W);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
        const size_t smem = sizeof(double) * (size_t)n;
        e = cudaFuncSetAttribute(apply_q2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int64_t blocks = n < sm_count() * 4 ? n : sm_count() * 4;
        apply_q2_kernel<<<(unsigned)blocks, kDenseThreads, smem, st>>>(Lq, u0b, cfb, w.perm, w.V, n, w.W);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // 5. extraction (k = 0: left to the caller, V in w.W and sigma in w.sigma)
    if (k > 0) {
        extract_kernel<<<(unsigned)k, kDenseThreads, sizeof(long long) * (size_t)n, st>>>(w.W, w.sigma, n, k, Vk, sigk);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (save_V) {
        copy_kernel<<<64, 256, 0, st>>>(w.W, n * n, save_V);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (save_sigma) {
        copy_kernel<<<1, 256, 0, st>>>(w.sigma, n, save_sigma);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace ns
