// ns_dense_cta.cuh -- Algorithm 1 lines 3-4 for one problem by ONE CTA (FP64):
// pivoted Householder QR of SA, QR of R^T, one-sided Jacobi on R2^T with one
// warp per pair, V = P Q2 Vx, and the k trailing right singular vectors
// (Drmac-Veselic preconditioning, as in ns_dense.cu).  Used by the batched
// solver and the AAA driver, where many small problems or a sequence of small
// problems run without grid-wide synchronisation.
#pragma once
#include "ns_device.cuh"
#include "ns_internal.h"

namespace ns {

constexpr int kBatchMaxSweeps = 30;

__device__ __forceinline__ long long abskey(double x) { return __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll; }

// Householder QR of W (rows x cols, ld = rows) by one CTA, optionally with
// column pivoting (physical swaps).  Reflector j: u = [u0[j]; W[j+1:, j]],
// H = I - cf[j] u u^T; R is the upper triangle of W afterwards.
static __device__ void qr_cta(double *W, int64_t rows, int64_t cols, bool pivot, double *u0, double *cf, int32_t *perm,
                       double *xs /* rows */, double *nrm /* cols */, double *nref /* cols */) {
    __shared__ double red[32];
    __shared__ long long redk[32];
    __shared__ double par[3];
    __shared__ int piv;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    for (int64_t l = tid; l < cols; l += blockDim.x) perm[l] = (int32_t)l;
    if (pivot) {
        for (int64_t l = wid; l < cols; l += nw) {
            double a = 0.0;
            for (int64_t i = lane; i < rows; i += 32) a = fma(W[i + l * rows], W[i + l * rows], a);
            a = warp_sum(a);
            if (lane == 0) {
                nrm[l] = a;
                nref[l] = a;
            }
        }
    }
    __syncthreads();
    const int64_t steps = rows < cols ? rows : cols;
    for (int64_t j = 0; j < steps; ++j) {
        if (pivot) {
            if (wid == 0) {  // argmax of the remaining norms, lowest index on ties
                double best = -1.0;
                int64_t bi = j;
                for (int64_t l = j + lane; l < cols; l += 32)
                    if (nrm[l] > best) {
                        best = nrm[l];
                        bi = l;
                    }
                for (int o = 16; o > 0; o >>= 1) {
                    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const long long oi = __shfl_xor_sync(0xffffffffu, (long long)bi, o);
                    if (ob > best || (ob == best && oi < bi)) {
                        best = ob;
                        bi = oi;
                    }
                }
                if (lane == 0) piv = (int)bi;
            }
            __syncthreads();
            const int64_t p = piv;
            if (p != j) {
                for (int64_t i = tid; i < rows; i += blockDim.x) {
                    const double a = W[i + j * rows];
                    W[i + j * rows] = W[i + p * rows];
                    W[i + p * rows] = a;
                }
                if (tid == 0) {
                    double a = nrm[j]; nrm[j] = nrm[p]; nrm[p] = a;
                    a = nref[j]; nref[j] = nref[p]; nref[p] = a;
                    const int32_t q = perm[j]; perm[j] = perm[p]; perm[p] = q;
                }
            }
            __syncthreads();
        }
        const int64_t len = rows - j;
        double *x = W + j + j * rows;
        long long key = 0;
        for (int64_t i = tid; i < len; i += blockDim.x) {
            const double a = x[i];
            xs[i] = a;
            key = max(key, abskey(a));
        }
        key = warp_max(key);
        if (lane == 0) redk[wid] = key;
        __syncthreads();
        long long kmax = redk[0];
        for (int w = 1; w < nw; ++w) kmax = max(kmax, redk[w]);
        double sc = 0.0;
        if (kmax != 0) {
            int se = 2046 - (int)((unsigned long long)kmax >> 52);
            se = se < 1 ? 1 : (se > 2045 ? 2045 : se);
            sc = __longlong_as_double((long long)se << 52);
        }
        double ss[1] = {0.0};
        if (sc != 0.0)
            for (int64_t i = 1 + tid; i < len; i += blockDim.x) {
                const double a = xs[i] * sc;
                ss[0] = fma(a, a, ss[0]);
            }
        block_sum_t0<1>(ss, red);
        if (tid == 0) {
            const double alpha = xs[0];
            if (sc == 0.0 || ss[0] == 0.0) {
                par[0] = 0.0;
                par[1] = alpha;
                par[2] = 0.0;
            } else {
                const double isc = __longlong_as_double((2046ll << 52) - __double_as_longlong(sc));
                const double as = alpha * sc;
                const double r = sqrt(fma(as, as, ss[0])) * isc;
                const double beta = alpha >= 0.0 ? -r : r;
                par[0] = 1.0 / (beta * (beta - alpha));
                par[1] = beta;
                par[2] = alpha - beta;
            }
        }
        __syncthreads();
        const double coef = par[0], beta = par[1], ua = par[2];
        // trailing columns, one warp per column
        if (coef != 0.0) {
            for (int64_t l = j + 1 + wid; l < cols; l += nw) {
                double *y = W + j + l * rows;
                double d = 0.0;
                for (int64_t i = 1 + lane; i < len; i += 32) d = fma(xs[i], y[i], d);
                d = warp_sum(d);
                const double f = coef * fma(ua, y[0], d);
                if (lane == 0) y[0] -= f * ua;
                for (int64_t i = 1 + lane; i < len; i += 32) y[i] = fma(-f, xs[i], y[i]);
                if (pivot) {
                    __syncwarp();
                    if (lane == 0) {
                        const double r0 = y[0];
                        nrm[l] -= r0 * r0;
                    }
                    __syncwarp();
                    if (!(nrm[l] > 1e-8 * nref[l])) {  // recompute from the remaining rows
                        double a = 0.0;
                        for (int64_t i = 1 + lane; i < len; i += 32) a = fma(y[i], y[i], a);
                        a = warp_sum(a);
                        if (lane == 0) {
                            nrm[l] = a;
                            nref[l] = a;
                        }
                    }
                }
            }
        } else if (pivot) {
            for (int64_t l = j + 1 + wid; l < cols; l += nw) {
                if (lane == 0) {
                    const double r0 = W[j + l * rows];
                    nrm[l] -= r0 * r0;
                }
            }
        }
        if (tid == 0) {
            x[0] = beta;
            u0[j] = ua;
            cf[j] = coef;
            if (pivot) nrm[j] = -1.0;
        }
        __syncthreads();
    }
}

// one-sided Jacobi on X (n x n) by one CTA, one warp per pair of each
// round-robin step; V receives the accumulated rotations.  Returns whether the
// iteration converged.  Same rotation rule as the cooperative kernel.
static __device__ bool jacobi_cta(double *X, double *V, int64_t n, double *sigma) {
    __shared__ unsigned int rot_sh;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const double tol = (double)n * 1.1102230246251565e-16, tol2 = tol * tol;
    for (int64_t i = tid; i < n * n; i += blockDim.x) V[i] = ((i % n) == (i / n)) ? 1.0 : 0.0;
    const int64_t n2 = n + (n & 1), npairs = n2 / 2, steps = n2 - 1;
    bool converged = n < 2;
    for (int sweep = 0; sweep < kBatchMaxSweeps && !converged; ++sweep) {
        if (tid == 0) rot_sh = 0;
        __syncthreads();
        unsigned int local = 0;
        for (int64_t step = 0; step < steps; ++step) {
            for (int64_t pi = wid; pi < npairs; pi += nw) {
                int64_t p = (pi == 0) ? 0 : 1 + (pi - 1 + step) % (n2 - 1);
                const int64_t qpos = n2 - 1 - pi;
                int64_t q = (qpos == 0) ? 0 : 1 + (qpos - 1 + step) % (n2 - 1);
                if (p > q) {
                    const int64_t tmp = p;
                    p = q;
                    q = tmp;
                }
                if (q >= n) continue;
                double *xp = X + p * n, *xq = X + q * n;
                double a = 0.0, b = 0.0, g = 0.0;
                for (int64_t i = lane; i < n; i += 32) {
                    const double u = xp[i], w = xq[i];
                    a = fma(u, u, a);
                    b = fma(w, w, b);
                    g = fma(u, w, g);
                }
                a = warp_sum(a);
                b = warp_sum(b);
                g = warp_sum(g);
                if (g == 0.0 || !(g * g > tol2 * a * b)) continue;
                const double zeta = (b - a) / (2.0 * g);
                const double t = (fabs(zeta) > 1e150) ? 0.5 / zeta
                                                      : copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
                const double cs = rsqrt(fma(t, t, 1.0)), sn = cs * t;
                double *vp = V + p * n, *vq = V + q * n;
                for (int64_t i = lane; i < n; i += 32) {
                    const double u = xp[i], w = xq[i];
                    xp[i] = fma(cs, u, -sn * w);
                    xq[i] = fma(sn, u, cs * w);
                    const double c0 = vp[i], d0 = vq[i];
                    vp[i] = fma(cs, c0, -sn * d0);
                    vq[i] = fma(sn, c0, cs * d0);
                }
                ++local;
            }
            __syncthreads();
        }
        if (lane == 0 && local) atomicAdd(&rot_sh, local);
        __syncthreads();
        converged = (rot_sh == 0);
        __syncthreads();
    }
    for (int64_t l = wid; l < n; l += nw) {
        double a = 0.0;
        for (int64_t i = lane; i < n; i += 32) a = fma(X[i + l * n], X[i + l * n], a);
        a = warp_sum(a);
        if (lane == 0) sigma[l] = sqrt(a);
    }
    __syncthreads();
    return converged;
}


struct DenseScratch {
    double *X, *V, *L;          // n x n each
    double *u0a, *cfa, *u0b, *cfb;  // n each
    double *sigma;              // n
    int32_t *perm;              // n
};

// SA (s x n, ld s) is destroyed.  Shared scratch: xs (s doubles), nrm and nref
// (n doubles each).  Writes Vk (n x k, ld n) and sigk (k); returns whether the
// Jacobi iteration converged.
static __device__ bool dense_solve_cta(double *SA, int64_t s, int64_t n, int32_t k, const DenseScratch &w, double *xs,
                                double *nrm, double *nref, double *Vk, double *sigk) {
    __shared__ int src_sh;
    __shared__ long long bk[32];
    __shared__ int bi_sh[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    // 1. SA P = Q1 R (pivoted), in place
    qr_cta(SA, s, n, true, w.u0a, w.cfa, w.perm, xs, nrm, nref);
    // 2. L = R^T
    for (int64_t idx = tid; idx < n * n; idx += blockDim.x) {
        const int64_t i = idx % n, j = idx / n;
        w.L[i + j * n] = (i >= j) ? SA[j + i * s] : 0.0;
    }
    __syncthreads();
    // 3. L = Q2 R2 (no pivoting); X = R2^T; perm of this QR is not used
    qr_cta(w.L, n, n, false, w.u0b, w.cfb, (int32_t *)w.sigma, xs, nrm, nref);
    for (int64_t idx = tid; idx < n * n; idx += blockDim.x) {
        const int64_t i = idx % n, j = idx / n;
        w.X[i + j * n] = (i >= j) ? w.L[j + i * n] : 0.0;
    }
    __syncthreads();
    // 4. Jacobi on X: Vx in V
    const bool conv = jacobi_cta(w.X, w.V, n, w.sigma);
    // 5. the k trailing columns of V = P Q2 Vx, one warp per column
    for (int32_t c = 0; c < k; ++c) {
        // source column: the singular value of rank n - k + c (non-increasing, ties to lower index)
        if (tid == 0) src_sh = -1;
        __syncthreads();
        for (int64_t i = tid; i < n; i += blockDim.x) {
            const double si = w.sigma[i];
            int64_t r = 0;
            for (int64_t jj = 0; jj < n; ++jj) {
                const double sj = w.sigma[jj];
                r += (sj > si || (sj == si && jj < i)) ? 1 : 0;
            }
            if (r == n - k + c) src_sh = (int)i;
        }
        __syncthreads();
        const int64_t src = src_sh;
        // column src of Vx -> apply H_{n-1} ... H_0 of the second QR (xs as the column)
        for (int64_t i = tid; i < n; i += blockDim.x) xs[i] = w.V[i + src * n];
        __syncthreads();
        for (int64_t j = n - 1; j >= 0; --j) {
            const double coef = w.cfb[j];
            if (coef == 0.0) continue;
            const double ua = w.u0b[j];
            double d[1] = {0.0};
            for (int64_t i = j + tid; i < n; i += blockDim.x) d[0] = fma(i == j ? ua : w.L[i + j * n], xs[i], d[0]);
            block_sum_t0<1>(d, (double *)bk);
            if (tid == 0) *(double *)&bk[31] = coef * d[0];
            __syncthreads();
            const double f = *(double *)&bk[31];
            for (int64_t i = j + tid; i < n; i += blockDim.x) xs[i] = fma(-f, i == j ? ua : w.L[i + j * n], xs[i]);
            __syncthreads();
        }
        // row i of Q2 Vx is row perm[i] of V; sign: largest |entry| positive (lowest index on ties)
        long long best = -1;
        int bi = 0;
        for (int64_t i = tid; i < n; i += blockDim.x) {
            const int64_t row = w.perm[i];
            const long long kk = abskey(xs[i]);
            if (kk > best || (kk == best && row < bi)) {
                best = kk;
                bi = (int)row;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (lane == 0) {
            bk[wid] = best;
            bi_sh[wid] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < nw; ++w)
                if (bk[w] > bk[0] || (bk[w] == bk[0] && bi_sh[w] < bi_sh[0])) {
                    bk[0] = bk[w];
                    bi_sh[0] = bi_sh[w];
                }
        }
        __syncthreads();
        const int brow = bi_sh[0];
        double sgn = 1.0;
        for (int64_t i = 0; i < n; ++i)
            if (w.perm[i] == brow) sgn = xs[i] < 0.0 ? -1.0 : 1.0;
        for (int64_t i = tid; i < n; i += blockDim.x) Vk[w.perm[i] + c * n] = sgn * xs[i];
        if (tid == 0) sigk[c] = w.sigma[src];
        __syncthreads();
    }
    return conv;
}

}  // namespace ns
