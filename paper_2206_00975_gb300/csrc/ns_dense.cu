// ns_dense.cu -- Algorithm 1 lines 3-4 on the GPU, FP64: Householder QR of SA
// (s x n), one-sided Jacobi SVD of the n x n factor R (SA and R share singular
// values and right singular vectors, proof of Theorem 3.2), and extraction of
// the k trailing right singular vectors (line 4).
//
// FP64 runs at ~2 FMA/clock/SM on this part, so even a 256 x 256 problem has
// to be spread over the whole GPU: both factorizations are cooperative
// launches whose CTAs own columns round-robin and meet at a bounded grid
// barrier once per Householder step / Jacobi step.
//
// Jacobi: pairs are scheduled by the round-robin (circle) ordering, n'/2
// disjoint pairs per step, n'-1 steps per sweep (n' = n rounded up to even; an
// odd n gets a phantom zero column).  A pair (p, q) is rotated when
// |gamma| > tol sqrt(alpha beta) with alpha = |x_p|^2, beta = |x_q|^2,
// gamma = x_p . x_q and tol = n 2^-53; the rotation (zeta = (beta-alpha)/(2
// gamma), t = sign(zeta)/(|zeta| + sqrt(1+zeta^2)), c = 1/sqrt(1+t^2), s = c t)
// makes the pair orthogonal.  A sweep without rotations ends the iteration;
// 30 sweeps without convergence report NS_ERR_NOCONV.
#include <cmath>
#include "ns_device.cuh"
#include "ns_internal.h"

namespace ns {

constexpr int kDenseThreads = 256;
constexpr int kMaxSweeps = 30;

size_t dense_work_bytes(int64_t s, int64_t n) {
    Carver c(nullptr);
    dense_carve(c, s, n);
    return c.used;
}

DenseWork dense_carve(Carver &c, int64_t s, int64_t n) {
    DenseWork w;
    w.W = c.take<double>((size_t)(s * n));
    w.tau = c.take<double>((size_t)n);
    w.X = c.take<double>((size_t)(n * n));
    w.V = c.take<double>((size_t)(n * n));
    w.sigma = c.take<double>((size_t)n);
    w.bar = c.take<unsigned int>(2 + 64);
    return w;
}

// scaled 2-norm of x[0..len) over the block (every thread gets it)
__device__ double block_norm2(const double *x, int64_t len, double *red) {
    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) mx = fmax(mx, fabs(__ldcg(x + i)));
    mx = block_max(mx, red);
    if (mx == 0.0) return 0.0;
    double v[1] = {0.0};
    const double inv = 1.0 / mx;
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        const double y = __ldcg(x + i) * inv;
        v[0] += y * y;
    }
    block_sum<1>(v, red);
    return mx * sqrt(v[0]);
}

// ------------------------------------------------------------------- QR ----
// Reflector for column j (LAPACK-style): x = W[j:s, j]; H = I - tau u u^T with
// u = [1; v]; afterwards W[j, j] = beta (= R[j, j]) and W[j+1:s, j] = v.
__device__ void householder_column(double *x, int64_t len, double *tau_out, double *red) {
    const double alpha = __ldcg(x);
    const double xnorm = (len > 1) ? block_norm2(x + 1, len - 1, red) : 0.0;
    if (xnorm == 0.0) {
        if (threadIdx.x == 0) *tau_out = 0.0;
        __syncthreads();
        return;
    }
    const double beta = -copysign(hypot(alpha, xnorm), alpha);
    const double tau = (beta - alpha) / beta;
    const double inv = 1.0 / (alpha - beta);
    for (int64_t i = 1 + threadIdx.x; i < len; i += blockDim.x) x[i] = __ldcg(x + i) * inv;
    if (threadIdx.x == 0) {
        x[0] = beta;
        *tau_out = tau;
    }
    __threadfence();
    __syncthreads();
}

__global__ void __launch_bounds__(kDenseThreads) qr_coop_kernel(double *W, int64_t s, int64_t n, double *tau,
                                                               double *X, GridBarrier bar) {
    extern __shared__ double vsh[];  // s doubles: the current reflector
    __shared__ double red[64];
    const int64_t G = gridDim.x, me = blockIdx.x;
    if (me == 0) householder_column(W, s, tau, red);
    for (int64_t j = 0; j < n; ++j) {
        if (!grid_sync(bar)) return;
        const int64_t len = s - j;
        const double tj = __ldcg(tau + j);
        // first owned column after j
        int64_t l0 = j + 1 + (((me - (j + 1)) % G) + G) % G;
        if (tj != 0.0 && l0 < n) {
            const double *v = W + j + j * s;
            for (int64_t i = threadIdx.x; i < len; i += blockDim.x) vsh[i] = (i == 0) ? 1.0 : __ldcg(v + i);
            __syncthreads();
            for (int64_t l = l0; l < n; l += G) {
                double *y = W + j + l * s;
                double w[1] = {0.0};
                for (int64_t i = threadIdx.x; i < len; i += blockDim.x) w[0] += vsh[i] * y[i];
                block_sum<1>(w, red);
                const double f = tj * w[0];
                for (int64_t i = threadIdx.x; i < len; i += blockDim.x) y[i] -= f * vsh[i];
                __syncthreads();
            }
        }
        __threadfence();
        // the owner of column j+1 forms its reflector (it applied H_j to it above)
        if (j + 1 < n && (j + 1) % G == me) householder_column(W + (j + 1) + (j + 1) * s, s - j - 1, tau + j + 1, red);
    }
    if (!grid_sync(bar)) return;
    // R = upper triangle of W
    for (int64_t l = me; l < n; l += G)
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) X[i + l * n] = (i <= l) ? __ldcg(W + i + l * s) : 0.0;
}

// --------------------------------------------------------------- Jacobi ----
__device__ __forceinline__ int64_t rr_player(int64_t pos, int64_t step, int64_t n2) {
    return pos == 0 ? 0 : 1 + (pos - 1 + step) % (n2 - 1);
}

__global__ void __launch_bounds__(kDenseThreads) jacobi_coop_kernel(double *X, double *V, int64_t n, double tol,
                                                                   GridBarrier bar, unsigned int *rotcount,
                                                                   double *sigma, int32_t *status) {
    __shared__ double red[96];
    const int64_t G = gridDim.x, me = blockIdx.x;
    for (int64_t l = me; l < n; l += G)
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) V[i + l * n] = (i == l) ? 1.0 : 0.0;
    const int64_t n2 = n + (n & 1), npairs = n2 / 2, steps = n2 - 1;
    bool converged = (n < 2);
    for (int sweep = 0; sweep < kMaxSweeps && !converged; ++sweep) {
        unsigned int local = 0;
        for (int64_t step = 0; step < steps; ++step) {
            if (!grid_sync(bar)) return;
            for (int64_t pi = me; pi < npairs; pi += G) {
                int64_t p = rr_player(pi, step, n2), q = rr_player(n2 - 1 - pi, step, n2);
                if (p > q) {
                    const int64_t tmp = p;
                    p = q;
                    q = tmp;
                }
                if (q >= n) continue;  // phantom column
                double *xp = X + p * n, *xq = X + q * n;
                double a3[3] = {0.0, 0.0, 0.0};
                for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
                    const double a = __ldcg(xp + i), b = __ldcg(xq + i);
                    a3[0] += a * a;
                    a3[1] += b * b;
                    a3[2] += a * b;
                }
                block_sum<3>(a3, red);
                const double alpha = a3[0], beta = a3[1], gamma = a3[2];
                if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta)) continue;
                const double zeta = (beta - alpha) / (2.0 * gamma);
                double t;
                if (fabs(zeta) > 1e150) t = 0.5 / zeta;
                else t = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + t * t);
                const double sn = cs * t;
                double *vp = V + p * n, *vq = V + q * n;
                for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
                    const double a = __ldcg(xp + i), b = __ldcg(xq + i);
                    xp[i] = cs * a - sn * b;
                    xq[i] = sn * a + cs * b;
                    const double c = __ldcg(vp + i), d = __ldcg(vq + i);
                    vp[i] = cs * c - sn * d;
                    vq[i] = sn * c + cs * d;
                }
                ++local;
            }
            __threadfence();
        }
        if (threadIdx.x == 0 && local) atomicAdd(rotcount + sweep, local);
        if (!grid_sync(bar)) return;
        converged = (*(volatile unsigned int *)(rotcount + sweep) == 0u);
    }
    if (!converged && me == 0 && threadIdx.x == 0) set_status(status, NS_ERR_NOCONV);
    for (int64_t l = me; l < n; l += G) {
        const double nv = block_norm2(X + l * n, n, red);
        if (threadIdx.x == 0) sigma[l] = nv;
    }
}

// ----------------------------------------------------------- extraction ----
// Order by non-increasing sigma (ties: lower index first); W = the last k
// columns; each returned column is signed so its entry of largest magnitude
// (lowest index on ties) is positive.
__global__ void __launch_bounds__(kDenseThreads) extract_kernel(const double *V, const double *sigma, int64_t n,
                                                               int32_t k, double *Vk, double *sigk, double *save_V,
                                                               double *save_sigma) {
    extern __shared__ int rank_sh[];  // n ints
    __shared__ double redv[32];
    __shared__ long long redi[32];
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double si = sigma[i];
        int r = 0;
        for (int64_t j = 0; j < n; ++j) {
            const double sj = sigma[j];
            r += (sj > si || (sj == si && j < i)) ? 1 : 0;
        }
        rank_sh[i] = r;
    }
    __syncthreads();
    if (save_V)
        for (int64_t i = threadIdx.x; i < n * n; i += blockDim.x) save_V[i] = V[i];
    if (save_sigma)
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) save_sigma[i] = sigma[i];
    for (int64_t src = 0; src < n; ++src) {
        const int r = rank_sh[src];
        if (r < n - k) continue;
        const int64_t col = r - (n - k);
        const double *v = V + src * n;
        // arg max |v| (lowest index on ties)
        double best = -1.0;
        long long bi = 0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const double a = fabs(v[i]);
            if (a > best) {
                best = a;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const long long oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            redv[threadIdx.x >> 5] = best;
            redi[threadIdx.x >> 5] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (redv[w] > redv[0] || (redv[w] == redv[0] && redi[w] < redi[0])) {
                    redv[0] = redv[w];
                    redi[0] = redi[w];
                }
        }
        __syncthreads();
        const double sg = (v[redi[0]] < 0.0) ? -1.0 : 1.0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) Vk[i + col * n] = sg * v[i];
        if (threadIdx.x == 0) sigk[col] = sigma[src];
        __syncthreads();
    }
}

static int coop_blocks(const void *fn, int threads, size_t smem, int64_t want) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    const int64_t cap = (int64_t)sms * (per_sm > 0 ? (per_sm > 1 ? 1 : per_sm) : 1);
    int64_t g = want < cap ? want : cap;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_dense_solve(const double *SA, int64_t s, int64_t n, int32_t k, const DenseWork &w, double *Vk,
                               double *sigk, double *save_V, double *save_sigma, int32_t *status, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(w.W, SA, sizeof(double) * (size_t)(s * n), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(w.bar, 0, sizeof(unsigned int) * 66, st);
    if (e != cudaSuccess) return e;
    GridBarrier bar{w.bar, w.bar + 1, status};
    // QR
    {
        const size_t smem = sizeof(double) * (size_t)s;
        e = cudaFuncSetAttribute(qr_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int G = coop_blocks((const void *)qr_coop_kernel, kDenseThreads, smem, n);
        double *W = w.W, *tau = w.tau, *X = w.X;
        int64_t s_ = s, n_ = n;
        void *args[] = {&W, &s_, &n_, &tau, &X, &bar};
        e = cudaLaunchCooperativeKernel((const void *)qr_coop_kernel, G, kDenseThreads, args, smem, st);
        if (e != cudaSuccess) return e;
    }
    // Jacobi
    {
        e = cudaMemsetAsync(w.bar, 0, sizeof(unsigned int) * 66, st);
        if (e != cudaSuccess) return e;
        const int64_t npairs = (n + (n & 1)) / 2;
        const int G = coop_blocks((const void *)jacobi_coop_kernel, kDenseThreads, 0, npairs);
        double *X = w.X, *V = w.V, *sigma = w.sigma;
        int64_t n_ = n;
        double tol = (double)n * std::ldexp(1.0, -53);
        unsigned int *rot = w.bar + 2;
        int32_t *status_ = status;
        void *args[] = {&X, &V, &n_, &tol, &bar, &rot, &sigma, &status_};
        e = cudaLaunchCooperativeKernel((const void *)jacobi_coop_kernel, G, kDenseThreads, args, 0, st);
        if (e != cudaSuccess) return e;
    }
    // extraction
    {
        const size_t smem = sizeof(int) * (size_t)n;
        e = cudaFuncSetAttribute(extract_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        extract_kernel<<<1, kDenseThreads, smem, st>>>(w.V, w.sigma, n, k, Vk, sigk, save_V, save_sigma);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace ns
