// ns_batched.cu -- ns_solve_batched: Algorithm 1 on many independent problems
// of different shapes, e.g. total least squares [X_i b_i] (Section 4): the
// trailing right singular vector v of the sketch gives x = -v(1:n-1)/v(n).
//
// Stages (all problems at once, no host round trips):
//   setup   one CTA: per-problem workspace offsets and work-item ranges
//           (prefix sums over the device problem array);
//   meta    one CTA per problem: SRHT signs and sample rows from its seed;
//   sketch  persistent CTAs take (problem, column) items from an atomic
//           counter (uneven problems balance dynamically) and run the exact
//           fixed-point SRHT pipeline over the column's blocks;
//   dense   persistent CTAs take whole problems from a second counter: pivoted
//           Householder QR, QR of R^T, one-sided Jacobi on R2^T with one warp
//           per pair, V = P Q2 Vx, extraction, TLS.
// Each problem's numerical status (non-finite input, no convergence, TLS
// without solution) goes to dev_status[i].
#include <cmath>
#include "ns_device.cuh"
#include "ns_internal.h"
#include "ns_srht_core.cuh"

namespace ns {

constexpr int kBatchThreads = 256;
constexpr int kBatchMaxSweeps = 30;

struct BatchSlot {
    int64_t off;       // byte offset of the problem's workspace
    int64_t item0;     // first sketch work item (one per column)
    int32_t nblk;      // 4096-row blocks of its padded length
    int32_t lg;        // m' = 2^lg
};

// per-problem workspace: signs, rows, SA (QR in place), X, V, L, reflector
// scalars, sigma, perm; every piece 256-byte aligned
__host__ __device__ inline int64_t a256(int64_t x) { return (x + 255) & ~(int64_t)255; }
__host__ __device__ inline int clog2(int64_t m) {
    int lg = 0;
    while (((int64_t)1 << lg) < m) ++lg;
    return lg;
}
__host__ __device__ inline int64_t problem_bytes(int64_t m, int64_t n, int64_t s) {
    const int64_t mp = (int64_t)1 << clog2(m);
    const int64_t words = (mp > 4096 ? mp : 4096) / 32;
    return a256(4 * words) + a256(4 * s) + a256(8 * s * n) + 3 * a256(8 * n * n) + a256(8 * 4 * n) + a256(8 * n) +
           a256(4 * n);
}

struct ProblemView {
    uint32_t *sign_words;
    int32_t *rows;
    double *SA, *X, *V, *L, *u0a, *cfa, *u0b, *cfb, *sigma;
    int32_t *perm;
};
__device__ inline ProblemView problem_view(char *base, int64_t m, int64_t n, int64_t s) {
    const int64_t mp = (int64_t)1 << clog2(m);
    const int64_t words = (mp > 4096 ? mp : 4096) / 32;
    ProblemView v;
    char *p = base;
    v.sign_words = (uint32_t *)p; p += a256(4 * words);
    v.rows = (int32_t *)p; p += a256(4 * s);
    v.SA = (double *)p; p += a256(8 * s * n);
    v.X = (double *)p; p += a256(8 * n * n);
    v.V = (double *)p; p += a256(8 * n * n);
    v.L = (double *)p; p += a256(8 * n * n);
    v.u0a = (double *)p; v.cfa = v.u0a + n; v.u0b = v.u0a + 2 * n; v.cfb = v.u0a + 3 * n; p += a256(8 * 4 * n);
    v.sigma = (double *)p; p += a256(8 * n);
    v.perm = (int32_t *)p;
    return v;
}

size_t batched_head_bytes(int32_t batch) { return align256(sizeof(BatchSlot) * (size_t)batch) + 256; }

// ------------------------------------------------------------------ setup ----
__global__ void __launch_bounds__(1024) batched_setup_kernel(const ns_problem *__restrict__ P, int32_t batch,
                                                             BatchSlot *slots, unsigned long long *counters,
                                                             int64_t head) {
    __shared__ int64_t part_b[1024], part_i[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t per = (batch + nt - 1) / nt;
    const int64_t i0 = tid * per, i1 = (i0 + per < batch) ? i0 + per : batch;
    int64_t sb = 0, si = 0;
    for (int64_t i = i0; i < i1; ++i) {
        sb += problem_bytes(P[i].m, P[i].n, P[i].s);
        si += P[i].n;
    }
    part_b[tid] = sb;
    part_i[tid] = si;
    __syncthreads();
    if (tid == 0) {
        int64_t ab = 0, ai = 0;
        for (int w = 0; w < nt; ++w) {
            const int64_t b = part_b[w], it = part_i[w];
            part_b[w] = ab;
            part_i[w] = ai;
            ab += b;
            ai += it;
        }
        counters[0] = 0;                      // sketch item counter
        counters[1] = 0;                      // dense problem counter
        counters[2] = (unsigned long long)ai; // total sketch items
    }
    __syncthreads();
    int64_t ob = head + part_b[tid], oi = part_i[tid];
    for (int64_t i = i0; i < i1; ++i) {
        const int lg = clog2(P[i].m);
        const int64_t mp = (int64_t)1 << lg;
        slots[i].off = ob;
        slots[i].item0 = oi;
        slots[i].nblk = (int32_t)(mp > kBlock ? mp / kBlock : 1);
        slots[i].lg = lg;
        ob += problem_bytes(P[i].m, P[i].n, P[i].s);
        oi += P[i].n;
    }
}

// ------------------------------------------------------------------- meta ----
__global__ void batched_meta_kernel(const ns_problem *__restrict__ P, const BatchSlot *__restrict__ slots, char *ws) {
    const int64_t i = blockIdx.x;
    const ns_problem pr = P[i];
    ProblemView v = problem_view(ws + slots[i].off, pr.m, pr.n, pr.s);
    const int lg = slots[i].lg;
    const int64_t mp = (int64_t)1 << lg;
    const int64_t words = (mp > 4096 ? mp : 4096) / 32;
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) {
        const u64x4 b = draw(pr.seed, (uint64_t)(w >> 3), 0, 0);
        const uint64_t word = b.w[(w & 7) >> 1];
        v.sign_words[w] = (w & 1) ? (uint32_t)(word >> 32) : (uint32_t)word;
    }
    for (int64_t t = threadIdx.x; t < pr.s; t += blockDim.x) v.rows[t] = (int32_t)sample_perm(pr.seed, lg, (uint32_t)t);
}

// ----------------------------------------------------------------- sketch ----
__global__ void __launch_bounds__(64) batched_sketch_kernel(const ns_problem *__restrict__ P, int32_t batch,
                                                            const BatchSlot *__restrict__ slots, char *ws,
                                                            unsigned long long *counters, int64_t smax,
                                                            int32_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    long long *Zs = (long long *)smem_raw;
    long long *acc = Zs + kBlock;                                   // smax
    unsigned long long *need = (unsigned long long *)(acc + smax);  // 64
    uint32_t *sgn = (uint32_t *)(need + 64);                        // 128
    int *red = (int *)(sgn + 128);                                  // 4
    int32_t *rows_s = (int32_t *)(red + 4);                         // smax
    __shared__ long long item_sh;
    const int t = threadIdx.x;
    const unsigned long long total = counters[2];
    while (true) {
        if (t == 0) item_sh = (long long)atomicAdd(counters, 1ull);
        __syncthreads();
        const long long item = item_sh;
        __syncthreads();
        if ((unsigned long long)item >= total) break;
        // problem of this item: last slot with item0 <= item
        int64_t lo = 0, hi = batch - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (slots[mid].item0 <= item) lo = mid;
            else hi = mid - 1;
        }
        const ns_problem pr = P[lo];
        const BatchSlot sl = slots[lo];
        const int64_t c = item - sl.item0;
        ProblemView v = problem_view(ws + sl.off, pr.m, pr.n, pr.s);
        const int64_t s = pr.s;
        for (int64_t i = t; i < s; i += 64) {
            rows_s[i] = v.rows[i];
            acc[i] = 0;
        }
        const unsigned long long myneed = srht_need_mask(rows_s, s, need);
        const double *Acol = (const double *)pr.A + c * pr.lda;
        const int vec_ok = ((((uintptr_t)pr.A) & 15) == 0 && (pr.lda & 1) == 0) ? 1 : 0;
        const int P_bits = 63 - kBlockLog - clog2(sl.nblk) - 1;
        int Erun = 0, nonfinite = 0;
        for (int64_t b = 0; b < sl.nblk; ++b)
            srht_f64_block(Acol, pr.m, s, b, P_bits, v.sign_words, rows_s, myneed, Zs, acc, sgn, red, vec_ok, Erun,
                           nonfinite);
        const double scale = ldexp(1.0, Erun - 1022 - P_bits) / sqrt((double)s);
        double *out = v.SA + c * s;
        for (int64_t i = t; i < s; i += 64) out[i] = (double)acc[i] * scale;
        if (nonfinite) atomicMax(status + lo, (int32_t)NS_ERR_NONFINITE);
        __syncthreads();
    }
}

// ------------------------------------------------------- one-CTA dense ----
__device__ __forceinline__ long long abskey(double x) { return __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll; }

// Householder QR of W (rows x cols, ld = rows) by one CTA, optionally with
// column pivoting (physical swaps).  Reflector j: u = [u0[j]; W[j+1:, j]],
// H = I - cf[j] u u^T; R is the upper triangle of W afterwards.
__device__ void qr_cta(double *W, int64_t rows, int64_t cols, bool pivot, double *u0, double *cf, int32_t *perm,
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
__device__ bool jacobi_cta(double *X, double *V, int64_t n, double *sigma) {
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

__global__ void __launch_bounds__(kBatchThreads) batched_dense_kernel(const ns_problem *__restrict__ P, int32_t batch,
                                                                      const BatchSlot *__restrict__ slots, char *ws,
                                                                      unsigned long long *counters, int32_t *status) {
    extern __shared__ double dsh[];  // xs (smax), nrm, nref (nmax each)
    __shared__ long long prob_sh;
    __shared__ int src_sh;
    __shared__ long long bk[32];
    __shared__ int bi_sh[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    while (true) {
        if (tid == 0) prob_sh = (long long)atomicAdd(counters + 1, 1ull);
        __syncthreads();
        const long long pi = prob_sh;
        __syncthreads();
        if (pi >= batch) break;
        const ns_problem pr = P[pi];
        const int64_t n = pr.n, s = pr.s;
        ProblemView v = problem_view(ws + slots[pi].off, pr.m, n, s);
        double *xs = dsh, *nrm = dsh + s, *nref = dsh + s + n;
        // 1. SA P = Q1 R (pivoted), in place
        qr_cta(v.SA, s, n, true, v.u0a, v.cfa, v.perm, xs, nrm, nref);
        // 2. L = R^T
        for (int64_t idx = tid; idx < n * n; idx += blockDim.x) {
            const int64_t i = idx % n, j = idx / n;
            v.L[i + j * n] = (i >= j) ? v.SA[j + i * s] : 0.0;
        }
        __syncthreads();
        // 3. L = Q2 R2 (no pivoting); X = R2^T; perm of this QR is not used
        qr_cta(v.L, n, n, false, v.u0b, v.cfb, (int32_t *)v.sigma, xs, nrm, nref);
        for (int64_t idx = tid; idx < n * n; idx += blockDim.x) {
            const int64_t i = idx % n, j = idx / n;
            v.X[i + j * n] = (i >= j) ? v.L[j + i * n] : 0.0;
        }
        __syncthreads();
        // 4. Jacobi on X: Vx in V
        const bool conv = jacobi_cta(v.X, v.V, n, v.sigma);
        if (!conv && tid == 0) atomicMax(status + pi, (int32_t)NS_ERR_NOCONV);
        // 5. the k trailing columns of V = P Q2 Vx, one warp per column
        for (int32_t c = 0; c < pr.k; ++c) {
            // source column: the singular value of rank n - k + c (non-increasing, ties to lower index)
            if (tid == 0) src_sh = -1;
            __syncthreads();
            for (int64_t i = tid; i < n; i += blockDim.x) {
                const double si = v.sigma[i];
                int64_t r = 0;
                for (int64_t jj = 0; jj < n; ++jj) {
                    const double sj = v.sigma[jj];
                    r += (sj > si || (sj == si && jj < i)) ? 1 : 0;
                }
                if (r == n - pr.k + c) src_sh = (int)i;
            }
            __syncthreads();
            const int64_t src = src_sh;
            // column src of Vx -> apply H_{n-1} ... H_0 of the second QR (xs as the column)
            for (int64_t i = tid; i < n; i += blockDim.x) xs[i] = v.V[i + src * n];
            __syncthreads();
            for (int64_t j = n - 1; j >= 0; --j) {
                const double coef = v.cfb[j];
                if (coef == 0.0) continue;
                const double ua = v.u0b[j];
                double d[1] = {0.0};
                for (int64_t i = j + tid; i < n; i += blockDim.x) d[0] = fma(i == j ? ua : v.L[i + j * n], xs[i], d[0]);
                block_sum_t0<1>(d, (double *)bk);
                if (tid == 0) *(double *)&bk[31] = coef * d[0];
                __syncthreads();
                const double f = *(double *)&bk[31];
                for (int64_t i = j + tid; i < n; i += blockDim.x) xs[i] = fma(-f, i == j ? ua : v.L[i + j * n], xs[i]);
                __syncthreads();
            }
            // row i of Q2 Vx is row perm[i] of V; sign: largest |entry| positive (lowest index on ties)
            long long best = -1;
            int bi = 0;
            for (int64_t i = tid; i < n; i += blockDim.x) {
                const int64_t row = v.perm[i];
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
                if (v.perm[i] == brow) sgn = xs[i] < 0.0 ? -1.0 : 1.0;
            for (int64_t i = tid; i < n; i += blockDim.x) pr.Vk[v.perm[i] + c * n] = sgn * xs[i];
            if (tid == 0) pr.sigk[c] = v.sigma[src];
            __syncthreads();
        }
        // 6. TLS: x = -v(1:n-1) / v(n)
        if (pr.tls && pr.x) {
            const double *w = pr.Vk;  // k = 1
            double ss[1] = {0.0};
            for (int64_t i = tid; i < n; i += blockDim.x) ss[0] = fma(w[i], w[i], ss[0]);
            block_sum_t0<1>(ss, (double *)bk);
            if (tid == 0) *(double *)&bk[31] = ss[0];
            __syncthreads();
            const double last = w[n - 1];
            if (fabs(last) < 1.1102230246251565e-16 * sqrt(*(double *)&bk[31])) {
                if (tid == 0) atomicMax(status + pi, (int32_t)NS_ERR_TLS_NOSOLUTION);
            }
            for (int64_t i = tid; i < n - 1; i += blockDim.x) pr.x[i] = -w[i] / last;
            __syncthreads();
        }
    }
}

static int sm_count_b() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

size_t batched_work_bytes(int32_t batch, const ns_problem *host) {
    int64_t total = (int64_t)batched_head_bytes(batch);
    for (int32_t i = 0; i < batch; ++i) total += problem_bytes(host[i].m, host[i].n, host[i].s);
    return (size_t)total;
}

cudaError_t launch_batched(int32_t batch, const ns_problem *host, const ns_problem *dev, int32_t *status, void *ws,
                           cudaStream_t st) {
    int64_t smax = 1, nmax = 1;
    for (int32_t i = 0; i < batch; ++i) {
        smax = host[i].s > smax ? host[i].s : smax;
        nmax = host[i].n > nmax ? host[i].n : nmax;
    }
    char *base = (char *)ws;
    BatchSlot *slots = (BatchSlot *)base;
    unsigned long long *counters = (unsigned long long *)(base + align256(sizeof(BatchSlot) * (size_t)batch));
    const int64_t head = (int64_t)batched_head_bytes(batch);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t) * (size_t)batch, st);
    if (e != cudaSuccess) return e;
    batched_setup_kernel<<<1, 1024, 0, st>>>(dev, batch, slots, counters, head);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    batched_meta_kernel<<<(unsigned)batch, 256, 0, st>>>(dev, slots, base);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = (size_t)kBlock * 8 + (size_t)smax * 8 + 64 * 8 + 128 * 4 + 16 + (size_t)smax * 4;
    e = cudaFuncSetAttribute(batched_sketch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_sketch_kernel, 64, smem);
    const int grid1 = sm_count_b() * (per_sm > 0 ? per_sm : 1);
    batched_sketch_kernel<<<grid1, 64, smem, st>>>(dev, batch, slots, base, counters, smax, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t dsmem = sizeof(double) * (size_t)(smax + 2 * nmax);
    e = cudaFuncSetAttribute(batched_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
    if (e != cudaSuccess) return e;
    int per_sm2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, batched_dense_kernel, kBatchThreads, dsmem);
    int64_t grid2 = (int64_t)sm_count_b() * (per_sm2 > 0 ? per_sm2 : 1);
    if (grid2 > batch) grid2 = batch;
    batched_dense_kernel<<<(unsigned)grid2, kBatchThreads, dsmem, st>>>(dev, batch, slots, base, counters, status);
    return cudaGetLastError();
}

}  // namespace ns
