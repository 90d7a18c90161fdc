// ns_aaa.cu -- AAA rational approximation with a reused SRHT sketch
// (Section 6.2), real points.
//
// Iteration k = 1..K:
//   1. the support point j_k maximises |f - r| over non-support points (lowest
//      index on ties); r_0 = mean(f);
//   2. row downdate of the existing sketch columns (Algorithm 3 and the
//      non-Gaussian rule of Section 5.3): SA(:, l) -= (S e_j) A(j, l), with the
//      closed form (S e_j)_t = d_j (-1)^popcount(r_t & j) / sqrt(s) -- O(s)
//      instead of the O(m log m) transform of e_j;
//   3. column update: the new Loewner column (f_i - f_j)/(x_i - x_j) (support
//      rows zero) is sketched with the FP64 SRHT kernels;
//   4. the weights w solve min |A w|, |w| = 1, on the first min(4k, s) rows of
//      the s-row sketch (Algorithm 1 on the sketch: one CTA while k is small,
//      the whole-GPU dense stage of ns_solve from kAaaWideFrom columns on);
//   5. r(x) = sum_l w_l f_l/(x - x_l) / sum_l w_l/(x - x_l) at every point, and
//      the largest error and its index (deterministic reduction).
// Every step reads the current support index from device memory, so the loop
// runs without host round trips and can be captured in a CUDA graph.
#include <cmath>
#include "ns_device.cuh"
#include "ns_internal.h"
#include "ns_dense_cta.cuh"

namespace ns {

constexpr int kAaaThreads = 256;
constexpr int kAaaEvalBlocks = 512;
constexpr int kAaaWideFrom = 24;  // iterations k >= this solve on the whole GPU

struct AaaWork {
    SrhtWork srht;
    double *col;        // m: current Loewner column
    double *err;        // m
    unsigned char *sup; // m: support flags
    double *SAk;        // smax x K: the updated sketch
    double *SAc;        // smax x K: the prefix copied for the dense solve
    double *X, *V, *L, *u0a, *cfa, *u0b, *cfb, *sigma;
    int32_t *perm;
    double *w;          // K
    double *sigk;       // 1
    double *bval;       // kAaaEvalBlocks
    long long *bidx;    // kAaaEvalBlocks
    long long *cur;     // current support index
    double *mean;       // 1
    DenseWork dw;       // smax x K: the whole-GPU dense solve of the larger iterations
};

static AaaWork aaa_carve(Carver &c, int64_t m, int64_t smax, int32_t K) {
    AaaWork w;
    w.srht = srht_carve(c, m, 1, smax);
    w.col = c.take<double>((size_t)m);
    w.err = c.take<double>((size_t)m);
    w.sup = c.take<unsigned char>((size_t)m);
    w.SAk = c.take<double>((size_t)(smax * K));
    w.SAc = c.take<double>((size_t)(smax * K));
    w.X = c.take<double>((size_t)K * K);
    w.V = c.take<double>((size_t)K * K);
    w.L = c.take<double>((size_t)K * K);
    w.u0a = c.take<double>((size_t)4 * K);
    w.cfa = w.u0a + K;
    w.u0b = w.u0a + 2 * K;
    w.cfb = w.u0a + 3 * K;
    w.sigma = c.take<double>((size_t)K);
    w.perm = c.take<int32_t>((size_t)K);
    w.w = c.take<double>((size_t)K);
    w.sigk = c.take<double>(1);
    w.bval = c.take<double>(kAaaEvalBlocks);
    w.bidx = c.take<long long>(kAaaEvalBlocks);
    w.cur = c.take<long long>(1);
    w.mean = c.take<double>(1);
    w.dw = dense_carve(c, smax, K);
    return w;
}

size_t aaa_work_bytes(int64_t m, int64_t smax, int32_t K) {
    Carver c(nullptr);
    aaa_carve(c, m, smax, K);
    return c.used;
}

// mean(f) in a fixed order (one CTA), err = |f - mean|, no support points
__global__ void __launch_bounds__(kAaaThreads) aaa_init_kernel(const double *__restrict__ f, int64_t m, double *mean,
                                                               double *err, unsigned char *sup) {
    __shared__ double red[32];
    double v[1] = {0.0};
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) v[0] += f[i];
    block_sum_t0<1>(v, red);
    __shared__ double mu;
    if (threadIdx.x == 0) {
        mu = v[0] / (double)m;
        *mean = mu;
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
        err[i] = fabs(f[i] - mu);
        sup[i] = 0;
    }
}

// per-block (max err, lowest index) over non-support points
__global__ void __launch_bounds__(kAaaThreads) aaa_argmax_blocks(const double *__restrict__ err,
                                                                 const unsigned char *__restrict__ sup, int64_t m,
                                                                 double *bval, long long *bidx) {
    double best = -1.0;
    long long bi = -1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        if (sup[i]) continue;
        const double e = err[i];
        if (e > best || (e == best && (bi < 0 || i < bi))) {
            best = e;
            bi = i;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const long long oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) {
            best = ob;
            bi = oi;
        }
    }
    __shared__ double sv[32];
    __shared__ long long si[32];
    if ((threadIdx.x & 31) == 0) {
        sv[threadIdx.x >> 5] = best;
        si[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (sv[w] > best || (sv[w] == best && si[w] >= 0 && (bi < 0 || si[w] < bi))) {
                best = sv[w];
                bi = si[w];
            }
        bval[blockIdx.x] = best;
        bidx[blockIdx.x] = bi;
    }
}

// final argmax over blocks (in block order); also the error of iteration kprev
__global__ void aaa_argmax_final(const double *bval, const long long *bidx, int nb, long long *cur, double *errmax,
                                 int32_t kprev) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double best = -1.0;
    long long bi = -1;
    for (int b = 0; b < nb; ++b)
        if (bval[b] > best || (bval[b] == best && bidx[b] >= 0 && (bi < 0 || bidx[b] < bi))) {
            best = bval[b];
            bi = bidx[b];
        }
    *cur = bi;
    if (kprev >= 1) errmax[kprev - 1] = best < 0.0 ? 0.0 : best;
}

// support point of iteration k, row downdate of the existing k-1 columns
__global__ void __launch_bounds__(kAaaThreads) aaa_downdate_kernel(
    const double *__restrict__ x, const double *__restrict__ f, int32_t k, const long long *forced, long long *cur,
    long long *support, unsigned char *sup, double *SAk, int64_t smax, const uint32_t *__restrict__ sign_words,
    const int32_t *__restrict__ rows) {
    __shared__ long long jsh;
    if (threadIdx.x == 0) {
        long long j = forced ? forced[k - 1] : *cur;
        *cur = j;
        support[k - 1] = j;
        jsh = j;
    }
    __syncthreads();
    const long long j = jsh;
    const double dj = ((sign_words[j >> 5] >> (j & 31)) & 1u) ? -1.0 : 1.0;
    const double inv = 1.0 / sqrt((double)smax);
    for (int64_t idx = threadIdx.x; idx < smax * (k - 1); idx += blockDim.x) {
        const int64_t t = idx % smax, l = idx / smax;
        const long long jl = support[l];
        const double a = (f[j] - f[jl]) / (x[j] - x[jl]);  // row j of column l
        const double e = ((__popcll((unsigned long long)(rows[t] & j)) & 1) ? -dj : dj) * inv;
        SAk[t + l * smax] -= e * a;
    }
    __syncthreads();
    if (threadIdx.x == 0) sup[j] = 1;
}

__global__ void aaa_column_kernel(const double *__restrict__ x, const double *__restrict__ f,
                                  const unsigned char *__restrict__ sup, const long long *cur, int64_t m,
                                  double *__restrict__ col) {
    const long long j = *cur;
    const double xj = x[j], fj = f[j];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        col[i] = sup[i] ? 0.0 : (f[i] - fj) / (x[i] - xj);
}

// weights of iteration k: Algorithm 1 on the first sk rows of the sketch (one CTA)
__global__ void __launch_bounds__(kAaaThreads) aaa_dense_kernel(const double *SAk, int64_t smax, int32_t k,
                                                                int64_t sk, AaaWork w, double *Wout, int32_t K,
                                                                int32_t *status) {
    extern __shared__ double dsh[];  // xs (sk), nrm, nref (k each)
    for (int64_t idx = threadIdx.x; idx < sk * k; idx += blockDim.x) {
        const int64_t t = idx % sk, l = idx / sk;
        w.SAc[t + l * sk] = SAk[t + l * smax];
    }
    __syncthreads();
    DenseScratch scr{w.X, w.V, w.L, w.u0a, w.cfa, w.u0b, w.cfb, w.sigma, w.perm};
    const bool conv = dense_solve_cta(w.SAc, sk, k, 1, scr, dsh, dsh + sk, dsh + sk + k, w.w, w.sigk);
    if (!conv && threadIdx.x == 0) atomicMax(status, (int32_t)NS_ERR_NOCONV);
    for (int32_t l = threadIdx.x; l < K; l += blockDim.x) Wout[(int64_t)(k - 1) * K + l] = (l < k) ? w.w[l] : 0.0;
}

// the first sk rows of the k sketch columns, contiguous (ld sk)
__global__ void aaa_prefix_kernel(const double *__restrict__ SAk, int64_t smax, int32_t k, int64_t sk,
                                  double *__restrict__ SAc) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < sk * k;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = idx % sk, l = idx / sk;
        SAc[t + l * sk] = SAk[t + l * smax];
    }
}

// weights of iteration k from the trailing right singular vector
__global__ void aaa_store_w_kernel(const double *__restrict__ vk, int32_t k, int32_t K, double *__restrict__ wts,
                                   double *__restrict__ Wout) {
    for (int32_t l = threadIdx.x; l < K; l += blockDim.x) {
        const double v = (l < k) ? vk[l] : 0.0;
        if (l < k) wts[l] = v;
        Wout[(int64_t)(k - 1) * K + l] = v;
    }
}

// r at every point and |f - r| (0 at support points)
__global__ void __launch_bounds__(kAaaThreads) aaa_eval_kernel(const double *__restrict__ x,
                                                               const double *__restrict__ f,
                                                               const unsigned char *__restrict__ sup,
                                                               const long long *__restrict__ support,
                                                               const double *__restrict__ wts, int32_t k, int64_t m,
                                                               double *__restrict__ err) {
    extern __shared__ double sh[];  // xs, fs, ws (k each)
    double *xs = sh, *fs = sh + k, *ws = sh + 2 * k;
    for (int32_t l = threadIdx.x; l < k; l += blockDim.x) {
        xs[l] = x[support[l]];
        fs[l] = f[support[l]];
        ws[l] = wts[l];
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        if (sup[i]) {
            err[i] = 0.0;
            continue;
        }
        const double xi = x[i];
        double num = 0.0, den = 0.0;
        for (int32_t l = 0; l < k; ++l) {
            const double cl = ws[l] / (xi - xs[l]);
            num += cl * fs[l];
            den += cl;
        }
        err[i] = fabs(f[i] - num / den);
    }
}

cudaError_t launch_aaa(uint64_t seed, const double *x, const double *f, int64_t m, int32_t K, int64_t smax,
                       const long long *forced, long long *support, double *Wout, double *errmax, double *SAk_out,
                       int32_t *status, void *ws, cudaStream_t st) {
    Carver c(ws);
    AaaWork w = aaa_carve(c, m, smax, K);
    const SrhtGeom g = srht_geom(m, 1);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(w.SAk, 0, sizeof(double) * (size_t)(smax * K), st);
    if (e != cudaSuccess) return e;
    e = launch_srht_meta(seed, g.lg, g.sign_words, smax, w.srht.sign_words, w.srht.rows, st);
    if (e != cudaSuccess) return e;
    aaa_init_kernel<<<1, kAaaThreads, 0, st>>>(f, m, w.mean, w.err, w.sup);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t dsmem = sizeof(double) * (size_t)(smax + 2 * K);
    e = cudaFuncSetAttribute(aaa_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
    if (e != cudaSuccess) return e;
    const int nb = kAaaEvalBlocks;
    for (int32_t k = 1; k <= K; ++k) {
        aaa_argmax_blocks<<<nb, kAaaThreads, 0, st>>>(w.err, w.sup, m, w.bval, w.bidx);
        aaa_argmax_final<<<1, 32, 0, st>>>(w.bval, w.bidx, nb, w.cur, errmax, k - 1);
        aaa_downdate_kernel<<<1, kAaaThreads, 0, st>>>(x, f, k, forced, w.cur, support, w.sup, w.SAk, smax,
                                                       w.srht.sign_words, w.srht.rows);
        aaa_column_kernel<<<nb, kAaaThreads, 0, st>>>(x, f, w.sup, w.cur, m, w.col);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        e = launch_srht_f64(w.col, m, 1, m, smax, w.srht, w.SAk + (int64_t)(k - 1) * smax, status, st);
        if (e != cudaSuccess) return e;
        const int64_t sk = (4 * (int64_t)k < smax) ? 4 * (int64_t)k : smax;
        if (k < kAaaWideFrom || sk < k) {  // small problems: one CTA, no grid-wide launches
            aaa_dense_kernel<<<1, kAaaThreads, dsmem, st>>>(w.SAk, smax, k, sk, w, Wout, K, status);
        } else {  // larger ones: the whole-GPU QR and cluster-ring Jacobi of ns_solve
            aaa_prefix_kernel<<<64, kAaaThreads, 0, st>>>(w.SAk, smax, k, sk, w.SAc);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            e = launch_dense_solve(w.SAc, sk, k, 1, w.dw, w.X, w.sigk, nullptr, nullptr, status, st);
            if (e != cudaSuccess) return e;
            aaa_store_w_kernel<<<1, kAaaThreads, 0, st>>>(w.X, k, K, w.w, Wout);
        }
        aaa_eval_kernel<<<nb, kAaaThreads, sizeof(double) * 3 * (size_t)k, st>>>(x, f, w.sup, support, w.w, k, m,
                                                                                 w.err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // error after the last iteration
    aaa_argmax_blocks<<<nb, kAaaThreads, 0, st>>>(w.err, w.sup, m, w.bval, w.bidx);
    aaa_argmax_final<<<1, 32, 0, st>>>(w.bval, w.bidx, nb, w.cur, errmax, K);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (SAk_out) e = cudaMemcpyAsync(SAk_out, w.SAk, sizeof(double) * (size_t)(smax * K), cudaMemcpyDeviceToDevice, st);
    return e;
}

}  // namespace ns
