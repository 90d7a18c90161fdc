// ns_batched.cu -- ns_solve_batched: Algorithm 1 on many independent problems
// of different shapes, e.g. total least squares [X_i b_i] (Section 4): the
// trailing right singular vector v of the sketch gives x = -v(1:n-1)/v(n).
//
// Stages (all problems at once, no host round trips):
//   setup   one CTA: per-problem workspace offsets and work-item ranges
//           (prefix sums over the device problem array);
//   meta    one CTA per problem: SRHT signs and sample rows from its seed;
//   sketch  persistent CTAs take (problem, panel of columns) items from an
//           atomic counter (uneven problems balance dynamically) and run, per
//           column, the exact fixed-point SRHT pipeline over its blocks (FP64
//           problems) or the FP32-stream pipeline (FP32 problems);
//   dense   persistent CTAs take whole problems from a second counter: pivoted
//           Householder QR, QR of R^T, one-sided Jacobi on R2^T with one warp
//           per pair, V = P Q2 Vx, extraction, TLS.
// Each problem's numerical status (non-finite input, no convergence, TLS
// without solution) goes to dev_status[i].
#include <cmath>
#include "ns_device.cuh"
#include "ns_internal.h"
#include "ns_srht_core.cuh"
#include "ns_dense_cta.cuh"

namespace ns {

constexpr int kBatchThreads = 256;

// Tuning of the batched launches (process-wide, set by ns_batched_tuning; 0 =
// the default).  None of them changes the arithmetic: a column is sketched and
// a problem solved the same way whatever the panel width or the grid sizes.
struct BatchTuning {
    int panel = 1;              // columns per sketch work item
    int sketch_ctas_per_sm = 0; // persistent sketch CTAs per SM (0: occupancy limit)
    int dense_ctas_per_sm = 0;  // persistent dense CTAs per SM (0: occupancy limit)
};
static BatchTuning g_batch_tuning;

bool set_batch_tuning(int panel, int sketch_cps, int dense_cps) {
    if (panel < 0 || panel > 64 || sketch_cps < 0 || sketch_cps > 64 || dense_cps < 0 || dense_cps > 64) return false;
    g_batch_tuning.panel = panel > 0 ? panel : 1;
    g_batch_tuning.sketch_ctas_per_sm = sketch_cps;
    g_batch_tuning.dense_ctas_per_sm = dense_cps;
    return true;
}

struct BatchSlot {
    int64_t off;       // byte offset of the problem's workspace
    int64_t item0;     // first sketch work item (one per panel of columns)
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
                                                             int64_t head, int panel) {
    __shared__ int64_t part_b[1024], part_i[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t per = (batch + nt - 1) / nt;
    const int64_t i0 = tid * per, i1 = (i0 + per < batch) ? i0 + per : batch;
    int64_t sb = 0, si = 0;
    for (int64_t i = i0; i < i1; ++i) {
        sb += problem_bytes(P[i].m, P[i].n, P[i].s);
        si += (P[i].n + panel - 1) / panel;
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
        oi += (P[i].n + panel - 1) / panel;
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
                                                            int32_t *status, int panel) {
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
        const int64_t c0 = (item - sl.item0) * panel;
        const int64_t c1 = (c0 + panel < pr.n) ? c0 + panel : pr.n;
        ProblemView v = problem_view(ws + sl.off, pr.m, pr.n, pr.s);
        const int64_t s = pr.s;
        for (int64_t i = t; i < s; i += 64) rows_s[i] = srht_pack_row(v.rows[i]);
        int nonfinite = 0;
        for (int64_t c = c0; c < c1; ++c) {
            double *out = v.SA + c * s;
            if (pr.dtype == NS_F32) {  // FP32-stream: FP32 butterflies and accumulation
                float *accf = (float *)acc;
                for (int64_t i = t; i < s; i += 64) accf[i] = 0.0f;
                __syncthreads();
                const float *Acol = (const float *)pr.A + c * pr.lda;
                const int vec_ok = ((((uintptr_t)pr.A) & 7) == 0 && (pr.lda & 1) == 0) ? 1 : 0;
                for (int64_t b = 0; b < sl.nblk; ++b)
                    srht_f32_block(Acol, pr.m, s, b, v.sign_words, rows_s, (float *)Zs, accf, sgn, vec_ok,
                                   nonfinite);
                const double scale = 1.0 / sqrt((double)s);
                for (int64_t i = t; i < s; i += 64) out[i] = (double)accf[i] * scale;
            } else {  // FP64: exact fixed point
                for (int64_t i = t; i < s; i += 64) acc[i] = 0;
                __syncthreads();
                const double *Acol = (const double *)pr.A + c * pr.lda;
                const int vec_ok = ((((uintptr_t)pr.A) & 15) == 0 && (pr.lda & 1) == 0) ? 1 : 0;
                const int P_bits = 63 - kBlockLog - clog2(sl.nblk);
                int Erun = 0;
                for (int64_t b = 0; b < sl.nblk; ++b)
                    srht_f64_block(Acol, pr.m, s, b, P_bits, v.sign_words, rows_s, Zs, acc, sgn, red, vec_ok, Erun,
                                   nonfinite, b + 1 < sl.nblk);
                const double scale = ldexp(1.0, Erun - 1022 - P_bits) / sqrt((double)s);
                for (int64_t i = t; i < s; i += 64) out[i] = (double)acc[i] * scale;
            }
            __syncthreads();
        }
        if (nonfinite) atomicMax(status + lo, (int32_t)NS_ERR_NONFINITE);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBatchThreads) batched_dense_kernel(const ns_problem *__restrict__ P, int32_t batch,
                                                                      const BatchSlot *__restrict__ slots, char *ws,
                                                                      unsigned long long *counters, int32_t *status) {
    extern __shared__ double dsh[];  // xs (smax), nrm, nref (nmax each)
    __shared__ long long prob_sh;
    __shared__ long long bk[32];
    const int tid = threadIdx.x;
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
        DenseScratch scr{v.X, v.V, v.L, v.u0a, v.cfa, v.u0b, v.cfb, v.sigma, v.perm};
        if (!dense_solve_cta(v.SA, s, n, pr.k, scr, xs, nrm, nref, pr.Vk, pr.sigk) && tid == 0)
            atomicMax(status + pi, (int32_t)NS_ERR_NOCONV);
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

static int sm_count_b() { return device_sm_count(); }

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
    const BatchTuning tu = g_batch_tuning;
    batched_setup_kernel<<<1, 1024, 0, st>>>(dev, batch, slots, counters, head, tu.panel);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    batched_meta_kernel<<<(unsigned)batch, 256, 0, st>>>(dev, slots, base);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = (size_t)kBlock * 8 + (size_t)smax * 8 + 64 * 8 + 128 * 4 + 16 + (size_t)smax * 4;
    e = cudaFuncSetAttribute(batched_sketch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_sketch_kernel, 64, smem);
    if (per_sm < 1) per_sm = 1;
    if (tu.sketch_ctas_per_sm > 0 && tu.sketch_ctas_per_sm < per_sm) per_sm = tu.sketch_ctas_per_sm;
    const int grid1 = sm_count_b() * per_sm;
    batched_sketch_kernel<<<grid1, 64, smem, st>>>(dev, batch, slots, base, counters, smax, status, tu.panel);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t dsmem = sizeof(double) * (size_t)(smax + 2 * nmax);
    e = cudaFuncSetAttribute(batched_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
    if (e != cudaSuccess) return e;
    int per_sm2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, batched_dense_kernel, kBatchThreads, dsmem);
    if (per_sm2 < 1) per_sm2 = 1;
    if (tu.dense_ctas_per_sm > 0 && tu.dense_ctas_per_sm < per_sm2) per_sm2 = tu.dense_ctas_per_sm;
    int64_t grid2 = (int64_t)sm_count_b() * per_sm2;
    if (grid2 > batch) grid2 = batch;
    batched_dense_kernel<<<(unsigned)grid2, kBatchThreads, dsmem, st>>>(dev, batch, slots, base, counters, status);
    return cudaGetLastError();
}

}  // namespace ns
