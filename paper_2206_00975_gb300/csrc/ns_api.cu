// ns_api.cu -- the extern "C" entry points of libns (see include/ns.h).
//
// Every entry point validates its arguments on the host, carves the caller's
// workspace, enqueues kernels on the caller's stream and returns; nothing is
// allocated, freed or synchronised here.
#include <cmath>
#include <cstring>
#include <mutex>
#include "ns_device.cuh"
#include "ns_internal.h"

namespace ns {

constexpr int64_t kMaxN = 4096;    // columns handled by the dense kernels

int device_sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 1;
    }
    if (cached[dev] > 0) return cached[dev];
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return 1;
    }
    cached[dev] = sms;
    return sms;
}

static bool desc_ok(const ns_sketch_desc *d) {
    if (!d) return false;
    if (d->kind < NS_SRHT || d->kind > NS_HRHT) return false;
    if (d->prec < NS_PREC_FP64 || d->prec > NS_PREC_BF16X3) return false;
    if (d->s < 1 || d->s > kMaxS) return false;
    if (d->kind == NS_SPARSE_SIGN && (d->zeta < 1 || d->zeta > 64 || d->zeta > d->s)) return false;
    if (d->max_sweeps < 0 || d->max_sweeps > 30) return false;
    return true;
}

// (kind, prec, dtype) triples with a GPU path
static bool path_ok(const ns_sketch_desc *d, int32_t dtype) {
    if (d->kind == NS_SRHT)
        return (d->prec == NS_PREC_FP64 && dtype == NS_F64) || (d->prec == NS_PREC_FP32_STREAM && dtype == NS_F32);
    if (d->kind == NS_SPARSE_SIGN) return d->prec == NS_PREC_FP64 && dtype == NS_F64;
    if (d->kind == NS_GAUSSIAN) return d->prec == NS_PREC_BF16X3 && dtype == NS_F32;
    if (d->kind == NS_HRHT) return d->prec == NS_PREC_FP64 && dtype == NS_F64;
    return false;
}

static bool shape_ok(const ns_sketch_desc *d, int64_t m, int64_t n, int64_t lda) {
    if (m < 1 || n < 1 || lda < m) return false;
    if (d->kind == NS_GAUSSIAN && n > 512) return false;
    if ((d->kind == NS_SRHT || d->kind == NS_HRHT) && d->s > ((int64_t)1 << ceil_log2(m))) return false;
    if (d->kind == NS_HRHT && ceil_log2(m) > 24) return false;  // at most 4096 blocks across
    return true;
}

struct SolveLayout {
    int32_t *status_word;
    SrhtWork srht;
    SparseWork sparse;
    HrhtWork hrht;
    float *gauss_partial;
    double *SA;
    DenseWork dense;
    size_t bytes;
};

// the sketch's scratch (and SA when need_sa) of one solve
static void carve_sketch(Carver &c, const ns_sketch_desc *d, int64_t m, int64_t n, bool need_sa, SolveLayout &L) {
    L.srht = SrhtWork{nullptr, nullptr, nullptr};
    L.sparse = SparseWork{nullptr, nullptr, nullptr};
    if (d->kind == NS_SRHT) L.srht = srht_carve(c, m, n, d->s);
    if (d->kind == NS_SPARSE_SIGN) L.sparse = sparse_carve(c, m, n, d->s, d->zeta);
    L.hrht = HrhtWork{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (d->kind == NS_HRHT) L.hrht = hrht_carve(c, m, n, d->s);
    L.gauss_partial = nullptr;
    if (d->kind == NS_GAUSSIAN) {
        const GaussGeom g = gauss_geom(m, n, d->s);
        L.gauss_partial = c.take<float>((size_t)(g.nsplit * n * d->s));
    }
    L.SA = need_sa ? c.take<double>((size_t)(d->s * n)) : nullptr;
}

static SolveLayout solve_layout(void *ws, const ns_sketch_desc *d, int64_t m, int64_t n, bool need_sa) {
    Carver c(ws);
    SolveLayout L;
    L.status_word = c.take<int32_t>(1);
    carve_sketch(c, d, m, n, need_sa, L);
    L.dense = dense_carve(c, d->s, n);
    L.bytes = c.used;
    return L;
}

// ns_solve_pipelined: kPipeLanes lanes, each with two sketch slots (scratch
// and SA) and a dense workspace, after one status word
constexpr int kPipeLanes = 3;
struct PipeLayout {
    int32_t *status_word;
    SolveLayout slot[kPipeLanes][2];
    DenseWork dense[kPipeLanes];
    size_t bytes;
};

static PipeLayout pipe_layout(void *ws, const ns_sketch_desc *d, int64_t m, int64_t n) {
    Carver c(ws);
    PipeLayout L;
    L.status_word = c.take<int32_t>(1);
    for (int l = 0; l < kPipeLanes; ++l) {
        for (int i = 0; i < 2; ++i) carve_sketch(c, d, m, n, true, L.slot[l][i]);
        L.dense[l] = dense_carve(c, d->s, n);
    }
    L.bytes = c.used;
    return L;
}

static ns_status cuda_status(cudaError_t e) { return e == cudaSuccess ? NS_OK : NS_ERR_CUDA; }

static ns_status run_sketch(const ns_sketch_desc *d, const void *A, int64_t m, int64_t n, int64_t lda, double *SA,
                            const SolveLayout &L, int32_t *status, cudaStream_t st) {
    if (d->kind == NS_GAUSSIAN)
        return cuda_status(launch_gauss_bf16x3(d->seed, (const float *)A, m, n, lda, d->s, L.gauss_partial, SA, status,
                                               st));
    if (d->kind == NS_HRHT)
        return cuda_status(launch_hrht_f64(d->seed, (const double *)A, m, n, lda, d->s, L.hrht, SA, status, st));
    if (d->kind == NS_SPARSE_SIGN)
        return cuda_status(launch_sparse_f64(d->seed, (const double *)A, m, n, lda, d->s, d->zeta, L.sparse, SA,
                                             status, st));
    const SrhtWork &w = L.srht;
    const SrhtGeom g = srht_geom(m, n);
    cudaError_t e = launch_srht_meta(d->seed, g.lg, g.sign_words, d->s, w.sign_words, w.rows, st);
    if (e != cudaSuccess) return NS_ERR_CUDA;
    if (d->prec == NS_PREC_FP32_STREAM)
        return cuda_status(launch_srht_f32((const float *)A, m, n, lda, d->s, w, SA, status, st));
    return cuda_status(launch_srht_f64((const double *)A, m, n, lda, d->s, w, SA, status, st));
}

// ---------------------------------------------------------------- residual --
// One thread per row: y = A(row, :) W, accumulated in FP64.  K is the number
// of columns of W rounded up to a power of two, so no predicated-off FP64 FMA
// occupies the (slow) FP64 pipe.
template <int K>
__global__ void __launch_bounds__(256) residual_rows_kernel(const double *__restrict__ A, int64_t m, int64_t n,
                                                            int64_t lda, const double *__restrict__ W, int32_t k,
                                                            double *__restrict__ partial) {
    extern __shared__ double wsh[];  // n * K, row-major: wsh[j * K + c]
    __shared__ double red[32];
    for (int64_t i = threadIdx.x; i < n * K; i += blockDim.x) {
        const int64_t j = i / K, c = i - j * K;
        wsh[i] = (c < k) ? W[j + c * n] : 0.0;
    }
    __syncthreads();
    double ss = 0.0;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < m; row += (int64_t)gridDim.x * blockDim.x) {
        double y[K];
#pragma unroll
        for (int c = 0; c < K; ++c) y[c] = 0.0;
        const double *a_row = A + row;
        int64_t j = 0;
        for (; j + 4 <= n; j += 4) {
            double a[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = __ldcs(a_row + (j + u) * lda);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int c = 0; c < K; ++c) y[c] = fma(a[u], wsh[(j + u) * K + c], y[c]);
        }
        for (; j < n; ++j) {
            const double a = __ldcs(a_row + j * lda);
#pragma unroll
            for (int c = 0; c < K; ++c) y[c] = fma(a, wsh[j * K + c], y[c]);
        }
#pragma unroll
        for (int c = 0; c < K; ++c) ss = fma(y[c], y[c], ss);
    }
    double v[1] = {ss};
    block_sum<1>(v, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = v[0];
}

__global__ void residual_final_kernel(const double *partial, int64_t np, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0;
        for (int64_t i = 0; i < np; ++i) a += partial[i];  // fixed order
        *out = sqrt(a);
    }
}

template <int K>
static cudaError_t launch_residual(const double *A, int64_t m, int64_t n, int64_t lda, const double *W, int32_t k,
                                   double *partial, int64_t blocks, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(residual_rows_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    residual_rows_kernel<K><<<(unsigned)blocks, 256, smem, st>>>(A, m, n, lda, W, k, partial);
    return cudaGetLastError();
}

}  // namespace ns

using namespace ns;

extern "C" {

const char *ns_status_string(int status) {
    switch (status) {
        case NS_OK: return "NS_OK";
        case NS_ERR_INVALID_ARG: return "NS_ERR_INVALID_ARG";
        case NS_ERR_WORKSPACE: return "NS_ERR_WORKSPACE";
        case NS_ERR_NONFINITE: return "NS_ERR_NONFINITE";
        case NS_ERR_NOCONV: return "NS_ERR_NOCONV";
        case NS_ERR_TLS_NOSOLUTION: return "NS_ERR_TLS_NOSOLUTION";
        case NS_ERR_TIMEOUT: return "NS_ERR_TIMEOUT";
        case NS_ERR_CUDA: return "NS_ERR_CUDA";
        default: return "NS_ERR_UNKNOWN";
    }
}

const char *ns_version(void) { return "libns 0.1 (sm_103a)"; }

int64_t ns_save_size(int64_t s, int64_t n) { return s * n + n * n + n; }

size_t ns_workspace_size(const ns_sketch_desc *d, int64_t m, int64_t n, int32_t k) {
    if (!desc_ok(d) || m < 1 || n < 1 || n > kMaxN || k < 0) return 0;
    size_t need = solve_layout(nullptr, d, m, n, true).bytes;
    const size_t resid = align256(sizeof(double) * 4096);
    need = need > resid ? need : resid;
    if (d->kind == NS_SRHT && k >= 1 && k < n) {
        const size_t bw = backward_work_bytes(m, n, d->s, k);
        need = need > bw ? need : bw;
    }
    return need;
}

ns_status ns_sketch(const ns_sketch_desc *d, const void *A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                    double *SA, void *ws, size_t ws_bytes, void *stream) {
    if (!desc_ok(d) || !A || !SA || !ws) return NS_ERR_INVALID_ARG;
    if (!path_ok(d, dtype) || !shape_ok(d, m, n, lda)) return NS_ERR_INVALID_ARG;
    if ((((uintptr_t)ws) & 255) != 0 || (((uintptr_t)A) & (dtype == NS_F32 ? 3 : 7)) != 0) return NS_ERR_INVALID_ARG;
    SolveLayout L = solve_layout(ws, d, m, n, false);
    if (L.bytes > ws_bytes) return NS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(L.status_word, 0, sizeof(int32_t), st) != cudaSuccess) return NS_ERR_CUDA;
    return run_sketch(d, A, m, n, lda, SA, L, L.status_word, st);
}

static bool rows_ok(const ns_sketch_desc *d, int32_t dtype, int64_t m_total, int64_t o, int64_t m_p, int64_t n) {
    if (!desc_ok(d) || d->prec != NS_PREC_FP64 || dtype != NS_F64) return false;
    if (d->kind != NS_SRHT && d->kind != NS_SPARSE_SIGN) return false;
    if (m_total < 1 || o < 0 || m_p < 1 || o + m_p > m_total || n < 1) return false;
    if (d->kind == NS_SRHT && d->s > ((int64_t)1 << ceil_log2(m_total))) return false;
    return true;
}

static size_t rows_layout(void *ws, const ns_sketch_desc *d, int64_t m_total, int64_t o, int64_t m_p, int64_t n,
                          int32_t **status_word, SrhtWork *sw, SparseWork *pw) {
    Carver c(ws);
    *status_word = c.take<int32_t>(1);
    if (d->kind == NS_SRHT) *sw = srht_rows_carve(c, m_total, o, o + m_p, n, d->s);
    else *pw = sparse_carve(c, m_p, n, d->s, d->zeta);
    return c.used;
}

size_t ns_sketch_rows_workspace_size(const ns_sketch_desc *d, int64_t m_total, int64_t o, int64_t m_p, int64_t n) {
    if (!d || !rows_ok(d, NS_F64, m_total, o, m_p, n)) return 0;
    int32_t *sw_;
    SrhtWork a;
    SparseWork b;
    return rows_layout(nullptr, d, m_total, o, m_p, n, &sw_, &a, &b);
}

ns_status ns_sketch_rows(const ns_sketch_desc *d, const void *A_p, int32_t dtype, int64_t m_total, int64_t o,
                         int64_t m_p, int64_t n, int64_t lda, double *SA_p, int32_t *dev_status, void *ws,
                         size_t ws_bytes, void *stream) {
    if (!d || !A_p || !SA_p || !ws || !rows_ok(d, dtype, m_total, o, m_p, n) || lda < m_p) return NS_ERR_INVALID_ARG;
    if ((((uintptr_t)ws) & 255) != 0 || (((uintptr_t)A_p) & 7) != 0) return NS_ERR_INVALID_ARG;
    int32_t *status_word;
    SrhtWork sw{nullptr, nullptr, nullptr};
    SparseWork pw{nullptr, nullptr, nullptr};
    if (rows_layout(ws, d, m_total, o, m_p, n, &status_word, &sw, &pw) > ws_bytes) return NS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *status = dev_status ? dev_status : status_word;
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return NS_ERR_CUDA;
    if (d->kind == NS_SPARSE_SIGN)
        return cuda_status(
            launch_sparse_f64(d->seed, (const double *)A_p, m_p, n, lda, d->s, d->zeta, pw, SA_p, status, st, o));
    const SrhtRowsGeom g = srht_rows_geom(m_total, o, o + m_p, n);
    if (launch_srht_meta(d->seed, g.lg, g.sign_words, d->s, sw.sign_words, sw.rows, st) != cudaSuccess)
        return NS_ERR_CUDA;
    return cuda_status(launch_srht_f64_rows((const double *)A_p, m_total, o, o + m_p, n, lda, d->s, sw, SA_p, status,
                                            st));
}

ns_status ns_solve(const ns_sketch_desc *d, const void *A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                   int32_t k, double *Vk, double *sigk, double *save, int32_t *dev_status, void *ws, size_t ws_bytes,
                   void *stream) {
    if (!desc_ok(d) || !A || !Vk || !sigk || !ws) return NS_ERR_INVALID_ARG;
    if (!path_ok(d, dtype) || !shape_ok(d, m, n, lda)) return NS_ERR_INVALID_ARG;
    if (m < n || n > d->s || n > kMaxN || k < 1 || k > n) return NS_ERR_INVALID_ARG;
    if ((((uintptr_t)ws) & 255) != 0 || (((uintptr_t)A) & (dtype == NS_F32 ? 3 : 7)) != 0) return NS_ERR_INVALID_ARG;
    SolveLayout L = solve_layout(ws, d, m, n, save == nullptr);
    if (L.bytes > ws_bytes) return NS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *status = dev_status ? dev_status : L.status_word;
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return NS_ERR_CUDA;
    double *SA = save ? save : L.SA;
    ns_status r = run_sketch(d, A, m, n, lda, SA, L, status, st);
    if (r != NS_OK) return r;
    double *save_V = save ? save + d->s * n : nullptr;
    double *save_sigma = save ? save + d->s * n + n * n : nullptr;
    return cuda_status(
        launch_dense_solve(SA, d->s, n, k, L.dense, Vk, sigk, save_V, save_sigma, status, st, d->max_sweeps));
}

size_t ns_solve_pipelined_workspace_size(const ns_sketch_desc *d, int64_t m, int64_t n) {
    if (!desc_ok(d) || m < 1 || n < 1 || n > kMaxN) return 0;
    return pipe_layout(nullptr, d, m, n).bytes;
}

// The library's streams per device: for each lane a dense stream (higher
// priority) and a sketch stream, and the events that order them.
struct PipeRes {
    cudaStream_t dense[kPipeLanes] = {}, sketch[kPipeLanes] = {};
    cudaEvent_t in = nullptr, out[kPipeLanes] = {}, after_qr[kPipeLanes] = {}, sk[kPipeLanes][2] = {};
};

static PipeRes *pipe_resources() {
    static std::mutex mu;
    static PipeRes res[64];
    static bool made[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!made[dev]) {
        int lo = 0, hi = 0;
        PipeRes r;
        if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) return nullptr;
        if (cudaEventCreateWithFlags(&r.in, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        for (int l = 0; l < kPipeLanes; ++l) {
            if (cudaStreamCreateWithPriority(&r.dense[l], cudaStreamNonBlocking, hi) != cudaSuccess ||
                cudaStreamCreateWithPriority(&r.sketch[l], cudaStreamNonBlocking, lo) != cudaSuccess)
                return nullptr;
            cudaEvent_t *evs[] = {&r.out[l], &r.after_qr[l], &r.sk[l][0], &r.sk[l][1]};
            for (cudaEvent_t *e : evs)
                if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        }
        res[dev] = r;
        made[dev] = true;
    }
    return &res[dev];
}

// Problems i = l, l + kPipeLanes, ... go to lane l, so several dense stages
// are in flight (the dense stage is bound by FP64 latency chains, and a few
// of them share the SMs well).  Within a lane, the sketch of the lane's next
// problem waits for the event the dense launcher records once the QRs are
// done, and runs at the lower priority beside the rest of that dense stage.
ns_status ns_solve_pipelined(const ns_sketch_desc *d, const void *const *A, int32_t count, int32_t dtype, int64_t m,
                             int64_t n, int64_t lda, int32_t k, double *Vk, double *sigk, int32_t *dev_status,
                             void *ws, size_t ws_bytes, void *stream) {
    if (!desc_ok(d) || !A || count < 1 || !Vk || !sigk || !ws) return NS_ERR_INVALID_ARG;
    if (!path_ok(d, dtype) || !shape_ok(d, m, n, lda)) return NS_ERR_INVALID_ARG;
    if (m < n || n > d->s || n > kMaxN || k < 1 || k > n) return NS_ERR_INVALID_ARG;
    if ((((uintptr_t)ws) & 255) != 0) return NS_ERR_INVALID_ARG;
    for (int32_t i = 0; i < count; ++i)
        if (!A[i] || (((uintptr_t)A[i]) & (dtype == NS_F32 ? 3 : 7)) != 0) return NS_ERR_INVALID_ARG;
    const PipeLayout L = pipe_layout(ws, d, m, n);
    if (L.bytes > ws_bytes) return NS_ERR_WORKSPACE;
    PipeRes *R = pipe_resources();
    if (!R) return NS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *status = dev_status ? dev_status : L.status_word;
    const size_t nstat = dev_status ? (size_t)count : 1;
    if (cudaMemsetAsync(status, 0, sizeof(int32_t) * nstat, st) != cudaSuccess) return NS_ERR_CUDA;
    if (cudaEventRecord(R->in, st) != cudaSuccess) return NS_ERR_CUDA;
    for (int l = 0; l < kPipeLanes; ++l)
        if (cudaStreamWaitEvent(R->dense[l], R->in, 0) != cudaSuccess ||
            cudaStreamWaitEvent(R->sketch[l], R->in, 0) != cudaSuccess)
            return NS_ERR_CUDA;
    auto stat = [&](int32_t i) { return dev_status ? dev_status + i : L.status_word; };
    const int lanes = count < kPipeLanes ? count : kPipeLanes;
    for (int l = 0; l < lanes; ++l) {  // each lane's first sketch
        const ns_status r = run_sketch(d, A[l], m, n, lda, L.slot[l][0].SA, L.slot[l][0], stat(l), R->sketch[l]);
        if (r != NS_OK) return r;
        if (cudaEventRecord(R->sk[l][0], R->sketch[l]) != cudaSuccess) return NS_ERR_CUDA;
    }
    for (int32_t i = 0; i < count; ++i) {
        const int l = i % kPipeLanes, p = (i / kPipeLanes) & 1;
        const int32_t next = i + kPipeLanes;  // the lane's next problem
        const bool more = next < count;
        if (cudaStreamWaitEvent(R->dense[l], R->sk[l][p], 0) != cudaSuccess) return NS_ERR_CUDA;
        const cudaError_t e = launch_dense_solve(L.slot[l][p].SA, d->s, n, k, L.dense[l], Vk + (int64_t)i * n * k,
                                                 sigk + (int64_t)i * k, nullptr, nullptr, stat(i), R->dense[l],
                                                 d->max_sweeps, true, more ? R->after_qr[l] : nullptr);
        if (e != cudaSuccess) return NS_ERR_CUDA;
        if (more) {
            // the lane's next sketch once this dense stage is past its QRs; its
            // slot's SA was last read by the lane's previous dense stage,
            // finished before this one began
            if (cudaStreamWaitEvent(R->sketch[l], R->after_qr[l], 0) != cudaSuccess) return NS_ERR_CUDA;
            const ns_status r = run_sketch(d, A[next], m, n, lda, L.slot[l][p ^ 1].SA, L.slot[l][p ^ 1], stat(next),
                                           R->sketch[l]);
            if (r != NS_OK) return r;
            if (cudaEventRecord(R->sk[l][p ^ 1], R->sketch[l]) != cudaSuccess) return NS_ERR_CUDA;
        }
    }
    for (int l = 0; l < kPipeLanes; ++l)
        if (cudaEventRecord(R->out[l], R->dense[l]) != cudaSuccess ||
            cudaStreamWaitEvent(st, R->out[l], 0) != cudaSuccess)
            return NS_ERR_CUDA;
    return NS_OK;
}

ns_status ns_solve_eps(const ns_sketch_desc *d, const void *A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                       double eps, double *Vk, double *sigk, int32_t *dev_k, double *save, int32_t *dev_status,
                       void *ws, size_t ws_bytes, void *stream) {
    if (!desc_ok(d) || !A || !Vk || !sigk || !dev_k || !ws) return NS_ERR_INVALID_ARG;
    if (!path_ok(d, dtype) || !shape_ok(d, m, n, lda)) return NS_ERR_INVALID_ARG;
    if (m < n || n > d->s || n > kMaxN || !(eps >= 0.0)) return NS_ERR_INVALID_ARG;
    if ((((uintptr_t)ws) & 255) != 0 || (((uintptr_t)A) & (dtype == NS_F32 ? 3 : 7)) != 0) return NS_ERR_INVALID_ARG;
    SolveLayout L = solve_layout(ws, d, m, n, save == nullptr);
    if (L.bytes > ws_bytes) return NS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *status = dev_status ? dev_status : L.status_word;
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return NS_ERR_CUDA;
    double *SA = save ? save : L.SA;
    ns_status r = run_sketch(d, A, m, n, lda, SA, L, status, st);
    if (r != NS_OK) return r;
    double *save_V = save ? save + d->s * n : nullptr;
    double *save_sigma = save ? save + d->s * n + n * n : nullptr;
    cudaError_t e =
        launch_dense_solve(SA, d->s, n, 0, L.dense, nullptr, nullptr, save_V, save_sigma, status, st, d->max_sweeps);
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(launch_dense_select_eps(L.dense, n, eps, Vk, sigk, dev_k, st));
}

ns_status ns_sketch_update(const ns_sketch_desc *d, int64_t m0, int32_t op, int64_t j, const double *row, int64_t n,
                           double *SA, void *stream) {
    if (!desc_ok(d) || !row || !SA) return NS_ERR_INVALID_ARG;
    if (m0 < 1 || n < 1 || j < 0 || (op != NS_ROW_APPEND && op != NS_ROW_REMOVE)) return NS_ERR_INVALID_ARG;
    if (op == NS_ROW_APPEND && j < m0) return NS_ERR_INVALID_ARG;
    if (d->kind == NS_HRHT) return NS_ERR_INVALID_ARG;
    if (d->kind == NS_SRHT && d->s > ((int64_t)1 << ceil_log2(m0 > kBlock ? m0 : kBlock))) return NS_ERR_INVALID_ARG;
    if (n > kMaxN * 64) return NS_ERR_INVALID_ARG;
    return cuda_status(launch_sketch_update(d->kind, d->seed, d->s, d->zeta, m0, op, j, row, n, SA,
                                            (cudaStream_t)stream));
}

ns_status ns_solve_sketched(const ns_sketch_desc *d, const double *SA, int64_t n, int32_t k, double *Vk, double *sigk,
                           double *save, int32_t *dev_status, void *ws, size_t ws_bytes, void *stream) {
    if (!desc_ok(d) || !SA || !Vk || !sigk || !ws) return NS_ERR_INVALID_ARG;
    if (n < 1 || n > d->s || n > kMaxN || k < 1 || k > n) return NS_ERR_INVALID_ARG;
    if ((((uintptr_t)ws) & 255) != 0) return NS_ERR_INVALID_ARG;
    Carver c(ws);
    int32_t *status_word = c.take<int32_t>(1);
    DenseWork w = dense_carve(c, d->s, n);
    if (c.used > ws_bytes) return NS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *status = dev_status ? dev_status : status_word;
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return NS_ERR_CUDA;
    double *save_V = nullptr, *save_sigma = nullptr;
    if (save) {
        if (cudaMemcpyAsync(save, SA, sizeof(double) * (size_t)(d->s * n), cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return NS_ERR_CUDA;
        save_V = save + d->s * n;
        save_sigma = save + d->s * n + n * n;
    }
    return cuda_status(launch_dense_solve(SA, d->s, n, k, w, Vk, sigk, save_V, save_sigma, status, st, d->max_sweeps));
}

ns_status ns_solve_stats(const ns_sketch_desc *d, int64_t m, int64_t n, const void *ws, int64_t *dev_out,
                         void *stream) {
    if (!desc_ok(d) || !ws || !dev_out || m < 1 || n < 1 || n > kMaxN) return NS_ERR_INVALID_ARG;
    SolveLayout L = solve_layout(const_cast<void *>(ws), d, m, n, true);
    return cuda_status(launch_dense_stats(L.dense, dev_out, (cudaStream_t)stream));
}

ns_status ns_sketched_stats(const ns_sketch_desc *d, int64_t n, const void *ws, int64_t *dev_out, void *stream) {
    if (!desc_ok(d) || !ws || !dev_out || n < 1 || n > kMaxN) return NS_ERR_INVALID_ARG;
    Carver c(const_cast<void *>(ws));
    c.take<int32_t>(1);
    DenseWork w = dense_carve(c, d->s, n);
    return cuda_status(launch_dense_stats(w, dev_out, (cudaStream_t)stream));
}

ns_status ns_backward(const ns_sketch_desc *d, int64_t m, int64_t n, int32_t k, const double *save, const double *Vk,
                      const double *dVk, double *dA, int64_t ldd, void *ws, size_t ws_bytes, void *stream) {
    if (!desc_ok(d) || d->kind != NS_SRHT || d->prec != NS_PREC_FP64) return NS_ERR_INVALID_ARG;
    if (!save || !Vk || !dVk || !dA || !ws) return NS_ERR_INVALID_ARG;
    if (m < n || n < 2 || n > kMaxN || k < 1 || k >= n || n > d->s || ldd < m) return NS_ERR_INVALID_ARG;
    if (d->s > ((int64_t)1 << ceil_log2(m))) return NS_ERR_INVALID_ARG;
    if ((((uintptr_t)ws) & 255) != 0) return NS_ERR_INVALID_ARG;
    Carver c(ws);
    BackwardWork w = backward_carve(c, m, n, d->s, k);
    if (c.used > ws_bytes) return NS_ERR_WORKSPACE;
    return cuda_status(launch_backward(d->seed, m, n, k, d->s, save, Vk, dVk, dA, ldd, w, (cudaStream_t)stream));
}

static bool problem_ok(const ns_problem &p) {
    if (!p.A || !p.Vk || !p.sigk) return false;
    if (p.dtype != NS_F64 && p.dtype != NS_F32) return false;
    if (p.m < 1 || p.n < 1 || p.m < p.n || p.lda < p.m || p.n > kMaxN) return false;
    if (p.s < p.n || p.s > kMaxS || p.s > ((int64_t)1 << ceil_log2(p.m))) return false;
    if (p.k < 1 || p.k > p.n) return false;
    if (p.tls && (p.k != 1 || p.n < 2 || !p.x)) return false;
    if ((((uintptr_t)p.A) & (p.dtype == NS_F32 ? 3 : 7)) != 0) return false;
    return true;
}

static bool batch_desc_ok(const ns_sketch_desc *d) {
    return d && d->kind == NS_SRHT && (d->prec == NS_PREC_FP64 || d->prec == NS_PREC_FP32_STREAM);
}

size_t ns_batched_workspace_size(const ns_sketch_desc *d, int32_t batch, const ns_problem *host) {
    if (!batch_desc_ok(d) || batch < 1 || !host) return 0;
    for (int32_t i = 0; i < batch; ++i)
        if (!problem_ok(host[i])) return 0;
    return batched_work_bytes(batch, host);
}

ns_status ns_solve_batched(const ns_sketch_desc *d, int32_t batch, const ns_problem *host, const ns_problem *dev,
                           int32_t *dev_status, void *ws, size_t ws_bytes, void *stream) {
    if (!batch_desc_ok(d)) return NS_ERR_INVALID_ARG;
    if (batch < 1 || !host || !dev || !dev_status || !ws) return NS_ERR_INVALID_ARG;
    if ((((uintptr_t)ws) & 255) != 0) return NS_ERR_INVALID_ARG;
    for (int32_t i = 0; i < batch; ++i)
        if (!problem_ok(host[i])) return NS_ERR_INVALID_ARG;
    if (batched_work_bytes(batch, host) > ws_bytes) return NS_ERR_WORKSPACE;
    return cuda_status(launch_batched(batch, host, dev, dev_status, ws, (cudaStream_t)stream));
}

static bool aaa_ok(const ns_sketch_desc *d, int64_t m, int32_t K) {
    if (!d || d->kind != NS_SRHT || d->prec != NS_PREC_FP64) return false;
    if (m < 2 || K < 1 || K > 1024 || d->s < K || d->s > kMaxS) return false;
    if (d->s > ((int64_t)1 << ceil_log2(m))) return false;
    return true;
}

size_t ns_aaa_workspace_size(const ns_sketch_desc *d, int64_t m, int32_t K) {
    if (!aaa_ok(d, m, K)) return 0;
    return aaa_work_bytes(m, d->s, K);
}

ns_status ns_aaa_real(const ns_sketch_desc *d, const double *x, const double *f, int64_t m, int32_t K,
                      const int64_t *forced, int64_t *support, double *W, double *errmax, double *SAk_out,
                      int32_t *dev_status, void *ws, size_t ws_bytes, void *stream) {
    if (!aaa_ok(d, m, K) || !x || !f || !support || !W || !errmax || !dev_status || !ws) return NS_ERR_INVALID_ARG;
    if ((((uintptr_t)ws) & 255) != 0) return NS_ERR_INVALID_ARG;
    if (aaa_work_bytes(m, d->s, K) > ws_bytes) return NS_ERR_WORKSPACE;
    return cuda_status(launch_aaa(d->seed, x, f, m, K, d->s, (const long long *)forced, (long long *)support, W,
                                  errmax, SAk_out, dev_status, ws, (cudaStream_t)stream));
}

ns_status ns_residual(const void *A, int32_t dtype, int64_t m, int64_t n, int64_t lda, const double *W, int32_t k,
                      double *out, void *ws, size_t ws_bytes, void *stream) {
    if (!A || !W || !out || !ws || dtype != NS_F64) return NS_ERR_INVALID_ARG;
    if (m < 1 || n < 1 || lda < m || k < 1 || k > 16 || n > kMaxN) return NS_ERR_INVALID_ARG;
    const int64_t blocks = 1024;
    if (ws_bytes < sizeof(double) * (size_t)blocks) return NS_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    double *partial = (double *)ws;
    const int K = k <= 1 ? 1 : k <= 2 ? 2 : k <= 4 ? 4 : k <= 8 ? 8 : 16;
    const size_t smem = sizeof(double) * (size_t)(n * K);
    if (smem > 200 * 1024) return NS_ERR_INVALID_ARG;
    cudaError_t e = cudaSuccess;
    switch (K) {
        case 1: e = launch_residual<1>((const double *)A, m, n, lda, W, k, partial, blocks, smem, st); break;
        case 2: e = launch_residual<2>((const double *)A, m, n, lda, W, k, partial, blocks, smem, st); break;
        case 4: e = launch_residual<4>((const double *)A, m, n, lda, W, k, partial, blocks, smem, st); break;
        case 8: e = launch_residual<8>((const double *)A, m, n, lda, W, k, partial, blocks, smem, st); break;
        default: e = launch_residual<16>((const double *)A, m, n, lda, W, k, partial, blocks, smem, st); break;
    }
    if (e != cudaSuccess) return NS_ERR_CUDA;
    residual_final_kernel<<<1, 32, 0, st>>>(partial, blocks, out);
    return cuda_status(cudaGetLastError());
}

ns_status ns_srht_meta(const ns_sketch_desc *d, int64_t m, uint32_t *sign_words, int32_t *rows, void *stream) {
    if (!desc_ok(d) || d->kind != NS_SRHT || m < 1) return NS_ERR_INVALID_ARG;
    const int lg = ceil_log2(m);
    if (d->s > ((int64_t)1 << lg)) return NS_ERR_INVALID_ARG;
    const int64_t nwords = (((int64_t)1 << lg) + 31) / 32;
    return cuda_status(launch_srht_meta(d->seed, lg, nwords, d->s, sign_words, rows, (cudaStream_t)stream));
}

ns_status ns_sparse_meta(const ns_sketch_desc *d, int64_t m, int32_t *rows, int8_t *signs, void *stream) {
    if (!desc_ok(d) || d->kind != NS_SPARSE_SIGN || m < 1 || !rows || !signs) return NS_ERR_INVALID_ARG;
    return cuda_status(launch_sparse_meta(d->seed, d->s, d->zeta, m, rows, signs, (cudaStream_t)stream));
}

ns_status ns_batched_tuning(int32_t panel, int32_t sketch_ctas_per_sm, int32_t dense_ctas_per_sm) {
    return set_batch_tuning(panel, sketch_ctas_per_sm, dense_ctas_per_sm) ? NS_OK : NS_ERR_INVALID_ARG;
}

ns_status ns_test_bounded_wait(int32_t which, int64_t limit, int32_t *dev_status, void *ws, size_t ws_bytes,
                               void *stream) {
    if ((which != 0 && which != 1) || limit < 1 || limit > ((int64_t)1 << 24) || !dev_status) return NS_ERR_INVALID_ARG;
    if (which == 0 && (!ws || ws_bytes < 256 || (((uintptr_t)ws) & 255) != 0)) return NS_ERR_INVALID_ARG;
    return cuda_status(launch_test_wait(which, (long long)limit, dev_status, (unsigned int *)ws, (cudaStream_t)stream));
}

}  // extern "C"
