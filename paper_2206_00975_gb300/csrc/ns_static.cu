// ns_static.cu -- ns_sketch_static: the SRHT sketch with its scratch memory in
// a fixed device array owned by this library, for callers that cannot
// allocate device memory themselves (see include/ns.h).
//
// The paper has no counterpart of this entry point; it exists only for
// embedding.  The scratch is a file-scope __device__ array of
// kStaticScratchBytes: every GPU that loads libns holds it until the process
// exits.  Host code may not pass the array's name to a kernel (on the host it
// is only a stand-in symbol), so the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, and cached.
#include <mutex>
#include "ns_device.cuh"
#include "ns_internal.h"

namespace ns {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void *g_static_ptr[kMaxDevices] = {nullptr};

// Device address of g_static_scratch on the current device (set up on the
// first call per device).  Returns nullptr if the lookup fails.
static void *static_scratch_address() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return nullptr;
        g_static_ptr[dev] = p;
    }
    return g_static_ptr[dev];
}

}  // namespace ns

using namespace ns;

extern "C" ns_status ns_sketch_static(const ns_sketch_desc *d, const void *A, int32_t dtype, int64_t m, int64_t n,
                                      int64_t lda, double *SA, void *stream) {
    if (!d || !A || !SA) return NS_ERR_INVALID_ARG;
    if (d->kind != NS_SRHT || d->prec != NS_PREC_FP64 || dtype != NS_F64) return NS_ERR_INVALID_ARG;
    if (d->s < 1 || d->s > 16384 || m < 1 || n < 1 || lda < m) return NS_ERR_INVALID_ARG;
    if (d->s > ((int64_t)1 << ceil_log2(m))) return NS_ERR_INVALID_ARG;
    if ((((uintptr_t)A) & 7) != 0) return NS_ERR_INVALID_ARG;
    // scratch needed: one status word, then the sketch's signs, rows and partial sums
    Carver sizing(nullptr);
    sizing.take<int32_t>(1);
    srht_carve(sizing, m, n, d->s);
    if (sizing.used > kStaticScratchBytes) return NS_ERR_WORKSPACE;
    void *base = static_scratch_address();
    if (!base) return NS_ERR_CUDA;
    Carver c(base);
    int32_t *status = c.take<int32_t>(1);
    SrhtWork w = srht_carve(c, m, n, d->s);
    cudaStream_t st = (cudaStream_t)stream;
    // the status word is the only scratch that must start at zero; the
    // kernels overwrite signs, rows and partial sums before reading them
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return NS_ERR_CUDA;
    const SrhtGeom g = srht_geom(m, n);
    if (launch_srht_meta(d->seed, g.lg, g.sign_words, d->s, w.sign_words, w.rows, st) != cudaSuccess)
        return NS_ERR_CUDA;
    return launch_srht_f64((const double *)A, m, n, lda, d->s, w, SA, status, st) == cudaSuccess ? NS_OK
                                                                                                   : NS_ERR_CUDA;
}
