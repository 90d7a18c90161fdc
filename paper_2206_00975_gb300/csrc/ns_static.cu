// ns_static.cu -- ns_sketch_static: the SRHT sketch with its scratch memory in
// a fixed device array owned by this library, for callers that cannot
// allocate device memory themselves (see include/ns.h).
//
// The paper has no counterpart of this entry point; it exists only for
// embedding.  The scratch is a file-scope __device__ array of
// kStaticScratchBytes: every GPU that loads libns holds it until the process
// exits.  Host code may not pass the array's name to a kernel (on the host it
// is only a stand-in symbol), so the device address is looked up with
// cudaGetSymbolAddress, with the device current, and cached per CUDA context:
// a context created after a cudaDeviceReset loads the module again, and the
// array may then sit at another address, so the cache entry is keyed on the
// context's unique id rather than on the device ordinal.
#include <mutex>
#include <cuda.h>
#include "ns_device.cuh"
#include "ns_internal.h"

namespace ns {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
struct StaticSlot {
    unsigned long long ctx_id;  // id of the context the address belongs to (0: none)
    void *ptr;
};
static StaticSlot g_static_slot[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (0 if it cannot be read).
// The driver entry points are resolved through the runtime, so libns needs no
// link against libcuda.
static unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {
        void *f0 = nullptr, *f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) == cudaSuccess &&
            q0 == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f0;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f1;
        resolved = true;
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_static_scratch in the current context (looked up on
// the first call in each context).  Returns nullptr if the lookup fails.
static void *static_scratch_address() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_static_mu);
    const unsigned long long id = current_ctx_id();  // 0 before the runtime has made a context current
    StaticSlot &slot = g_static_slot[dev];
    if (!slot.ptr || id == 0 || slot.ctx_id != id) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return nullptr;
        slot.ptr = p;
        slot.ctx_id = current_ctx_id();  // the lookup has made the device's context current
    }
    return slot.ptr;
}

}  // namespace ns

using namespace ns;

extern "C" ns_status ns_sketch_static(const ns_sketch_desc *d, const void *A, int32_t dtype, int64_t m, int64_t n,
                                      int64_t lda, double *SA, int32_t *dev_status, void *stream) {
    if (!d || !A || !SA) return NS_ERR_INVALID_ARG;
    if (d->kind != NS_SRHT || d->prec != NS_PREC_FP64 || dtype != NS_F64) return NS_ERR_INVALID_ARG;
    if (d->s < 1 || d->s > kMaxS || m < 1 || n < 1 || lda < m) return NS_ERR_INVALID_ARG;
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
    int32_t *own_status = c.take<int32_t>(1);
    SrhtWork w = srht_carve(c, m, n, d->s);
    int32_t *status = dev_status ? dev_status : own_status;
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
