// ns_internal.h -- host-side declarations shared by the libns translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/ns.h"

namespace ns {

constexpr int kBlockLog = 12;                 // FWHT block: 4096 rows of one column
constexpr int64_t kBlock = 1 << kBlockLog;
constexpr int kMaxChunkBlocks = 16;           // blocks summed per fixed-point accumulator
constexpr int64_t kMaxS = 16384;              // sketch rows held in one CTA's shared memory

inline int ceil_log2(int64_t m) {
    int lg = 0;
    while (((int64_t)1 << lg) < m) ++lg;
    return lg;
}
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Streaming multiprocessors of the current device (queried once per device;
// 1 if no device can be queried, e.g. when only workspace sizes are asked for
// on a machine without a GPU: geometries derived from it then stay valid, they
// only spread work less widely).
int device_sm_count();

// Carves consecutive 256-byte-aligned pieces out of the caller's workspace.
struct Carver {
    char *base;
    size_t used = 0;
    explicit Carver(void *p) : base((char *)p) {}
    template <typename T>
    T *take(size_t count) {
        T *p = base ? (T *)(base + used) : nullptr;
        used += align256(count * sizeof(T));
        return p;
    }
};

// SRHT forward geometry: the padded length m' is split into blocks of 4096
// rows (a single, zero-padded block when m' <= 4096); consecutive blocks of a
// column are grouped into chunks that share one fixed-point accumulator.
struct SrhtGeom {
    int lg;            // m' = 2^lg
    int64_t nblk;      // blocks per column
    int chunk;         // blocks per chunk
    int64_t nchunk;    // chunks per column
    int fx_bits;       // fixed-point magnitude bits P
    int64_t sign_words;  // uint32 words of sign bits kept in workspace
};
SrhtGeom srht_geom(int64_t m, int64_t n);

struct SrhtWork {
    uint32_t *sign_words;
    int32_t *rows;
    double *partial;
};
size_t srht_work_bytes(int64_t m, int64_t n, int64_t s);
SrhtWork srht_carve(Carver &c, int64_t m, int64_t n, int64_t s);

// SRHT of a row window [lo, hi) of A (the partial sketch of a row block):
// global blocks b0 .. b_end - 1 in nchunk chunks of `chunk` blocks
struct SrhtRowsGeom {
    int lg;
    int64_t b0, b_end;
    int chunk;
    int64_t nchunk;
    int fx_bits;
    int64_t sign_words;
};
SrhtRowsGeom srht_rows_geom(int64_t m_total, int64_t lo, int64_t hi, int64_t n);
SrhtWork srht_rows_carve(Carver &c, int64_t m_total, int64_t lo, int64_t hi, int64_t n, int64_t s);

// launches (return cudaGetLastError())
cudaError_t launch_srht_meta(uint64_t seed, int lg, int64_t nsign_words, int64_t s, uint32_t *sign_words,
                             int32_t *rows, cudaStream_t st);
cudaError_t launch_srht_f64(const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, const SrhtWork &w,
                            double *SA, int32_t *status, cudaStream_t st);
cudaError_t launch_srht_f32(const float *A, int64_t m, int64_t n, int64_t lda, int64_t s, const SrhtWork &w,
                            double *SA, int32_t *status, cudaStream_t st);
// SA[t, c] = scale * sum over nchunk partials (chunk-major, s x n each), in chunk order
cudaError_t launch_srht_f64_rows(const double *A_p, int64_t m_total, int64_t lo, int64_t hi, int64_t n, int64_t lda,
                                 int64_t s, const SrhtWork &w, double *SA_p, int32_t *status, cudaStream_t st);
cudaError_t launch_srht_reduce(const double *partial, int64_t n, int64_t s, int64_t nchunk, double scale, double *SA,
                               cudaStream_t st);

// H-RHT geometry: B = m'/4096 blocks per column (1 when m' <= 4096), slabs of
// W = 2^lw consecutive lo across all blocks, nseg segments of sps slabs per
// column, one pass-2 CTA and one FP64 partial per (column, segment).
struct HrhtGeom {
    int lg;              // m' = 2^lg
    int64_t mp;
    int64_t B;           // blocks per column
    int LB;              // log2 B
    int lw;              // log2 W = 12 - LB
    int nseg;            // segments per column
    int64_t sps;         // slabs per segment (B / nseg)
    int64_t sign_words;  // uint32 words of sign bits
};
struct HrhtWork {
    uint32_t *sign_words;
    uint32_t *hash;      // m': h(i) | (sign < 0) << 31
    unsigned int *cmax;  // largest bucket count of any segment
    int2 *blk;           // n * B: (quantum exponent, top exponent) of each Z_b
    long long *Z;        // n * B * 4096: pass-1 blocks
    double *partial;     // nseg * n * s
};
HrhtGeom hrht_geom(int64_t m, int64_t n);
HrhtWork hrht_carve(Carver &c, int64_t m, int64_t n, int64_t s);
cudaError_t launch_hrht_f64(uint64_t seed, const double *A, int64_t m, int64_t n, int64_t lda, int64_t s,
                            const HrhtWork &w, double *SA, int32_t *status, cudaStream_t st);

struct SparseGeom {
    int64_t ntile;        // 128-row tiles of A
    int64_t nent;         // entries per tile (128 * zeta)
    int64_t ntgrp;        // target groups of 1024 output rows (one accumulator each)
    int64_t nbucket;      // entry buckets per tile: ntgrp * 32 owners
    int64_t ncolgrp;      // 16-column groups
    int64_t chunk_tiles;  // tiles per accumulator chunk
    int64_t nchunk;
    int fx_bits;          // fixed-point magnitude bits P
};
struct SparseWork {
    uint32_t *entries;
    int32_t *offsets;
    double *partial;
};
SparseGeom sparse_geom(int64_t m, int64_t n, int64_t s, int zeta);
SparseWork sparse_carve(Carver &c, int64_t m, int64_t n, int64_t s, int zeta);
cudaError_t launch_sparse_meta(uint64_t seed, int64_t s, int zeta, int64_t m, int32_t *rows, int8_t *signs,
                               cudaStream_t st);
// j0: global index of row 0 of A (the columns of S follow the global row index;
// a row block [j0, j0 + m) gives its partial sketch)
cudaError_t launch_sparse_f64(uint64_t seed, const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, int zeta,
                              const SparseWork &w, double *SA, int32_t *status, cudaStream_t st, int64_t j0 = 0);

struct BackwardWork {
    uint32_t *sign_words;
    int32_t *rows;
    int32_t *rank;
    double *Y;         // n x k
    double *P;         // s x 2k: SA Y, SA W
    long long *q;      // s x n fixed-point image of dL/dSA / sqrt(s)
    int32_t *colexp;   // n: fixed-point scale exponents
};
size_t backward_work_bytes(int64_t m, int64_t n, int64_t s, int32_t k);
BackwardWork backward_carve(Carver &c, int64_t m, int64_t n, int64_t s, int32_t k);
cudaError_t launch_backward(uint64_t seed, int64_t m, int64_t n, int32_t k, int64_t s, const double *save,
                            const double *Vk, const double *dVk, double *dA, int64_t ldd, const BackwardWork &w,
                            cudaStream_t st);

size_t batched_work_bytes(int32_t batch, const ns_problem *host);
bool set_batch_tuning(int panel, int sketch_cps, int dense_cps);
cudaError_t launch_batched(int32_t batch, const ns_problem *host, const ns_problem *dev, int32_t *status, void *ws,
                           cudaStream_t st);

size_t aaa_work_bytes(int64_t m, int64_t smax, int32_t K);
cudaError_t launch_aaa(uint64_t seed, const double *x, const double *f, int64_t m, int32_t K, int64_t smax,
                       const long long *forced, long long *support, double *Wout, double *errmax, double *SAk_out,
                       int32_t *status, void *ws, cudaStream_t st);

struct GaussGeom {
    int64_t mtiles;   // 128-row tiles of G
    int NP;           // n rounded up to 16
    int64_t kper;     // K (= rows of A) per split
    int64_t nsplit;
};
GaussGeom gauss_geom(int64_t m, int64_t n, int64_t s);
size_t gauss_work_bytes(int64_t m, int64_t n, int64_t s);
cudaError_t launch_gauss_bf16x3(uint64_t seed, const float *A, int64_t m, int64_t n, int64_t lda, int64_t s,
                                float *partial, double *SA, int32_t *status, cudaStream_t st);

struct DenseWork {
    double *W;        // s x n working copy of SA (QR in place); later V (n x n)
    double *tau;      // 2n: reflector factors of both QRs
    double *X;        // n x n: R, then X = R2^T rotated into U Sigma
    double *V;        // n x n: R2, then the accumulated rotations Vx
    double *sigma;    // n
    double *L;        // n x 2n: [R^T | I] for the second QR (n x n R^T and its reflectors on the coop fallback)
    double *R2;       // n x 2n: [R2 | Q2^T] from the pipelined second QR
    double *U;        // s x n: reflectors published by the pipelined QRs
    int32_t *perm;    // n: column pivots of the first QR
    unsigned long long *pivslot;  // n + 1: pivot candidates (atomic max)
    unsigned int *bar;  // grid barrier words (2), rotation counters (64), check flags (64)
    unsigned int *colver;  // n + 32: per-column write versions of the ring Jacobi
};
size_t dense_work_bytes(int64_t s, int64_t n);
DenseWork dense_carve(Carver &c, int64_t s, int64_t n);
cudaError_t launch_dense_stats(const DenseWork &w, int64_t *out, cudaStream_t st);
// failure-detection test hook: which 0 = grid barrier (limit in polls), 1 = cluster-peer mbarrier wait (limit
// in clock cycles); word: one device word of scratch for the barrier
cudaError_t launch_test_wait(int which, long long limit, int32_t *status, unsigned int *word, cudaStream_t st);
// Section 5 row updates of a sketch (op 0: append row index j, 1: remove row j)
cudaError_t launch_sketch_update(int kind, uint64_t seed, int64_t s, int zeta, int64_t m0, int op, int64_t j,
                                 const double *row, int64_t n, double *SA, cudaStream_t st);
// after launch_dense_solve with k = 0: the tolerance selection (Vk n x n, sigk n, k in *dev_k)
cudaError_t launch_dense_select_eps(const DenseWork &w, int64_t n, double eps, double *Vk, double *sigk,
                                    int32_t *dev_k, cudaStream_t st);
// max_sweeps: Jacobi sweep limit (30 when 0 or out of range); the solve reports
// NS_ERR_NOCONV, with the partial result written, when the limit is reached
// fp32_phase: run the linear phase of the Jacobi iteration in FP32 first
// (ns_jacobi32.cu) where it applies (pipelined QRs, 64 <= n <= 256)
// after_qr: if set, recorded on st once the QRs and X0 = R2^T, V = Q2 are in
// place (from then on the stage no longer needs every SM at once)
cudaError_t launch_dense_solve(const double *SA, int64_t s, int64_t n, int32_t k, const DenseWork &w, double *Vk,
                               double *sigk, double *save_V, double *save_sigma, int32_t *status, cudaStream_t st,
                               int max_sweeps = 0, bool fp32_phase = true, cudaEvent_t after_qr = nullptr);
// FP32 linear phase of the Jacobi iteration on X = w.X (n x n) with V = w.V
// holding Q2: X <- X V0, V <- Q2 V0 (V0 orthogonal in FP64); ctl[0] = 1 if it
// ran, ctl[1..2] its sweeps and rotations.  Scratch: w.L, w.U, w.W.
bool jacobi32_applicable(int64_t n);
cudaError_t launch_jacobi32_precondition(const DenseWork &w, int64_t n, unsigned int *ctl, cudaStream_t st);

}  // namespace ns
