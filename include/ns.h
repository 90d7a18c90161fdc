/*
 * ns.h -- C ABI of libns: GB300 (sm_103a) sketch-and-solve approximate null
 * space, after Park & Nakatsukasa, "A Fast Randomized Algorithm for Computing
 * an Approximate Null Space".
 *
 * The problem (Problem 2.1): given A (m x n, m >= n) and k, find W (n x k)
 * minimising ||A W||_F over W^T W = I_k.  Algorithm 1 solves it approximately:
 * draw a sketch S (s x m), form SA, take the SVD of SA and return its k
 * trailing right singular vectors.  Here the SVD of SA is a Householder QR
 * SA = QR followed by a one-sided Jacobi SVD of R (SA and R share singular
 * values and right singular vectors, proof of Theorem 3.2).
 *
 * Conventions for every call:
 *  - Matrices are column-major.  A has leading dimension lda >= m.  Sketch
 *    outputs SA are s x n with leading dimension s.
 *  - Every pointer argument named A, SA, Vk, sigk, save, dA, dVk, ws,
 *    dev_status, problems or any output array is a DEVICE pointer on the
 *    current CUDA device; sketch descriptors are HOST pointers.
 *  - The caller owns all memory.  The library never allocates, frees or
 *    synchronises; it enqueues kernels on `stream` (a cudaStream_t, 0 = the
 *    legacy default stream) and returns.  Scratch space comes from the
 *    caller's workspace `ws` of `ws_bytes` bytes (>= the size reported by the
 *    matching *_workspace_size call, 256-byte aligned).
 *  - Argument errors are detected on the host before any launch and returned
 *    (NS_ERR_INVALID_ARG, NS_ERR_WORKSPACE); nothing is enqueued then.  A
 *    failed launch returns NS_ERR_CUDA.  Numerical conditions found by the
 *    kernels (non-finite input, Jacobi not converged, TLS without solution,
 *    a bounded device wait that ran out) are written to *dev_status (a device
 *    int32, 0 on success) for the caller to read after synchronising; the
 *    outputs are still written on a best-effort basis.
 *  - Calls that share a workspace must not overlap on the GPU.
 */
#ifndef NS_H
#define NS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NS_OK = 0,
    NS_ERR_INVALID_ARG = 1,     /* bad size, pointer, alignment or option */
    NS_ERR_WORKSPACE = 2,       /* ws_bytes below the required size */
    NS_ERR_NONFINITE = 3,       /* (device status) A holds Inf or NaN */
    NS_ERR_NOCONV = 4,          /* (device status) Jacobi hit its sweep limit */
    NS_ERR_TLS_NOSOLUTION = 5,  /* (device status) v_{n+1} = 0, Section 4 */
    NS_ERR_TIMEOUT = 6,         /* (device status) a bounded device wait ran out */
    NS_ERR_CUDA = 7             /* a CUDA launch or attribute call failed */
} ns_status;

/* Sketch families (Sections 1-2). */
typedef enum {
    NS_SRHT = 0,        /* S = (1/sqrt s) R H D: the SRFT of Section 2 with the
                           Sylvester Walsh-Hadamard matrix H on m' = 2^ceil(log2 m) */
    NS_SPARSE_SIGN = 1, /* zeta entries +-1/sqrt(zeta) per column of S (sparse
                           sketch of the kind Section 1 names, CountSketch-like) */
    NS_GAUSSIAN = 2,    /* S = G/sqrt(s), G standard Gaussian (Theorem 2.1) */
    NS_HRHT = 3         /* S = S_h (1/sqrt m') H D: the SRFT with R replaced by a
                           1-hashing matrix S_h (Section 2, after Theorem 2.2), one
                           +-1 per column of S_h; an embedding at s = O(n) also for
                           coherent A, where the SRHT needs s = O(n log n) */
} ns_sketch_kind;

typedef enum { NS_F64 = 0, NS_F32 = 1 } ns_dtype;

/* Arithmetic used to form SA.  The dense stage does not depend on it: the QRs
 * run in FP64, and the one-sided Jacobi takes its linear phase in FP32 (graded
 * rotations accumulated exactly) and finishes in FP64 (first-order completions,
 * a Gram-matrix convergence test and, where pairs remain, FP64 sweeps), so V
 * and sigma carry FP64 accuracy. */
typedef enum {
    NS_PREC_FP64 = 0,        /* exact +-1 transforms on a 64-bit fixed-point
                                image of A; FP64 results */
    NS_PREC_FP32_STREAM = 1, /* SRHT streamed in FP32 with FP32 accumulation */
    NS_PREC_BF16X3 = 2       /* Gaussian: 3-term BF16 split products, FP32
                                accumulation, on the tensor cores */
} ns_prec;

/* Sketch descriptor (host memory).  seed selects the realisation of S; the
 * same (kind, s, zeta, seed) and m always give the same S. */
typedef struct {
    int32_t kind;    /* ns_sketch_kind */
    int32_t zeta;    /* nonzeros per column of S for NS_SPARSE_SIGN (1..64) */
    int64_t s;       /* sketch size, n <= s; SRHT also needs s <= m' */
    uint64_t seed;
    int32_t prec;    /* ns_prec */
    int32_t max_sweeps; /* Jacobi sweep limit of the solves, 0 = the default 30;
                           a limit the iteration reaches makes the solve report
                           NS_ERR_NOCONV with its partial result written (the
                           failure-detection tests force this with 1) */
} ns_sketch_desc;

/* Human-readable name of a status code (static storage). */
const char *ns_status_string(int status);

/* Library version string. */
const char *ns_version(void);

/* Bytes of workspace needed by ns_sketch / ns_solve / ns_backward / ns_residual
 * for this descriptor and shape (the maximum over the calls).  Returns 0 for
 * an invalid combination. */
size_t ns_workspace_size(const ns_sketch_desc *desc, int64_t m, int64_t n, int32_t k);

/* Number of doubles in the `save` buffer of ns_solve: SA (s x n), V (n x n),
 * sigma (n), in that order. */
int64_t ns_save_size(int64_t s, int64_t n);

/*
 * ns_sketch -- Algorithm 1, line 2: SA = S A.
 *   A      device, m x n (dtype), column-major, leading dimension lda >= m.
 *   SA     device, s x n FP64 output, leading dimension s.
 * SRHT (Section 2, with H in place of F): SA = (1/sqrt s) R H_{m'} D [A; 0].
 * Sparse sign: SA = sum_j S(:, j) A(j, :), zeta entries per column of S.
 * Gaussian: SA = G A / sqrt(s).
 * H-RHT: SA = S_h (1/sqrt m') H_{m'} D [A; 0]; coordinate i of the transform
 *   goes to row h(i) = floor(s (w mod 2^32) / 2^32) with the sign of bit 63 of
 *   w, w = word (i mod 4) of the stream-4 Philox block i/4.  Exact fixed-point
 *   arithmetic with two roundings (the input onto 2^-50 of its 4096-row
 *   block's largest magnitude; the block transforms onto 2^-P of the column's
 *   largest, P = 62 - log2(m'/4096) - ceil(log2(largest count of rows one
 *   pass-2 segment sends to one bucket)), about 47 at m' = 2^20, s = 1024).
 *   Its workspace holds the m' x n transformed blocks (8 m' n bytes).
 * Errors: NS_ERR_INVALID_ARG for m < 1, n < 1, s < 1, lda < m, SRHT or H-RHT
 * s > m', H-RHT m' > 2^24,
 * zeta outside 1..min(64, s), an unsupported (kind, prec, dtype) triple, or a
 * NULL pointer; NS_ERR_WORKSPACE for a short workspace.
 */
ns_status ns_sketch(const ns_sketch_desc *desc, const void *A, int32_t dtype, int64_t m, int64_t n,
                    int64_t lda, double *SA, void *ws, size_t ws_bytes, void *stream);

/*
 * ns_sketch_rows -- the share of one row block of A in its sketch, for A split
 * by rows across devices or streamed in row blocks (Section 1: A need only be
 * read once, in any order; Section 5: a sketch is a sum over the rows of A):
 * SA_p = S[:, o:o+m_p] A[o:o+m_p, :], with S the sketch of the whole m_total x n
 * matrix.  The sum of the SA_p of blocks that cover rows 0..m_total-1 is
 * ns_sketch's SA up to the rounding of the sum (exactly, for integer data).
 * For the SRHT, H_{m'} = H_{m'/4096} (x) H_4096: the block is transformed in its
 * 4096-row blocks with their global indices (rows of a block outside
 * [o, o + m_p) count as zero); for the sparse sign, column j of S belongs to
 * global row j.
 *   desc      NS_SRHT (NS_PREC_FP64) or NS_SPARSE_SIGN (NS_PREC_FP64).
 *   A_p       device, m_p x n FP64, column-major, leading dimension lda >= m_p:
 *             rows o .. o + m_p - 1 of A (o = row_offset).
 *   m_total   rows of the whole A (sets m' and the sketch's columns).
 *   SA_p      device, s x n FP64 output, leading dimension s.
 *   dev_status  device int32 or NULL: 0, or NS_ERR_NONFINITE.
 *   ws        ns_sketch_rows_workspace_size(desc, m_total, row_offset, m_p, n)
 *             bytes, 256-byte aligned.
 * Errors: NS_ERR_INVALID_ARG for another kind or precision, row_offset < 0,
 * m_p < 1, row_offset + m_p > m_total, n < 1, lda < m_p, SRHT s > m', or a
 * NULL pointer; NS_ERR_WORKSPACE for a short workspace.
 */
size_t ns_sketch_rows_workspace_size(const ns_sketch_desc *desc, int64_t m_total, int64_t row_offset, int64_t m_p,
                                     int64_t n);
ns_status ns_sketch_rows(const ns_sketch_desc *desc, const void *A_p, int32_t dtype, int64_t m_total,
                         int64_t row_offset, int64_t m_p, int64_t n, int64_t lda, double *SA_p, int32_t *dev_status,
                         void *ws, size_t ws_bytes, void *stream);

/*
 * ns_solve -- Algorithm 1 end to end: sketch, QR of SA, one-sided Jacobi SVD
 * of R, and W = V(:, n-k+1:n) (line 4).
 *   Vk    device, n x k FP64 output: the k trailing right singular vectors of
 *         SA, ordered by non-increasing singular value (the last column
 *         belongs to the smallest); each column is signed so that its entry of
 *         largest magnitude (lowest index on ties) is positive.
 *   sigk  device, k FP64 output: the matching singular values of SA.
 *   save  device, ns_save_size(s, n) doubles or NULL: SA, V, sigma, kept for
 *         ns_backward.
 *   dev_status  device int32 (may be NULL): 0, or NS_ERR_NONFINITE /
 *         NS_ERR_NOCONV (sweep limit 30) / NS_ERR_TIMEOUT.
 * Requires 1 <= k <= n <= s and m >= n.
 */
ns_status ns_solve(const ns_sketch_desc *desc, const void *A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                   int32_t k, double *Vk, double *sigk, double *save, int32_t *dev_status, void *ws,
                   size_t ws_bytes, void *stream);

/*
 * ns_solve_pipelined -- Algorithm 1 (as ns_solve) for `count` independent
 * problems of the same shape, dtype and lda: a throughput form for a stream
 * of problems.  Problems go round-robin to three lanes, so several solves are
 * in flight (the dense stage is bound by FP64 latency chains, and a few of
 * them share the SMs well); within a lane the sketch of its next problem runs
 * while the current dense stage is past its two QRs.  The library runs the
 * lanes on streams of its own (per device; dense stages at the higher
 * priority), ordered after all work already enqueued on `stream`; every
 * result is complete before work enqueued on `stream` later.
 *   A      host array of `count` device pointers, problem i = A[i] (m x n,
 *          column-major, leading dimension lda, dtype as ns_solve).
 *   Vk     device, count * n * k FP64: problem i at Vk + i n k (n x k each,
 *          ordered and signed as ns_solve).
 *   sigk   device, count * k FP64: problem i at sigk + i k.
 *   dev_status  device int32[count] (may be NULL): problem i's status.
 *   ws     ns_solve_pipelined_workspace_size(desc, m, n) bytes, 256-byte
 *          aligned (per lane two sketch slots and a dense workspace).
 * The results are those of ns_solve on each problem, bit for bit (the same
 * kernels in the same order per problem).  Not re-entrant for one device
 * from several host threads at once (the library's streams are shared).
 * Errors: NS_ERR_INVALID_ARG as ns_solve, and for count < 1 or a null or
 * misaligned A[i]; NS_ERR_WORKSPACE; NS_ERR_CUDA.
 */
size_t ns_solve_pipelined_workspace_size(const ns_sketch_desc *desc, int64_t m, int64_t n);
ns_status ns_solve_pipelined(const ns_sketch_desc *desc, const void *const *A, int32_t count, int32_t dtype,
                             int64_t m, int64_t n, int64_t lda, int32_t k, double *Vk, double *sigk,
                             int32_t *dev_status, void *ws, size_t ws_bytes, void *stream);

/*
 * ns_solve_eps -- the tolerance version of Algorithm 1 (Section 2, the remark
 * after Algorithm 1): instead of k, W is every right singular vector of SA
 * whose singular value is below eps (eps = O(u) sigma_1 gives the numerical
 * null space).
 *   eps    absolute tolerance, eps >= 0 (the comparison is sigma_i < eps).
 *   Vk     device, n x n FP64 output: columns 0..k-1 receive W, ordered and
 *          signed as ns_solve (the last column belongs to the smallest
 *          singular value); the other columns are left as they were.
 *   sigk   device, n FP64 output: entries 0..k-1 receive the matching
 *          singular values.
 *   dev_k  device int32 output: k = #{i : sigma_i < eps}, 0 <= k <= n.
 * Everything else as ns_solve (workspace: ns_workspace_size with any k).
 * Errors: NS_ERR_INVALID_ARG as ns_solve, and for eps < 0 or NaN.
 */
ns_status ns_solve_eps(const ns_sketch_desc *desc, const void *A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                       double eps, double *Vk, double *sigk, int32_t *dev_k, double *save, int32_t *dev_status,
                       void *ws, size_t ws_bytes, void *stream);

/*
 * ns_sketch_update -- keep a sketch SA current when A gains or loses a row
 * (Section 5: Algorithms 2 and 3, and the rule for non-Gaussian sketches).
 *   m0    the row count SA was sketched with (sets m' and which columns of S
 *         are SRHT or sparse-sign columns).
 *   op    NS_ROW_APPEND: A gains the row `row` with index j >= m0 (appended
 *         rows are numbered m0, m0 + 1, ...); S gains the column g / sqrt(s),
 *         g the Gaussian sketch's column j for desc->seed (Philox stream 3),
 *         and SA += g row / sqrt(s).
 *         NS_ROW_REMOVE: A loses row j, whose entries are `row`; SA -= (S e_j)
 *         row, with S e_j regenerated from desc: the SRHT column
 *         d_j (-1)^popcount(r_t & j) / sqrt(s) or the sparse-sign column for
 *         j < m0, the Gaussian column j for a row appended earlier (j >= m0) and
 *         for the Gaussian kind.
 *   row   device, n FP64 (the row's entries).
 *   SA    device, s x n FP64, leading dimension s, updated in place.
 * O(s n) work, enqueued on stream.  A column of A is added by sketching it
 * with ns_sketch (n = 1, the same desc and m0) and appending it to SA; a column
 * is removed by dropping it from SA.
 * Errors: NS_ERR_INVALID_ARG for a bad desc or op, j < 0, an append with
 * j < m0, m0 < 1, n < 1, an SRHT s > m', the H-RHT kind (its column S e_j
 * takes all m' coordinates, not O(s) work), or a NULL pointer.
 */
enum { NS_ROW_APPEND = 0, NS_ROW_REMOVE = 1 };
ns_status ns_sketch_update(const ns_sketch_desc *desc, int64_t m0, int32_t op, int64_t j, const double *row,
                           int64_t n, double *SA, void *stream);

/*
 * ns_solve_sketched -- Algorithm 1 lines 3-4 on a sketch the caller already
 * holds: SA (device, s x n FP64, ld s, s = desc->s) -> QR, Jacobi SVD, the k
 * trailing right singular vectors.  Outputs as ns_solve (save receives a copy
 * of SA, then V and sigma).  SA is not modified.
 */
ns_status ns_solve_sketched(const ns_sketch_desc *desc, const double *SA, int64_t n, int32_t k, double *Vk,
                           double *sigk, double *save, int32_t *dev_status, void *ws, size_t ws_bytes,
                           void *stream);

/*
 * ns_solve_stats / ns_sketched_stats -- statistics of the Jacobi iteration of
 * the last ns_solve (ns_solve_sketched) that ran in workspace ws with the same
 * desc and shape: dev_out (device int64[8]) receives the number of full FP64
 * sweeps, the number of FP64 rotations, the number of barrier-free check
 * passes, the kernel that ran (the cluster size, 8 or 16, of the cluster-ring
 * Jacobi, or 0: the barrier-separated one), the sweeps and rotations of the
 * FP32 linear phase that precedes the FP64 iteration for 64 <= n <= 256 (0
 * and 0 when it did not run), how many of the two first-order completions
 * that follow the phase formed their K^4 and K^6 terms, and 1 if the
 * iteration's convergence test ran on the Gram matrix X^T X after the last
 * completion (else 0; when it finds no pair above the tolerance the FP64
 * iteration runs no sweep).
 * Enqueued on stream after that call.
 */
ns_status ns_solve_stats(const ns_sketch_desc *desc, int64_t m, int64_t n, const void *ws, int64_t *dev_out,
                         void *stream);
ns_status ns_sketched_stats(const ns_sketch_desc *desc, int64_t n, const void *ws, int64_t *dev_out, void *stream);

/*
 * ns_backward -- adjoint of ns_solve for a loss L that depends on W only
 * through the projector W W^T (a loss that is invariant under W -> W Q).
 * With M = SA^T SA = V Sigma^2 V^T, T the trailing k indices and N the others:
 *   dL/dM  = sum_{i in T, j in N} c_ji (v_j v_i^T + v_i v_j^T),
 *   c_ji   = (v_j . g_i) / (2 (sigma_i^2 - sigma_j^2)),  g_i = dL/dW(:, i),
 *   dL/dSA = 2 SA dL/dM,    dL/dA = S^T dL/dSA.
 * For the SRHT, S^T = (1/sqrt s) D H R^T is applied by regenerating D and R
 * from the seed (nothing of the forward transform is stored).  Components of
 * dL/dW along span(W) are ignored (they cannot change W W^T).
 *   save  device: the buffer ns_solve filled.   Vk: the returned W.
 *   dVk   device n x k: dL/dW.   dA: device m x n output, leading dim ldd >= m.
 * Only NS_SRHT with NS_PREC_FP64 is supported; requires 1 <= k < n.
 */
ns_status ns_backward(const ns_sketch_desc *desc, int64_t m, int64_t n, int32_t k, const double *save,
                      const double *Vk, const double *dVk, double *dA, int64_t ldd, void *ws, size_t ws_bytes,
                      void *stream);

/*
 * One problem of a batch (ns_solve_batched).  Pointers are DEVICE pointers.
 * For total least squares (Section 4) A = [X b] with n = n_X + 1 columns, k = 1
 * and tls != 0: then x = -v(1:n-1)/v(n) is written to x (n-1 doubles), v the
 * trailing right singular vector of the sketch.
 */
typedef struct {
    const void *A;   /* m x n, column-major, leading dimension lda >= m; FP64 or FP32 (dtype) */
    int64_t m, n, lda;
    int64_t s;       /* SRHT sketch size: n <= s <= min(m', 16384) */
    int32_t k;       /* trailing vectors, 1 <= k <= n */
    int32_t tls;     /* nonzero: also solve the TLS problem (needs k = 1, n >= 2, x) */
    uint64_t seed;   /* realisation of this problem's sketch */
    double *Vk;      /* n x k out (ordering and signs as ns_solve) */
    double *sigk;    /* k out */
    double *x;       /* n - 1 out when tls != 0, else unused */
    int32_t dtype;   /* NS_F64: exact fixed-point sketch (NS_PREC_FP64); NS_F32:
                        the FP32-stream sketch (NS_PREC_FP32_STREAM); QR and
                        Jacobi run in FP64 either way */
    int32_t reserved;  /* 0 */
} ns_problem;

/* Workspace bytes for ns_solve_batched; host_problems is a HOST copy of the
 * problem array.  Returns 0 if any problem is invalid. */
size_t ns_batched_workspace_size(const ns_sketch_desc *desc, int32_t batch, const ns_problem *host_problems);

/*
 * ns_solve_batched -- Algorithm 1 (SRHT sketch, QR, Jacobi SVD, trailing
 * vectors) on `batch` independent problems of arbitrary shapes in one
 * sequence of launches with no host round trip: a persistent sketch kernel
 * takes (problem, column) items from a device work counter, a persistent dense
 * kernel takes whole problems.  desc: kind NS_SRHT, prec NS_PREC_FP64 or
 * NS_PREC_FP32_STREAM (its s and seed are unused; each problem has its own
 * size, seed and dtype).  host_problems and dev_problems
 * hold the same array (host copy for validation and sizing, device copy for
 * the kernels).  dev_status: device int32[batch], per-problem status
 * (0, NS_ERR_NONFINITE, NS_ERR_NOCONV, NS_ERR_TLS_NOSOLUTION).
 */
ns_status ns_solve_batched(const ns_sketch_desc *desc, int32_t batch, const ns_problem *host_problems,
                           const ns_problem *dev_problems, int32_t *dev_status, void *ws, size_t ws_bytes,
                           void *stream);

/*
 * ns_batched_tuning -- launch geometry of ns_solve_batched, chosen by the
 * autotuner of the Python package (paper_2206_00975_gb300.autotune) and cached
 * per (architecture, m' of the largest problem, column panel, dtype):
 *   panel               columns per sketch work item (1..64; 0 = 1);
 *   sketch_ctas_per_sm  persistent sketch CTAs per SM (0 = the occupancy limit);
 *   dense_ctas_per_sm   persistent dense CTAs per SM (0 = the occupancy limit).
 * None of them changes the arithmetic: the results are bit-identical for every
 * setting.  The setting is process-wide and read when ns_solve_batched
 * launches; calls that change it must not race with those launches.
 * Errors: NS_ERR_INVALID_ARG for a value outside its range.
 */
ns_status ns_batched_tuning(int32_t panel, int32_t sketch_ctas_per_sm, int32_t dense_ctas_per_sm);

/*
 * ns_aaa_real -- AAA rational approximation of f on real points x (Section
 * 6) with a reused SRHT sketch: K iterations; iteration k picks the support
 * point maximising |f - r| (r_0 = mean f; lowest index on ties), downdates the
 * sketch by the new support row (Algorithm 3 with the non-Gaussian rule of
 * Section 5.3; S e_j in closed form), sketches the new Loewner column
 * (f_i - f_j)/(x_i - x_j), and takes the barycentric weights w as the trailing
 * right singular vector of the first min(4k, s) rows of the s-row sketch
 * (Algorithm 1 on the sketch).  Everything stays on the device: the call only
 * enqueues kernels, so it can be captured in a CUDA graph (make one un-captured
 * call first).
 *   desc    NS_SRHT, NS_PREC_FP64, s = the sketch rows (K <= s <= m').
 *   x, f    device, m FP64 (distinct points).
 *   forced  device int64[K] or NULL: support points to use instead of the
 *           greedy choice (teacher forcing).
 *   support device int64[K] out; W device FP64 K x K out, row k-1 = weights of
 *           iteration k (zero padded); errmax device FP64[K] out, max |f - r|
 *           after iteration k; SAk_out device FP64 s x K or NULL (final sketch).
 */
size_t ns_aaa_workspace_size(const ns_sketch_desc *desc, int64_t m, int32_t K);
ns_status ns_aaa_real(const ns_sketch_desc *desc, const double *x, const double *f, int64_t m, int32_t K,
                      const int64_t *forced, int64_t *support, double *W, double *errmax, double *SAk_out,
                      int32_t *dev_status, void *ws, size_t ws_bytes, void *stream);

/*
 * ns_residual -- the objective of Problem 2.1, ||A W||_F, in one streaming
 * pass over A (evaluation only).  W is device n x k FP64 (1 <= k <= 16 and
 * n * k' <= 25600 with k' = k rounded up to a power of two; A FP64 only);
 * *out (device double) receives the result.  ws needs 8 KiB.  One thread per
 * row of A accumulates A(row, :) W in FP64.
 */
ns_status ns_residual(const void *A, int32_t dtype, int64_t m, int64_t n, int64_t lda, const double *W, int32_t k,
                      double *out, void *ws, size_t ws_bytes, void *stream);

/*
 * ns_srht_meta -- the realisation of the SRHT's random ingredients, for
 * inspection and tests: sign_words (device, ceil(m'/32) uint32; bit i set
 * means d_i = -1) and rows (device, s int32: the coordinates kept by R, in
 * draw order).  Either pointer may be NULL.
 */
ns_status ns_srht_meta(const ns_sketch_desc *desc, int64_t m, uint32_t *sign_words, int32_t *rows, void *stream);

/*
 * ns_sparse_meta -- the realisation of the sparse-sign sketch, column by column
 * of S: rows (device, m*zeta int32) and signs (device, m*zeta int8); entries
 * j*zeta .. j*zeta+zeta-1 describe column j of S: zeta distinct rows in [0, s)
 * in draw order, each with value signs[.]/sqrt(zeta).
 */
ns_status ns_sparse_meta(const ns_sketch_desc *desc, int64_t m, int32_t *rows, int8_t *signs, void *stream);

/*
 * ns_sketch_static -- the SRHT sketch of ns_sketch (FP64 input, NS_SRHT with
 * NS_PREC_FP64 only, bit-identical result) without a caller-supplied
 * workspace.  The paper has no counterpart of this call; it exists for
 * callers that cannot allocate device memory: code embedded in a host
 * application whose device memory is owned by the application's own pool
 * allocator, or a service that must not allocate after start-up because an
 * allocation can fail, block or fragment memory at an unpredictable moment.
 * Such callers still pass A and SA, but need no scratch of their own.
 *
 * The scratch lives in one fixed device array of 16 MiB inside libns; every
 * GPU on which the library is used holds those 16 MiB until the process
 * exits.  A problem whose scratch (sign words, sample rows and per-chunk
 * partial sums, about 8 * n * s * (number of 65536-row chunks) bytes) does not
 * fit returns NS_ERR_WORKSPACE; use ns_sketch with a workspace instead.  The
 * call allocates nothing (no cudaMalloc, no cudaFree, no allocating library
 * routine).
 *
 *   dev_status  device int32 owned by the caller, or NULL: receives 0, or
 *               NS_ERR_NONFINITE when A holds an Inf or a NaN (SA is then not
 *               meaningful).  With NULL the word inside the library's array
 *               is used and non-finite input is NOT reported to the caller.
 *
 * The first call in each CUDA context looks up the array's device address
 * (with the device current) and caches it under the context's id, so a call
 * after cudaDeviceReset (a new context, possibly another address) looks it up
 * again; make the first call in a context before any stream capture.  Every
 * call shares the one array and leaves its contents behind: calls whose work
 * overlaps on the GPU (two streams, or two threads) race on it and must be
 * serialised by the caller.
 */
ns_status ns_sketch_static(const ns_sketch_desc *desc, const void *A, int32_t dtype, int64_t m, int64_t n,
                           int64_t lda, double *SA, int32_t *dev_status, void *stream);

/*
 * ns_test_bounded_wait -- failure-detection test hook; the paper has no
 * counterpart.  Every spin wait in the library's kernels is bounded; this call
 * launches one of those waits on something nothing completes, with a short
 * limit, so the wait runs out, the kernel writes NS_ERR_TIMEOUT to
 * *dev_status and returns, and the stream stays usable.  Nothing faults or
 * hangs.
 *   which   0: the grid barrier of the cooperative kernels (two CTAs, the
 *              second leaves without arriving; limit = polls of the barrier
 *              word; ws: 256 bytes of device scratch, 256-byte aligned);
 *           1: the cluster-peer mbarrier wait of the ring Jacobi (a cluster
 *              of two CTAs, the first waits for a phase the second never
 *              completes; limit = clock cycles; ws unused), after which both
 *              CTAs meet at the final cluster barrier.
 *   limit   1 .. 2^24.
 *   dev_status  device int32, set to NS_ERR_TIMEOUT (callers zero it first).
 * Errors: NS_ERR_INVALID_ARG for another `which`, a limit out of range, a
 * NULL dev_status, or (which 0) a missing or short workspace.
 */
ns_status ns_test_bounded_wait(int32_t which, int64_t limit, int32_t *dev_status, void *ws, size_t ws_bytes,
                               void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NS_H */
