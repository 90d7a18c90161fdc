/*
 * oracle.c -- plain, slow, obviously-correct FP64 CPU reference for the
 * sketch-and-solve approximate null-space method of Park & Nakatsukasa,
 * "A Fast Randomized Algorithm for Computing an Approximate Null Space".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke() check and
 * the benchmark's CPU-baseline leg may load this library.  The GPU library
 * shares no code, header, table or constant generator with this file.
 *
 * Every routine below follows one passage of the paper (cited per function)
 * in the paper's order and notation, with no blocking, fusion or reordering.
 * All matrices are column-major; "ld" is the leading dimension.
 *
 * Readings where the paper is silent (all listed in the design notes):
 *  - the transform of the SRFT (Section 2) is the Sylvester-ordered,
 *    unnormalised Walsh-Hadamard matrix H[i,j] = (-1)^popcount(i&j) on the
 *    zero-padded length m' = 2^ceil(log2 m); S = (1/sqrt s) R H D;
 *  - R samples s of the m' coordinates uniformly without replacement; the
 *    sample is the first s images of a keyed 4-round Feistel permutation of
 *    [0, m') whose round function is Philox4x64-10 (stream 1);
 *  - the sparse-sign sketch has zeta distinct rows per column of S, chosen
 *    by Floyd's sampling algorithm, with values +-1/sqrt(zeta);
 *  - the Gaussian sketch is G/sqrt(s) with G from Box-Muller on Philox words;
 *  - the H-RHT (Section 2) is S_h (1/sqrt m') H D with the 1-hashing S_h:
 *    coordinate i goes to row floor(s (w mod 2^32) / 2^32) with the sign of
 *    bit 63 of w, w a stream-4 Philox word;
 *  - random numbers come from Philox4x64-10 (Salmon et al., SC'11) with
 *    key = (seed, 0) and counter = (index, aux, stream, 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_INVALID_ARG 1
#define OR_ERR_NOCONV 4
#define OR_ERR_TLS_NOSOLUTION 5

/* ------------------------------------------------------------------------ */
/* Philox4x64-10, written from its published definition (Salmon, Moraes,     */
/* Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).        */
/* ------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    __uint128_t p = (__uint128_t)a * (__uint128_t)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void or_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint64_t k[2] = {key_in[0], key_in[1]};
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k[0] += W0; k[1] += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c[0], &hi0, &lo0);
        mulhilo64(M1, c[2], &hi1, &lo1);
        uint64_t n0 = hi1 ^ c[1] ^ k[0];
        uint64_t n2 = hi0 ^ c[3] ^ k[1];
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* One block of stream `stream`: counter (c0, c1, stream, 0), key (seed, 0). */
static void draw(uint64_t seed, uint64_t c0, uint64_t c1, uint64_t stream, uint64_t w[4]) {
    uint64_t ctr[4] = {c0, c1, stream, 0};
    uint64_t key[2] = {seed, 0};
    or_philox4x64_10(ctr, key, w);
}

int or_ceil_log2(int64_t m) {
    int lg = 0;
    while (((int64_t)1 << lg) < m) lg++;
    return lg;
}

/* ------------------------------------------------------------------------ */
/* SRFT ingredients (Section 2): the random diagonal D of +-1 entries and    */
/* the restriction R to s coordinates chosen uniformly at random.            */
/* ------------------------------------------------------------------------ */

/* d[i] = +1 or -1: bit (i mod 64) of word ((i mod 256) / 64) of block i/256
 * of stream 0 (a set bit means -1). */
void or_signs(uint64_t seed, int64_t len, int8_t *d) {
    uint64_t w[4];
    for (int64_t i = 0; i < len; i++) {
        draw(seed, (uint64_t)(i / 256), 0, 0, w);
        int bit = (int)((w[(i % 256) / 64] >> (i % 64)) & 1u);
        d[i] = bit ? -1 : +1;
    }
}

/* Keyed permutation of [0, 2^lg): four Feistel rounds on the high half L
 * (lg - lg/2 bits) and low half Rr (lg/2 bits); even rounds update Rr from L,
 * odd rounds update L from Rr; round function word 0 of stream-1 block
 * (v, round).  Each round is invertible, so the map is a bijection. */
int64_t or_prp(uint64_t seed, int lg, int64_t x) {
    int br = lg / 2, bl = lg - br;
    uint64_t maskR = br ? ((1ULL << br) - 1) : 0;
    uint64_t maskL = bl ? ((1ULL << bl) - 1) : 0;
    uint64_t L = (uint64_t)x >> br, Rr = (uint64_t)x & maskR;
    uint64_t w[4];
    for (int round = 0; round < 4; round++) {
        if (round % 2 == 0) { draw(seed, L, (uint64_t)round, 1, w); Rr ^= w[0] & maskR; }
        else                { draw(seed, Rr, (uint64_t)round, 1, w); L ^= w[0] & maskL; }
    }
    return (int64_t)((L << br) | Rr);
}

/* r[t], t < s: the sampled coordinates of R, in draw order (distinct). */
void or_sample_rows(uint64_t seed, int lg, int64_t s, int64_t *r) {
    for (int64_t t = 0; t < s; t++) r[t] = or_prp(seed, lg, t);
}

/* Walsh-Hadamard transform in Sylvester order, written as the recursion
 * H_{2h} [x1; x2] = [H_h x1 + H_h x2; H_h x1 - H_h x2]. */
static void fwht_rec(double *x, int64_t len) {
    if (len <= 1) return;
    int64_t h = len / 2;
    fwht_rec(x, h);
    fwht_rec(x + h, h);
    for (int64_t i = 0; i < h; i++) {
        double a = x[i], b = x[i + h];
        x[i] = a + b;
        x[i + h] = a - b;
    }
}

void or_fwht(double *x, int64_t len) { fwht_rec(x, len); }

/* Algorithm 1 line 2 with the SRFT of Section 2: SA = (1/sqrt s) R H D [A;0].
 * With scaled = 0 the 1/sqrt(s) factor is left out (integer inputs then give
 * integer outputs). SA is s x n with leading dimension s. */
int or_srht(uint64_t seed, int64_t s, const double *A, int64_t m, int64_t n, int64_t lda,
            int scaled, double *SA) {
    int lg = or_ceil_log2(m);
    int64_t mp = (int64_t)1 << lg;
    if (s < 1 || s > mp || lda < m) return OR_ERR_INVALID_ARG;
    int8_t *d = (int8_t *)malloc((size_t)mp);
    int64_t *r = (int64_t *)malloc(sizeof(int64_t) * (size_t)s);
    double *buf = (double *)malloc(sizeof(double) * (size_t)mp);
    or_signs(seed, mp, d);
    or_sample_rows(seed, lg, s, r);
    double scale = scaled ? 1.0 / sqrt((double)s) : 1.0;
    for (int64_t j = 0; j < n; j++) {
        for (int64_t i = 0; i < mp; i++) buf[i] = (i < m) ? d[i] * A[i + j * lda] : 0.0;
        fwht_rec(buf, mp);
        for (int64_t t = 0; t < s; t++) SA[t + j * s] = scale * buf[r[t]];
    }
    free(d); free(r); free(buf);
    return OR_OK;
}

/* The explicit unscaled SRHT matrix for small m: S[t, j] = d_j (-1)^popcount(r_t & j),
 * j < m (s x m, leading dimension s). */
int or_srht_explicit(uint64_t seed, int64_t s, int64_t m, double *S) {
    int lg = or_ceil_log2(m);
    int64_t mp = (int64_t)1 << lg;
    if (s < 1 || s > mp) return OR_ERR_INVALID_ARG;
    int8_t *d = (int8_t *)malloc((size_t)mp);
    int64_t *r = (int64_t *)malloc(sizeof(int64_t) * (size_t)s);
    or_signs(seed, mp, d);
    or_sample_rows(seed, lg, s, r);
    for (int64_t j = 0; j < m; j++)
        for (int64_t t = 0; t < s; t++)
            S[t + j * s] = d[j] * ((__builtin_popcountll((uint64_t)(r[t] & j)) & 1) ? -1.0 : 1.0);
    free(d); free(r);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* H-RHT (Section 2, after Theorem 2.2): the SRFT with its restriction R     */
/* replaced by a random 1-hashing matrix, S = S_h (1/sqrt m') H D.  Column i */
/* of S_h has one nonzero, sg[i] = +-1, in row h[i].                         */
/* ------------------------------------------------------------------------ */

/* h[i], sg[i] for i < mp: word w = word (i mod 4) of stream-4 block i/4;
 * h[i] = floor(s (w mod 2^32) / 2^32), sg[i] = -1 if bit 63 of w is set. */
void or_hash_rows(uint64_t seed, int64_t s, int64_t mp, int64_t *h, int8_t *sg) {
    uint64_t w[4];
    for (int64_t i = 0; i < mp; i++) {
        draw(seed, (uint64_t)(i / 4), 0, 4, w);
        uint64_t word = w[i % 4];
        h[i] = (int64_t)(((word & 0xFFFFFFFFULL) * (uint64_t)s) >> 32);
        sg[i] = (word >> 63) ? -1 : +1;
    }
}

/* SA = S_h (1/sqrt m') H D [A; 0]: per column, the sign flip, the full
 * recursive transform of length m', then each coordinate i added with its
 * sign into row h[i], in i order.  With scaled = 0 the 1/sqrt(m') factor is
 * left out (integer inputs then give integer outputs). */
int or_hrht(uint64_t seed, int64_t s, const double *A, int64_t m, int64_t n, int64_t lda, int scaled,
            double *SA) {
    int lg = or_ceil_log2(m);
    int64_t mp = (int64_t)1 << lg;
    if (s < 1 || s > mp || lda < m) return OR_ERR_INVALID_ARG;
    int8_t *d = (int8_t *)malloc((size_t)mp);
    int8_t *sg = (int8_t *)malloc((size_t)mp);
    int64_t *h = (int64_t *)malloc(sizeof(int64_t) * (size_t)mp);
    double *buf = (double *)malloc(sizeof(double) * (size_t)mp);
    or_signs(seed, mp, d);
    or_hash_rows(seed, s, mp, h, sg);
    double scale = scaled ? 1.0 / sqrt((double)mp) : 1.0;
    for (int64_t j = 0; j < n; j++) {
        for (int64_t i = 0; i < mp; i++) buf[i] = (i < m) ? d[i] * A[i + j * lda] : 0.0;
        fwht_rec(buf, mp);
        for (int64_t t = 0; t < s; t++) SA[t + j * s] = 0.0;
        for (int64_t i = 0; i < mp; i++) SA[h[i] + j * s] += sg[i] * buf[i];
        for (int64_t t = 0; t < s; t++) SA[t + j * s] *= scale;
    }
    free(d); free(sg); free(h); free(buf);
    return OR_OK;
}

/* The explicit unscaled H-RHT matrix for small m:
 * S[t, j] = d_j sum over i with h[i] = t of sg[i] (-1)^popcount(i & j), j < m. */
int or_hrht_explicit(uint64_t seed, int64_t s, int64_t m, double *S) {
    int lg = or_ceil_log2(m);
    int64_t mp = (int64_t)1 << lg;
    if (s < 1 || s > mp) return OR_ERR_INVALID_ARG;
    int8_t *d = (int8_t *)malloc((size_t)mp);
    int8_t *sg = (int8_t *)malloc((size_t)mp);
    int64_t *h = (int64_t *)malloc(sizeof(int64_t) * (size_t)mp);
    or_signs(seed, mp, d);
    or_hash_rows(seed, s, mp, h, sg);
    for (int64_t j = 0; j < m; j++) {
        for (int64_t t = 0; t < s; t++) S[t + j * s] = 0.0;
        for (int64_t i = 0; i < mp; i++)
            S[h[i] + j * s] += d[j] * sg[i] * ((__builtin_popcountll((uint64_t)(i & j)) & 1) ? -1.0 : 1.0);
    }
    free(d); free(sg); free(h);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Sparse sketching matrix (Section 1 and 2 name CountSketch-type sparse     */
/* sketches): column j of S has zeta nonzeros +-1/sqrt(zeta) in distinct     */
/* rows drawn by Floyd's algorithm from stream 2.                            */
/* ------------------------------------------------------------------------ */
void or_sparse_sign_cols(uint64_t seed, int64_t s, int32_t zeta, int64_t m, int32_t *rows, int8_t *sg) {
    uint64_t w[4 * 16];
    for (int64_t j = 0; j < m; j++) {
        for (int q = 0; q < (zeta + 3) / 4; q++) draw(seed, (uint64_t)j, (uint64_t)q, 2, w + 4 * q);
        for (int i = 0; i < zeta; i++) {
            int64_t bound = s - zeta + i;               /* draw uniformly from [0, bound] */
            uint64_t hi, lo;
            mulhilo64(w[i], (uint64_t)(bound + 1), &hi, &lo);
            int64_t t = (int64_t)hi;
            for (int u = 0; u < i; u++)
                if (rows[j * zeta + u] == t) { t = bound; break; }
            rows[j * zeta + i] = (int32_t)t;
            sg[j * zeta + i] = (w[i] & 1u) ? -1 : +1;
        }
    }
}

int or_sparse_sign(uint64_t seed, int64_t s, int32_t zeta, const double *A, int64_t m, int64_t n,
                   int64_t lda, int scaled, double *SA) {
    if (zeta < 1 || zeta > 64 || zeta > s || lda < m) return OR_ERR_INVALID_ARG;
    int32_t *rows = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m * zeta));
    int8_t *sg = (int8_t *)malloc((size_t)(m * zeta));
    or_sparse_sign_cols(seed, s, zeta, m, rows, sg);
    double v = scaled ? 1.0 / sqrt((double)zeta) : 1.0;
    memset(SA, 0, sizeof(double) * (size_t)(s * n));
    for (int64_t c = 0; c < n; c++)
        for (int64_t j = 0; j < m; j++)
            for (int i = 0; i < zeta; i++)
                SA[rows[j * zeta + i] + c * s] += sg[j * zeta + i] * v * A[j + c * lda];
    free(rows); free(sg);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Gaussian sketch G/sqrt(s) (Theorem 2.1 and the scaling of Section 5).     */
/* Entry G[r, j]: block (r, j/8) of stream 3 gives four 64-bit words; word    */
/* q = (j mod 8)/2 supplies u_a = (lo32 + 1/2)/2^32 and u_b = (hi32 + 1/2)/2^32 */
/* and Box-Muller gives sqrt(-2 ln u_a) cos(2 pi u_b) for even j and          */
/* sqrt(-2 ln u_a) sin(2 pi u_b) for odd j.                                   */
/* ------------------------------------------------------------------------ */
double or_gaussian_entry(uint64_t seed, int64_t r, int64_t j) {
    uint64_t w[4];
    draw(seed, (uint64_t)r, (uint64_t)(j / 8), 3, w);
    uint64_t word = w[(j % 8) / 2];
    double ua = ((double)(uint32_t)word + 0.5) / 4294967296.0;
    double ub = ((double)(uint32_t)(word >> 32) + 0.5) / 4294967296.0;
    double rad = sqrt(-2.0 * log(ua));
    double ang = 2.0 * 3.14159265358979323846 * ub;
    return (j % 2 == 0) ? rad * cos(ang) : rad * sin(ang);
}

/* SA = G A / sqrt(s), computed for the columns listed in cols (ncols of them;
 * cols == NULL means all n columns).  SA column c lands at SA + c*s. */
int or_gaussian(uint64_t seed, int64_t s, const double *A, int64_t m, int64_t n, int64_t lda,
                const int64_t *cols, int64_t ncols, double *SA) {
    if (s < 1 || lda < m) return OR_ERR_INVALID_ARG;
    if (!cols) ncols = n;
    double scale = 1.0 / sqrt((double)s);
    double *g = (double *)malloc(sizeof(double) * (size_t)s);
    double *acc = (double *)calloc((size_t)(s * ncols), sizeof(double));
    for (int64_t j = 0; j < m; j++) {
        for (int64_t r = 0; r < s; r++) g[r] = or_gaussian_entry(seed, r, j);
        for (int64_t ci = 0; ci < ncols; ci++) {
            int64_t c = cols ? cols[ci] : ci;
            double a = A[j + c * lda];
            for (int64_t r = 0; r < s; r++) acc[r + ci * s] += g[r] * a;
        }
    }
    for (int64_t ci = 0; ci < ncols; ci++) {
        int64_t c = cols ? cols[ci] : ci;
        for (int64_t r = 0; r < s; r++) SA[r + c * s] = scale * acc[r + ci * s];
    }
    free(g); free(acc);
    return OR_OK;
}

/* Rows rows[0..nrows) of SA = G A / sqrt(s) (Theorem 2.1 scaling), every
 * column: out[i + c*nrows] = sum_j G(rows[i], j) A(j, c) / sqrt(s), summed over
 * j in increasing order as or_gaussian does (so the two agree bit for bit).
 * mag[i + c*nrows] (if not NULL) receives sqrt(sum_j (G(rows[i], j) A(j, c))^2)
 * / sqrt(s): the size of the terms, the scale against which the rounding
 * error of any evaluation of that entry is judged. */
int or_gaussian_rows(uint64_t seed, int64_t s, const double *A, int64_t m, int64_t n, int64_t lda,
                     const int64_t *rows, int64_t nrows, double *out, double *mag) {
    if (s < 1 || lda < m || nrows < 0) return OR_ERR_INVALID_ARG;
    for (int64_t i = 0; i < nrows; i++)
        if (rows[i] < 0 || rows[i] >= s) return OR_ERR_INVALID_ARG;
    double scale = 1.0 / sqrt((double)s);
    double *acc = (double *)calloc((size_t)(nrows * n), sizeof(double));
    double *sq = (double *)calloc((size_t)(nrows * n), sizeof(double));
    for (int64_t j = 0; j < m; j++) {
        for (int64_t i = 0; i < nrows; i++) {
            double g = or_gaussian_entry(seed, rows[i], j);
            for (int64_t c = 0; c < n; c++) {
                double t = g * A[j + c * lda];
                acc[i + c * nrows] += t;
                sq[i + c * nrows] += t * t;
            }
        }
    }
    for (int64_t q = 0; q < nrows * n; q++) {
        out[q] = scale * acc[q];
        if (mag) mag[q] = scale * sqrt(sq[q]);
    }
    free(acc); free(sq);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 line 3: SVD of SA, taken as Householder QR SA = QR followed   */
/* by a one-sided (Hestenes) Jacobi SVD of R; SA and R share singular values */
/* and right singular vectors (the argument in the proof of Theorem 3.2).    */
/* ------------------------------------------------------------------------ */

static double norm2_scaled(const double *x, int64_t len) {
    double mx = 0.0;
    for (int64_t i = 0; i < len; i++) if (fabs(x[i]) > mx) mx = fabs(x[i]);
    if (mx == 0.0) return 0.0;
    double ss = 0.0;
    for (int64_t i = 0; i < len; i++) { double y = x[i] / mx; ss += y * y; }
    return mx * sqrt(ss);
}

/* R (n x n, leading dimension n) of the Householder QR of B (s x n, s >= n). */
int or_householder_qr(const double *B, int64_t s, int64_t n, int64_t ldb, double *R) {
    if (s < n || ldb < s) return OR_ERR_INVALID_ARG;
    double *W = (double *)malloc(sizeof(double) * (size_t)(s * n));
    double *v = (double *)malloc(sizeof(double) * (size_t)s);
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < s; i++) W[i + j * s] = B[i + j * ldb];
    for (int64_t j = 0; j < n; j++) {
        int64_t len = s - j;
        double *x = W + j + j * s;
        double normx = norm2_scaled(x, len);
        if (normx == 0.0) continue;              /* column already zero: H_j = I */
        double alpha = (x[0] >= 0.0) ? -normx : normx;
        for (int64_t i = 0; i < len; i++) v[i] = x[i];
        v[0] -= alpha;
        double vv = 0.0;
        for (int64_t i = 0; i < len; i++) vv += v[i] * v[i];
        for (int64_t l = j + 1; l < n; l++) {
            double *y = W + j + l * s;
            double w = 0.0;
            for (int64_t i = 0; i < len; i++) w += v[i] * y[i];
            double f = 2.0 * w / vv;
            for (int64_t i = 0; i < len; i++) y[i] -= f * v[i];
        }
        x[0] = alpha;
        for (int64_t i = 1; i < len; i++) x[i] = 0.0;
    }
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < n; i++) R[i + j * n] = (i <= j) ? W[i + j * s] : 0.0;
    free(W); free(v);
    return OR_OK;
}

/* One-sided Jacobi SVD (Hestenes; Demmel & Veselic 1992) of the n x n matrix
 * in X (overwritten by X V = U Sigma).  Cyclic-by-rows order of the pairs
 * (p, q), p < q.  A pair is rotated when |gamma| > tol sqrt(alpha beta), with
 * alpha = |x_p|^2, beta = |x_q|^2, gamma = x_p . x_q.  The rotation makes the
 * pair orthogonal: zeta = (beta - alpha)/(2 gamma), t = sign(zeta)/(|zeta| +
 * sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), sn = c t.  Stops after a sweep with
 * no rotation, or after max_sweeps sweeps (status OR_ERR_NOCONV). */
int or_jacobi(double *X, int64_t n, double *V, double *sigma, double tol, int max_sweeps, int *sweeps_out) {
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < n; i++) V[i + j * n] = (i == j) ? 1.0 : 0.0;
    int sweeps = 0, converged = 0;
    while (sweeps < max_sweeps && !converged) {
        int64_t rotations = 0;
        for (int64_t p = 0; p < n - 1; p++) {
            for (int64_t q = p + 1; q < n; q++) {
                double *xp = X + p * n, *xq = X + q * n;
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int64_t i = 0; i < n; i++) {
                    alpha += xp[i] * xp[i];
                    beta += xq[i] * xq[i];
                    gamma += xp[i] * xq[i];
                }
                if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta)) continue;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t;
                if (fabs(zeta) > 1e150) t = 0.5 / zeta;
                else t = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double sn = c * t;
                for (int64_t i = 0; i < n; i++) {
                    double a = xp[i], b = xq[i];
                    xp[i] = c * a - sn * b;
                    xq[i] = sn * a + c * b;
                }
                double *vp = V + p * n, *vq = V + q * n;
                for (int64_t i = 0; i < n; i++) {
                    double a = vp[i], b = vq[i];
                    vp[i] = c * a - sn * b;
                    vq[i] = sn * a + c * b;
                }
                rotations++;
            }
        }
        sweeps++;
        if (rotations == 0) converged = 1;
    }
    for (int64_t j = 0; j < n; j++) sigma[j] = norm2_scaled(X + j * n, n);
    if (sweeps_out) *sweeps_out = sweeps;
    return converged ? OR_OK : OR_ERR_NOCONV;
}

/* Algorithm 1 line 4: W = V(:, n-k+1:n).  Singular values are ordered
 * non-increasingly (ties to the lower index); each returned vector is signed
 * so that its entry of largest magnitude (ties to the lower index) is
 * positive. */
void or_extract(const double *sigma, const double *V, int64_t n, int32_t k, double *Vk, double *sigk,
                int64_t *order_out) {
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; i++) order[i] = i;
    /* insertion sort: descending sigma, stable */
    for (int64_t i = 1; i < n; i++) {
        int64_t cur = order[i];
        int64_t j = i - 1;
        while (j >= 0 && sigma[order[j]] < sigma[cur]) { order[j + 1] = order[j]; j--; }
        order[j + 1] = cur;
    }
    for (int32_t c = 0; c < k; c++) {
        int64_t src = order[n - k + c];
        const double *v = V + src * n;
        int64_t imax = 0;
        for (int64_t i = 1; i < n; i++) if (fabs(v[i]) > fabs(v[imax])) imax = i;
        double sgn = (v[imax] < 0.0) ? -1.0 : 1.0;
        for (int64_t i = 0; i < n; i++) Vk[i + c * n] = sgn * v[i];
        sigk[c] = sigma[src];
    }
    if (order_out) memcpy(order_out, order, sizeof(int64_t) * (size_t)n);
    free(order);
}

/* The tolerance version of Algorithm 1 (Section 2, the remark after
 * Algorithm 1): the number of singular values below eps.  W is then the
 * trailing k = #{i : sigma_i < eps} columns in the order of or_extract. */
int32_t or_count_below(const double *sigma, int64_t n, double eps) {
    int32_t k = 0;
    for (int64_t i = 0; i < n; i++)
        if (sigma[i] < eps) k++;
    return k;
}

/* Sketch kinds. */
#define OR_SRHT 0
#define OR_SPARSE_SIGN 1
#define OR_GAUSSIAN 2
#define OR_HRHT 3

int or_sketch(int kind, uint64_t seed, int64_t s, int32_t zeta, const double *A, int64_t m, int64_t n,
              int64_t lda, double *SA) {
    if (kind == OR_SRHT) return or_srht(seed, s, A, m, n, lda, 1, SA);
    if (kind == OR_SPARSE_SIGN) return or_sparse_sign(seed, s, zeta, A, m, n, lda, 1, SA);
    if (kind == OR_GAUSSIAN) return or_gaussian(seed, s, A, m, n, lda, NULL, n, SA);
    if (kind == OR_HRHT) return or_hrht(seed, s, A, m, n, lda, 1, SA);
    return OR_ERR_INVALID_ARG;
}

/* Section 5, row updates of a sketch SA (s x n) of an m0-row A.
 * op 0 (Algorithm 2): A gains `row` as row j >= m0; S gains the column
 *   g / sqrt(s), g_r = G(r, j) (the Gaussian sketch's column j), and
 *   SA += g row / sqrt(s).
 * op 1 (Algorithm 3 and the non-Gaussian rule): A loses row j; SA -= (S e_j)
 *   row, where S e_j is the sketch of the unit vector e_j of length m0 for
 *   j < m0 (the SRHT or sparse-sign column), the Gaussian column j otherwise. */
int or_sketch_update(int kind, uint64_t seed, int64_t s, int32_t zeta, int64_t m0, int op, int64_t j,
                     const double *row, int64_t n, double *SA) {
    if (s < 1 || m0 < 1 || n < 1 || j < 0 || (op != 0 && op != 1) || (op == 0 && j < m0))
        return OR_ERR_INVALID_ARG;
    double *col = (double *)calloc((size_t)s, sizeof(double));
    int st = OR_OK;
    if (op == 0 || j >= m0 || kind == OR_GAUSSIAN) {
        for (int64_t r = 0; r < s; r++) col[r] = or_gaussian_entry(seed, r, j) / sqrt((double)s);
    } else {
        double *e = (double *)calloc((size_t)m0, sizeof(double));
        e[j] = 1.0;
        st = or_sketch(kind, seed, s, zeta, e, m0, 1, m0, col);
        free(e);
    }
    const double sign = (op == 0) ? 1.0 : -1.0;
    if (st == OR_OK)
        for (int64_t c = 0; c < n; c++)
            for (int64_t r = 0; r < s; r++) SA[r + c * s] += sign * col[r] * row[c];
    free(col);
    return st;
}

/* Algorithm 1 on an already-formed sketch SA (s x n, leading dimension s):
 * QR, Jacobi SVD of R, extraction.  V_full (n x n) and sigma_full (n) receive
 * the Jacobi result (may be NULL). */
int or_solve_sketched(const double *SA, int64_t s, int64_t n, int32_t k, double *Vk, double *sigk,
                      double *V_full, double *sigma_full, int *sweeps_out) {
    if (k < 1 || k > n || s < n) return OR_ERR_INVALID_ARG;
    double *R = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *V = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *sig = (double *)malloc(sizeof(double) * (size_t)n);
    int st = or_householder_qr(SA, s, n, s, R);
    if (st == OR_OK) {
        double tol = (double)n * ldexp(1.0, -53);
        st = or_jacobi(R, n, V, sig, tol, 30, sweeps_out);
        or_extract(sig, V, n, k, Vk, sigk, NULL);
        if (V_full) memcpy(V_full, V, sizeof(double) * (size_t)(n * n));
        if (sigma_full) memcpy(sigma_full, sig, sizeof(double) * (size_t)n);
    }
    free(R); free(V); free(sig);
    return st;
}

/* Algorithm 1 end to end.  SA_out (s x n) may be NULL. */
int or_solve(int kind, uint64_t seed, int64_t s, int32_t zeta, const double *A, int64_t m, int64_t n,
             int64_t lda, int32_t k, double *Vk, double *sigk, double *SA_out, double *V_full,
             double *sigma_full) {
    if (m < n || s < n || k < 1 || k > n) return OR_ERR_INVALID_ARG;
    double *SA = SA_out ? SA_out : (double *)malloc(sizeof(double) * (size_t)(s * n));
    int st = or_sketch(kind, seed, s, zeta, A, m, n, lda, SA);
    if (st == OR_OK) st = or_solve_sketched(SA, s, n, k, Vk, sigk, V_full, sigma_full, NULL);
    if (!SA_out) free(SA);
    return st;
}

/* ||A W||_F, the objective of the null-space problem (Problem 2.1). */
double or_residual(const double *A, int64_t m, int64_t n, int64_t lda, const double *W, int32_t k) {
    double ss = 0.0;
    for (int32_t c = 0; c < k; c++) {
        for (int64_t i = 0; i < m; i++) {
            double y = 0.0;
            for (int64_t j = 0; j < n; j++) y += A[i + j * lda] * W[j + c * n];
            ss += y * y;
        }
    }
    return sqrt(ss);
}

/* ------------------------------------------------------------------------ */
/* Total least squares (Section 4, Golub & Van Loan): the trailing right     */
/* singular vector v of [X b] ((n+1) columns) gives x = -v(1:n)/v(n+1).      */
/* The solution does not exist when v(n+1) vanishes.                         */
/* ------------------------------------------------------------------------ */
int or_tls(uint64_t seed, int64_t s, const double *Xb, int64_t m, int64_t n1, int64_t lda, double *x,
           double *v_out) {
    double *v = (double *)malloc(sizeof(double) * (size_t)n1);
    double sig;
    int st = or_solve(OR_SRHT, seed, s, 0, Xb, m, n1, lda, 1, v, &sig, NULL, NULL, NULL);
    if (st == OR_OK) {
        double nv = norm2_scaled(v, n1);
        double last = v[n1 - 1];
        if (fabs(last) < ldexp(1.0, -53) * nv) st = OR_ERR_TLS_NOSOLUTION;
        for (int64_t i = 0; i < n1 - 1; i++) x[i] = -v[i] / last;
    }
    if (v_out) memcpy(v_out, v, sizeof(double) * (size_t)n1);
    free(v);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Backward pass of Algorithm 1 for a loss that depends on W only through    */
/* W W^T.  With M = SA^T SA = V Sigma^2 V^T, T the trailing k indices and N   */
/* the rest, dL/dM = sum_{i in T, j in N} c_ji (v_j v_i^T + v_i v_j^T) with   */
/* c_ji = (1/2) (v_j . g_i)/(sigma_i^2 - sigma_j^2), g_i = dL/dw_i;           */
/* dL/dSA = 2 SA dL/dM; dL/dA = S^T dL/dSA with S^T = (1/sqrt s) D H R^T.     */
/* ------------------------------------------------------------------------ */
int or_backward_srht(uint64_t seed, int64_t s, int64_t m, int64_t n, int32_t k, const double *SA,
                     const double *V, const double *sigma, const double *Vk, const double *dVk,
                     double *dA, int64_t ldd) {
    if (k < 1 || k >= n || ldd < m) return OR_ERR_INVALID_ARG;
    int lg = or_ceil_log2(m);
    int64_t mp = (int64_t)1 << lg;
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *tmpV = (double *)malloc(sizeof(double) * (size_t)(n * k));
    double *tmps = (double *)malloc(sizeof(double) * (size_t)k);
    or_extract(sigma, V, n, k, tmpV, tmps, order);
    double *GM = (double *)calloc((size_t)(n * n), sizeof(double));
    for (int32_t ci = 0; ci < k; ci++) {
        const double *vi = Vk + ci * n;          /* returned (signed) trailing vector */
        const double *gi = dVk + ci * n;
        double si = sigma[order[n - k + ci]];
        for (int64_t jj = 0; jj < n - k; jj++) {
            const double *vj = V + order[jj] * n;
            double sj = sigma[order[jj]];
            double dot = 0.0;
            for (int64_t r = 0; r < n; r++) dot += vj[r] * gi[r];
            double c = 0.5 * dot / (si * si - sj * sj);
            for (int64_t b = 0; b < n; b++)
                for (int64_t a = 0; a < n; a++)
                    GM[a + b * n] += c * (vj[a] * vi[b] + vi[a] * vj[b]);
        }
    }
    /* dL/dSA = 2 SA GM  (s x n) */
    double *GB = (double *)calloc((size_t)(s * n), sizeof(double));
    for (int64_t b = 0; b < n; b++)
        for (int64_t a = 0; a < n; a++) {
            double g = 2.0 * GM[a + b * n];
            for (int64_t t = 0; t < s; t++) GB[t + b * s] += SA[t + a * s] * g;
        }
    /* dL/dA = (1/sqrt s) D H R^T dL/dSA, truncated to the first m rows */
    int8_t *d = (int8_t *)malloc((size_t)mp);
    int64_t *r = (int64_t *)malloc(sizeof(int64_t) * (size_t)s);
    double *buf = (double *)malloc(sizeof(double) * (size_t)mp);
    or_signs(seed, mp, d);
    or_sample_rows(seed, lg, s, r);
    double scale = 1.0 / sqrt((double)s);
    for (int64_t c = 0; c < n; c++) {
        for (int64_t i = 0; i < mp; i++) buf[i] = 0.0;
        for (int64_t t = 0; t < s; t++) buf[r[t]] = GB[t + c * s];
        fwht_rec(buf, mp);
        for (int64_t i = 0; i < m; i++) dA[i + c * ldd] = scale * d[i] * buf[i];
    }
    free(order); free(tmpV); free(tmps); free(GM); free(GB); free(d); free(r); free(buf);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* AAA with a reused SRHT sketch (Section 6.2, with Algorithm 3 and the      */
/* non-Gaussian row downdate of Section 5.3), real points.                    */
/*  - r_0 = mean(f); the first support point maximises |f - mean f|.         */
/*  - iteration k: the Loewner matrix gains the column (f_i - f_j)/(x_i - x_j) */
/*    of the new support point j and loses row j.  The sketch is updated as  */
/*    [SA - (S e_j) A(j,:), S c_k]: S e_j is the sketch of the unit vector.   */
/*  - the weights w solve min |A w| over |w| = 1 on the first min(4k, smax)   */
/*    rows of the smax-row sketch (Algorithm 1 on the sketch).                */
/*  - r(x) = sum w_l f_l/(x - x_l) / sum w_l/(x - x_l); the next support      */
/*    point maximises |f - r| over non-support points (lowest index on ties). */
/* With forced != NULL the support points are taken from forced[0..K-1].     */
/* Outputs: support[K], weights W[K*K] (row k-1 holds w of iteration k),     */
/* errmax[K] = max |f - r| after iteration k; SAk_out (smax x K, may be NULL) */
/* receives the final updated sketch.                                        */
/* ------------------------------------------------------------------------ */
int or_aaa(uint64_t seed, const double *x, const double *f, int64_t m, int32_t K, int64_t smax,
           const int64_t *forced, int64_t *support, double *W, double *errmax, double *SAk_out) {
    int lg = or_ceil_log2(m);
    int64_t mp = (int64_t)1 << lg;
    if (K < 1 || smax < K || smax > mp || m < 2) return OR_ERR_INVALID_ARG;
    double *SAk = (double *)calloc((size_t)(smax * K), sizeof(double));
    double *col = (double *)malloc(sizeof(double) * (size_t)m);
    double *ej = (double *)malloc(sizeof(double) * (size_t)m);
    double *Se = (double *)malloc(sizeof(double) * (size_t)smax);
    double *Sc = (double *)malloc(sizeof(double) * (size_t)smax);
    double *err = (double *)malloc(sizeof(double) * (size_t)m);
    char *is_sup = (char *)calloc((size_t)m, 1);
    double *w = (double *)malloc(sizeof(double) * (size_t)K);
    double *Sk = (double *)malloc(sizeof(double) * (size_t)(smax * K));
    int st = OR_OK;
    double mean = 0.0;
    for (int64_t i = 0; i < m; i++) mean += f[i];
    mean /= (double)m;
    for (int64_t i = 0; i < m; i++) err[i] = fabs(f[i] - mean);
    for (int32_t k = 1; k <= K; k++) {
        int64_t j;
        if (forced) j = forced[k - 1];
        else {
            j = -1;
            for (int64_t i = 0; i < m; i++)
                if (!is_sup[i] && (j < 0 || err[i] > err[j])) j = i;
        }
        support[k - 1] = j;
        /* row downdate of the existing k-1 columns (Algorithm 3, Section 5.3) */
        if (k > 1) {
            for (int64_t i = 0; i < m; i++) ej[i] = (i == j) ? 1.0 : 0.0;
            or_srht(seed, smax, ej, m, 1, m, 1, Se);
            for (int32_t l = 0; l < k - 1; l++) {
                int64_t jl = support[l];
                double a = (f[j] - f[jl]) / (x[j] - x[jl]);
                for (int64_t t = 0; t < smax; t++) SAk[t + l * smax] -= Se[t] * a;
            }
        }
        is_sup[j] = 1;
        /* column update: sketch of the new Loewner column */
        for (int64_t i = 0; i < m; i++) col[i] = is_sup[i] ? 0.0 : (f[i] - f[j]) / (x[i] - x[j]);
        or_srht(seed, smax, col, m, 1, m, 1, Sc);
        for (int64_t t = 0; t < smax; t++) SAk[t + (k - 1) * smax] = Sc[t];
        /* null vector of the first s_k rows */
        int64_t sk = 4 * (int64_t)k < smax ? 4 * (int64_t)k : smax;
        for (int32_t l = 0; l < k; l++)
            for (int64_t t = 0; t < sk; t++) Sk[t + l * sk] = SAk[t + l * smax];
        double sg;
        if (k == 1) { w[0] = 1.0; }
        else {
            int s2 = or_solve_sketched(Sk, sk, k, 1, w, &sg, NULL, NULL, NULL);
            if (s2 != OR_OK) st = s2;
        }
        for (int32_t l = 0; l < K; l++) W[(k - 1) * K + l] = (l < k) ? w[l] : 0.0;
        /* barycentric evaluation and error */
        double emax = 0.0;
        for (int64_t i = 0; i < m; i++) {
            if (is_sup[i]) { err[i] = 0.0; continue; }
            double num = 0.0, den = 0.0;
            for (int32_t l = 0; l < k; l++) {
                double cl = w[l] / (x[i] - x[support[l]]);
                num += cl * f[support[l]];
                den += cl;
            }
            err[i] = fabs(f[i] - num / den);
            if (err[i] > emax) emax = err[i];
        }
        errmax[k - 1] = emax;
    }
    if (SAk_out) memcpy(SAk_out, SAk, sizeof(double) * (size_t)(smax * K));
    free(SAk); free(col); free(ej); free(Se); free(Sc); free(err); free(is_sup); free(w); free(Sk);
    return st;
}
