// ns_jacobi32.cu -- the linear phase of the one-sided Jacobi SVD in FP32, as a
// preconditioner for the FP64 iteration of ns_dense.cu (Algorithm 1 line 3:
// the SVD of SA, through R and X = R2^T).
//
// One-sided Jacobi converges linearly over its first sweeps and quadratically
// once the columns are nearly orthogonal.  On this part FP32 arithmetic runs
// at 64 times the FP64 rate and an FP32 column takes half the bytes, so the
// linear phase runs in FP32 and the FP64 ring only finishes the job:
//
//   1. Y = X0 in FP32 (columns of X0 = R2^T scaled by one power of two);
//      columns whose norm is below 2^-60 of the largest are left out (zero in
//      Y, identity in W), so that no FP32 square underflows.  Numerically null
//      columns (~u of the largest) take part: left out, they would need FP64
//      sweeps of their own among themselves.
//   2. One-sided Jacobi sweeps on Y in FP32, the rotations accumulated in W
//      (FP32, from I), with the rotation threshold |y_a . y_b| > tau |y_a||y_b|,
//      tau = 2^-17, until a sweep rotates fewer than half of the pairs (the
//      iteration has left its linear phase) or 8 sweeps.  W is held
//      graded, W~[i, j] = W[i, j] d_i / d_j with d the column norms of X0 (a
//      rotation (c, s) of columns a, b then uses s d_b/d_a and s d_a/d_b, see
//      j32_pair): one-sided Jacobi keeps W[i, j] ~ d_j/d_i between columns of
//      very different size, so W~ is O(1) and its FP32 rounding is relative to
//      the column it lands in (plain FP32 W would carry an absolute ~1e-7 that
//      X0 W spreads from the largest columns over the smallest).
//   3. V0 = W made orthogonal in FP64: E = I - W^T W (about 1e-6), and
//      V0 = W (I + E/2 + 3 E^2 / 8), the series of (W^T W)^(-1/2) to second
//      order (the remainder is of order E^3).
//   4. X1 = X0 V0 and V = Q2 V0 in FP64: nearly orthogonal columns (cosines
//      ~ tau), where the rotations still to come are small.
//   5. Two first-order completions (see completion below): the rotation that
//      diagonalises G = X^T X to first order, made exactly orthogonal to
//      working accuracy, applied to X and V as one FP64 product each.  On the
//      benchmark's spectrum the FP64 ring then only runs its convergence check
//      (seven sweeps and a check without steps 1-5, two sweeps and a check
//      without step 5).
//
// Step 2 runs on one cluster of 8 CTAs (n <= 256): the 256 columns of Y and W
// are 16 blocks of 16 columns, two blocks per CTA in shared memory.  A sweep is
// one round-robin tournament of the blocks (15 outer steps, block pairs; the
// pairs inside each block at the first); inside an outer step the 256 pairs
// between the CTA's two blocks take 16 rounds of 16 disjoint pairs, one warp
// per pair, separated by CTA barriers only.  Between outer steps each CTA pulls
// its next blocks from its neighbours' shared memory (distributed shared
// memory loads, one cluster barrier per exchange, two slot parities).
//
// Accuracy.  W~ carries FP32 rounding relative to its O(1) entries, so
// W[i, j] is off by ~2^-24 d_j/d_i and column j of X0 W by ~2^-24 sqrt(n) d_j:
// the columns of X1 are orthogonal to ~1e-6 relative to their own sizes, and
// the FP64 corrections of step 3 (E[a, b] ~ 2^-24 d_b/d_a) keep that grading.
// Rounding in the FP64 products adds ~n u d_j to column j.  Columns below
// 2^-60 d_max keep their X0 column unchanged.  The FP64 iteration is then the
// usual one and fixes the final accuracy.
#include <cmath>
#include "ns_device.cuh"
#include "ns_internal.h"

namespace ns {

constexpr int kJ32Cta = 8;                     // CTAs per cluster
constexpr int kJ32B = 16;                      // columns per block
constexpr int kJ32Blocks = 2 * kJ32Cta;        // 16 blocks
constexpr int kJ32N = kJ32B * kJ32Blocks;      // 256 columns (n <= 256)
constexpr int kJ32Rows = 256;                  // rows of Y and of W
constexpr int kJ32Col = 2 * kJ32Rows;          // floats per column: y (256), then w (256)
constexpr int kJ32Slot = kJ32B * kJ32Col;      // floats per block slot (32 KB)
constexpr int kJ32Threads = kJ32B * 32;        // one warp per pair of a round
constexpr int kJ32Steps = kJ32Blocks - 1;      // outer steps per sweep
constexpr int kJ32MaxSweeps = 8;
constexpr float kJ32Tau = 1.0f / 131072.0f;    // 2^-17
constexpr double kJ32Keep = 7.52316384526264e-37;   // 2^-120: kept columns have |x| >= 2^-60 max |x|
constexpr size_t kJ32Smem = (size_t)4 * kJ32Slot * sizeof(float);

// slot index in the per-CTA array of four block slots: parity p holds
// top (2 p) and bottom (2 p + 1)
__device__ __forceinline__ float *j32_slot(float *base, int idx) { return base + (size_t)idx * kJ32Slot; }

// player of tournament position `pos` at step `step` (16 players, player 0 fixed)
__device__ __forceinline__ int j32_rr(int pos, int step) {
    return pos == 0 ? 0 : 1 + (pos - 1 + step) % (kJ32B - 1);
}

// One pair (columns a, b: pointers to their y rows; w~ follows at +kJ32Rows;
// da, db their scales d), one warp; returns 1 (in every lane) if the pair was
// rotated.
__device__ __forceinline__ unsigned int j32_pair(float *a, float *b, float da, float db, float tau2) {
    const int lane = threadIdx.x & 31;
    // lane l holds rows 4l..4l+3 and 128+4l..128+4l+3: each float4 access of the
    // warp covers 512 contiguous bytes (no bank conflicts)
    const float4 a0 = *(const float4 *)(a + 4 * lane), a1 = *(const float4 *)(a + 128 + 4 * lane);
    const float4 b0 = *(const float4 *)(b + 4 * lane), b1 = *(const float4 *)(b + 128 + 4 * lane);
    float al = a0.x * a0.x, be = b0.x * b0.x, ga = a0.x * b0.x;
    al = fmaf(a0.y, a0.y, al); be = fmaf(b0.y, b0.y, be); ga = fmaf(a0.y, b0.y, ga);
    al = fmaf(a0.z, a0.z, al); be = fmaf(b0.z, b0.z, be); ga = fmaf(a0.z, b0.z, ga);
    al = fmaf(a0.w, a0.w, al); be = fmaf(b0.w, b0.w, be); ga = fmaf(a0.w, b0.w, ga);
    al = fmaf(a1.x, a1.x, al); be = fmaf(b1.x, b1.x, be); ga = fmaf(a1.x, b1.x, ga);
    al = fmaf(a1.y, a1.y, al); be = fmaf(b1.y, b1.y, be); ga = fmaf(a1.y, b1.y, ga);
    al = fmaf(a1.z, a1.z, al); be = fmaf(b1.z, b1.z, be); ga = fmaf(a1.z, b1.z, ga);
    al = fmaf(a1.w, a1.w, al); be = fmaf(b1.w, b1.w, be); ga = fmaf(a1.w, b1.w, ga);
    // butterfly sums: every lane ends with the same totals (addition commutes)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        al += __shfl_xor_sync(0xffffffffu, al, o);
        be += __shfl_xor_sync(0xffffffffu, be, o);
        ga += __shfl_xor_sync(0xffffffffu, ga, o);
    }
    // |gamma| > tau sqrt(alpha beta), as (gamma/alpha)(gamma/beta) > tau^2: the
    // product alpha beta of two columns ~2^-60 of the largest would underflow
    if (!(ga != 0.0f && al > 0.0f && be > 0.0f && __fdividef(ga, al) * __fdividef(ga, be) > tau2)) return 0u;
    // the rotation of the FP64 kernel: zeta = (beta - alpha) / (2 gamma),
    // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = c t;
    // a <- c a - s b, b <- s a + c b
    // (fast division and square root: the angle needs modest accuracy only; the
    // applied (c, s) satisfy c^2 + s^2 = 1 to FP32 rounding whatever t is)
    const float z = __fdividef(be - al, 2.0f * ga), az = fabsf(z);
    const float w1 = fmaf(z, z, 1.0f);
    const float t = (az > 1e18f) ? __fdividef(0.5f, z) : copysignf(__fdividef(1.0f, az + w1 * rsqrtf(w1)), z);
    const float c = rsqrtf(fmaf(t, t, 1.0f)), s = c * t;
    // graded W~: w~_a <- c w~_a - (s d_b/d_a) w~_b,  w~_b <- (s d_a/d_b) w~_a + c w~_b
    const float sab = s * __fdividef(db, da), sba = s * __fdividef(da, db);
    float4 na0, na1, nb0, nb1;
    na0.x = c * a0.x - s * b0.x; nb0.x = s * a0.x + c * b0.x;
    na0.y = c * a0.y - s * b0.y; nb0.y = s * a0.y + c * b0.y;
    na0.z = c * a0.z - s * b0.z; nb0.z = s * a0.z + c * b0.z;
    na0.w = c * a0.w - s * b0.w; nb0.w = s * a0.w + c * b0.w;
    na1.x = c * a1.x - s * b1.x; nb1.x = s * a1.x + c * b1.x;
    na1.y = c * a1.y - s * b1.y; nb1.y = s * a1.y + c * b1.y;
    na1.z = c * a1.z - s * b1.z; nb1.z = s * a1.z + c * b1.z;
    na1.w = c * a1.w - s * b1.w; nb1.w = s * a1.w + c * b1.w;
    *(float4 *)(a + 4 * lane) = na0;
    *(float4 *)(a + 128 + 4 * lane) = na1;
    *(float4 *)(b + 4 * lane) = nb0;
    *(float4 *)(b + 128 + 4 * lane) = nb1;
    float *aw = a + kJ32Rows, *bw = b + kJ32Rows;
    const float4 p0 = *(const float4 *)(aw + 4 * lane), p1 = *(const float4 *)(aw + 128 + 4 * lane);
    const float4 q0 = *(const float4 *)(bw + 4 * lane), q1 = *(const float4 *)(bw + 128 + 4 * lane);
    na0.x = c * p0.x - sab * q0.x; nb0.x = sba * p0.x + c * q0.x;
    na0.y = c * p0.y - sab * q0.y; nb0.y = sba * p0.y + c * q0.y;
    na0.z = c * p0.z - sab * q0.z; nb0.z = sba * p0.z + c * q0.z;
    na0.w = c * p0.w - sab * q0.w; nb0.w = sba * p0.w + c * q0.w;
    na1.x = c * p1.x - sab * q1.x; nb1.x = sba * p1.x + c * q1.x;
    na1.y = c * p1.y - sab * q1.y; nb1.y = sba * p1.y + c * q1.y;
    na1.z = c * p1.z - sab * q1.z; nb1.z = sba * p1.z + c * q1.z;
    na1.w = c * p1.w - sab * q1.w; nb1.w = sba * p1.w + c * q1.w;
    *(float4 *)(aw + 4 * lane) = na0;
    *(float4 *)(aw + 128 + 4 * lane) = na1;
    *(float4 *)(bw + 4 * lane) = nb0;
    *(float4 *)(bw + 128 + 4 * lane) = nb1;
    return 1u;
}

// The 16 rounds of cross pairs of one outer step (all warps of the CTA): warp w
// keeps top column T[w] (y and w~, 8 + 8 values per lane) and its squared norm
// in registers; in round r it pairs with bottom column B[(w + r) mod 16], read
// from and written back to shared memory with its squared norm in bn[].  Only
// the inner product needs a warp reduction: a rotation that zeroes gamma maps
// the squared norms to alpha - t gamma and beta + t gamma exactly (the
// one-sided Jacobi identity), and both are recomputed from the columns at the
// start of every outer step, so rounding does not accumulate.  Returns the
// warp's rotations.
__device__ __forceinline__ unsigned int j32_cross_rounds(float *T, float *B, float dt, const float *dB, float *bn,
                                                         float tau2) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float *tc = T + w * kJ32Col;
    float4 ty0 = *(const float4 *)(tc + 4 * lane), ty1 = *(const float4 *)(tc + 128 + 4 * lane);
    float4 tw0 = *(const float4 *)(tc + kJ32Rows + 4 * lane), tw1 = *(const float4 *)(tc + kJ32Rows + 128 + 4 * lane);
    float al, be;
    {   // exact squared norms: this warp's top column, and bottom column w into bn[w]
        const float *bc = B + w * kJ32Col;
        const float4 b0 = *(const float4 *)(bc + 4 * lane), b1 = *(const float4 *)(bc + 128 + 4 * lane);
        al = ty0.x * ty0.x; be = b0.x * b0.x;
        al = fmaf(ty0.y, ty0.y, al); be = fmaf(b0.y, b0.y, be);
        al = fmaf(ty0.z, ty0.z, al); be = fmaf(b0.z, b0.z, be);
        al = fmaf(ty0.w, ty0.w, al); be = fmaf(b0.w, b0.w, be);
        al = fmaf(ty1.x, ty1.x, al); be = fmaf(b1.x, b1.x, be);
        al = fmaf(ty1.y, ty1.y, al); be = fmaf(b1.y, b1.y, be);
        al = fmaf(ty1.z, ty1.z, al); be = fmaf(b1.z, b1.z, be);
        al = fmaf(ty1.w, ty1.w, al); be = fmaf(b1.w, b1.w, be);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            al += __shfl_xor_sync(0xffffffffu, al, o);
            be += __shfl_xor_sync(0xffffffffu, be, o);
        }
        if (lane == 0) bn[w] = be;
    }
    const float inv_dt = __fdividef(1.0f, dt);
    __syncthreads();
    unsigned int rots = 0;
    for (int r = 0; r < kJ32B; ++r) {
        const int bq = (w + r) & (kJ32B - 1);
        float *bc = B + bq * kJ32Col;
        float4 by0 = *(const float4 *)(bc + 4 * lane), by1 = *(const float4 *)(bc + 128 + 4 * lane);
        const float4 bw0 = *(const float4 *)(bc + kJ32Rows + 4 * lane);
        const float4 bw1 = *(const float4 *)(bc + kJ32Rows + 128 + 4 * lane);
        const float bb = bn[bq], db = dB[bq];
        float ga = ty0.x * by0.x;
        ga = fmaf(ty0.y, by0.y, ga);
        ga = fmaf(ty0.z, by0.z, ga);
        ga = fmaf(ty0.w, by0.w, ga);
        ga = fmaf(ty1.x, by1.x, ga);
        ga = fmaf(ty1.y, by1.y, ga);
        ga = fmaf(ty1.z, by1.z, ga);
        ga = fmaf(ty1.w, by1.w, ga);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
        const bool rot = ga != 0.0f && al > 0.0f && bb > 0.0f && __fdividef(ga, al) * __fdividef(ga, bb) > tau2;
        if (rot) {  // warp-uniform: every lane holds the same sums
            const float z = __fdividef(bb - al, 2.0f * ga), az = fabsf(z);
            const float w1 = fmaf(z, z, 1.0f);
            const float t = (az > 1e18f) ? __fdividef(0.5f, z) : copysignf(__fdividef(1.0f, az + w1 * rsqrtf(w1)), z);
            const float cs = rsqrtf(fmaf(t, t, 1.0f)), sn = cs * t;
            const float sab = sn * db * inv_dt, sba = sn * dt * __fdividef(1.0f, db);
            float4 na0, na1;
            na0.x = cs * ty0.x - sn * by0.x; by0.x = sn * ty0.x + cs * by0.x;
            na0.y = cs * ty0.y - sn * by0.y; by0.y = sn * ty0.y + cs * by0.y;
            na0.z = cs * ty0.z - sn * by0.z; by0.z = sn * ty0.z + cs * by0.z;
            na0.w = cs * ty0.w - sn * by0.w; by0.w = sn * ty0.w + cs * by0.w;
            na1.x = cs * ty1.x - sn * by1.x; by1.x = sn * ty1.x + cs * by1.x;
            na1.y = cs * ty1.y - sn * by1.y; by1.y = sn * ty1.y + cs * by1.y;
            na1.z = cs * ty1.z - sn * by1.z; by1.z = sn * ty1.z + cs * by1.z;
            na1.w = cs * ty1.w - sn * by1.w; by1.w = sn * ty1.w + cs * by1.w;
            ty0 = na0;
            ty1 = na1;
            float4 nb0, nb1;
            na0.x = cs * tw0.x - sab * bw0.x; nb0.x = sba * tw0.x + cs * bw0.x;
            na0.y = cs * tw0.y - sab * bw0.y; nb0.y = sba * tw0.y + cs * bw0.y;
            na0.z = cs * tw0.z - sab * bw0.z; nb0.z = sba * tw0.z + cs * bw0.z;
            na0.w = cs * tw0.w - sab * bw0.w; nb0.w = sba * tw0.w + cs * bw0.w;
            na1.x = cs * tw1.x - sab * bw1.x; nb1.x = sba * tw1.x + cs * bw1.x;
            na1.y = cs * tw1.y - sab * bw1.y; nb1.y = sba * tw1.y + cs * bw1.y;
            na1.z = cs * tw1.z - sab * bw1.z; nb1.z = sba * tw1.z + cs * bw1.z;
            na1.w = cs * tw1.w - sab * bw1.w; nb1.w = sba * tw1.w + cs * bw1.w;
            tw0 = na0;
            tw1 = na1;
            *(float4 *)(bc + 4 * lane) = by0;
            *(float4 *)(bc + 128 + 4 * lane) = by1;
            *(float4 *)(bc + kJ32Rows + 4 * lane) = nb0;
            *(float4 *)(bc + kJ32Rows + 128 + 4 * lane) = nb1;
            const float tg = t * ga;
            al -= tg;
            if (lane == 0) bn[bq] = bb + tg;
            ++rots;
        }
        __syncthreads();
    }
    *(float4 *)(tc + 4 * lane) = ty0;
    *(float4 *)(tc + 128 + 4 * lane) = ty1;
    *(float4 *)(tc + kJ32Rows + 4 * lane) = tw0;
    *(float4 *)(tc + kJ32Rows + 128 + 4 * lane) = tw1;
    __syncthreads();
    return rots;
}

// (not volatile, no memory clobber: the blocks it reads were completed before
// the cluster barrier that precedes the exchange, so the compiler may issue all
// of a thread's loads before its stores)
__device__ __forceinline__ float4 ld_peer_f4(uint32_t addr) {
    float4 v;
    asm("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}

__device__ __forceinline__ void st_peer_u32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void st_peer_f32(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_peer_f64(uint32_t addr, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

// X (n x n FP64, column-major) -> V0 (n x n FP64: the accumulated FP32
// rotations W, exactly), ctl[0] = 1 if the phase ran (0: it was skipped and V0
// is not written), ctl[1] = sweeps, ctl[2] = rotations.
// At most 64 registers a thread (no spills): a CTA of the phase then leaves
// half of its SM's registers, room for a fused-QR CTA of another solve in
// flight beside it.
__global__ void __cluster_dims__(kJ32Cta, 1, 1) __maxnreg__(64)
    jacobi32_phase_kernel(const double *__restrict__ X, int64_t n, double *__restrict__ V0, unsigned int *ctl) {
    extern __shared__ __align__(16) float j32_smem[];
    __shared__ double s_nrm[2 * kJ32B];
    __shared__ double s_max[kJ32Cta];
    __shared__ unsigned int s_cnt[kJ32Cta];
    __shared__ unsigned int s_rot[kJ32Cta];
    __shared__ unsigned int s_local;
    __shared__ float s_d[4][kJ32B];  // column scales d of the four block slots (moved with the blocks)
    __shared__ float d_all[kJ32N];   // column scales d of every column (rows of W)
    __shared__ float s_bn[kJ32B];    // squared norms of the bottom block's columns during the cross rounds
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int c = (int)cluster_rank();
    const int btop = c, bbot = kJ32Blocks - 1 - c;  // blocks held at the start of every sweep
    cluster_sync_all();  // every CTA of the cluster has started before any distributed access
    // ---- column norms of this CTA's 32 columns (FP64), cluster-wide maximum
    for (int q = w; q < 2 * kJ32B; q += kJ32Threads / 32) {
        const int64_t j = (int64_t)(q < kJ32B ? btop : bbot) * kJ32B + (q % kJ32B);
        double a = 0.0;
        if (j < n)
            for (int64_t r = lane; r < n; r += 32) {
                const double x = X[r + j * n];
                a = fma(x, x, a);
            }
        a = warp_sum(a);
        if (lane == 0) s_nrm[q] = a;
    }
    __syncthreads();
    if (tid == 0) {
        double mx = 0.0;
        for (int q = 0; q < 2 * kJ32B; ++q) mx = fmax(mx, s_nrm[q]);
        for (int r = 0; r < kJ32Cta; ++r) st_peer_f64(peer_addr(shared_addr(&s_max[c]), r), mx);
    }
    __syncthreads();
    cluster_sync_all();
    double gmax = 0.0;
    for (int r = 0; r < kJ32Cta; ++r) gmax = fmax(gmax, s_max[r]);
    const double keep = gmax * kJ32Keep;
    // scale: the largest column norm lands in [0.5, 1)
    int e2 = 0;
    frexp(sqrt(gmax), &e2);
    const double sc = ldexp(1.0, -e2);
    // column scales d (1 for the columns left out) into this CTA's two slots and
    // into every CTA's d_all; the kept count into every CTA's s_cnt
    if (tid < 2 * kJ32B) {
        const int sl = tid / kJ32B, i = tid % kJ32B;
        const int64_t j = (int64_t)(sl == 0 ? btop : bbot) * kJ32B + i;
        const double nr = s_nrm[tid];
        const float dv = (nr > 0.0 && nr >= keep && gmax < 1e300) ? (float)(sqrt(nr) * sc) : 1.0f;
        s_d[sl][i] = dv;
        for (int r = 0; r < kJ32Cta; ++r) st_peer_f32(peer_addr(shared_addr(&d_all[j]), r), dv);
    }
    if (tid == 0) {
        unsigned int cnt = 0;
        for (int q = 0; q < 2 * kJ32B; ++q) cnt += (s_nrm[q] > 0.0 && s_nrm[q] >= keep) ? 1u : 0u;
        for (int r = 0; r < kJ32Cta; ++r) st_peer_u32(peer_addr(shared_addr(&s_cnt[c]), r), cnt);
    }
    __syncthreads();
    cluster_sync_all();
    unsigned int kept = 0;
    for (int r = 0; r < kJ32Cta; ++r) kept += s_cnt[r];
    if (!(gmax > 0.0) || !(gmax < 1e300) || 2 * (int64_t)kept < n) {  // nothing to gain (or nothing finite)
        if (c == 0 && tid == 0) ctl[0] = 0u;
        return;  // no CTA touched a peer after the last cluster barrier
    }
    // ---- Y and W~ = I into the parity-0 slots
    for (int sl = 0; sl < 2; ++sl) {
        float *S = j32_slot(j32_smem, sl);
        const int blk = sl == 0 ? btop : bbot;
        for (int idx = tid; idx < kJ32Slot; idx += kJ32Threads) {
            const int i = idx / kJ32Col, e = idx % kJ32Col;
            const int64_t j = (int64_t)blk * kJ32B + i;
            const bool inc = j < n && s_nrm[sl * kJ32B + i] > 0.0 && s_nrm[sl * kJ32B + i] >= keep;
            float v;
            if (e < kJ32Rows) v = (inc && e < n) ? (float)(X[e + j * n] * sc) : 0.0f;
            else v = (e - kJ32Rows == j) ? 1.0f : 0.0f;
            S[idx] = v;
        }
    }
    if (tid == 0) s_local = 0u;
    __syncthreads();
    const float tau2 = kJ32Tau * kJ32Tau;
    int par = 0, sweeps = 0;
    unsigned int rot_total = 0;
    for (int sweep = 0; sweep < kJ32MaxSweeps; ++sweep) {
        ++sweeps;
        unsigned int mine = 0;  // rotations of this warp (lane values agree)
        for (int step = 0; step < kJ32Steps; ++step) {
            float *T = j32_slot(j32_smem, 2 * par), *B = j32_slot(j32_smem, 2 * par + 1);
            if (step == 0) {  // pairs inside each block: the first half of the warps the top block
                constexpr int kHalf = kJ32B / 2;
                float *M = w < kHalf ? T : B;
                const float *dM = s_d[w < kHalf ? 2 * par : 2 * par + 1];
                const int q = w & (kHalf - 1);
                for (int r = 0; r < kJ32B - 1; ++r) {
                    const int pa = j32_rr(q, r), pb = j32_rr(kJ32B - 1 - q, r);
                    mine += j32_pair(M + pa * kJ32Col, M + pb * kJ32Col, dM[pa], dM[pb], tau2);
                    __syncthreads();
                }
            }
            // the 256 pairs between the two blocks: warp w holds top column w in
            // registers for all 16 rounds; bottom column (w + r) mod 16 visits it
            // through shared memory with its squared norm
            mine += j32_cross_rounds(T, B, s_d[2 * par][w], s_d[2 * par + 1], s_bn, tau2);
            if (step == kJ32Steps - 1) {  // publish this CTA's rotation count of the sweep
                if (lane == 0) atomicAdd(&s_local, mine);
                __syncthreads();
                if (tid == 0) {
                    for (int r = 0; r < kJ32Cta; ++r) st_peer_u32(peer_addr(shared_addr(&s_rot[c]), r), s_local);
                    s_local = 0u;
                }
                __syncthreads();
            }
            // ---- exchange: position p takes the block of position p - 1 (1 after 15; 0 stays)
            cluster_sync_all();
            const int np = par ^ 1;
            float *dT = j32_slot(j32_smem, 2 * np), *dB = j32_slot(j32_smem, 2 * np + 1);
            // sources: new top <- (c == 0: own top; c == 1: CTA 0's bottom; else CTA c-1's top)
            //          new bottom <- (c == 7: own top; else CTA c+1's bottom)
            const int st_rank = c == 0 ? 0 : (c == 1 ? 0 : c - 1);
            const int st_slot = c == 0 ? 2 * par : (c == 1 ? 2 * par + 1 : 2 * par);
            const int sb_rank = c == kJ32Cta - 1 ? c : c + 1;
            const int sb_slot = c == kJ32Cta - 1 ? 2 * par : 2 * par + 1;
            const uint32_t srcT = peer_addr(shared_addr(j32_slot(j32_smem, st_slot)), (uint32_t)st_rank);
            const uint32_t srcB = peer_addr(shared_addr(j32_slot(j32_smem, sb_slot)), (uint32_t)sb_rank);
            if (tid < 2 * kJ32B) {  // the blocks' column scales travel with them
                const int h = tid / kJ32B, i = tid % kJ32B;
                const uint32_t src = peer_addr(shared_addr(&s_d[h ? sb_slot : st_slot][i]),
                                               (uint32_t)(h ? sb_rank : st_rank));
                float v;
                asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(src) : "memory");
                s_d[2 * np + h][i] = v;
            }
            {
                constexpr int kPer = kJ32Slot / 4 / kJ32Threads;  // float4 per thread and block (4)
                float4 x[kPer], y[kPer];
#pragma unroll
                for (int u = 0; u < kPer; ++u) {
                    x[u] = ld_peer_f4(srcT + 16u * (uint32_t)(tid + u * kJ32Threads));
                    y[u] = ld_peer_f4(srcB + 16u * (uint32_t)(tid + u * kJ32Threads));
                }
#pragma unroll
                for (int u = 0; u < kPer; ++u) {
                    ((float4 *)dT)[tid + u * kJ32Threads] = x[u];
                    ((float4 *)dB)[tid + u * kJ32Threads] = y[u];
                }
            }
            __syncthreads();
            par = np;
        }
        // every CTA reads the same counts (published before the last cluster barrier)
        unsigned int tot = 0;
        for (int r = 0; r < kJ32Cta; ++r) tot += s_rot[r];
        rot_total += tot;
        // a sweep that rotated fewer than half of the pairs has left the linear
        // phase: the FP64 iteration converges quadratically from here
        if (2ull * tot < (unsigned long long)kept * (kept - 1) / 2) break;
    }
    // ---- blocks are back where they started: W = D^-1 W~ D -> V0 (FP64); the
    // scale of row r (column r of X0) is read from the slot that holds it
    for (int sl = 0; sl < 2; ++sl) {
        const float *S = j32_slot(j32_smem, 2 * par + sl);
        const int blk = sl == 0 ? btop : bbot;
        for (int idx = tid; idx < kJ32B * kJ32Rows; idx += kJ32Threads) {
            const int i = idx / kJ32Rows, r = idx % kJ32Rows;
            const int64_t j = (int64_t)blk * kJ32B + i;
            if (j < n && r < n) {
                const double wv = (double)S[i * kJ32Col + kJ32Rows + r];
                V0[r + j * n] = wv == 0.0 ? 0.0 : wv * ((double)s_d[2 * par + sl][i] / (double)d_all[r]);
            }
        }
    }
    if (c == 0 && tid == 0) {
        ctl[0] = 1u;
        ctl[1] = (unsigned int)sweeps;
        ctl[2] = rot_total;
    }
    __syncthreads();
    cluster_sync_all();  // no CTA leaves while a peer may still read its shared memory
}

// ----------------------------------------------------- small FP64 GEMMs ----
// C (M x N, column-major, leading dimension ldc) = op(A) B with op(A) = A
// (M x K) or A^T (A: K x M), B (K x N).  One 8 x 8 tile per CTA of 128
// threads: two threads per output, one summing the even chunks of 8 k, the
// other the odd ones (each an FMA chain in increasing k), then their sum.
// The products run in T: double, or float where the FP32 error (2^-24 times
// the sum of the |terms|) stays below 2^-53 once the series' coefficient is
// applied: E^2 in the series for (W^T W)^(-1/2) (|E| ~ 3e-6, n <= 256: sums
// below 2^-28) and K^4, K^6 of the completion (sums below b^2 <= 2^-26, t^4 b^2
// once scaled).
// Small tiles and the split of K keep enough independent chains in flight on
// each SM sub-partition's FP64 pipe even for a symmetric product of n = 256
// (528 tiles).  Skipped when *ctl == 0 (the FP32 phase did not run).
//   EPI 0: C = AB;  1: C = I - AB;  2: C = I + E/2 + (3/8) AB;
//   EPI 3: C = Q = I + t K + t^2 K2/2 - t^4 K4/8 + t^6 AB/16, the
//          completion's rotation (K's diagonal slots hold other data and
//          count as 0; t and the skip of the last two terms follow from the
//          bound b, see completion).
//   EPI 4: C = AB unless the completion's bound b says the K^4 term is
//          negligible (then nothing runs).
//   DZ: the diagonal entries of A and B count as 0 (K held in place of G).
//   SYM: the product is symmetric.  Only the tiles on and above the diagonal
//        run (a triangular grid); each writes its mirror image, with K's sign
//        flipped for EPI 3, and on a diagonal tile the upper entry defines
//        both, so the result is exactly symmetric (apart from K).
//   blockIdx.z picks one of two (A, C) pairs: X Q and V Q in one launch.
constexpr int kG64T = 8;

struct G64Args {
    const double *A[2];
    int64_t lda;
    const double *B;
    int64_t ldb;
    double *C[2];
    int64_t ldc;
    const double *E;      // EPI 2: E (M x N, ld ldc)
    const double *Km;     // EPI 3: K off the diagonal (ld ldc)
    const double *K2;     // EPI 3: K^2 (ld ldc)
    const double *K4;     // EPI 3: K^4 (ld ldc)
    const unsigned long long *bnd;  // EPI 3, 4: the completion's bound b (bits of a double)
    unsigned int *verdict;          // EPI 3: where the last completion writes its verdict, else null
    unsigned int *ran;              // EPI 4: set to 1 when the product ran
    const unsigned int *cnt;        // EPI 3: pairs left out, then max |K| (bits) at cnt + 2
    const unsigned int *gate;       // if set: the product runs only when *gate == 2
    int64_t M, N, K;
    const unsigned int *ctl;
};

// Entries of |K| above this are left to the FP64 sweeps (pairs whose squared
// norms are too close for the first-order rotation to be small).
constexpr double kCorrKappa = 0.00390625;      // 2^-8
constexpr double kCorrBmax = 1.220703125e-4;   // 2^-13: largest b taken with t = 1
constexpr double kCorrSmall = 1.862645149230957e-9;  // 2^-29: below, the K^4, K^6 terms are < 2^-60
constexpr double kCorrDone = 9.5367431640625e-7;     // 2^-20

__device__ __forceinline__ double corr_bound(const unsigned long long *bnd) {
    return __longlong_as_double((long long)*(volatile const unsigned long long *)bnd);
}

template <typename T, bool TA, int EPI, bool SYM, bool DZ>
__global__ void __launch_bounds__(2 * kG64T * kG64T) gemm64_kernel(const G64Args g) {
    if (g.ctl && *(volatile const unsigned int *)g.ctl == 0u) return;
    if (g.gate && *(volatile const unsigned int *)g.gate != 2u) return;
    bool skip_k = false;  // EPI 3, 4: the K^4 and K^6 terms are negligible
    if (EPI == 3 || EPI == 4) skip_k = corr_bound(g.bnd) <= kCorrSmall;
    if (EPI == 4 && skip_k) return;
    if (EPI == 4 && blockIdx.x == 0 && threadIdx.x == 0) *g.ran = 1u;
    __shared__ T As[2][kG64T][kG64T + 1];  // As[h][k][i] = op(A)[i, k] of chunk h
    __shared__ T Bs[2][kG64T][kG64T + 1];  // Bs[h][k][j] = B[k, j] of chunk h
    __shared__ T part[kG64T * kG64T];      // the odd chunks' sums
    int64_t bx = blockIdx.x, by = blockIdx.y;
    if (SYM) {  // triangular index -> tile (bx, by), bx <= by
        int64_t t = blockIdx.x;
        by = 0;
        while (t > by) {
            t -= by + 1;
            ++by;
        }
        bx = t;
    }
    const double *A = g.A[blockIdx.z];
    double *C = g.C[blockIdx.z];
    const int h = threadIdx.x / (kG64T * kG64T), tl = threadIdx.x % (kG64T * kG64T);
    const int tx = tl % kG64T, ty = tl / kG64T;
    const int64_t i = bx * kG64T + tx, j = by * kG64T + ty;
    const int64_t M = g.M, N = g.N, K = skip_k ? 0 : g.K;
    T acc = T(0);
    for (int64_t k00 = 0; k00 < K; k00 += 2 * kG64T) {
        {   // half h loads chunk k00 + h*8: op(A)[bx*8 + ?, k + ?] and B[k + ?, by*8 + ?]
            const int64_t k0 = k00 + h * kG64T;
            const int64_t ai = bx * kG64T + (TA ? ty : tx), ak = k0 + (TA ? tx : ty);
            double av = 0.0;
            if (ai < M && ak < K && !(DZ && ai == ak)) av = TA ? A[ak + ai * g.lda] : A[ai + ak * g.lda];
            if (TA) As[h][tx][ty] = (T)av;
            else As[h][ty][tx] = (T)av;
            const int64_t bk = k0 + tx, bj = by * kG64T + ty;
            Bs[h][tx][ty] = (T)((bk < K && bj < N && !(DZ && bk == bj)) ? g.B[bk + bj * g.ldb] : 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kG64T; ++kk) acc = fma(As[h][kk][tx], Bs[h][kk][ty], acc);
        __syncthreads();
    }
    if (h == 1) part[tl] = acc;
    __syncthreads();
    if (h == 1) return;
    acc += part[tl];
    const double accd = (double)acc;
    if (EPI == 3 && g.verdict && blockIdx.x == 0 && threadIdx.x == 0) {
        // verdict for the FP64 iteration: 2 (start with the convergence check)
        // when the full step was taken, no pair was left out and every
        // rotation was tiny
        const double b = corr_bound(g.bnd);
        const double mk = __longlong_as_double((long long)*(volatile const unsigned long long *)(g.cnt + 2));
        *g.verdict = (b <= kCorrBmax && g.cnt[0] == 0u && mk <= kCorrDone) ? 2u : 0u;
    }
    if (i >= M || j >= N) return;
    if (SYM && bx == by && i > j) return;  // the upper entry writes both
    const double id = (i == j) ? 1.0 : 0.0;
    const int64_t ld = g.ldc;
    double v = accd, vm = accd;  // C[i, j] and its mirror C[j, i]
    if (EPI == 1) v = vm = id - accd;
    if (EPI == 2) v = vm = id + 0.5 * g.E[i + j * ld] + 0.375 * accd;
    if (EPI == 3) {
        const double b = corr_bound(g.bnd);
        const double t = (b > kCorrBmax) ? sqrt(kCorrBmax / b) : 1.0, t2 = t * t;
        const double kij = (i == j) ? 0.0 : t * g.Km[i + j * ld];
        double sym = 0.5 * t2 * g.K2[i + j * ld];
        if (!skip_k) {
            const double t4 = t2 * t2;
            sym += -0.125 * t4 * g.K4[i + j * ld] + 0.0625 * (t4 * t2) * accd;
        }
        v = (id + kij) + sym;
        vm = (id - kij) + sym;
    }
    C[i + j * ld] = v;
    if (SYM && i != j) C[j + i * ld] = vm;
}

__global__ void copy_if_kernel(const double *__restrict__ a, int64_t len, double *__restrict__ b,
                               const unsigned int *ctl) {
    if (*(volatile const unsigned int *)ctl == 0u) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

template <bool TA, int EPI, bool SYM, bool DZ = false, typename T = double>
static cudaError_t gemm64(const G64Args &g, bool dual, cudaStream_t st) {
    const int64_t mt = (g.M + kG64T - 1) / kG64T, nt = (g.N + kG64T - 1) / kG64T;
    const dim3 grid = SYM ? dim3((unsigned)(mt * (mt + 1) / 2), 1, dual ? 2 : 1)
                          : dim3((unsigned)mt, (unsigned)nt, dual ? 2 : 1);
    gemm64_kernel<T, TA, EPI, SYM, DZ><<<grid, 2 * kG64T * kG64T, 0, st>>>(g);
    return cudaGetLastError();
}

static G64Args g64(const double *A, int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc, int64_t n,
                   const unsigned int *ctl) {
    G64Args g = {};
    g.A[0] = g.A[1] = A;
    g.lda = lda;
    g.B = B;
    g.ldb = ldb;
    g.C[0] = g.C[1] = C;
    g.ldc = ldc;
    g.M = g.N = g.K = n;
    g.ctl = ctl;
    return g;
}

// -------------------------------------------- first-order completion ----
// After the FP32 phase the columns of X are orthogonal to ~1e-5 relative to
// their sizes, so G = X^T X is diagonal up to small off-diagonal entries.  For
// such a nearly diagonal symmetric matrix the rotation that diagonalises it is,
// to first order, exp(K) with K skew, K[p, q] = G[p, q] / (G[q, q] - G[p, p])
// (the first-order completion of a nearly diagonal eigenproblem, Davies and
// Modi, Linear Algebra Appl. 77 (1986)).  It is applied as the orthogonal
//   Q = K + (I + K^2)^(1/2),
// (Q^T Q = (A - K)(A + K) = A^2 - K^2 = I for A = (I + K^2)^(1/2), which
// commutes with K), the square root by its binomial series to K^6:
// A = I + K^2/2 - K^4/8 + K^6/16, so that Q^T Q = I + O(5 K^8 / 64).  The
// step is scaled, K -> t K, so that this remainder stays below 2^-55:
// b = max_j sum_i |K^2[i, j]| bounds ||K||_2^2 and t = min(1, sqrt(bmax / b)).
// Pairs whose |K| exceeds kCorrKappa (close squared norms) keep K = 0 and are
// left to the FP64 sweeps.  After two completions the cosines on the
// benchmark's spectrum fall from ~1e-5 to ~1e-9 and ~1e-16.
//
// Control words of one completion (from cw, zeroed with the barrier words):
// cw[0] pairs left out, cw[1] 1 if the K^4 and K^6 terms were formed,
// cw[2..3] max |K| kept, cw[4..5] the bound b (doubles as bits: non-negative doubles order like their bit patterns, so integer
// atomic max gives a deterministic result).

// K in place of G off the diagonal (the diagonal keeps G's), with the count of
// pairs left out and the largest |K| kept.
__global__ void __launch_bounds__(256) corr_k_kernel(double *GK, int64_t n, unsigned int *cw,
                                                     const unsigned int *ctl) {
    if (*(volatile const unsigned int *)ctl == 0u) return;
    unsigned int out = 0;
    double mk = 0.0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx % n, j = idx / n;
        if (i == j) continue;
        const double g = GK[idx];
        double k = 0.0;
        if (g != 0.0) {
            const double den = GK[j + j * n] - GK[i + i * n];
            if (fabs(g) <= kCorrKappa * fabs(den)) {
                k = g / den;
                mk = fmax(mk, fabs(k));
            } else if (i < j) {
                ++out;  // also Inf and NaN
            }
        }
        GK[idx] = k;
    }
    for (int o = 16; o > 0; o >>= 1) {
        out += __shfl_xor_sync(0xffffffffu, out, o);
        mk = fmax(mk, __shfl_xor_sync(0xffffffffu, mk, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (out) atomicAdd(cw, out);
        atomicMax((unsigned long long *)(cw + 2), (unsigned long long)__double_as_longlong(mk));
    }
}

// b = max_j sum_i |K2[i, j]|, one warp per column
__global__ void __launch_bounds__(256) corr_bound_kernel(const double *K2, int64_t n, unsigned int *cw,
                                                         const unsigned int *ctl) {
    if (*(volatile const unsigned int *)ctl == 0u) return;
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= n) return;
    double sum = 0.0;
    for (int64_t i = lane; i < n; i += 32) sum += fabs(K2[i + j * n]);
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) atomicMax((unsigned long long *)(cw + 4), (unsigned long long)__double_as_longlong(sum));
}

// The FP64 iteration's convergence test on the Gram matrix of the final X
// (G = X^T X, only when the last completion's verdict is 2): a pair needs a
// rotation when G[p, q] != 0 and G[p, q]^2 > tol^2 G[p, p] G[q, q], the rule of
// the iteration's own check pass; any such pair sets ctl[16].
__global__ void __launch_bounds__(256) corr_check_kernel(const double *G, int64_t n, double tol2,
                                                         unsigned int *ctl) {
    if (*(volatile const unsigned int *)ctl == 0u || *(volatile const unsigned int *)(ctl + 3) != 2u) return;
    int bad = 0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = idx % n, q = idx / n;
        if (p >= q) continue;
        const double g = G[idx];
        if (g != 0.0 && g * g > tol2 * G[p + p * n] * G[q + q * n]) bad = 1;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(ctl + 16, 1u);
}

// (Xo, Vo) = (Xi, Vi) Q for one completion; scratch: G (then K) and K^2
// (n x n each, in R2), K^4 (n x n), Q (n x n); cw: this completion's control
// words; verdict: where the last completion writes its verdict, else null.
static cudaError_t completion(const double *Xi, const double *Vi, double *Xo, double *Vo, int64_t n, double *GKm,
                              double *K2m, double *K4m, double *Qm, unsigned int *cw, unsigned int *verdict,
                              const unsigned int *ctl, cudaStream_t st) {
    cudaError_t e;
    const unsigned long long *bnd = reinterpret_cast<const unsigned long long *>(cw + 4);
    G64Args g = g64(Xi, n, Xi, n, GKm, n, n, ctl);  // G = X^T X
    if ((e = gemm64<true, 0, true>(g, false, st)) != cudaSuccess) return e;
    corr_k_kernel<<<64, 256, 0, st>>>(GKm, n, cw, ctl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    g = g64(GKm, n, GKm, n, K2m, n, n, ctl);  // K^2 (K's diagonal slots read as 0)
    if ((e = gemm64<false, 0, true, true>(g, false, st)) != cudaSuccess) return e;
    corr_bound_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(K2m, n, cw, ctl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    g = g64(K2m, n, K2m, n, K4m, n, n, ctl);  // K^4 (skipped when negligible)
    g.bnd = bnd;
    g.ran = cw + 1;
    if ((e = gemm64<false, 4, true, false, float>(g, false, st)) != cudaSuccess) return e;
    g = g64(K2m, n, K4m, n, Qm, n, n, ctl);  // Q from K, K^2, K^4 and K^6 = K^2 K^4
    g.Km = GKm;
    g.K2 = K2m;
    g.K4 = K4m;
    g.bnd = bnd;
    g.verdict = verdict;
    g.cnt = cw;
    if ((e = gemm64<false, 3, true, false, float>(g, false, st)) != cudaSuccess) return e;
    g = g64(Xi, n, Qm, n, Xo, n, n, ctl);  // X Q and V Q
    g.A[1] = Vi;
    g.C[1] = Vo;
    return gemm64<false, 0, false>(g, true, st);
}

bool jacobi32_applicable(int64_t n) { return n >= 64 && n <= kJ32N; }

cudaError_t launch_jacobi32_precondition(const DenseWork &w, int64_t n, unsigned int *ctl, cudaStream_t st) {
    // the phase is an optimisation: if the cluster cannot be placed, the FP64
    // iteration runs alone (ctl[0] stays 0, the products below are skipped)
    static int state[64] = {0};  // per device: 0 unknown, 1 usable, -1 not usable
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaSuccess;
    if (state[dev] < 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (state[dev] == 0) {
        if (cudaFuncSetAttribute(jacobi32_phase_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kJ32Smem) != cudaSuccess ||
            (kJ32Cta > 8 && cudaFuncSetAttribute(jacobi32_phase_kernel,
                                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
            cudaGetLastError();
            state[dev] = -1;
            return cudaSuccess;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kJ32Cta, 1, 1);
        cfg.blockDim = dim3(kJ32Threads, 1, 1);
        cfg.dynamicSmemBytes = kJ32Smem;
        cfg.stream = st;
        int maxc = 0;
        if (cudaOccupancyMaxActiveClusters(&maxc, (void *)jacobi32_phase_kernel, &cfg) != cudaSuccess || maxc < 1) {
            cudaGetLastError();
            state[dev] = -1;
            return cudaSuccess;
        }
        state[dev] = 1;
    }
    double *V0 = w.L, *Em = w.L + n * n, *Mm = w.U, *V0p = w.W, *X1 = w.U, *V1 = w.L;
    jacobi32_phase_kernel<<<kJ32Cta, kJ32Threads, kJ32Smem, st>>>(w.X, n, V0, ctl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // E = I - V0^T V0;  M = I + E/2 + (3/8) E^2 (both symmetric);  V0' = V0 M
    G64Args g = g64(V0, n, V0, n, Em, n, n, ctl);
    if ((e = gemm64<true, 1, true>(g, false, st)) != cudaSuccess) return e;
    g = g64(Em, n, Em, n, Mm, n, n, ctl);
    g.E = Em;
    if ((e = gemm64<false, 2, true, false, float>(g, false, st)) != cudaSuccess) return e;
    g = g64(V0, n, Mm, n, V0p, n, n, ctl);
    if ((e = gemm64<false, 0, false>(g, false, st)) != cudaSuccess) return e;
    // X1 = X0 V0' (into U), V1 = Q2 V0' (into L)
    g = g64(w.X, n, V0p, n, X1, n, n, ctl);
    g.A[1] = w.V;
    g.C[1] = V1;
    if ((e = gemm64<false, 0, false>(g, true, st)) != cudaSuccess) return e;
    // two first-order completions: (U, L) -> (X, V) -> (U, L); scratch G (then
    // K) and K^2 in R2, K^4 in the second half of L, Q in W
    double *GKm = w.R2, *K2m = w.R2 + n * n, *K4m = w.L + n * n, *Qm = w.W;
    unsigned int *cw0 = ctl + 4, *cw1 = ctl + 10, *verdict = ctl + 3;
    if ((e = completion(X1, V1, w.X, w.V, n, GKm, K2m, K4m, Qm, cw0, nullptr, ctl, st)) != cudaSuccess) return e;
    if ((e = completion(w.X, w.V, X1, V1, n, GKm, K2m, K4m, Qm, cw1, verdict, ctl, st)) != cudaSuccess) return e;
    // the FP64 iteration's convergence test, on G = X^T X of the final X when
    // the last completion expects convergence (tolerance n 2^-53, as there)
    g = g64(X1, n, X1, n, GKm, n, n, ctl);
    g.gate = verdict;
    if ((e = gemm64<true, 0, true>(g, false, st)) != cudaSuccess) return e;
    const double tol = (double)n * std::ldexp(1.0, -53);
    corr_check_kernel<<<64, 256, 0, st>>>(GKm, n, tol * tol, ctl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    copy_if_kernel<<<64, 256, 0, st>>>(X1, n * n, w.X, ctl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    copy_if_kernel<<<64, 256, 0, st>>>(V1, n * n, w.V, ctl);
    return cudaGetLastError();
}

}  // namespace ns
