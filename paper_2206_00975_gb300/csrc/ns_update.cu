// ns_update.cu -- keeping a sketch current under row changes of A (Section 5):
//   row append (Algorithm 2): S gains the column g / sqrt(s), g a standard
//     Gaussian vector independent of S, and SA += g a / sqrt(s).  For the SRHT
//     and sparse-sign kinds this is the rule Section 5 proposes for
//     non-Gaussian sketches;
//   row removal (Algorithm 3 and the non-Gaussian rule): SA -= (S e_j) A(j, :),
//     with S e_j regenerated from the seed in O(s): the SRHT column
//     d_j (-1)^popcount(r_t & j) / sqrt(s), the sparse-sign column (zeta
//     entries +-1/sqrt(zeta)), or the Gaussian column.
// The Gaussian column of an appended row with index j is column j of the
// Gaussian sketch with the same seed (Philox stream 3, block (r, j/8)), here
// evaluated in FP64, so appending row m to a Gaussian sketch of m rows gives
// the Gaussian sketch of the m + 1 rows.  Column changes need no kernel: a new
// column of A is sketched with ns_sketch (n = 1) and appended to SA; a removed
// column is dropped from SA.
#include <cmath>
#include "ns_device.cuh"
#include "ns_internal.h"

namespace ns {

// G(r, j) in FP64: word (j mod 8)/2 of stream-3 block (r, j/8) gives u_a
// (low half) and u_b (high half), each (w + 1/2) 2^-32; Box-Muller
// sqrt(-2 ln u_a) cos(2 pi u_b) for even j, sin for odd j.
__device__ __forceinline__ double gauss_entry64(uint64_t seed, int64_t r, int64_t j) {
    const u64x4 b = draw(seed, (uint64_t)r, (uint64_t)(j / 8), 3);
    const uint64_t w = b.w[(j % 8) / 2];
    const double ua = ((double)(uint32_t)w + 0.5) * 0x1p-32, ub = ((double)(uint32_t)(w >> 32) + 0.5) * 0x1p-32;
    const double rad = sqrt(-2.0 * log(ua));
    double sn, cs;
    sincospi(2.0 * ub, &sn, &cs);
    return (j % 2 == 0) ? rad * cs : rad * sn;
}

// Dense column (SRHT column j < m0, or a Gaussian column): thread r forms
// coefficient r and adds coef * row into row r of SA.
__global__ void update_dense_kernel(int gaussian, uint64_t seed, int64_t s, int lg, int64_t j, double scale,
                                    const double *__restrict__ row, int64_t n, double *__restrict__ SA) {
    extern __shared__ double rsh[];  // n
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) rsh[c] = row[c];
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= s) return;
    double coef;
    if (gaussian) {
        coef = gauss_entry64(seed, r, j);
    } else {
        // d_j: bit j % 64 of word (j % 256) / 64 of stream-0 block j / 256 (set: -1)
        const u64x4 sb = draw(seed, (uint64_t)(j >> 8), 0, 0);
        const int dneg = (int)((sb.w[(j & 255) >> 6] >> (j & 63)) & 1ull);
        const uint32_t rt = sample_perm(seed, lg, (uint32_t)r);
        coef = (((__popcll((unsigned long long)rt & (unsigned long long)j) & 1) ^ dneg) != 0) ? -1.0 : 1.0;
    }
    coef *= scale;
    for (int64_t c = 0; c < n; ++c) SA[r + c * s] = fma(coef, rsh[c], SA[r + c * s]);
}

// Sparse-sign column j: zeta rows, one thread per column of SA.
__global__ void update_sparse_kernel(uint64_t seed, int64_t s, int zeta, int64_t j, double scale,
                                     const double *__restrict__ row, int64_t n, double *__restrict__ SA) {
    __shared__ int32_t rr[64];
    __shared__ int8_t sg[64];
    if (threadIdx.x == 0) sparse_column(seed, s, zeta, j, rr, sg);
    __syncthreads();
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const double a = row[c];
        for (int i = 0; i < zeta; ++i) SA[rr[i] + c * s] = fma(sg[i] * scale, a, SA[rr[i] + c * s]);
    }
}

cudaError_t launch_sketch_update(int kind, uint64_t seed, int64_t s, int zeta, int64_t m0, int op, int64_t j,
                                 const double *row, int64_t n, double *SA, cudaStream_t st) {
    const double sign = (op == 0) ? 1.0 : -1.0;  // 0: append, 1: remove
    const bool gaussian_col = (op == 0) || (j >= m0) || (kind == NS_GAUSSIAN);
    if (!gaussian_col && kind == NS_SPARSE_SIGN) {
        update_sparse_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(seed, s, zeta, j,
                                                                          sign / std::sqrt((double)zeta), row, n, SA);
        return cudaGetLastError();
    }
    const size_t smem = sizeof(double) * (size_t)n;
    cudaError_t e = cudaFuncSetAttribute(update_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    update_dense_kernel<<<(unsigned)((s + 255) / 256), 256, smem, st>>>(
        gaussian_col ? 1 : 0, seed, s, ceil_log2(m0), j, sign / std::sqrt((double)s), row, n, SA);
    return cudaGetLastError();
}

}  // namespace ns
