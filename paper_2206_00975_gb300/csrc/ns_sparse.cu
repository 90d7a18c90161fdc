// ns_sparse.cu -- sparse-sign sketch SA = S A: column j of S holds zeta entries
// +-1/sqrt(zeta) in distinct rows (a sparse sketch of the CountSketch kind that
// the paper names in Sections 1-2; zeta rows per column drawn by Floyd's
// algorithm from Philox stream 2, block (j, q) for q < ceil(zeta/4); row i
// draws t = floor(w_i (b+1) / 2^64) with b = s - zeta + i and keeps t unless
// already taken, else b; sign = low bit of w_i).
//
// Deterministic bucketed reduction without floating-point atomics:
//   1. for every 128-row tile of A the (row, sign) pairs of its 128 columns of S
//      are generated and sorted by output row (one CTA per tile, bitonic sort of
//      keys r*256 + j_local*2 + sign); offsets per 16-row group are kept;
//   2. a CTA of 16 warps owns 256 output rows x 32 columns of A for a chunk of
//      tiles: it maps each 128 x 32 tile of A exactly onto 64-bit fixed point in
//      shared memory (per-column running exponent, as for the SRHT), and each
//      warp adds the tile's entries of its 16 rows into integer accumulators in
//      registers (lane = column), walking the sorted entries;
//   3. one FP64 partial per chunk is summed over chunks in a fixed order.
// Integer addition is exact and associative, so the result does not depend on
// the order of the updates.
#include <cmath>
#include "ns_device.cuh"
#include "ns_internal.h"

namespace ns {

constexpr int kSpTile = 128;         // rows of A per tile
constexpr int kSpRowsPerWarp = 16;
constexpr int kSpWarps = 16;
constexpr int kSpRowGroup = kSpRowsPerWarp * kSpWarps;  // 256 output rows per CTA
constexpr int kSpCols = 32;          // columns of A per CTA (lane = column)

SparseGeom sparse_geom(int64_t m, int64_t n, int64_t s, int zeta) {
    SparseGeom g;
    g.ntile = (m + kSpTile - 1) / kSpTile;
    g.nent = (int64_t)kSpTile * zeta;
    g.nsort = 1;
    while (g.nsort < g.nent) g.nsort <<= 1;
    g.ngrp16 = (s + kSpRowsPerWarp - 1) / kSpRowsPerWarp;
    g.nrowgrp = (s + kSpRowGroup - 1) / kSpRowGroup;
    g.ncolgrp = (n + kSpCols - 1) / kSpCols;
    // about 1024 CTAs; chunks of whole tiles
    int64_t per = g.nrowgrp * g.ncolgrp;
    int64_t want_chunks = 1024 / (per > 0 ? per : 1);
    if (want_chunks < 1) want_chunks = 1;
    g.chunk_tiles = (g.ntile + want_chunks - 1) / want_chunks;
    if (g.chunk_tiles < 8) g.chunk_tiles = g.ntile < 8 ? g.ntile : 8;
    g.nchunk = (g.ntile + g.chunk_tiles - 1) / g.chunk_tiles;
    // |acc| <= rows per chunk * 2^P < 2^63
    g.fx_bits = 62 - ceil_log2(g.chunk_tiles * kSpTile);
    return g;
}

SparseWork sparse_carve(Carver &c, int64_t m, int64_t n, int64_t s, int zeta) {
    SparseGeom g = sparse_geom(m, n, s, zeta);
    SparseWork w;
    w.entries = c.take<uint32_t>((size_t)(g.ntile * g.nent));
    w.offsets = c.take<int32_t>((size_t)(g.ntile * (g.ngrp16 + 1)));
    w.partial = c.take<double>((size_t)(g.nchunk * n * s));
    return w;
}

// Floyd's sampling of zeta distinct rows of [0, s) for column j of S.
__device__ __forceinline__ void sparse_column(uint64_t seed, int64_t s, int zeta, int64_t j, int32_t *rows,
                                              int8_t *signs) {
    uint64_t w[64];
    for (int q = 0; q < (zeta + 3) / 4; ++q) {
        const u64x4 b = draw(seed, (uint64_t)j, (uint64_t)q, 2);
        w[4 * q + 0] = b.w[0];
        w[4 * q + 1] = b.w[1];
        w[4 * q + 2] = b.w[2];
        w[4 * q + 3] = b.w[3];
    }
    for (int i = 0; i < zeta; ++i) {
        const int64_t bound = s - zeta + i;
        int64_t t = (int64_t)__umul64hi(w[i], (uint64_t)(bound + 1));
        for (int u = 0; u < i; ++u)
            if (rows[u] == t) {
                t = bound;
                break;
            }
        rows[i] = (int32_t)t;
        signs[i] = (w[i] & 1ull) ? -1 : 1;
    }
}

__global__ void sparse_meta_kernel(uint64_t seed, int64_t s, int zeta, int64_t m, int32_t *rows, int8_t *signs) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    int32_t r[64];
    int8_t g[64];
    sparse_column(seed, s, zeta, j, r, g);
    for (int i = 0; i < zeta; ++i) {
        rows[j * zeta + i] = r[i];
        signs[j * zeta + i] = g[i];
    }
}

// one CTA per tile: generate, sort by (row, j_local), store entries and the
// offsets of every 16-row group
__global__ void __launch_bounds__(256) sparse_tile_sort_kernel(uint64_t seed, int64_t s, int zeta, int64_t m,
                                                               int64_t nent, int64_t nsort, int64_t ngrp16,
                                                               uint32_t *entries, int32_t *offsets) {
    extern __shared__ uint32_t keys[];  // nsort
    const int64_t tile = blockIdx.x;
    const int tid = threadIdx.x;
    for (int64_t i = tid; i < nsort; i += blockDim.x) keys[i] = 0xFFFFFFFFu;
    __syncthreads();
    for (int jl = tid; jl < kSpTile; jl += blockDim.x) {
        const int64_t j = tile * kSpTile + jl;
        if (j >= m) continue;
        int32_t r[64];
        int8_t g[64];
        sparse_column(seed, s, zeta, j, r, g);
        for (int i = 0; i < zeta; ++i)
            keys[jl * zeta + i] = ((uint32_t)r[i] << 8) | ((uint32_t)jl << 1) | (g[i] < 0 ? 1u : 0u);
    }
    __syncthreads();
    // bitonic sort of nsort keys (padding keys sort last)
    for (int64_t k = 2; k <= nsort; k <<= 1) {
        for (int64_t jj = k >> 1; jj > 0; jj >>= 1) {
            for (int64_t i = tid; i < nsort; i += blockDim.x) {
                const int64_t l = i ^ jj;
                if (l > i) {
                    const uint32_t a = keys[i], b = keys[l];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int64_t i = tid; i < nent; i += blockDim.x) entries[tile * nent + i] = keys[i];
    // offsets: first entry whose row >= 16 g, for g = 0..ngrp16 (binary search)
    for (int64_t gI = tid; gI <= ngrp16; gI += blockDim.x) {
        const uint32_t lim = (uint32_t)(gI * kSpRowsPerWarp) << 8;
        int64_t lo = 0, hi = nent;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (keys[mid] < lim) lo = mid + 1;
            else hi = mid;
        }
        offsets[tile * (ngrp16 + 1) + gI] = (int32_t)lo;
    }
}

__global__ void __launch_bounds__(kSpWarps * 32, 2) sparse_f64_kernel(
    const double *__restrict__ A, int64_t m, int64_t n, int64_t lda, int64_t s, int64_t nent, int64_t ngrp16,
    int64_t chunk_tiles, int64_t ntile, int P, const uint32_t *__restrict__ entries,
    const int32_t *__restrict__ offsets, double *__restrict__ partial, int32_t *status) {
    __shared__ long long tq[kSpTile][kSpCols + 1];  // quantised tile, [row][column]
    __shared__ int Ecol[kSpCols], Enew[kSpCols];
    __shared__ int nonfinite;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t rg = blockIdx.x, cg = blockIdx.y, ch = blockIdx.z;
    const int64_t col = cg * kSpCols + lane;
    const int64_t row0 = rg * kSpRowGroup + (int64_t)wid * kSpRowsPerWarp;  // this warp's first output row
    const int64_t g16 = row0 / kSpRowsPerWarp;
    if (tid < kSpCols) Ecol[tid] = 0;
    if (tid == 0) nonfinite = 0;
    long long acc[kSpRowsPerWarp];
#pragma unroll
    for (int r = 0; r < kSpRowsPerWarp; ++r) acc[r] = 0;
    int Emine = 0;  // running exponent of this lane's column (mirrors Ecol[lane])
    const int64_t t0 = ch * chunk_tiles, t1 = (t0 + chunk_tiles < ntile) ? t0 + chunk_tiles : ntile;
    for (int64_t t = t0; t < t1; ++t) {
        __syncthreads();
        // ---- load the tile (raw bits), 128 rows x 32 columns; column c handled by
        // 16 threads, 8 rows each (coalesced along rows)
        const int c = tid >> 4, part = tid & 15;
        const int64_t gc = cg * kSpCols + c;
        long long raw[8];
        int emax = 1;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int jl = part + 16 * q;
            const int64_t j = t * kSpTile + jl;
            long long v = 0;
            if (gc < n && j < m) v = __double_as_longlong(__ldcs(A + j + gc * lda));
            raw[q] = v;
            const int e = (int)((unsigned long long)v >> 52) & 0x7FF;
            if (e == 0x7FF) nonfinite = 1;
            else emax = max(emax, e);
        }
        // column max exponent over its 16 threads (a half warp)
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        if (part == 0) Enew[c] = max(Ecol[c], emax);
        __syncthreads();
        const int E = Enew[c];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int jl = part + 16 * q;
            const unsigned long long b = (unsigned long long)raw[q];
            const int e = (int)(b >> 52) & 0x7FF;
            const unsigned long long frac = b & 0x000FFFFFFFFFFFFFull;
            const unsigned long long mant = e ? (frac | 0x0010000000000000ull) : frac;
            const int sh = E - (e ? e : 1) + 53 - P;
            unsigned long long q64 = (sh >= 64 || e == 0x7FF) ? 0ull
                                     : (sh <= 0 ? (mant << (-sh)) : ((mant + (1ull << (sh - 1))) >> sh));
            tq[jl][c] = (b >> 63) ? -(long long)q64 : (long long)q64;
        }
        __syncthreads();
        // ---- rescale this lane's accumulators if its column's exponent grew
        const int En = Enew[lane];
        if (En > Emine) {
            if (Emine > 0) {
                const int d = En - Emine;
#pragma unroll
                for (int r = 0; r < kSpRowsPerWarp; ++r) acc[r] = (d >= 63) ? (acc[r] >> 63) : (acc[r] >> d);
            }
            Emine = En;
        }
        if (tid < kSpCols) Ecol[tid] = Enew[tid];
        // ---- this warp's entries: rows row0 .. row0+15, sorted by row
        if (row0 < s) {
            const uint32_t *ent = entries + t * nent;
            int64_t e = offsets[t * (ngrp16 + 1) + g16];
            const int64_t e_end = offsets[t * (ngrp16 + 1) + g16 + 1];
#pragma unroll
            for (int r = 0; r < kSpRowsPerWarp; ++r) {
                const uint32_t rk = (uint32_t)(row0 + r);
                while (e < e_end) {
                    const uint32_t k = __ldg(ent + e);
                    if ((k >> 8) != rk) break;
                    const long long v = tq[(k >> 1) & 127][lane];
                    acc[r] += (k & 1u) ? -v : v;
                    ++e;
                }
            }
        }
    }
    // chunk partial in FP64: value = acc * 2^(E - 1022 - P)
    if (col < n && Emine > 0) {
        const double scale = ldexp(1.0, Emine - 1022 - P);
        double *out = partial + (ch * n + col) * s;
#pragma unroll
        for (int r = 0; r < kSpRowsPerWarp; ++r)
            if (row0 + r < s) out[row0 + r] = (double)acc[r] * scale;
    } else if (col < n) {
        double *out = partial + (ch * n + col) * s;
        for (int r = 0; r < kSpRowsPerWarp; ++r)
            if (row0 + r < s) out[row0 + r] = 0.0;
    }
    __syncthreads();
    if (tid == 0 && nonfinite) set_status(status, NS_ERR_NONFINITE);
}

__global__ void chunk_reduce_kernel(const double *__restrict__ partial, int64_t n, int64_t s, int64_t nchunk,
                                    double scale, double *__restrict__ SA) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * s) return;
    const int64_t c = idx / s, t = idx - c * s;
    double a = 0.0;
    for (int64_t ch = 0; ch < nchunk; ++ch) a += partial[(ch * n + c) * s + t];
    SA[t + c * s] = a * scale;
}

cudaError_t launch_sparse_meta(uint64_t seed, int64_t s, int zeta, int64_t m, int32_t *rows, int8_t *signs,
                               cudaStream_t st) {
    sparse_meta_kernel<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(seed, s, zeta, m, rows, signs);
    return cudaGetLastError();
}

cudaError_t launch_sparse_f64(uint64_t seed, const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, int zeta,
                              const SparseWork &w, double *SA, int32_t *status, cudaStream_t st) {
    const SparseGeom g = sparse_geom(m, n, s, zeta);
    const size_t sort_smem = sizeof(uint32_t) * (size_t)g.nsort;
    cudaError_t e =
        cudaFuncSetAttribute(sparse_tile_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem);
    if (e != cudaSuccess) return e;
    sparse_tile_sort_kernel<<<(unsigned)g.ntile, 256, sort_smem, st>>>(seed, s, zeta, m, g.nent, g.nsort, g.ngrp16,
                                                                        w.entries, w.offsets);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 grid((unsigned)g.nrowgrp, (unsigned)g.ncolgrp, (unsigned)g.nchunk);
    sparse_f64_kernel<<<grid, kSpWarps * 32, 0, st>>>(A, m, n, lda, s, g.nent, g.ngrp16, g.chunk_tiles, g.ntile,
                                                      g.fx_bits, w.entries, w.offsets, w.partial, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    chunk_reduce_kernel<<<(unsigned)((n * s + 255) / 256), 256, 0, st>>>(w.partial, n, s, g.nchunk,
                                                                          1.0 / std::sqrt((double)zeta), SA);
    return cudaGetLastError();
}

}  // namespace ns
