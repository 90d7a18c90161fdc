// ns_sparse.cu -- sparse-sign sketch SA = S A: column j of S holds zeta entries
// +-1/sqrt(zeta) in distinct rows (a sparse sketch of the CountSketch kind that
// the paper names in Sections 1-2; zeta rows per column drawn by Floyd's
// algorithm from Philox stream 2, block (j, q) for q < ceil(zeta/4); row i
// draws t = floor(w_i (b+1) / 2^64) with b = s - zeta + i and keeps t unless
// already taken, else b; sign = low bit of w_i).
//
// Deterministic reduction without floating-point atomics:
//   1. for every 128-row tile of A the tile's (target row, row, sign) entries
//      are generated and bucketed by owner, bucket = (r / 1024) * 32 + r % 32
//      (counting sort; the order inside a bucket is irrelevant, see below);
//   2. a CTA of 16 warps owns 16 columns of A, one group of 1024 target rows
//      and a chunk of tiles.  It keeps the 1024 x 16 accumulator in shared
//      memory as 64-bit fixed point (per-column running exponent, as for the
//      SRHT), quantises each 128 x 16 tile of A into shared memory (each entry
//      with both signs, so the key indexes the signed value), and half
//      warp h of warp w (lane = column) applies the entries of owner 2w + h,
//      two per step: the two halves of a warp never touch the same target
//      row, and one half walks its entries in order, so no update races.
//      The next tile's A values, offsets and entries are loaded while this
//      tile is applied;
//   3. one FP64 partial per chunk is summed over chunks in a fixed order.
// Integer addition is exact and associative, so the result does not depend on
// the order of the updates.
#include <cmath>
#include "ns_device.cuh"
#include "ns_internal.h"

namespace ns {

constexpr int kSpTile = 128;      // rows of A per tile
constexpr int kSpCols = 16;       // columns of A per CTA (lane % 16 = column)
constexpr int kSpWarps = 16;      // owners 2w, 2w + 1 per warp
constexpr int kSpOwners = 2 * kSpWarps;
constexpr int kSpGroup = 1024;    // target rows per accumulator
constexpr int kSpThreads = kSpWarps * 32;
constexpr int kSpTileStride = 2 * kSpTile + 1;  // per column: +v, -v of each row, padded (conflict-free reads)
constexpr int kSpMaxEntPerThread = kSpTile * 64 / kSpThreads;  // zeta <= 64

SparseGeom sparse_geom(int64_t m, int64_t n, int64_t s, int zeta) {
    SparseGeom g;
    g.ntile = (m + kSpTile - 1) / kSpTile;
    g.nent = (int64_t)kSpTile * zeta;
    g.ntgrp = (s + kSpGroup - 1) / kSpGroup;
    g.nbucket = g.ntgrp * kSpOwners;
    g.ncolgrp = (n + kSpCols - 1) / kSpCols;
    // about two CTAs per SM over (column group, target group, chunk)
    const int64_t per = g.ncolgrp * g.ntgrp;
    int64_t want = (2 * (int64_t)device_sm_count() + per - 1) / per;
    if (want < 1) want = 1;
    if (want > g.ntile) want = g.ntile;
    g.chunk_tiles = (g.ntile + want - 1) / want;
    g.nchunk = (g.ntile + g.chunk_tiles - 1) / g.chunk_tiles;
    // |acc| <= rows per chunk * 2^P < 2^63; at most the 52 bits of the mantissa
    g.fx_bits = 62 - ceil_log2(g.chunk_tiles * kSpTile);
    if (g.fx_bits > 52) g.fx_bits = 52;
    return g;
}

SparseWork sparse_carve(Carver &c, int64_t m, int64_t n, int64_t s, int zeta) {
    SparseGeom g = sparse_geom(m, n, s, zeta);
    SparseWork w;
    w.entries = c.take<uint32_t>((size_t)(g.ntile * g.nent));
    w.offsets = c.take<int32_t>((size_t)(g.ntile * (g.nbucket + 1)));
    w.partial = c.take<double>((size_t)(g.nchunk * n * s));
    return w;
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

// one CTA per tile: generate the tile's entries, key (r << 8) | (j_local << 1)
// | sign, and bucket them by owner (counting sort); offsets[tile][b] is the
// first entry of bucket b, offsets[tile][nbucket] = nent
__global__ void __launch_bounds__(256) sparse_bucket_kernel(uint64_t seed, int64_t s, int zeta, int64_t m,
                                                            int64_t nent, int64_t nbucket, uint32_t *entries,
                                                            int32_t *offsets, int64_t j0) {
    extern __shared__ int32_t cnt[];  // nbucket + 1
    __shared__ uint32_t keys[kSpTile * 64];
    const int64_t tile = blockIdx.x;
    const int tid = threadIdx.x;
    for (int64_t b = tid; b <= nbucket; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    for (int jl = tid; jl < kSpTile; jl += blockDim.x) {
        const int64_t j = tile * kSpTile + jl;
        if (j >= m) continue;
        int32_t r[64];
        int8_t g[64];
        sparse_column(seed, s, zeta, j0 + j, r, g);  // column j0 + j of S (global row index)
        for (int i = 0; i < zeta; ++i) {
            const uint32_t key = ((uint32_t)r[i] << 8) | ((uint32_t)jl << 1) | (g[i] < 0 ? 1u : 0u);
            keys[jl * zeta + i] = key;
            atomicAdd(&cnt[(r[i] >> 10) * kSpOwners + (r[i] & (kSpOwners - 1))], 1);
        }
    }
    __syncthreads();
    if (tid == 0) {  // exclusive prefix sum (nbucket <= 512)
        int32_t run = 0;
        for (int64_t b = 0; b < nbucket; ++b) {
            const int32_t c = cnt[b];
            cnt[b] = run;
            run += c;
        }
        cnt[nbucket] = run;
    }
    __syncthreads();
    int32_t *off = offsets + tile * (nbucket + 1);
    for (int64_t b = tid; b <= nbucket; b += blockDim.x) off[b] = cnt[b];
    __syncthreads();
    uint32_t *ent = entries + tile * nent;
    const int64_t live = ((tile + 1) * kSpTile <= m ? kSpTile : m - tile * kSpTile) * zeta;
    for (int64_t e = tid; e < live; e += blockDim.x) {
        const uint32_t key = keys[e];
        const int r = (int)(key >> 8);
        const int pos = atomicAdd(&cnt[(r >> 10) * kSpOwners + (r & (kSpOwners - 1))], 1);
        ent[pos] = key;
    }
}

// grid (column group, target group, chunk); 16 warps; EPT >= entries per
// tile / threads (a tile holds kSpTile * zeta entries)
template <int EPT>
__global__ void __launch_bounds__(kSpThreads, 1) sparse_acc_kernel(
    const double *__restrict__ A, int64_t m, int64_t n, int64_t lda, int64_t s, int64_t nent, int64_t nbucket,
    int64_t chunk_tiles, int64_t ntile, int P, const uint32_t *__restrict__ entries,
    const int32_t *__restrict__ offsets, double *__restrict__ partial, int32_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    long long *acc = (long long *)smem_raw;                        // kSpGroup x kSpCols
    long long *tq = acc + kSpGroup * kSpCols;                      // kSpCols x kSpTileStride (signed pairs)
    uint32_t *ents = (uint32_t *)(tq + kSpCols * kSpTileStride);   // this tile's entries of the target group
    __shared__ int32_t boff[kSpOwners + 1];
    __shared__ int Ecol[kSpCols];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t cg = blockIdx.x, tg = blockIdx.y, ch = blockIdx.z;
    const int c = lane & (kSpCols - 1), h = lane >> 4;  // column of this lane, owner half
    const int64_t col = cg * kSpCols + c;
    const int64_t lcol = cg * kSpCols + w;               // column this warp loads
    for (int i = tid; i < kSpGroup * kSpCols; i += kSpThreads) acc[i] = 0;
    if (tid < kSpCols) Ecol[tid] = 0;
    int nonfinite = 0;
    const int64_t t0 = ch * chunk_tiles, t1 = (t0 + chunk_tiles < ntile) ? t0 + chunk_tiles : ntile;
    __syncthreads();
    // Software pipeline: tile t + 1's values of A, bucket offsets and entries
    // are loaded while tile t is applied.
    long long raw[4];
    uint32_t pre[EPT];
    int32_t e0 = 0, e1 = 0, myoff = 0;
    auto load_tile = [&](int64_t t, long long (&rv)[4], uint32_t (&pv)[EPT], int32_t &f0, int32_t &f1,
                         int32_t &fo) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t j = t * kSpTile + lane + 32 * q;
            rv[q] = (lcol < n && j < m) ? __double_as_longlong(__ldcs(A + j + lcol * lda)) : 0;
        }
        const int32_t *off = offsets + t * (nbucket + 1) + tg * kSpOwners;
        f0 = __ldg(off);
        f1 = __ldg(off + kSpOwners);
        fo = (tid <= kSpOwners) ? __ldg(off + tid) : 0;
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int32_t e = f0 + tid + q * kSpThreads;
            pv[q] = (e < f1) ? __ldg(entries + t * nent + e) : 0u;
        }
    };
    if (t0 < t1) load_tile(t0, raw, pre, e0, e1, myoff);
    for (int64_t t = t0; t < t1; ++t) {
        int emax = 1;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = (int)((unsigned long long)raw[q] >> 52) & 0x7FF;
            emax = (e == 0x7FF) ? emax : max(emax, e);
            nonfinite |= (e == 0x7FF);
        }
        emax = warp_max(emax);
        __syncthreads();  // the previous tile is fully applied
        if (tid <= kSpOwners) boff[tid] = myoff;
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int32_t e = e0 + tid + q * kSpThreads;
            if (e < e1) ents[e - e0] = pre[q];
        }
        // ---- running exponent of the warp's column; rescale its accumulator
        const int Eold = Ecol[w];
        const int E = max(Eold, emax);
        if (E > Eold && Eold > 0) {
            const int d = E - Eold;
            for (int r = lane; r < kSpGroup; r += 32) {
                long long &a = acc[r * kSpCols + w];
                a = (d >= 63) ? (a >> 63) : (a >> d);
            }
        }
        // quantise at 2^(E - 1022 - P), magnitude rounded to nearest
        const int sh1b = E + 52 - P;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const unsigned long long b = (unsigned long long)raw[q];
            const uint32_t hi = (uint32_t)(b >> 32);
            const int e = (int)((hi >> 20) & 0x7FF), e1b = max(e, 1);
            const uint32_t sh1 = (uint32_t)(sh1b - e1b);
            const unsigned long long mant = (b & 0x000FFFFFFFFFFFFFull) | ((unsigned long long)(1 - (e1b - e)) << 52);
            unsigned long long q1;
            asm("shr.b64 %0, %1, %2;" : "=l"(q1) : "l"(mant), "r"(sh1));
            unsigned long long qv = (q1 + 1ull) >> 1;
            if (e == 0x7FF) qv = 0ull;
            const long long msk = (long long)(int)(hi & 0x80000000u) >> 31;
            const long long zq = ((long long)qv ^ msk) - msk;
            long long *dst = tq + w * kSpTileStride + 2 * (lane + 32 * q);
            dst[0] = zq;
            dst[1] = -zq;
        }
        if (lane == 0) Ecol[w] = E;
        __syncthreads();  // tile, entries, offsets and exponents in place
        if (t + 1 < t1) load_tile(t + 1, raw, pre, e0, e1, myoff);  // lands while this tile is applied
        // ---- half warp h of warp w applies the entries of owner 2w + h
        const int o = 2 * w + h;
        const int32_t b0 = boff[o] - boff[0], cntme = boff[o + 1] - boff[o];
        const int cnt_other = __shfl_xor_sync(0xffffffffu, cntme, 16);
        const int steps = max(cntme, cnt_other);
        const long long *tqc = tq + c * kSpTileStride;  // +v at 2 jl, -v at 2 jl + 1
        long long *accc = acc + c;
        // two entries per step: both accumulators are read before either is
        // written (their updates overlap), and two entries for the same target
        // row are summed first; an inactive slot writes nothing
        for (int i = 0; i < steps; i += 2) {
            const bool a0 = i < cntme, a1 = i + 1 < cntme;
            const uint32_t k0 = a0 ? ents[b0 + i] : 0u, k1 = a1 ? ents[b0 + i + 1] : 0u;
            const int r0 = (int)((k0 >> 8) & (kSpGroup - 1)) * kSpCols, r1 = (int)((k1 >> 8) & (kSpGroup - 1)) * kSpCols;
            const long long v0 = tqc[k0 & (2 * kSpTile - 1)], v1 = tqc[k1 & (2 * kSpTile - 1)];
            if (a1) {
                if (r0 == r1) {
                    accc[r0] += v0 + v1;
                } else {
                    const long long x0 = accc[r0], x1 = accc[r1];
                    accc[r0] = x0 + v0;
                    accc[r1] = x1 + v1;
                }
            } else if (a0) {
                accc[r0] += v0;
            }
        }
    }
    __syncthreads();
    // chunk partial in FP64: value = acc * 2^(E - 1022 - P)
    if (col < n) {
        const int E = Ecol[c];
        const double scale = E > 0 ? ldexp(1.0, E - 1022 - P) : 0.0;
        double *out = partial + (ch * n + col) * s;
        for (int r = w * 2 + h; r < kSpGroup; r += 2 * kSpWarps) {
            const int64_t rg = tg * kSpGroup + r;
            if (rg < s) out[rg] = (double)acc[r * kSpCols + c] * scale;
        }
    }
    if (nonfinite) set_status(status, NS_ERR_NONFINITE);
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
                              const SparseWork &w, double *SA, int32_t *status, cudaStream_t st, int64_t j0) {
    const SparseGeom g = sparse_geom(m, n, s, zeta);
    const size_t bsmem = sizeof(int32_t) * (size_t)(g.nbucket + 1);
    sparse_bucket_kernel<<<(unsigned)g.ntile, 256, bsmem, st>>>(seed, s, zeta, m, g.nent, g.nbucket, w.entries,
                                                                w.offsets, j0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(long long) * (size_t)(kSpGroup * kSpCols + kSpCols * kSpTileStride) +
                        sizeof(uint32_t) * (size_t)g.nent;
    const int64_t need = (g.nent + kSpThreads - 1) / kSpThreads;  // entries per thread, at most
    const int ept = need <= 1 ? 1 : need <= 2 ? 2 : need <= 4 ? 4 : need <= 8 ? 8 : kSpMaxEntPerThread;
    auto kern = ept == 1 ? sparse_acc_kernel<1>
                : ept == 2 ? sparse_acc_kernel<2>
                : ept == 4 ? sparse_acc_kernel<4>
                : ept == 8 ? sparse_acc_kernel<8>
                           : sparse_acc_kernel<kSpMaxEntPerThread>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)g.ncolgrp, (unsigned)g.ntgrp, (unsigned)g.nchunk);
    kern<<<grid, kSpThreads, smem, st>>>(A, m, n, lda, s, g.nent, g.nbucket, g.chunk_tiles, g.ntile, g.fx_bits,
                                         w.entries, w.offsets, w.partial, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    chunk_reduce_kernel<<<(unsigned)((n * s + 255) / 256), 256, 0, st>>>(w.partial, n, s, g.nchunk,
                                                                          1.0 / std::sqrt((double)zeta), SA);
    return cudaGetLastError();
}

}  // namespace ns
