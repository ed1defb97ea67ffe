// Global merge level of the keys merge sort (one level of Algorithm 1's
// "Merge" over the whole array), tiled form: 16-byte aligned buffers and
// n % 4 == 0.  This is the dominant kernel of the 2^28-key sort: one launch
// per level reads and writes every key once.
//
// One CTA per output tile of TO = NT*EO keys (the partition pass gives its
// merge-path split), many CTAs per SM for latency hiding.  The tile's A and B
// ranges are staged in shared memory by 16-byte asynchronous copies
// (cp.async) of their 16-byte-aligned covers; each thread then forms its EO
// outputs by a bitonic merge of its windows, the outputs are staged in shared
// memory (odd stride EO: conflict-free) and leave as 16-byte streaming stores.
#pragma once

#include "hs_internal.h"
#include "hs_merge_prims.cuh"

namespace hs {

// Window form: each thread merges the EO-key windows of A and B at its split
// (reads up to 2*EO keys for EO outputs).
template <int NT, int EO>
struct TileMerge {
    static constexpr int EOUT = EO;
    static constexpr int P = pow2_at_least(EO);
    static constexpr int TO = NT * EO;
    static constexpr int REG = TO + 8 + P;  // aligned cover + window slack
    static constexpr int SMEM_BYTES = 2 * REG * 4;
};

template <int NT, int EO>
__global__ void __launch_bounds__(NT)
    k_merge_tile(const int32_t *in, int32_t *out, int64_t n, int64_t w, const int64_t *part,
                 int tpg, int32_t *samp) {
    using C = TileMerge<NT, EO>;
    constexpr int TO = C::TO, P = C::P;
    extern __shared__ __align__(16) int32_t smem[];
    const int64_t g = blockIdx.x / tpg;
    const int t = blockIdx.x - (int)(g * tpg);
    const MergeGeom m = merge_geom(g, n, w);
    const int64_t glen = m.alen + m.blen;
    const int64_t o0 = (int64_t)t * TO;
    const int64_t o1 = (o0 + TO) < glen ? (o0 + TO) : glen;
    const int64_t a0 = part[blockIdx.x];
    const int64_t a1 = (o1 == glen) ? m.alen : part[blockIdx.x + 1];
    const int na = (int)(a1 - a0);
    const int tot = (int)(o1 - o0);
    const int nb = tot - na;
    // 16-byte aligned covers of [A + a0, + na) and [B + b0, + nb).
    const int64_t ga = m.gs + a0, gb = m.gs + w + (o0 - a0);
    const int64_t ca = ga & ~int64_t(3), cb = gb & ~int64_t(3);
    const int nca = (int)(((ga + na + 3) & ~int64_t(3)) - ca) / 4;
    const int ncb = (int)(((gb + nb + 3) & ~int64_t(3)) - cb) / 4;
    int32_t *sA = smem, *sB = smem + C::REG;
    for (int q = threadIdx.x; q < nca + ncb; q += NT) {
        if (q < nca) cp_async16(sA + 4 * q, in + ca + 4 * q);
        else cp_async16(sB + 4 * (q - nca), in + cb + 4 * (q - nca));
    }
    cp_async_wait_all();
    __syncthreads();
    const int32_t *A = sA + (int)(ga - ca), *B = sB + (int)(gb - cb);

    const int diag = threadIdx.x * EO;
    int32_t o[P];
    if (diag < tot) {
        int lo = diag > nb ? diag - nb : 0, hi = diag < na ? diag : na;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A[mid] <= B[diag - 1 - mid]) lo = mid + 1;
            else hi = mid;
        }
        const int32_t *wA = A + lo, *wB = B + (diag - lo);
        const int ra = na - lo, rb = nb - (diag - lo);
        if (ra >= EO && rb >= EO) {
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const int j = P - 1 - i;
                o[i] = hs_min(i < EO ? wA[i] : kKeyMax, j < EO ? wB[j] : kKeyMax);
            }
        } else {
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const int j = P - 1 - i;
                const int32_t x = (i < EO && i < ra) ? wA[i] : kKeyMax;
                const int32_t y = (j < EO && j < rb) ? wB[j] : kKeyMax;
                o[i] = hs_min(x, y);
            }
        }
        bitonic_half_clean<P>(o);
    }
    __syncthreads();
    if (diag < tot) {
#pragma unroll
        for (int k = 0; k < EO; ++k) sA[diag + k] = o[k];
    }
    __syncthreads();
    int32_t *dst = out + m.gs + o0;  // 16-byte aligned: gs and o0 are multiples of 4
    store_tile_out<NT>(dst, sA, tot, samp, m.gs + o0);
}

// Exact-window form (the default): each thread merges exactly its own EO
// keys; its end split comes from the next lane (a shuffle), or for a warp's
// last lane from the next warp's first lane through shared memory, so the
// windows read each key once.  A's and B's covers sit back to back in one
// region: na + nb = TO keys plus at most 3 extra keys at each end of each.
template <int NT, int EO>
struct TileMerge2 {
    static constexpr int EOUT = EO;
    static constexpr int P = pow2_at_least(EO);
    static constexpr int TO = NT * EO;
    // Covers (at most TO + 12 words) plus the P words of slack that the
    // window loads of exact_window_merge may touch past the last B key.
    static constexpr int REG = TO + 16 + P;
    static constexpr int SMEM_BYTES = REG * 4;
};

template <int NT, int EO>
__global__ void __launch_bounds__(NT)
    k_merge_tile2(const int32_t *in, int32_t *out, int64_t n, int64_t w, const int64_t *part,
                  int tpg, int32_t *samp) {
    using C = TileMerge2<NT, EO>;
    constexpr int TO = C::TO, P = C::P;
    extern __shared__ __align__(16) int32_t smem[];
    const int64_t g = blockIdx.x / tpg;
    const int t = blockIdx.x - (int)(g * tpg);
    const MergeGeom m = merge_geom(g, n, w);
    const int64_t glen = m.alen + m.blen;
    const int64_t o0 = (int64_t)t * TO;
    const int64_t o1 = (o0 + TO) < glen ? (o0 + TO) : glen;
    const int64_t a0 = part[blockIdx.x];
    const int64_t a1 = (o1 == glen) ? m.alen : part[blockIdx.x + 1];
    const int na = (int)(a1 - a0);
    const int tot = (int)(o1 - o0);
    const int nb = tot - na;
    const int64_t ga = m.gs + a0, gb = m.gs + w + (o0 - a0);
    const int64_t ca = ga & ~int64_t(3), cb = gb & ~int64_t(3);
    const int nca = (int)(((ga + na + 3) & ~int64_t(3)) - ca) / 4;
    const int ncb = (int)(((gb + nb + 3) & ~int64_t(3)) - cb) / 4;
    int32_t *sA = smem, *sB = smem + 4 * nca;  // B's cover right after A's
    for (int q = threadIdx.x; q < nca + ncb; q += NT) {
        if (q < nca) cp_async16(sA + 4 * q, in + ca + 4 * q);
        else cp_async16(sB + 4 * (q - nca), in + cb + 4 * (q - nca));
    }
    cp_async_wait_all();
    __syncthreads();
    const int32_t *A = sA + (int)(ga - ca), *B = sB + (int)(gb - cb);

    const int diag = threadIdx.x * EO;
    const int lane = threadIdx.x & 31;
    const int dcl = diag < tot ? diag : tot;
    int lo = dcl > nb ? dcl - nb : 0, hi = dcl < na ? dcl : na;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A[mid] <= B[dcl - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    __shared__ int wsplit[NT / 32 + 1];
    int end = __shfl_down_sync(0xffffffffu, lo, 1);
    if (lane == 0) wsplit[threadIdx.x >> 5] = lo;
    if (threadIdx.x == 0) wsplit[NT / 32] = na;
    __syncthreads();
    const int dend = (diag + EO) < tot ? (diag + EO) : tot;
    if (lane == 31) end = wsplit[(threadIdx.x >> 5) + 1];
    if (dend == tot) end = na;
    int32_t x[P];
    const int cnt = dend - dcl;
    if (cnt > 0) exact_window_merge<EO, P>(A, lo, B, dcl - lo, end - lo, cnt, x);
    __syncthreads();
    if (cnt > 0) {
#pragma unroll
        for (int k = 0; k < EO; ++k)
            if (k < cnt) sA[diag + k] = x[k];
    }
    __syncthreads();
    int32_t *dst = out + m.gs + o0;  // 16-byte aligned: gs and o0 are multiples of 4
    store_tile_out<NT>(dst, sA, tot, samp, m.gs + o0);
}

// Partition pass + one tiled merge launch for one level.  With samp (samples
// of kin at stride kSampleStride) the partition searches the samples first,
// and the merge writes the samples of kout for the next level.
template <auto KERN, class C>
static hs_status launch_tile(const int32_t *kin, int32_t *kout, int64_t n, int64_t w,
                             int64_t *part, int32_t *samp, cudaStream_t st) {
    static_assert(C::TO % kSampleStride == 0, "output tiles start on sample positions");
    const LevelTiles lt = level_tiles(n, w, C::TO);
    LaunchToken t = launch_begin(K_MERGE_PARTITION, st);
    const unsigned pgrid = (unsigned)((lt.nblocks + 255) / 256);
    if (samp)
        k_merge_partition_sampled<<<pgrid, 256, 0, st>>>(kin, samp, n, w, C::TO, (int)lt.tpg,
                                                          lt.nblocks, part);
    else
        k_merge_partition<<<pgrid, 256, 0, st>>>(kin, n, w, C::TO, (int)lt.tpg, lt.nblocks, part);
    hs_status r = launch_end(t);
    if (r != HS_OK) return r;
    if ((r = ensure_smem((const void *)KERN, C::SMEM_BYTES)) != HS_OK) return r;
    constexpr int NTH = C::TO / C::EOUT;
    t = launch_begin(K_MERGE_KEYS, st);
    KERN<<<(unsigned)lt.nblocks, NTH, C::SMEM_BYTES, st>>>(kin, kout, n, w, part, (int)lt.tpg, samp);
    return launch_end(t);
}

constexpr int kDefaultMergeTile = 5;

// One tiled keys level; `shape` is the option "merge_tile": 5 (the default,
// 96 threads x 31 keys, exact windows: small CTAs, many per SM, so loads,
// merges and stores of neighbouring CTAs overlap), 0 (window form, 256 x 15),
// and the exact-window variants 1 (64 x 31), 2 (128 x 31), 3 (64 x 63),
// 4 (128 x 23), 6 (192 x 31), 7 (256 x 31).
static hs_status launch_keys_tile_level(int shape, const int32_t *kin, int32_t *kout, int64_t n,
                                        int64_t w, int64_t *part, int32_t *samp, cudaStream_t st) {
    switch (shape) {
        case 0: return launch_tile<k_merge_tile<256, 15>, TileMerge<256, 15>>(kin, kout, n, w, part, samp, st);
        case 1: return launch_tile<k_merge_tile2<64, 31>, TileMerge2<64, 31>>(kin, kout, n, w, part, samp, st);
        case 2: return launch_tile<k_merge_tile2<128, 31>, TileMerge2<128, 31>>(kin, kout, n, w, part, samp, st);
        case 3: return launch_tile<k_merge_tile2<64, 63>, TileMerge2<64, 63>>(kin, kout, n, w, part, samp, st);
        case 4: return launch_tile<k_merge_tile2<128, 23>, TileMerge2<128, 23>>(kin, kout, n, w, part, samp, st);
        case 6: return launch_tile<k_merge_tile2<192, 31>, TileMerge2<192, 31>>(kin, kout, n, w, part, samp, st);
        case 7: return launch_tile<k_merge_tile2<256, 31>, TileMerge2<256, 31>>(kin, kout, n, w, part, samp, st);
        default: return launch_tile<k_merge_tile2<96, 31>, TileMerge2<96, 31>>(kin, kout, n, w, part, samp, st);
    }
}

}  // namespace hs
