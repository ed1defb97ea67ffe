// Binary global merge level of the keys merge sort (one level of Algorithm
// 1's "Merge" over the whole array), tiled form: 16-byte aligned buffers and
// n % 4 == 0.  One launch per level reads and writes every key once.
//
// One CTA per output tile of TO = NT*EO keys (the partition pass gives its
// merge-path split), many CTAs per SM for latency hiding.  The tile's A and B
// ranges arrive in shared memory as their 16-byte-aligned covers by bulk
// copies; each thread forms its EO outputs by a bitonic merge of its exact
// windows, the outputs are staged in shared memory (odd stride EO:
// conflict-free) and leave as one bulk store.
#pragma once

#include "hs_bulk.cuh"
#include "hs_internal.h"
#include "hs_merge_prims.cuh"

namespace hs {

// Exact windows: each thread merges exactly its own EO keys; its end split
// comes from the next lane (a shuffle), or for a warp's last lane from the
// next warp's first lane through shared memory, so the windows read each key
// once.  A's and B's covers sit back to back in one region: na + nb = TO keys
// plus at most 3 extra keys at each end of each.
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

// One thread issues the two cover copies (cp.async.bulk, completion counted
// on an mbarrier) and, once the tile is merged, one bulk store of the whole
// output tile; each thread writes the samples that fall among its own
// outputs straight from registers.  The load/store units then carry only the
// merge's own shared-memory traffic.
//
// SELF_SPLIT: the CTA finds its own two merge-path splits (warps 0 and 1,
// one boundary each, by 32-ary searches of about four dependent load rounds)
// instead of reading them from a partition pass.  Used when a level's tiles
// fit one wave of CTAs: the partition launch and its dependency then cost
// more than the duplicated searches (part is unused).
template <int NT, int EO, bool SELF_SPLIT = false>
__global__ void __launch_bounds__(NT)
    k_merge_tile_bulk(const int32_t *in, int32_t *out, int64_t n, int64_t w, const int64_t *part,
                      int tpg, int32_t *samp, unsigned *status, int64_t block0) {
    using C = TileMerge2<NT, EO>;
    constexpr int TO = C::TO, P = C::P;
    static_assert(kSampleStride == 32, "sample positions are multiples of 32");
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int wsplit[NT / 32 + 1];
    const int64_t b = block0 + blockIdx.x;  // output tile (a launch may cover a range of them)
    const int64_t g = b / tpg;
    const int t = (int)(b - g * tpg);
    const MergeGeom m = merge_geom(g, n, w);
    const int64_t glen = m.alen + m.blen;
    const int64_t o0 = (int64_t)t * TO;
    const int64_t o1 = (o0 + TO) < glen ? (o0 + TO) : glen;
    int64_t a0, a1;
    if constexpr (SELF_SPLIT) {
        static_assert(NT >= 64, "two warps search the tile's two splits");
        tile_self_split(in, m.gs, w, m.alen, m.blen, o0, o1, &a0, &a1);
    } else {
        a0 = part[b];
        a1 = (o1 == glen) ? m.alen : part[b + 1];
    }
    const int na = (int)(a1 - a0);
    const int tot = (int)(o1 - o0);
    const int nb = tot - na;
    const int64_t ga = m.gs + a0, gb = m.gs + w + (o0 - a0);
    const int64_t ca = ga & ~int64_t(3), cb = gb & ~int64_t(3);
    const int nca = (int)(((ga + na + 3) & ~int64_t(3)) - ca) / 4;
    const int ncb = (int)(((gb + nb + 3) & ~int64_t(3)) - cb) / 4;
    int32_t *sA = smem, *sB = smem + 4 * nca;
    const uint64_t pol = l2_evict_first_policy();
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    // Bulk copies need 16-byte aligned ends: the covers are whole 16-byte
    // words of 16-byte aligned arrays, and this re-checks it before issuing.
    const bool aligned16 = ((smem_addr(sA) | smem_addr(sB)) & 15u) == 0 &&
                           ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
    if (threadIdx.x == 0 && aligned16) {
        mbar_arrive_expect_tx(&bar, (unsigned)(nca + ncb) * 16u);
        if (nca > 0) bulk_load(sA, in + ca, (unsigned)nca * 16u, &bar, pol);
        if (ncb > 0) bulk_load(sB, in + cb, (unsigned)ncb * 16u, &bar, pol);
    }
    if (!aligned16) {  // uniform across the CTA: nothing was issued
        if (threadIdx.x == 0) atomicOr(status, kStatusMisaligned);
        return;
    }
    const bool ok = mbar_wait(&bar, 0);
    if (__syncthreads_or(!ok)) {  // a copy never landed: report, drain, leave
        if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
        if (!ok) mbar_wait(&bar, 0);
        return;
    }
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
        fence_proxy_async_smem();
        if (samp) {
            // Output positions m.gs + o0 + diag + k; m.gs + o0 is a multiple of 32.
#pragma unroll
            for (int j = 0; j < (EO + 31) / 32; ++j) {
                const int k = ((-diag) & 31) + 32 * j;
                if (k < cnt) samp[(m.gs + o0 + diag + k) / kSampleStride] = select_dyn(x, k);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // 16-byte aligned: m.gs + o0 and tot are multiples of 4 keys.
        bulk_store(out + m.gs + o0, sA, (unsigned)tot * 4u, pol);
        bulk_wait_read();
    }
}



// Partition pass of one tiled level: part[b] = A keys before output tile b.
// With samp (samples of kin at stride kSampleStride) it searches the samples
// first.
static hs_status launch_partition(const int32_t *kin, int64_t n, int64_t w, int to,
                                  const LevelTiles &lt, int64_t *part, const int32_t *samp,
                                  cudaStream_t st) {
    LaunchToken t = launch_begin(K_MERGE_PARTITION, st);
    const unsigned pgrid = (unsigned)((lt.nblocks + 255) / 256);
    if (samp)
        k_merge_partition_sampled<<<pgrid, 256, 0, st>>>(kin, samp, n, w, to, (int)lt.tpg,
                                                          lt.nblocks, part);
    else
        k_merge_partition<<<pgrid, 256, 0, st>>>(kin, n, w, to, (int)lt.tpg, lt.nblocks, part);
    return launch_end(t);
}

// Partition pass + one tiled merge launch for one level (the merge also
// writes the samples of kout for the next level when samp is given, and
// takes the device status word for its bounded copy wait).
template <int NT, int EO>
static hs_status launch_tile_bulk(const int32_t *kin, int32_t *kout, int64_t n, int64_t w,
                                  int64_t *part, int32_t *samp, cudaStream_t st) {
    using C = TileMerge2<NT, EO>;
    static_assert(C::TO % kSampleStride == 0, "output tiles start on sample positions");
    unsigned *status = nullptr;
    hs_status r = device_status(&status);
    if (r != HS_OK) return r;
    const LevelTiles lt = level_tiles(n, w, C::TO);
    if (lt.nblocks <= kSelfSplitMaxTiles) {
        auto kern = k_merge_tile_bulk<NT, EO, true>;
        if ((r = ensure_smem((const void *)kern, C::SMEM_BYTES)) != HS_OK) return r;
        LaunchToken t = launch_begin(K_MERGE_KEYS, st);
        kern<<<(unsigned)lt.nblocks, NT, C::SMEM_BYTES, st>>>(kin, kout, n, w, nullptr, (int)lt.tpg,
                                                              samp, status, int64_t(0));
        return launch_end(t);
    }
    if ((r = launch_partition(kin, n, w, C::TO, lt, part, samp, st)) != HS_OK) return r;
    auto kern = k_merge_tile_bulk<NT, EO>;
    if ((r = ensure_smem((const void *)kern, C::SMEM_BYTES)) != HS_OK) return r;
    LaunchToken t = launch_begin(K_MERGE_KEYS, st);
    kern<<<(unsigned)lt.nblocks, NT, C::SMEM_BYTES, st>>>(kin, kout, n, w, part, (int)lt.tpg, samp,
                                                          status, int64_t(0));
    return launch_end(t);
}

// One tiled keys level: 128 threads x 31 keys per tile (3968 keys), moved in
// and out by the copy engine; small CTAs keep many tiles in flight per SM.
static hs_status launch_keys_tile_level(const int32_t *kin, int32_t *kout, int64_t n, int64_t w,
                                        int64_t *part, int32_t *samp, cudaStream_t st) {
    return launch_tile_bulk<128, 31>(kin, kout, n, w, part, samp, st);
}

}  // namespace hs
