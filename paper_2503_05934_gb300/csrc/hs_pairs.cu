// Stable key/value merge sort (Algorithm 1 on (key, value) pairs): block sort
// on (key, position) words, then global merge levels that keep equal keys in
// input order.  Keys and values live in separate int32 arrays; each level
// reads and writes both once.
#include <algorithm>

#include "hs_bulk.cuh"
#include "hs_internal.h"
#include "hs_blocksort.cuh"
#include "hs_merge4.cuh"

namespace hs {

// ---------------------------------------------------------------------------
// Tiled pairs level (16-byte aligned key and value buffers, n % 4 == 0).  One
// CTA per output tile of TO = NT*EO pairs: one thread issues the four cover
// copies (keys and values of A and B, cp.async.bulk, completion counted on an
// mbarrier); each thread finds its merge-path split, takes its end split from
// the next lane, and merges exactly its own outputs serially (stable: A's
// element on ties), picking each value by the same decision; once the tile
// is merged, one bulk store each of the output keys and values leaves, and
// each thread writes the samples among its own outputs from registers.
template <int NT, int EO>
struct TileMergePairs {
    static constexpr int EOUT = EO;
    static constexpr int TO = NT * EO;
    static constexpr int REG = TO + 16;  // A and B covers back to back
    static constexpr int SMEM_BYTES = 2 * REG * 4;  // keys, values
};

// SELF_SPLIT: the CTA searches its own two splits (tile_self_split), for
// levels small enough to need no partition pass (part is unused).
template <int NT, int EO, bool SELF_SPLIT = false>
__global__ void __launch_bounds__(NT)
    k_merge_tile_pairs_bulk(const int32_t *kin, int32_t *kout, const int32_t *vin, int32_t *vout,
                            int64_t n, int64_t w, const int64_t *part, int tpg, int32_t *samp,
                            unsigned *status) {
    using C = TileMergePairs<NT, EO>;
    constexpr int TO = C::TO;
    static_assert(kSampleStride == 32, "sample positions are multiples of 32");
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int wsplit[NT / 32 + 1];
    int32_t *sK = smem, *sV = smem + C::REG;
    const int64_t g = blockIdx.x / tpg;
    const int t = blockIdx.x - (int)(g * tpg);
    const MergeGeom m = merge_geom(g, n, w);
    const int64_t glen = m.alen + m.blen;
    const int64_t o0 = (int64_t)t * TO;
    const int64_t o1 = (o0 + TO) < glen ? (o0 + TO) : glen;
    int64_t a0, a1;
    if constexpr (SELF_SPLIT) {
        static_assert(NT >= 64, "two warps search the tile's two splits");
        tile_self_split(kin, m.gs, w, m.alen, m.blen, o0, o1, &a0, &a1);
    } else {
        a0 = part[blockIdx.x];
        a1 = (o1 == glen) ? m.alen : part[blockIdx.x + 1];
    }
    const int na = (int)(a1 - a0);
    const int tot = (int)(o1 - o0);
    const int nb = tot - na;
    const int64_t ga = m.gs + a0, gb = m.gs + w + (o0 - a0);
    const int64_t ca = ga & ~int64_t(3), cb = gb & ~int64_t(3);
    const int nca = (int)(((ga + na + 3) & ~int64_t(3)) - ca) / 4;
    const int ncb = (int)(((gb + nb + 3) & ~int64_t(3)) - cb) / 4;
    const uint64_t pol = l2_evict_first_policy();
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    // C::REG is a multiple of 4 words, so sV and both B covers start on 16 bytes.
    const bool aligned16 = ((smem_addr(sK) | smem_addr(sV)) & 15u) == 0 &&
                           ((reinterpret_cast<uintptr_t>(kin) | reinterpret_cast<uintptr_t>(kout) |
                             reinterpret_cast<uintptr_t>(vin) | reinterpret_cast<uintptr_t>(vout)) & 15u) == 0;
    if (!aligned16) {  // uniform across the CTA: nothing was issued
        if (threadIdx.x == 0) atomicOr(status, kStatusMisaligned);
        return;
    }
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, (unsigned)(nca + ncb) * 32u);
        if (nca > 0) {
            bulk_load(sK, kin + ca, (unsigned)nca * 16u, &bar, pol);
            bulk_load(sV, vin + ca, (unsigned)nca * 16u, &bar, pol);
        }
        if (ncb > 0) {
            bulk_load(sK + 4 * nca, kin + cb, (unsigned)ncb * 16u, &bar, pol);
            bulk_load(sV + 4 * nca, vin + cb, (unsigned)ncb * 16u, &bar, pol);
        }
    }
    const bool ok = mbar_wait(&bar, 0);
    if (__syncthreads_or(!ok)) {  // a copy never landed: report, drain, leave
        if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
        if (!ok) mbar_wait(&bar, 0);
        return;
    }
    const int offA = (int)(ga - ca), offB = 4 * nca + (int)(gb - cb);
    const int32_t *A = sK + offA, *B = sK + offB;
    const int32_t *VA = sV + offA, *VB = sV + offB;

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
    const int cnt = dend - dcl;

    // Serial stable merge of A[lo, end) and B[dcl - lo, dcl - lo + cnt - (end - lo)).
    // A read at ia == end or ib == eb lands inside the covers (each run is
    // followed by at least one staged word), and its key is never taken.
    int32_t ok_[EO], ov[EO];
    {
        int ia = lo, ib = dcl - lo;
        const int eb = ib + cnt - (end - lo);
        int32_t ka = A[ia], kb = B[ib];
#pragma unroll
        for (int k = 0; k < EO; ++k) {
            const bool take_b = (ib < eb) && ((ia >= end) || (kb < ka));
            ok_[k] = take_b ? kb : ka;
            ov[k] = take_b ? VB[ib] : VA[ia];
            ib += take_b;
            ia += !take_b;
            const int32_t nx = take_b ? B[ib] : A[ia];
            kb = take_b ? nx : kb;
            ka = take_b ? ka : nx;
        }
    }
    __syncthreads();
    if (cnt > 0) {
#pragma unroll
        for (int k = 0; k < EO; ++k) {
            if (k < cnt) {
                sK[diag + k] = ok_[k];
                sV[diag + k] = ov[k];
            }
        }
        fence_proxy_async_smem();
        if (samp) {
#pragma unroll
            for (int j = 0; j < (EO + 31) / 32; ++j) {
                const int k = ((-diag) & 31) + 32 * j;
                if (k < cnt) samp[(m.gs + o0 + diag + k) / kSampleStride] = select_dyn(ok_, k);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // 16-byte aligned: m.gs + o0 and tot are multiples of 4 pairs.
        bulk_store(kout + m.gs + o0, sK, (unsigned)tot * 4u, pol);
        bulk_store(vout + m.gs + o0, sV, (unsigned)tot * 4u, pol);
        bulk_wait_read();
    }
}

// ---------------------------------------------------------------------------
// Four-way pairs level: two of Algorithm 1's merge levels per read and write
// of the keys and values (runs of w -> 4w), as the keys' four-way level does:
// the four-way split of each output tile (on the keys, equal keys in run
// order) from k_merge4_partition, the tile's four key ranges and four value
// ranges in by bulk copies, then two stages of stable serial merges in
// shared memory (runs 0 and 1, runs 2 and 3; then the two results), each
// thread merging exactly its own outputs, values following their keys.

template <int NT, int EO>
struct TileMerge4Pairs {
    static constexpr int TO = ((NT - 1) * EO) / kSampleStride * kSampleStride;
    static_assert((TO - 2) / EO + 2 <= NT, "the two stage-1 merges fit the CTA's threads");
    // Four 16-byte covers (each at most 6 words beyond its keys) and a few
    // words of slack for the serial merge's read past a run's end.
    static constexpr int REG = TO + 24 + 8;
    static constexpr int SMEM_BYTES = 2 * REG * 4;  // keys, values
};

// One thread's cnt (<= EO) outputs of the stable merge of (A, VA)[0, na) and
// (B, VB)[0, nb) at output diagonal diag: merge-path split, end split from
// the next thread (or na when `last`), then a serial merge taking A's element
// on ties.  Every thread of the CTA calls this (it holds a barrier).
template <int NT, int EO>
HS_DEV void stage_merge_pairs(const int32_t *A, const int32_t *VA, int na, const int32_t *B,
                              const int32_t *VB, int nb, int diag, int cnt, bool last,
                              int *wsplit, int32_t (&ok)[EO], int32_t (&ov)[EO]) {
    const int lane = threadIdx.x & 31;
    const int dcl = hs_min(hs_max(diag, 0), na + nb);
    int lo = dcl > nb ? dcl - nb : 0, hi = dcl < na ? dcl : na;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A[mid] <= B[dcl - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    int end = __shfl_down_sync(0xffffffffu, lo, 1);
    if (lane == 0) wsplit[threadIdx.x >> 5] = lo;
    __syncthreads();
    if (lane == 31 && threadIdx.x + 1 < NT) end = wsplit[(threadIdx.x >> 5) + 1];
    if (last) end = na;
    if (cnt <= 0) return;
    // A read at ia == end or ib == eb lands inside the staged buffer and its
    // key is never taken.
    int ia = lo, ib = dcl - lo;
    const int eb = ib + cnt - (end - lo);
    int32_t ka = A[ia], kb = B[ib];
#pragma unroll
    for (int k = 0; k < EO; ++k) {
        const bool take_b = (ib < eb) && ((ia >= end) || (kb < ka));
        ok[k] = take_b ? kb : ka;
        ov[k] = take_b ? VB[ib] : VA[ia];
        ib += take_b;
        ia += !take_b;
        const int32_t nx = take_b ? B[ib] : A[ia];
        kb = take_b ? nx : kb;
        ka = take_b ? ka : nx;
    }
}

template <int NT, int EO>
__global__ void __launch_bounds__(NT)
    k_merge4_pairs_bulk(const int32_t *kin, int32_t *kout, const int32_t *vin, int32_t *vout,
                        int64_t n, int64_t w, const int64_t *part, int64_t tpg, int32_t *samp,
                        unsigned *status) {
    using C = TileMerge4Pairs<NT, EO>;
    constexpr int TO = C::TO;
    static_assert(kSampleStride == 32, "sample positions are multiples of 32");
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int wsplit[NT / 32 + 1];
    int32_t *sK = smem, *sV = smem + C::REG;
    const int64_t b = blockIdx.x;
    const int64_t g = b / tpg;
    const int64_t t = b - g * tpg;
    int64_t start[4], len[4];
    kway_runs_geom<4>(g, n, w, start, len);
    const int64_t glen = len[0] + len[1] + len[2] + len[3];
    const int64_t o0 = t * TO;
    const int64_t o1 = hs_min(o0 + TO, glen);
    const bool last_tile = o1 == glen;
    int cnt[4], off[4];
    int64_t src[4];
    int ncov[4];
    int pos = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t s0 = part[4 * b + i];
        const int64_t e0 = last_tile ? len[i] : part[4 * (b + 1) + i];
        cnt[i] = (int)(e0 - s0);
        src[i] = start[i] + s0;
        const int64_t c0 = src[i] & ~int64_t(3);
        ncov[i] = cnt[i] > 0 ? (int)(((src[i] + cnt[i] + 3) & ~int64_t(3)) - c0) / 4 : 0;
        off[i] = pos + (int)(src[i] - c0);
        pos += 4 * ncov[i];
    }
    const int tot = (int)(o1 - o0);
    const uint64_t pol = l2_evict_first_policy();
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    // C::REG is a multiple of 4 words, so sV starts on 16 bytes like sK.
    const bool fits = pos <= TO + 24 && tot <= TO && tot > 0 &&
                      tot == cnt[0] + cnt[1] + cnt[2] + cnt[3] && cnt[0] >= 0 && cnt[1] >= 0 &&
                      cnt[2] >= 0 && cnt[3] >= 0;
    const bool aligned16 = ((smem_addr(sK) | smem_addr(sV)) & 15u) == 0 &&
                           ((reinterpret_cast<uintptr_t>(kin) | reinterpret_cast<uintptr_t>(kout) |
                             reinterpret_cast<uintptr_t>(vin) | reinterpret_cast<uintptr_t>(vout)) & 15u) == 0;
    if (!aligned16 || !fits) {  // uniform across the CTA: nothing was issued
        if (threadIdx.x == 0) atomicOr(status, aligned16 ? kStatusInconsistent : kStatusMisaligned);
        return;
    }
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, (unsigned)pos * 8u);
        int so = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (ncov[i] > 0) {
                const int64_t c0 = src[i] & ~int64_t(3);
                bulk_load(sK + so, kin + c0, (unsigned)ncov[i] * 16u, &bar, pol);
                bulk_load(sV + so, vin + c0, (unsigned)ncov[i] * 16u, &bar, pol);
            }
            so += 4 * ncov[i];
        }
    }
    const bool ok_wait = mbar_wait(&bar, 0);
    if (__syncthreads_or(!ok_wait)) {  // a copy never landed: report, drain, leave
        if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
        if (!ok_wait) mbar_wait(&bar, 0);
        return;
    }

    // Stage 1: X = merge(R0, R1) on threads [0, tx), Y = merge(R2, R3) after.
    const int nx = cnt[0] + cnt[1], ny = cnt[2] + cnt[3];
    const int tx = (nx + EO - 1) / EO;
    const bool in_x = (int)threadIdx.x < tx;
    const int d1 = in_x ? (int)threadIdx.x * EO : ((int)threadIdx.x - tx) * EO;
    const int gl = in_x ? nx : ny;
    const int c1 = hs_max(hs_min(EO, gl - d1), 0);
    const int ia = in_x ? off[0] : off[2], ib = in_x ? off[1] : off[3];
    int32_t ok[EO], ov[EO];
    stage_merge_pairs<NT, EO>(sK + ia, sV + ia, in_x ? cnt[0] : cnt[2], sK + ib, sV + ib,
                              in_x ? cnt[1] : cnt[3], d1, c1, d1 + EO >= gl, wsplit, ok, ov);
    __syncthreads();  // every read of the staged covers is done
    if (c1 > 0) {
        const int o = (in_x ? 0 : nx) + d1;
#pragma unroll
        for (int k = 0; k < EO; ++k)
            if (k < c1) {
                sK[o + k] = ok[k];
                sV[o + k] = ov[k];
            }
    }
    __syncthreads();

    // Stage 2: the tile = merge(X, Y), X = [0, nx), Y = [nx, tot).
    const int d2 = (int)threadIdx.x * EO;
    const int c2 = hs_max(hs_min(EO, tot - d2), 0);
    stage_merge_pairs<NT, EO>(sK, sV, nx, sK + nx, sV + nx, ny, d2, c2, d2 + EO >= tot, wsplit,
                              ok, ov);
    __syncthreads();
    if (c2 > 0) {
#pragma unroll
        for (int k = 0; k < EO; ++k)
            if (k < c2) {
                sK[d2 + k] = ok[k];
                sV[d2 + k] = ov[k];
            }
        fence_proxy_async_smem();
        if (samp) {
            const int64_t ob = g * 4 * w + o0;  // a multiple of 32
#pragma unroll
            for (int j = 0; j < (EO + 31) / 32; ++j) {
                const int k = ((-d2) & 31) + 32 * j;
                if (k < c2) samp[(ob + d2 + k) / kSampleStride] = select_dyn(ok, k);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // 16-byte aligned: g*4w + o0 and tot are multiples of 4 pairs.
        bulk_store(kout + g * 4 * w + o0, sK, (unsigned)tot * 4u, pol);
        bulk_store(vout + g * 4 * w + o0, sV, (unsigned)tot * 4u, pol);
        bulk_wait_read();
    }
}

// ---------------------------------------------------------------------------
// Planner.

// Block sort: 256 threads x 4 leaves (tiles of 256 * (4L - 1) pairs).
constexpr int PB_NT = 256;
int64_t pairs_tile(int L) { return (int64_t)PB_NT * (4 * L - 1); }

// 16-byte aligned key and value arrays (vec) use the bulk-copy block sort
// (k_blocksort_pairs_bulk), others the thread-staged one.
template <int NT, int L, int LEAVES>
static hs_status launch_pairs_blocksort_t(const int32_t *kin, int32_t *kout, const int32_t *vin,
                                          int32_t *vout, int64_t n, hs_netset s, int vec,
                                          int32_t *samp, cudaStream_t st) {
    using C = BlockSortPairs<NT, L, LEAVES>;
    const int64_t grid = (n + C::T - 1) / C::T;
    hs_status r;
    if constexpr (C::BULK_OK) {
        if (vec) {
            unsigned *status = nullptr;
            if ((r = device_status(&status)) != HS_OK) return r;
            auto kern = k_blocksort_pairs_bulk<NT, L, LEAVES>;
            if ((r = ensure_smem((const void *)kern, C::SMEM_BYTES)) != HS_OK) return r;
            LaunchToken t = launch_begin(K_BLOCKSORT_PAIRS, st);
            kern<<<(unsigned)grid, NT, C::SMEM_BYTES, st>>>(kin, kout, vin, vout, n, s, samp, status);
            return launch_end(t);
        }
    }
    auto kern = k_blocksort_pairs<NT, L, LEAVES>;
    if ((r = ensure_smem((const void *)kern, C::SMEM_BYTES)) != HS_OK) return r;
    LaunchToken t = launch_begin(K_BLOCKSORT_PAIRS, st);
    kern<<<(unsigned)grid, NT, C::SMEM_BYTES, st>>>(kin, kout, vin, vout, n, s, vec, samp);
    return launch_end(t);
}

template <int NT, int LEAVES>
static hs_status launch_pairs_blocksort_nt(int L, const int32_t *kin, int32_t *kout,
                                           const int32_t *vin, int32_t *vout, int64_t n,
                                           hs_netset s, int vec, int32_t *samp, cudaStream_t st) {
    switch (L) {
        case 1: return launch_pairs_blocksort_t<NT, 1, LEAVES>(kin, kout, vin, vout, n, s, vec, samp, st);
        case 3: return launch_pairs_blocksort_t<NT, 3, LEAVES>(kin, kout, vin, vout, n, s, vec, samp, st);
        case 4: return launch_pairs_blocksort_t<NT, 4, LEAVES>(kin, kout, vin, vout, n, s, vec, samp, st);
        case 5: return launch_pairs_blocksort_t<NT, 5, LEAVES>(kin, kout, vin, vout, n, s, vec, samp, st);
        case 6: return launch_pairs_blocksort_t<NT, 6, LEAVES>(kin, kout, vin, vout, n, s, vec, samp, st);
        case 7: return launch_pairs_blocksort_t<NT, 7, LEAVES>(kin, kout, vin, vout, n, s, vec, samp, st);
        case 8: return launch_pairs_blocksort_t<NT, 8, LEAVES>(kin, kout, vin, vout, n, s, vec, samp, st);
    }
    return fail(HS_ERR_INVALID_ARG, "leaf size outside 1, 3..8");
}

constexpr int PG_NT = 256, PG_E = 8;  // generic level

// Tiled pairs level: 128 threads x 31 pairs, sampled partition searches.
constexpr int PM_NT = 128, PM_EO = 31;

static hs_status launch_pairs_tile(const int32_t *kin, int32_t *kout, const int32_t *vin,
                                   int32_t *vout, int64_t n, int64_t w, int64_t *part,
                                   int32_t *samp, cudaStream_t st) {
    using C = TileMergePairs<PM_NT, PM_EO>;
    static_assert(C::TO % kSampleStride == 0, "output tiles start on sample positions");
    const LevelTiles lt = level_tiles(n, w, C::TO);
    if (lt.nblocks <= kSelfSplitMaxTiles) {
        unsigned *status = nullptr;
        hs_status r = device_status(&status);
        if (r != HS_OK) return r;
        auto kern = k_merge_tile_pairs_bulk<PM_NT, PM_EO, true>;
        if ((r = ensure_smem((const void *)kern, C::SMEM_BYTES)) != HS_OK) return r;
        LaunchToken t = launch_begin(K_MERGE_PAIRS, st);
        kern<<<(unsigned)lt.nblocks, PM_NT, C::SMEM_BYTES, st>>>(kin, kout, vin, vout, n, w, nullptr,
                                                                 (int)lt.tpg, samp, status);
        return launch_end(t);
    }
    LaunchToken t = launch_begin(K_MERGE_PARTITION, st);
    k_merge_partition_sampled<<<(unsigned)((lt.nblocks + 255) / 256), 256, 0, st>>>(
        kin, samp, n, w, C::TO, (int)lt.tpg, lt.nblocks, part);
    hs_status r = launch_end(t);
    if (r != HS_OK) return r;
    unsigned *status = nullptr;
    if ((r = device_status(&status)) != HS_OK) return r;
    auto kern = k_merge_tile_pairs_bulk<PM_NT, PM_EO>;
    if ((r = ensure_smem((const void *)kern, C::SMEM_BYTES)) != HS_OK) return r;
    t = launch_begin(K_MERGE_PAIRS, st);
    kern<<<(unsigned)lt.nblocks, PM_NT, C::SMEM_BYTES, st>>>(kin, kout, vin, vout, n, w, part,
                                                             (int)lt.tpg, samp, status);
    return launch_end(t);
}

static bool pairs_tiled(int64_t n, int vec) { return vec && (n % 4) == 0; }

// Four-way pair levels (option merge_fanin: 4 always, 2 never, 0 from
// kPairsFourWayMinPairs pairs on).  The pair levels are HBM-bound, so saving
// passes pays off earlier than for keys.  Whole pair sorts measured on GB300
// with four-way / binary levels: 0.36 / 0.25 ms at 2^21 pairs, 0.68 / 0.57 at
// 2^23, 1.07 / 1.02 at 2^24, 1.78 / 1.87 at 2^25, 3.20 / 3.62 at 2^26 and
// 6.14 / 7.27 ms at 2^27.
constexpr int64_t kPairsFourWayMinPairs = int64_t(1) << 25;
static bool pairs_four_way(int64_t n, int vec) {
    if (!pairs_tiled(n, vec) || merge_fanin() == 2) return false;
    return merge_fanin() == 4 || n >= kPairsFourWayMinPairs;
}

constexpr int P4_NT = kMerge4Threads, P4_EO = kMerge4Keys;

static hs_status launch_pairs_level4(const int32_t *kin, int32_t *kout, const int32_t *vin,
                                     int32_t *vout, int64_t n, int64_t w, int64_t *part,
                                     int64_t part_cap, int32_t *samp, cudaStream_t st) {
    using C = TileMerge4Pairs<P4_NT, P4_EO>;
    static_assert(C::TO % kSampleStride == 0, "output tiles start on sample positions");
    unsigned *status = nullptr;
    hs_status r = device_status(&status);
    if (r != HS_OK) return r;
    const LevelTiles lt = level_tiles_span(n, 4 * w, C::TO);
    if (4 * (lt.nblocks + 1) > part_cap)
        return fail(HS_ERR_INVALID_ARG, "pair sort: workspace too small for the four-way partitions");
    LaunchToken t = launch_begin(K_MERGE_PARTITION, st);
    k_merge4_partition<4><<<(unsigned)((lt.nblocks + 127) / 128), 128, 0, st>>>(
        kin, samp, n, w, C::TO, lt.tpg, lt.nblocks, part);
    if ((r = launch_end(t)) != HS_OK) return r;
    auto kern = k_merge4_pairs_bulk<P4_NT, P4_EO>;
    if ((r = ensure_smem((const void *)kern, C::SMEM_BYTES)) != HS_OK) return r;
    t = launch_begin(K_MERGE_PAIRS, st);
    kern<<<(unsigned)lt.nblocks, P4_NT, C::SMEM_BYTES, st>>>(kin, kout, vin, vout, n, w, part,
                                                              lt.tpg, samp, status);
    return launch_end(t);
}

static hs_status launch_pairs_level(const int32_t *kin, int32_t *kout, const int32_t *vin,
                                    int32_t *vout, int64_t n, int64_t w, int64_t *part,
                                    int32_t *samp, int vec, cudaStream_t st) {
    if (pairs_tiled(n, vec)) return launch_pairs_tile(kin, kout, vin, vout, n, w, part, samp, st);
    const LevelTiles lt = level_tiles(n, w, PG_NT * PG_E);
    LaunchToken t = launch_begin(K_MERGE_PARTITION, st);
    k_merge_partition<<<(unsigned)((lt.nblocks + 255) / 256), 256, 0, st>>>(
        kin, n, w, PG_NT * PG_E, (int)lt.tpg, lt.nblocks, part);
    hs_status r = launch_end(t);
    if (r != HS_OK) return r;
    const int smem = merge_smem_words<PG_NT, PG_E>() * (int)sizeof(int32_t) * 2;
    auto kern = k_merge_pass<PG_NT, PG_E, true>;
    if ((r = ensure_smem((const void *)kern, smem)) != HS_OK) return r;
    t = launch_begin(K_MERGE_PAIRS, st);
    kern<<<(unsigned)lt.nblocks, PG_NT, smem, st>>>(kin, kout, vin, vout, n, w, part, (int)lt.tpg,
                                                     vec);
    return launch_end(t);
}

hs_status pairs_sort(int32_t *d_keys, int32_t *d_vals, size_t n_, hs_netset s, void *d_ws,
                     size_t ws_bytes, cudaStream_t st) {
    const int64_t n = (int64_t)n_;
    const int L = leaf_size(s);
    const int64_t T = pairs_tile(L);
    int doublings = 0;
    for (int64_t w = T; w < n; w *= 2) ++doublings;

    int32_t *kbuf = nullptr, *vbuf = nullptr, *samp = nullptr;
    int64_t *part = nullptr;
    const int vec = aligned(d_keys, 16) && aligned(d_vals, 16) ? 1 : 0;
    if (doublings > 0) {
        if (!d_ws || ws_bytes < merge_workspace_bytes(n_, 1))
            return fail(HS_ERR_INVALID_ARG, "pair sort: workspace smaller than hs_sort_workspace_bytes");
        if (!aligned(d_ws, 16)) return fail(HS_ERR_INVALID_ARG, "pair sort: workspace not 16-byte aligned");
        char *p = static_cast<char *>(d_ws);
        const size_t kb = merge_ws_keys_bytes(n_);
        kbuf = reinterpret_cast<int32_t *>(p);
        vbuf = reinterpret_cast<int32_t *>(p + kb);
        part = reinterpret_cast<int64_t *>(p + 2 * kb);
        if (pairs_tiled(n, vec))
            samp = reinterpret_cast<int32_t *>(p + 2 * kb + merge_ws_part_bytes(n_));
    }

    // With an even number of level launches the block sort writes in place,
    // so the last level lands in the caller's arrays.
    const bool four = pairs_four_way(n, vec);
    const int launches = four ? doublings / 2 + doublings % 2 : doublings;
    int32_t *kcur = (launches % 2 == 0) ? d_keys : kbuf;
    int32_t *vcur = (launches % 2 == 0) ? d_vals : vbuf;
    int32_t *kalt = (kcur == d_keys) ? kbuf : d_keys;
    int32_t *valt = (vcur == d_vals) ? vbuf : d_vals;

    hs_status r = launch_pairs_blocksort_nt<PB_NT, 4>(L, d_keys, kcur, d_vals, vcur, n, s, vec, samp, st);
    if (r != HS_OK) return r;
    // A binary level first when the number of doublings is odd, then four-way
    // levels (or binary levels throughout).
    int64_t w = T;
    for (int d = doublings; d > 0;) {
        if (four && d % 2 == 0) {
            r = launch_pairs_level4(kcur, kalt, vcur, valt, n, w, part,
                                    (int64_t)merge_ws_part_entries(n_), samp, st);
            w *= 4;
            d -= 2;
        } else {
            r = launch_pairs_level(kcur, kalt, vcur, valt, n, w, part, samp, vec, st);
            w *= 2;
            d -= 1;
        }
        if (r != HS_OK) return r;
        std::swap(kcur, kalt);
        std::swap(vcur, valt);
    }
    return HS_OK;
}

}  // namespace hs
