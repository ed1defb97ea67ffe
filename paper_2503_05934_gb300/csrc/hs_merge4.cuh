// Four-way global merge level of the keys merge sort: two levels of
// Algorithm 1's "Merge" (runs of w -> 2w -> 4w) in one read and one write of
// every key, which halves the HBM passes above the block sort.
//
// Group g holds the four runs R_i = [g*4w + i*w, + w) (clipped to n).  Its
// output is the stable merge of the four: equal keys keep the order of their
// runs, which is the order the two binary levels it replaces would give (the
// left run wins every tie).  Output tiles of TO keys are cut by a four-way
// merge-path split (kway_split below, one thread per tile boundary); a CTA
// stages its tile's four input ranges in shared memory by bulk copies, merges
// R_0 with R_1 and R_2 with R_3 (stage 1), then the two results (stage 2),
// and leaves by one bulk store.
#pragma once

#include "hs_bulk.cuh"
#include "hs_internal.h"
#include "hs_merge_prims.cuh"

namespace hs {

// ---------------------------------------------------------------------------
// K-way merge-path split.
//
// For an output rank k of the stable merge of K sorted runs, a_i = the number
// of elements of run i among the first k outputs.  The order is the total
// order on (key, run, position): that of the stable merge.
//
// The search refines over resolutions r = 2^m, ..., 2, 1.  At resolution r
// the samples of run i are its keys at positions 0, r, 2r, ..., and U(r) is
// the set of the ceil(k / r) smallest samples of all runs (it holds a prefix
// of each run's samples; u_i counts them).  U(1) is the first k outputs, so
// u_i = a_i at the end.  Going from r to h = r / 2: every sample of U(r)
// belongs to U(h) (U(h) holds at least ceil(k / r) of the resolution-r
// samples, and those are the smallest), so does everything before it in its
// run, which is the first max(0, 2u_i - 1) resolution-h samples of run i.
// The rest of U(h) (at most K samples) is added one at a time, each the
// smallest sample not yet taken: the smallest of the K runs' next samples.
// Each round therefore reads two new samples per run (and rarely a third),
// independent of each other, and decides with K-way minimums.
//
// At resolutions of kSampleStride and above every position read is a
// multiple of it, and the sample array (every 32nd key, L2-resident) is read
// when the caller has one.

// A sample as one unsigned word ordered like the stable merge: the key (sign
// bit flipped) above the run index, and past the end of its run a word above
// every key.
constexpr uint64_t kSplitPastEnd = uint64_t(1) << 40;
HS_HD uint64_t split_word(int32_t key, int run) {
    return ((uint64_t)((uint32_t)key ^ 0x80000000u) << 8) | (uint64_t)run;
}

template <int K>
struct KwayRuns {
    const int32_t *keys;  // the level's input
    const int32_t *samp;  // samp[j] = keys[j * kSampleStride], or null
    int64_t start[K];     // run starts (multiples of kSampleStride when samp is used)
    int64_t len[K];
    // Sample word of run i at position p; from_samp: p is a multiple of
    // kSampleStride and the sample array is read.
    HS_HD uint64_t word(int i, int64_t p, bool from_samp) const {
        if (p >= len[i]) return kSplitPastEnd | (uint64_t)i;
        const int64_t gpos = start[i] + p;
        return split_word(from_samp ? samp[gpos >> 5] : keys[gpos], i);
    }
};

template <int K>
HS_HD uint64_t min_word(const uint64_t (&v)[K]) {
    uint64_t m = v[0];
#pragma unroll
    for (int i = 1; i < K; ++i) m = hs_min(m, v[i]);
    return m;
}

// U(2^lg) for rank k with lg >= ceil(log2(longest run)), where each run has
// one sample (position 0): u[i] = 1 for the ceil(k / 2^lg) (at most K) runs
// with the smallest first keys.  cur[i] = each run's first untaken sample.
template <int K, class Src>
HS_HD void kway_split_init(const Src &R, int64_t k, int lg, bool fs, int64_t (&u)[K],
                           uint64_t (&cur)[K]) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
        u[i] = 0;
        cur[i] = R.word(i, 0, fs);
    }
    for (int64_t need = (k + (int64_t(1) << lg) - 1) >> lg; need > 0; --need) {
        const int b = (int)(min_word<K>(cur) & 0xFF);
#pragma unroll
        for (int i = 0; i < K; ++i)
            if (i == b) {
                u[i] += 1;
                cur[i] = R.word(i, u[i] << lg, fs);
            }
    }
}

// Each round halves the resolution and preloads two samples per run after
// its first untaken one.  Measured on GB300 at 2^28 keys (partition time
// per sort, seven four-way levels): 0.65 ms; one sample preloaded 0.73 ms;
// rounds of 4-fold refinement with 3 or 5 preloaded 0.90 / 0.84 ms; 8-fold
// with 7 or 9 preloaded 1.21 / 1.18 ms (longer serial additions per round).
constexpr int kSplitLR = 1;  // each round refines 2^kSplitLR-fold
constexpr int kSplitWN = 2;  // samples preloaded per run and round after its first untaken one

// Refines U(2^lg) (u, cur) to U(1), 2^LR-fold per round (lg a multiple of
// LR): going from r to h = r / 2^LR, a run with u samples in U(r) has its
// first max(0, 2^LR (u - 1) + 1) resolution-h samples in U(h) (those up to
// its last sample of U(r)); the rest of U(h) is added one sample at a time,
// each the smallest first untaken sample of the K runs.  Each round reads,
// per run, its first untaken sample and the WN after it (independent loads;
// one of them is the resolution-r sample already held), and loads further
// ones only when its run advances past them.  fs_min: the lowest
// resolution exponent at which positions are read from the sample array.
template <int K, int LR, int WN, class Src>
HS_HD void kway_split_refine(const Src &R, int64_t k, int lg, int fs_min, int64_t (&u)[K],
                             uint64_t (&cur)[K]) {
    constexpr int64_t RR = int64_t(1) << LR;
    for (; lg > 0; lg -= LR) {
        const int lh = lg - LR;
        const bool fs = lh >= fs_min;
        int64_t v[K];
        int d[K];
        uint64_t c[K][WN];  // c[i][j]: run i's sample at index v + 1 + j
        int64_t taken = 0;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const uint64_t old = cur[i];
            v[i] = u[i] == 0 ? 0 : RR * (u[i] - 1) + 1;
            if (u[i] > 0) cur[i] = R.word(i, v[i] << lh, fs);  // else index 0 is old
#pragma unroll
            for (int j = 0; j < WN; ++j)
                c[i][j] = (u[i] > 0 && j == RR - 2) ? old : R.word(i, (v[i] + 1 + j) << lh, fs);
            d[i] = 0;
            taken += v[i];
        }
        for (int64_t need = ((k + (int64_t(1) << lh) - 1) >> lh) - taken; need > 0; --need) {
            const int b = (int)(min_word<K>(cur) & 0xFF);
#pragma unroll
            for (int i = 0; i < K; ++i)
                if (i == b) {
                    d[i] += 1;
                    cur[i] = d[i] <= WN ? select_dyn(c[i], d[i] - 1) : R.word(i, (v[i] + d[i]) << lh, fs);
                }
        }
#pragma unroll
        for (int i = 0; i < K; ++i) u[i] = v[i] + d[i];
    }
}

// Exponent of the coarsest resolution the search starts from: each run has
// one sample there; a multiple of kSplitLR.
template <int K>
HS_HD int kway_split_top(const int64_t (&len)[K]) {
    int64_t mx = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) mx = hs_max(mx, len[i]);
    int lg = 0;
    while ((int64_t(1) << lg) < mx) lg += kSplitLR;
    return lg;
}

// a[i] = elements of run i among the first k outputs (0 <= k <= sum of len).
template <int K>
HS_HD void kway_split(const KwayRuns<K> &R, int64_t k, int64_t (&a)[K]) {
    static_assert(K <= 255, "run index fits the sample word");
    const int fs_min = R.samp ? 5 : 64;
    const int lg = kway_split_top<K>(R.len);
    int64_t u[K];
    uint64_t cur[K];
    kway_split_init<K>(R, k, lg, lg >= fs_min, u, cur);
    kway_split_refine<K, kSplitLR, kSplitWN>(R, k, lg, fs_min, u, cur);
#pragma unroll
    for (int i = 0; i < K; ++i) a[i] = u[i];
}

// ---------------------------------------------------------------------------
// Level geometry: group g merges K runs of w starting at g*K*w.

template <int K>
HS_HD void kway_runs_geom(int64_t g, int64_t n, int64_t w, int64_t (&start)[K], int64_t (&len)[K]) {
    const int64_t gs = g * K * w;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int64_t s = gs + i * w;
        start[i] = s;
        len[i] = s >= n ? 0 : (n - s < w ? n - s : w);
    }
}

// Output tiles of a K-way level: groups of K*w keys cut into tiles of TO.
HS_HD LevelTiles level_tiles_span(int64_t n, int64_t span, int64_t to) {
    const int64_t ngroups = (n + span - 1) / span;
    const int64_t last = n - (ngroups - 1) * span;
    LevelTiles t;
    t.tpg = (span + to - 1) / to;
    t.nblocks = (ngroups - 1) * t.tpg + (last + to - 1) / to;
    return t;
}

// part[K*b + i] = elements of run i before output tile b's first output;
// one thread per tile boundary b.
template <int K>
static __global__ void k_merge4_partition(const int32_t *in, const int32_t *samp, int64_t n,
                                          int64_t w, int to, int64_t tpg, int64_t nblocks,
                                          int64_t *part) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const int64_t g = b / tpg, t = b - g * tpg;
    KwayRuns<K> R;
    R.keys = in;
    R.samp = samp;
    kway_runs_geom<K>(g, n, w, R.start, R.len);
    int64_t glen = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) glen += R.len[i];
    const int64_t k = hs_min(t * (int64_t)to, glen);
    int64_t a[K];
    kway_split<K>(R, k, a);
#pragma unroll
    for (int i = 0; i < K; ++i) part[K * b + i] = a[i];
}

// ---------------------------------------------------------------------------
// The four-way merge tile.  NT threads x EO outputs per stage; the tile holds
// TO keys, a multiple of kSampleStride small enough that the two stage-1
// merges (whose outputs each start on a fresh thread) fit in NT threads.

template <int NT, int EO>
struct TileMerge4 {
    static constexpr int P = pow2_at_least(EO);
    static constexpr int TO = ((NT - 1) * EO) / kSampleStride * kSampleStride;
    static_assert((TO - 2) / EO + 2 <= NT, "the two stage-1 merges fit the CTA's threads");
    // Four 16-byte covers (each at most 6 words beyond its keys), then the P
    // words of slack that exact-window loads may touch past the last key.
    static constexpr int REG = TO + 24 + P + 8;
    static constexpr int SMEM_BYTES = REG * 4;
};

// One thread's EO outputs of the stable merge of A[0, na) and B[0, nb) at
// output diagonal diag (cnt = outputs it owns, 0 if none): its merge-path
// split, its end split from the next thread (a shuffle, or the next warp's
// first thread through wsplit; `last` threads take na), and the exact-window
// merge.  Every thread of the CTA calls this (it holds a barrier).
template <int NT, int EO, int P>
HS_DEV int stage_merge(const int32_t *A, int na, const int32_t *B, int nb, int diag, int cnt,
                       bool last, int *wsplit, int32_t (&x)[P]) {
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
    if (cnt > 0) exact_window_merge<EO, P>(A, lo, B, dcl - lo, end - lo, cnt, x);
    return cnt;
}

template <int NT, int EO>
__global__ void __launch_bounds__(NT)
    k_merge4_tile_bulk(const int32_t *in, int32_t *out, int64_t n, int64_t w, const int64_t *part,
                       int64_t tpg, int32_t *samp, unsigned *status, int64_t block0) {
    using C = TileMerge4<NT, EO>;
    constexpr int TO = C::TO, P = C::P;
    static_assert(kSampleStride == 32, "sample positions are multiples of 32");
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int wsplit[NT / 32 + 1];

    const int64_t b = block0 + blockIdx.x;  // output tile (a launch may cover a range of them)
    const int64_t g = b / tpg;
    const int64_t t = b - g * tpg;
    int64_t start[4], len[4];
    kway_runs_geom<4>(g, n, w, start, len);
    const int64_t glen = len[0] + len[1] + len[2] + len[3];
    const int64_t o0 = t * TO;
    const int64_t o1 = hs_min(o0 + TO, glen);
    const bool last_tile = o1 == glen;
    int cnt[4], off[4];
    int64_t src[4];  // global position of each range's first key
    int ncov[4];     // 16-byte words of each range's cover
    int pos = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t s = part[4 * b + i];
        const int64_t e = last_tile ? len[i] : part[4 * (b + 1) + i];
        cnt[i] = (int)(e - s);
        src[i] = start[i] + s;
        const int64_t c0 = src[i] & ~int64_t(3);
        ncov[i] = cnt[i] > 0 ? (int)(((src[i] + cnt[i] + 3) & ~int64_t(3)) - c0) / 4 : 0;
        off[i] = pos + (int)(src[i] - c0);  // the range's first key in shared memory
        pos += 4 * ncov[i];
    }
    const int tot = (int)(o1 - o0);
    const uint64_t pol = l2_evict_first_policy();
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    // Bulk copies need 16-byte aligned ends: whole 16-byte words of 16-byte
    // aligned arrays; this re-checks it, and that the covers fit the buffer.
    const bool fits = pos <= TO + 24 && tot <= TO && tot == cnt[0] + cnt[1] + cnt[2] + cnt[3] &&
                      cnt[0] >= 0 && cnt[1] >= 0 && cnt[2] >= 0 && cnt[3] >= 0;
    const bool aligned16 = (smem_addr(smem) & 15u) == 0 &&
                           ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
    if (!aligned16 || !fits) {  // uniform across the CTA: nothing was issued
        if (threadIdx.x == 0) atomicOr(status, aligned16 ? kStatusInconsistent : kStatusMisaligned);
        return;
    }
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, (unsigned)pos * 4u);
        int so = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (ncov[i] > 0)
                bulk_load(smem + so, in + (src[i] & ~int64_t(3)), (unsigned)ncov[i] * 16u, &bar, pol);
            so += 4 * ncov[i];
        }
    }
    const bool ok = mbar_wait(&bar, 0);
    if (__syncthreads_or(!ok)) {  // a copy never landed: report, drain, leave
        if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
        if (!ok) mbar_wait(&bar, 0);
        return;
    }

    // Stage 1: X = merge(R0, R1) on threads [0, tx), Y = merge(R2, R3) on the
    // threads after them.
    const int nx = cnt[0] + cnt[1], ny = cnt[2] + cnt[3];
    const int tx = (nx + EO - 1) / EO;
    const bool in_x = (int)threadIdx.x < tx;
    const int d1 = in_x ? (int)threadIdx.x * EO : ((int)threadIdx.x - tx) * EO;
    const int gl = in_x ? nx : ny;  // length of this thread's merge
    const int c1 = hs_max(hs_min(EO, gl - d1), 0);
    int32_t x[P];
    stage_merge<NT, EO, P>(smem + (in_x ? off[0] : off[2]), in_x ? cnt[0] : cnt[2],
                           smem + (in_x ? off[1] : off[3]), in_x ? cnt[1] : cnt[3], d1, c1,
                           d1 + EO >= gl, wsplit, x);
    __syncthreads();  // every window read is done: the buffer is free
    if (c1 > 0) {
        int32_t *dst = smem + (in_x ? 0 : nx) + d1;
#pragma unroll
        for (int k = 0; k < EO; ++k)
            if (k < c1) dst[k] = x[k];
    }
    __syncthreads();

    // Stage 2: the tile = merge(X, Y), X = smem[0, nx), Y = smem[nx, tot).
    const int d2 = (int)threadIdx.x * EO;
    const int c2 = hs_max(hs_min(EO, tot - d2), 0);
    stage_merge<NT, EO, P>(smem, nx, smem + nx, ny, d2, c2, d2 + EO >= tot, wsplit, x);
    __syncthreads();
    if (c2 > 0) {
#pragma unroll
        for (int k = 0; k < EO; ++k)
            if (k < c2) smem[d2 + k] = x[k];
        fence_proxy_async_smem();
        if (samp) {
            // Output positions g*4w + o0 + d2 + k; g*4w + o0 is a multiple of 32.
            const int64_t ob = g * 4 * w + o0;
#pragma unroll
            for (int j = 0; j < (EO + 31) / 32; ++j) {
                const int k = ((-d2) & 31) + 32 * j;
                if (k < c2) samp[(ob + d2 + k) / kSampleStride] = select_dyn(x, k);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && tot > 0) {
        // 16-byte aligned: g*4w + o0 and tot are multiples of 4 keys.
        bulk_store(out + g * 4 * w + o0, smem, (unsigned)tot * 4u, pol);
        bulk_wait_read();
    }
}

// The launch shape of the four-way tile: 128 threads x 31 keys, 3936 keys
// per tile.  With 192 or 256 threads (5920 / 7904 keys) the partitions shrink
// in number but the merge slows more: 4.26 / 4.36 ms of four-way levels per
// 2^28 sort against 4.02 ms.
constexpr int kMerge4Threads = 128, kMerge4Keys = 31;

}  // namespace hs
