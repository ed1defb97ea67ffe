// Block sort: the first pass of Algorithm 1 on the GPU.  One CTA sorts one
// tile of the array: every thread sorts its leaves in registers with the
// fixed networks ("ApplySortingNetwork" on subarrays of 3..8 keys), merges
// them in registers, and log2(NT) merge-path levels in shared memory merge
// the threads' runs into one sorted tile (the bottom levels of "Merge").
//
//  * keys (block_sort_tile3): int32 keys.
//  * pairs (block_sort_pairs_tile): 64-bit sort words (key, position in the
//    tile), so every network and merge orders equal keys by input position,
//    which makes the result the stable order; the values stay in shared
//    memory and are gathered once, by position, at the end.
#pragma once

#include "hs_bulk.cuh"
#include "hs_merge_prims.cuh"
#include "hs_networks.cuh"

namespace hs {

// Compare-exchange on one register array of sort words (keys or pair words).
template <class K>
struct WordCE {
    K *k;
    template <int i, int j>
    HS_HD void ce() {
        K a = k[i], b = k[j];
        k[i] = hs_min(a, b);
        k[j] = hs_max(a, b);
    }
};

// Sorts leaf x[0..N) in registers (N live slots; r of them real).  A leaf of
// r keys uses the size-r network when the set has one, else the next size up
// with the missing keys padded by +infinity sentinels (never stored).
template <int N, class K>
HS_DEV void sort_leaf(K *x, int r, uint32_t netset) {
    if (r <= 1) return;
    const int m = ragged_net_size(r, netset);
    if (m == N && r == N) {
        WordCE<K> op{x};
        network<N>(op);
        return;
    }
    K t[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) t[i] = (i < N && i < r) ? x[i < N ? i : 0] : word_max<K>();
    WordCE<K> op{t};
    network_dyn(m, op);
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = t[i];
}

// Bitonic merge of sorted x[0..N1) and x[N1..N1+N2) (N1, N2 <= P/2) in
// registers; the ascending result goes back to x[0..N1+N2).
template <int N1, int N2, int P, class K>
HS_DEV void register_merge(K *x) {
    K lo[P / 2], hi[P / 2];
#pragma unroll
    for (int i = 0; i < P / 2; ++i) {
        const K a = i < N1 ? x[i] : word_max<K>();
        const int j = P / 2 - 1 - i;  // second run, reversed
        const K b = j < N2 ? x[N1 + (j < N2 ? j : 0)] : word_max<K>();
        lo[i] = hs_min(a, b);
        hi[i] = hs_max(a, b);
    }
    bitonic_half_clean<P / 2>(lo);
    bitonic_half_clean<P / 2>(hi);
#pragma unroll
    for (int i = 0; i < N1 + N2; ++i) x[i] = i < P / 2 ? lo[i] : hi[i - P / 2];
}

// A thread's leaves: two (L, L - 1 keys) or four (L, L, L, L - 1 keys), each
// sorted by its network, then merged in registers into one run of EO keys.
// A leaf size that is not in the set is padded up to the next size that is,
// the same rule as a ragged leaf; for the {6,7,8} set the leaves are 8 and 7
// keys, both in the set.  avail = live keys from the thread's first slot.
template <int L, int LEAVES, int P, class K>
HS_DEV void sort_thread_leaves(K *k, int avail, uint32_t netset) {
    if constexpr (LEAVES == 2) {
        if constexpr (L > 1) {
            sort_leaf<L>(k, hs_min(hs_max(avail, 0), L), netset);
            sort_leaf<L - 1>(k + L, hs_min(hs_max(avail - L, 0), L - 1), netset);
            register_merge<L, L - 1, P>(k);
        }
    } else {
        if constexpr (L > 1) {
#pragma unroll
            for (int h = 0; h < 3; ++h)
                sort_leaf<L>(k + h * L, hs_min(hs_max(avail - h * L, 0), L), netset);
            sort_leaf<L - 1>(k + 3 * L, hs_min(hs_max(avail - 3 * L, 0), L - 1), netset);
        }
        register_merge<L, L, P / 2>(k);
        register_merge<L, L - 1, P / 2>(k + 2 * L);
        register_merge<2 * L, 2 * L - 1, P>(k);
    }
}

// The shared-memory merge levels: runs of w -> 2w over the tile s[0..T).
// Every thread finds its merge-path split and forms its EO outputs as the
// exact-window merge of its own keys; its end split is the next lane's start
// (a shuffle), or for a warp's last lane the next warp's first lane's start,
// passed through wsplit.  Because EO is odd, neighbouring threads' windows
// and their own EO-key slots fall on different banks, so the tile is stored
// unpadded.  NT need not be a power of two: the last group of a level may
// hold a short B run or none (then its keys stay as they are).  On return k
// holds the thread's EO keys of the sorted tile.
//
// WARP: the tile belongs to one warp alone (NT = 32, s is that warp's own
// buffer), every barrier is a warp barrier, and other warps of the block may
// be sorting other tiles meanwhile.
// First merge level in registers: lanes 2j and 2j+1 merge their EO-key runs
// (A = the even lane's, B = the odd lane's) without shared memory.  Each lane
// gets the other's run by shuffles and applies the first half-cleaner of the
// bitonic merge of A and reversed B (both padded to P with +infinity): the
// even lane keeps the minima, the odd lane the maxima (in reverse order,
// still bitonic), and each sorts its P words with the remaining half-cleaner
// stages.  The even lane's P smallest words are the P smallest of the pair;
// it keeps EO of them and hands the other P - EO to the odd lane, whose EO
// outputs are those followed by the real words of its maxima.
template <int EO, int P, class K>
HS_DEV void shuffle_first_level(K (&k)[EO], bool odd) {
    constexpr int X = P - EO;  // words the even lane hands to the odd lane
    K z[P];
#pragma unroll
    for (int i = 0; i < P; ++i) z[i] = i < EO ? k[i < EO ? i : 0] : word_max<K>();
    // Slots i and P-1-i meet the partner's P-1-i and i: both are updated in
    // one step, so only the P-word array stays live (no copy of the partner's
    // run).  Padding slots hold +infinity on both lanes and need no shuffle.
#pragma unroll
    for (int i = 0; i < P / 2; ++i) {
        const int j = P - 1 - i;
        const K a = z[i], b = z[j];
        const K pb = j < EO ? __shfl_xor_sync(0xffffffffu, b, 1) : word_max<K>();  // partner's z[j]
        const K pa = i < EO ? __shfl_xor_sync(0xffffffffu, a, 1) : word_max<K>();  // partner's z[i]
        z[i] = odd ? hs_max(a, pb) : hs_min(a, pb);
        z[j] = odd ? hs_max(b, pa) : hs_min(b, pa);
    }
    if constexpr (P == 1) z[0] = odd ? hs_max(z[0], __shfl_xor_sync(0xffffffffu, z[0], 1))
                                    : hs_min(z[0], __shfl_xor_sync(0xffffffffu, z[0], 1));
    bitonic_half_clean<P>(z);
    if constexpr (X > 0) {
        K e[X];
#pragma unroll
        for (int q = 0; q < X; ++q) e[q] = __shfl_xor_sync(0xffffffffu, z[EO + q], 1);
#pragma unroll
        for (int q = 0; q < EO; ++q) k[q] = odd ? (q < X ? e[q < X ? q : 0] : z[q - X < 0 ? 0 : q - X]) : z[q];
    } else {
#pragma unroll
        for (int q = 0; q < EO; ++q) k[q] = z[q];
    }
}

template <int NT, int EO, int P, bool SKIP, class K, bool WARP = false>
HS_DEV void block_merge_levels(K *s, int *wsplit, K (&k)[EO], int cnt) {
    static_assert(!WARP || NT == 32, "a warp-owned tile has 32 threads");
    constexpr int T = NT * EO;
    const int tid = WARP ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
    const int my0 = tid * EO;
    // 4-byte keys: runs of EO -> 2EO in registers (pairs of adjacent lanes),
    // then the shared-memory levels from 2EO on.  cnt is uniform, so every
    // lane of a warp takes the same branch.  8-byte words keep the shared-
    // memory first level: the register form needs about 14 more registers
    // per thread there, which costs the int64 block sort a resident CTA per
    // SM (7.41 against 7.15 ms at 2^27 keys).
    constexpr bool kRegisterLevel = sizeof(K) == 4;
    if constexpr (kRegisterLevel)
        if (EO < T && EO < cnt) shuffle_first_level<EO, P>(k, (tid & 1) != 0);
    constexpr int W0 = kRegisterLevel ? 2 * EO : EO;
    for (int w = W0; w < T && w < cnt; w *= 2) {
        // While a group of two runs lies inside one warp's slots, the warp
        // only reads what its own lanes wrote: a warp barrier suffices.  The
        // first stores still wait for the whole block, because the caller may
        // have staged the tile in this buffer in another layout (the pair
        // sort reads int32 keys from slots the 64-bit words then overwrite).
        const bool in_warp = 2 * w <= 32 * EO;
        if (WARP || (in_warp && w != W0)) __syncwarp();
        else __syncthreads();
#pragma unroll
        for (int j = 0; j < EO; ++j) s[my0 + j] = k[j];
        if (WARP || in_warp) __syncwarp();
        else __syncthreads();
        const int gs = (my0 / (2 * w)) * (2 * w);
        const int diag = my0 - gs;
        const int alen = hs_min(w, T - gs);
        const int blen = hs_max(hs_min(w, T - gs - w), 0);
        // With no B run (a short last group) B points at A, so the unused
        // window slots still read inside the tile.
        const K *A = s + gs, *B = s + (blen > 0 ? gs + w : gs);
        // A group that starts at or past the live keys holds only sentinels
        // (merges permute keys within their group), so it is already merged:
        // with SKIP (for tiles that are often partly empty) it is left alone.
        const bool live = !SKIP || gs < cnt;
        int lo = diag > blen ? diag - blen : 0;
        int hi = diag < alen ? diag : alen;
        if (!live) lo = hi;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A[mid] <= B[diag - 1 - mid]) lo = mid + 1;
            else hi = mid;
        }
        int end = __shfl_down_sync(0xffffffffu, lo, 1);
        const int dend = diag + EO;  // runs and groups are multiples of EO
        const bool last = dend == alen + blen;
        if (!WARP && 2 * w > 32 * EO) {  // groups span warps: exchange warp-boundary splits
            if ((threadIdx.x & 31) == 0) wsplit[threadIdx.x >> 5] = lo;
            __syncthreads();
            if ((threadIdx.x & 31) == 31 && !last) end = wsplit[(threadIdx.x >> 5) + 1];
        }
        if (last) end = alen;
        if (live) {
            K o[P];
            exact_window_merge<EO, P>(A, lo, B, diag - lo, end - lo, EO, o);
#pragma unroll
            for (int j = 0; j < EO; ++j) k[j] = o[j];
        }
    }
}

// ---------------------------------------------------------------------------
// Keys.  NT threads x EO = LEAVES*L - 1 keys per tile.

template <int NT, int L, int LEAVES = 2>
struct BlockSort3 {
    static_assert(LEAVES == 2 || LEAVES == 4, "two or four leaves per thread");
    static constexpr int EO = LEAVES * L - 1;
    static constexpr int P = pow2_at_least(EO);
    static constexpr int T = NT * EO;
    static constexpr int SZ = T + P + 32 + NT / 32 + 1;  // tile + window slack + warp splits
    static constexpr int SMEM_BYTES = SZ * 4;
};

// With samp, also writes the tile's samples (every kSampleStride-th key,
// samp[(base + q) / S] for q % S == 0; base % S == 0).  SKIP: threads past
// the live keys skip their leaves and merges (for tiles that are often partly
// empty, such as small segments).
template <int NT, int L, int LEAVES = 2, bool SKIP = false>
HS_DEV void block_sort_tile3(const int32_t *kin, int32_t *kout, int cnt, uint32_t netset,
                             bool vec, int32_t *s, int32_t *samp = nullptr, int64_t base = 0) {
    using C = BlockSort3<NT, L, LEAVES>;
    constexpr int EO = C::EO, P = C::P, T = C::T;
    int *wsplit = s + C::T + C::P + 32;  // one split per warp

    if (vec && cnt == T && (T % 4) == 0) {
        const int4 *s4 = reinterpret_cast<const int4 *>(kin);
#pragma unroll 4
        for (int q = threadIdx.x; q < T / 4; q += NT)
            *reinterpret_cast<int4 *>(s + 4 * q) = ld_stream(s4 + q);
    } else {
        for (int i = threadIdx.x; i < T; i += NT) {
            if (i < cnt) cp_async4(s + i, kin + i);
            else s[i] = kKeyMax;
        }
        cp_async_wait_all();
    }
    __syncthreads();

    const int my0 = threadIdx.x * EO;
    int32_t k[EO];
#pragma unroll
    for (int j = 0; j < EO; ++j) k[j] = s[my0 + j];
    if (!SKIP || my0 < cnt) sort_thread_leaves<L, LEAVES, P>(k, cnt - my0, netset);
    block_merge_levels<NT, EO, P, SKIP>(s, wsplit, k, cnt);

    __syncthreads();
#pragma unroll
    for (int j = 0; j < EO; ++j) s[my0 + j] = k[j];
    __syncthreads();
    if (vec && (T % 4) == 0) {
        store_tile_out<NT>(kout, s, cnt, samp, base);
    } else {
        int32_t *sp = samp ? samp + base / kSampleStride : nullptr;
        for (int i = threadIdx.x; i < cnt; i += NT) {
            kout[i] = s[i];
            if (sp && i % kSampleStride == 0) sp[i / kSampleStride] = s[i];
        }
    }
}

// Tile t covers keys [t*T, (t+1)*T); the last tile may be short.  kin/kout
// may alias: each CTA reads its whole tile into shared memory before writing.
// Resident CTAs per SM the register budget must allow (about as many as the
// shared tiles fit): 5 of up to 288 threads, 3 of 512, 2 of 576.
constexpr int blocksort_min_ctas(int nt) { return nt <= 288 ? 5 : nt <= 512 ? 3 : nt <= 576 ? 2 : 1; }

template <int NT, int L, int LEAVES = 2>
__global__ void __launch_bounds__(NT, blocksort_min_ctas(NT))
    k_blocksort3(const int32_t *kin, int32_t *kout, int64_t n, uint32_t netset, int vec,
                 int32_t *samp) {
    constexpr int T = BlockSort3<NT, L, LEAVES>::T;
    static_assert(T % kSampleStride == 0, "tiles start on sample positions");
    extern __shared__ __align__(16) int32_t smem[];
    const int64_t base = (int64_t)blockIdx.x * T;
    const int cnt = (int)((n - base) < T ? (n - base) : T);
    block_sort_tile3<NT, L, LEAVES>(kin + base, kout + base, cnt, netset, vec != 0, smem, samp,
                                    base);
}

// A whole small array [0, n) (n <= the tile) sorted by one CTA of NT
// threads in one launch: leaves and every merge level in shared memory; the
// threads and groups past the live keys skip their work (SKIP).
template <int NT, int L, int LEAVES>
__global__ void __launch_bounds__(NT, 1)
    k_blocksort_small(const int32_t *kin, int32_t *kout, int n, uint32_t netset, int vec) {
    extern __shared__ __align__(16) int32_t smem[];
    block_sort_tile3<NT, L, LEAVES, true>(kin, kout, n, netset, vec != 0, smem);
}

// Bulk-copy form for 16-byte aligned arrays: a full tile arrives by one bulk
// copy (completion counted on an mbarrier) and leaves by one bulk store, and
// each thread writes the samples among its own keys from registers, so the
// load/store units carry only the merge levels' shared-memory traffic.  A
// partial last tile takes block_sort_tile3's plain path.  Same results as
// k_blocksort3.
template <int NT, int L, int LEAVES = 2>
__global__ void __launch_bounds__(NT, blocksort_min_ctas(NT))
    k_blocksort3_bulk(const int32_t *kin, int32_t *kout, int64_t n, uint32_t netset,
                      int32_t *samp, unsigned *status) {
    using C = BlockSort3<NT, L, LEAVES>;
    constexpr int EO = C::EO, P = C::P, T = C::T;
    static_assert(T % kSampleStride == 0 && kSampleStride == 32, "tiles start on sample positions");
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ __align__(8) uint64_t bar;
    const int64_t base = (int64_t)blockIdx.x * T;
    const int cnt = (int)((n - base) < T ? (n - base) : T);
    if (cnt < T) {  // uniform across the CTA
        block_sort_tile3<NT, L, LEAVES>(kin + base, kout + base, cnt, netset, true, smem, samp,
                                        base);
        return;
    }
    int *wsplit = smem + T + P + 32;
    const uint64_t pol = l2_evict_first_policy();
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    // T % 4 == 0 and the arrays are 16-byte aligned: both ends of each copy are.
    const bool aligned16 = (smem_addr(smem) & 15u) == 0 &&
                           ((reinterpret_cast<uintptr_t>(kin + base) |
                             reinterpret_cast<uintptr_t>(kout + base)) & 15u) == 0;
    if (!aligned16) {  // uniform across the CTA: nothing was issued
        if (threadIdx.x == 0) atomicOr(status, kStatusMisaligned);
        return;
    }
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, (unsigned)T * 4u);
        bulk_load(smem, kin + base, (unsigned)T * 4u, &bar, pol);
    }
    const bool ok = mbar_wait(&bar, 0);
    if (__syncthreads_or(!ok)) {  // the copy never landed: report, drain, leave
        if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
        if (!ok) mbar_wait(&bar, 0);
        return;
    }
    const int my0 = threadIdx.x * EO;
    int32_t k[EO];
#pragma unroll
    for (int j = 0; j < EO; ++j) k[j] = smem[my0 + j];
    sort_thread_leaves<L, LEAVES, P>(k, T - my0, netset);
    block_merge_levels<NT, EO, P, false>(smem, wsplit, k, T);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < EO; ++j) smem[my0 + j] = k[j];
    fence_proxy_async_smem();
    if (samp) {
#pragma unroll
        for (int j = 0; j < (EO + 31) / 32; ++j) {
            const int q = ((-my0) & 31) + 32 * j;
            if (q < EO) samp[(base + my0 + q) / kSampleStride] = select_dyn(k, q);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bulk_store(kout + base, smem, (unsigned)T * 4u, pol);
        bulk_wait_read();
    }
}

// ---------------------------------------------------------------------------
// Pairs.  Shared layout: W = sort words [T + P + 32] (int64; during the load
// and the final store its first 2T int32 slots hold keys, then output keys
// and output values), V = input values [T] (int32), then the warp splits.

template <int NT, int L, int LEAVES = 2>
struct BlockSortPairs {
    static_assert(LEAVES == 2 || LEAVES == 4, "two or four leaves per thread");
    static constexpr int EO = LEAVES * L - 1;
    static constexpr int P = pow2_at_least(EO);
    static constexpr int T = NT * EO;
    static constexpr int W_WORDS = T + P + 32;
    static constexpr int SMEM_BYTES = W_WORDS * 8 + T * 4 + (NT / 32 + 1) * 4;
    // The bulk-copy form needs 16-byte aligned key, value and output regions.
    static constexpr bool BULK_OK = T % 4 == 0 && W_WORDS % 2 == 0;
};

template <int NT, int L, int LEAVES = 2>
HS_DEV void block_sort_pairs_tile(const int32_t *kin, int32_t *kout, const int32_t *vin,
                                  int32_t *vout, int cnt, uint32_t netset, bool vec,
                                  int64_t *sw, int32_t *samp, int64_t base) {
    using C = BlockSortPairs<NT, L, LEAVES>;
    constexpr int EO = C::EO, P = C::P, T = C::T;
    int32_t *s32 = reinterpret_cast<int32_t *>(sw);  // 2 * W_WORDS int32 slots
    int32_t *sv = reinterpret_cast<int32_t *>(sw + C::W_WORDS);
    int *wsplit = sv + T;

    if (vec && cnt == T && (T % 4) == 0) {
        const int4 *k4 = reinterpret_cast<const int4 *>(kin);
        const int4 *v4 = reinterpret_cast<const int4 *>(vin);
#pragma unroll 4
        for (int q = threadIdx.x; q < T / 4; q += NT) {
            *reinterpret_cast<int4 *>(s32 + 4 * q) = ld_stream(k4 + q);
            *reinterpret_cast<int4 *>(sv + 4 * q) = ld_stream(v4 + q);
        }
    } else {
        for (int i = threadIdx.x; i < cnt; i += NT) {
            s32[i] = kin[i];
            sv[i] = vin[i];
        }
    }
    __syncthreads();

    const int my0 = threadIdx.x * EO;
    int64_t k[EO];
#pragma unroll
    for (int j = 0; j < EO; ++j)
        k[j] = (my0 + j < cnt) ? pack_word(s32[my0 + j], (uint32_t)(my0 + j)) : word_max<int64_t>();
    sort_thread_leaves<L, LEAVES, P>(k, cnt - my0, netset);
    block_merge_levels<NT, EO, P, false>(sw, wsplit, k, cnt);

    // Output keys to s32[0, T), values (gathered by position) to s32[T, 2T).
    __syncthreads();
#pragma unroll
    for (int j = 0; j < EO; ++j) {
        if (my0 + j < cnt) {
            s32[my0 + j] = word_key(k[j]);
            s32[T + my0 + j] = sv[word_tag(k[j])];
        }
    }
    __syncthreads();
    if (vec && (T % 4) == 0) {
        store_tile_out<NT>(kout, s32, cnt, samp, base);
        store_tile_out<NT>(vout, s32 + T, cnt, nullptr, 0);
    } else {
        int32_t *sp = samp ? samp + base / kSampleStride : nullptr;
        for (int i = threadIdx.x; i < cnt; i += NT) {
            kout[i] = s32[i];
            vout[i] = s32[T + i];
            if (sp && i % kSampleStride == 0) sp[i / kSampleStride] = s32[i];
        }
    }
}

template <int NT, int L, int LEAVES = 2>
__global__ void __launch_bounds__(NT)
    k_blocksort_pairs(const int32_t *kin, int32_t *kout, const int32_t *vin, int32_t *vout,
                      int64_t n, uint32_t netset, int vec, int32_t *samp) {
    constexpr int T = BlockSortPairs<NT, L, LEAVES>::T;
    static_assert(T % kSampleStride == 0, "tiles start on sample positions");
    extern __shared__ __align__(16) int64_t smem64[];
    const int64_t base = (int64_t)blockIdx.x * T;
    const int cnt = (int)((n - base) < T ? (n - base) : T);
    block_sort_pairs_tile<NT, L, LEAVES>(kin + base, kout + base, vin + base, vout + base, cnt,
                                         netset, vec != 0, smem64, samp, base);
}

// Bulk-copy form of the pair block sort for 16-byte aligned arrays: a full
// tile's keys and values arrive by two bulk copies (completion counted on an
// mbarrier) and the sorted keys and gathered values leave by two bulk stores;
// each thread writes the samples among its own keys from registers.  A
// partial last tile takes block_sort_pairs_tile's plain path.  Same results
// as k_blocksort_pairs.
template <int NT, int L, int LEAVES = 2>
__global__ void __launch_bounds__(NT)
    k_blocksort_pairs_bulk(const int32_t *kin, int32_t *kout, const int32_t *vin, int32_t *vout,
                           int64_t n, uint32_t netset, int32_t *samp, unsigned *status) {
    using C = BlockSortPairs<NT, L, LEAVES>;
    constexpr int EO = C::EO, P = C::P, T = C::T;
    static_assert(T % kSampleStride == 0 && kSampleStride == 32, "tiles start on sample positions");
    static_assert(C::BULK_OK, "16-byte aligned key, value and output regions");
    extern __shared__ __align__(16) int64_t smem64[];
    __shared__ __align__(8) uint64_t bar;
    const int64_t base = (int64_t)blockIdx.x * T;
    const int cnt = (int)((n - base) < T ? (n - base) : T);
    if (cnt < T) {  // uniform across the CTA
        block_sort_pairs_tile<NT, L, LEAVES>(kin + base, kout + base, vin + base, vout + base, cnt,
                                             netset, true, smem64, samp, base);
        return;
    }
    int32_t *s32 = reinterpret_cast<int32_t *>(smem64);  // keys in, then output keys and values
    int32_t *sv = reinterpret_cast<int32_t *>(smem64 + C::W_WORDS);  // input values
    int *wsplit = sv + T;
    const uint64_t pol = l2_evict_first_policy();
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    const bool aligned16 = ((smem_addr(s32) | smem_addr(sv)) & 15u) == 0 &&
                           ((reinterpret_cast<uintptr_t>(kin + base) |
                             reinterpret_cast<uintptr_t>(kout + base) |
                             reinterpret_cast<uintptr_t>(vin + base) |
                             reinterpret_cast<uintptr_t>(vout + base)) & 15u) == 0;
    if (!aligned16) {  // uniform across the CTA: nothing was issued
        if (threadIdx.x == 0) atomicOr(status, kStatusMisaligned);
        return;
    }
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, (unsigned)T * 8u);
        bulk_load(s32, kin + base, (unsigned)T * 4u, &bar, pol);
        bulk_load(sv, vin + base, (unsigned)T * 4u, &bar, pol);
    }
    const bool ok = mbar_wait(&bar, 0);
    if (__syncthreads_or(!ok)) {  // a copy never landed: report, drain, leave
        if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
        if (!ok) mbar_wait(&bar, 0);
        return;
    }
    const int my0 = threadIdx.x * EO;
    int64_t k[EO];
#pragma unroll
    for (int j = 0; j < EO; ++j) k[j] = pack_word(s32[my0 + j], (uint32_t)(my0 + j));
    sort_thread_leaves<L, LEAVES, P>(k, T - my0, netset);
    block_merge_levels<NT, EO, P, false>(smem64, wsplit, k, T);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < EO; ++j) {
        s32[my0 + j] = word_key(k[j]);
        s32[T + my0 + j] = sv[word_tag(k[j])];
    }
    fence_proxy_async_smem();
    if (samp) {
#pragma unroll
        for (int j = 0; j < (EO + 31) / 32; ++j) {
            const int q = ((-my0) & 31) + 32 * j;
            if (q < EO) samp[(base + my0 + q) / kSampleStride] = word_key(select_dyn(k, q));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bulk_store(kout + base, s32, (unsigned)T * 4u, pol);
        bulk_store(vout + base, s32 + T, (unsigned)T * 4u, pol);
        bulk_wait_read();
    }
}

}  // namespace hs
