// Merge-sort kernels: the GPU form of Algorithm 1 (Optimized Merge Sort with
// Sorting Networks).
//
//  * k_blocksort: one CTA sorts a tile of NT*L keys.  Each thread's L
//    consecutive keys form one leaf, sorted in registers by the size-L network
//    ("ApplySortingNetwork"); then log2(NT) merge-path levels in shared memory
//    merge the leaves into one sorted tile ("Merge", bottom levels).
//  * k_merge_partition + k_merge_pass: one global level of Merge.  Runs of
//    width w are merged pairwise into runs of 2w; each CTA writes one output
//    tile of NT*E keys whose inputs are located by a merge-path search.
//
// Stability (pairs): networks order (key, position); every merge takes the
// left run's element on ties, which keeps equal keys in input order.
#pragma once

#include "hs_common.cuh"
#include "hs_networks.cuh"

namespace hs {

// Sorts a bitonic sequence x[0..E) ascending (half-cleaners of decreasing
// distance, Batcher 1968).
template <int E>
HS_DEV void bitonic_half_clean(int32_t (&x)[E]) {
#pragma unroll
    for (int d = E / 2; d > 0; d >>= 1) {
#pragma unroll
        for (int i = 0; i < E; ++i) {
            if ((i & d) == 0) {
                int32_t lo = hs_min(x[i], x[i + d]);
                int32_t hi = hs_max(x[i], x[i + d]);
                x[i] = lo;
                x[i + d] = hi;
            }
        }
    }
}

// Merge-path split (Odeh, Green, Mwassi, Shmueli, Birk, "Merge Path -
// Parallel Merging Made Simple", IPDPSW 2012): the number of elements of run
// A among the first `diag` outputs of the stable merge of A and B.
template <bool PAD>
HS_DEV int merge_path(const int32_t *s, int a0, int na, int b0, int nb, int diag) {
    int lo = diag > nb ? diag - nb : 0;
    int hi = diag < na ? diag : na;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int ia = a0 + mid, ib = b0 + diag - 1 - mid;
        int32_t ka = s[PAD ? pad32(ia) : ia];
        int32_t kb = s[PAD ? pad32(ib) : ib];
        if (ka <= kb) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The cnt (<= EO) outputs of one thread as a sorted run: its merge-path split
// (ai, bi) and end split (ai + na) are known, so it reads exactly its na keys
// of A (ascending) and cnt - na keys of B (descending), with +infinity padding
// between them, which is one bitonic sequence of P keys; a P-wide bitonic
// merge sorts it.  Only ties between equal keys can land in either order,
// which keys alone cannot show.
template <int EO, int P>
HS_DEV void exact_window_merge(const int32_t *A, int ai, const int32_t *B, int bi, int na,
                               int cnt, int32_t (&x)[P]) {
    const int tb = P - (cnt - na);  // first slot of the descending B part
    const int32_t *pa = A + ai, *pb = B + bi;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        // One load per slot, always inside the thread's own keys: A ascending,
        // B descending, +infinity in between (those slots load B[bi] and
        // discard it).
        const int32_t v = (i < na) ? pa[i] : pb[(i >= tb) ? (P - 1 - i) : 0];
        x[i] = (i < na || i >= tb) ? v : kKeyMax;
    }
    bitonic_half_clean<P>(x);
}

// Merge-path split of two separate sorted arrays.
HS_DEV int merge_path2(const int32_t *A, int na, const int32_t *B, int nb, int diag) {
    int lo = diag > nb ? diag - nb : 0;
    int hi = diag < na ? diag : na;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (A[mid] <= B[diag - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Sequential stable merge of E outputs from shared memory, starting at the
// merge-path split (ai in A = [.., aend), bi in B = [.., bend)).  One shared
// load per output; it may read one element past either run, so every buffer
// keeps one word of slack.
template <int E, bool PAD, bool PAIRS>
HS_DEV void serial_merge(const int32_t *sk, const int32_t *sv, int ai, int aend, int bi,
                         int bend, int32_t (&k)[E], int32_t (&v)[E]) {
    int32_t ka = sk[PAD ? pad32(ai) : ai];
    int32_t kb = sk[PAD ? pad32(bi) : bi];
#pragma unroll
    for (int j = 0; j < E; ++j) {
        bool take_b = (bi < bend) && ((ai >= aend) || (kb < ka));
        int src = take_b ? bi : ai;
        k[j] = take_b ? kb : ka;
        if constexpr (PAIRS) v[j] = sv[PAD ? pad32(src) : src];
        bi += take_b;
        ai += !take_b;
        int nxt = take_b ? bi : ai;
        int32_t kn = sk[PAD ? pad32(nxt) : nxt];
        kb = take_b ? kn : kb;
        ka = take_b ? ka : kn;
    }
}

// Tile loader into padded shared memory; keys past cnt become `fill`.
template <int T, int NT>
HS_DEV void load_tile_padded(const int32_t *src, int cnt, int32_t *s, bool vec, int32_t fill) {
    if (vec && cnt == T) {
        const int4 *s4 = reinterpret_cast<const int4 *>(src);
#pragma unroll 4
        for (int q = threadIdx.x; q < T / 4; q += NT) {
            int4 x = ld_stream(s4 + q);
            int i = 4 * q;
            s[pad32(i)] = x.x;
            s[pad32(i + 1)] = x.y;
            s[pad32(i + 2)] = x.z;
            s[pad32(i + 3)] = x.w;
        }
    } else {
        for (int i = threadIdx.x; i < T; i += NT) s[pad32(i)] = i < cnt ? src[i] : fill;
    }
}

// Writes the first cnt keys of a padded shared tile to global memory.
template <int NT>
HS_DEV void store_tile_padded(int32_t *dst, int cnt, const int32_t *s, bool vec) {
    int start = 0;
    if (vec) {
        int n4 = cnt >> 2;
        int4 *d4 = reinterpret_cast<int4 *>(dst);
        for (int q = threadIdx.x; q < n4; q += NT) {
            int i = 4 * q;
            int4 x = make_int4(s[pad32(i)], s[pad32(i + 1)], s[pad32(i + 2)], s[pad32(i + 3)]);
            st_stream(d4 + q, x);
        }
        start = n4 * 4;
    }
    for (int i = start + threadIdx.x; i < cnt; i += NT) dst[i] = s[pad32(i)];
}

template <int NT, int L>
constexpr int blocksort_smem_words() {
    return NT * L + (NT * L) / 32 + 1;
}

// ---------------------------------------------------------------------------
// Block sort of one tile of cnt <= NT*L keys (kin -> kout, which may alias;
// values ride along when PAIRS).  Positions past cnt are padded with
// sentinels and never written back.  Merge levels stop once one run covers
// every live key: the remaining runs hold only sentinels.
template <int NT, int L, bool PAIRS>
HS_DEV void block_sort_tile(const int32_t *kin, int32_t *kout, const int32_t *vin,
                            int32_t *vout, int cnt, uint32_t netset, bool vec, int32_t *smem) {
    constexpr int T = NT * L;
    constexpr int SZ = blocksort_smem_words<NT, L>();
    int32_t *sk = smem;
    int32_t *sv = smem + SZ;

    load_tile_padded<T, NT>(kin, cnt, sk, vec, kKeyMax);
    if constexpr (PAIRS) load_tile_padded<T, NT>(vin, cnt, sv, vec, 0);
    __syncthreads();

    const int my0 = threadIdx.x * L;
    int32_t k[L], v[L], p[L];
#pragma unroll
    for (int j = 0; j < L; ++j) {
        k[j] = sk[pad32(my0 + j)];
        if constexpr (PAIRS) {
            v[j] = sv[pad32(my0 + j)];
            p[j] = my0 + j;
        }
    }

    // Leaves: "if size matches a sorting network size, apply it".
    if constexpr (L > 1) {
        if constexpr (PAIRS) {
            PairCE op{k, v, p};
            if (my0 + L <= cnt) network<L>(op);
            else if (my0 < cnt) network_dyn(ragged_net_size(cnt - my0, netset), op);
        } else {
            KeyCE op{k};
            if (my0 + L <= cnt) network<L>(op);
            else if (my0 < cnt) network_dyn(ragged_net_size(cnt - my0, netset), op);
        }
    }

    // Merge levels inside the tile: runs of w keys -> 2w keys.
    for (int w = L; w < T && w < cnt; w *= 2) {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < L; ++j) {
            sk[pad32(my0 + j)] = k[j];
            if constexpr (PAIRS) sv[pad32(my0 + j)] = v[j];
        }
        __syncthreads();
        const int gs = (my0 / (2 * w)) * (2 * w);
        const int diag = my0 - gs;
        const int ai = merge_path<true>(sk, gs, w, gs + w, w, diag);
        serial_merge<L, true, PAIRS>(sk, sv, gs + ai, gs + w, gs + w + diag - ai, gs + 2 * w,
                                     k, v);
    }

    __syncthreads();
#pragma unroll
    for (int j = 0; j < L; ++j) {
        sk[pad32(my0 + j)] = k[j];
        if constexpr (PAIRS) sv[pad32(my0 + j)] = v[j];
    }
    __syncthreads();
    store_tile_padded<NT>(kout, cnt, sk, vec);
    if constexpr (PAIRS) store_tile_padded<NT>(vout, cnt, sv, vec);
}

// Block sort.  Tile t covers keys [t*NT*L, (t+1)*NT*L); the last tile may be
// short.  kin/kout may alias: each CTA reads its whole tile into shared
// memory before writing.
template <int NT, int L, bool PAIRS>
__global__ void __launch_bounds__(NT)
    k_blocksort(const int32_t *kin, int32_t *kout, const int32_t *vin, int32_t *vout,
                int64_t n, uint32_t netset, int vec) {
    constexpr int T = NT * L;
    extern __shared__ int32_t smem[];
    const int64_t base = (int64_t)blockIdx.x * T;
    const int cnt = (int)((n - base) < T ? (n - base) : T);
    block_sort_tile<NT, L, PAIRS>(kin + base, kout + base, PAIRS ? vin + base : nullptr,
                                  PAIRS ? vout + base : nullptr, cnt, netset, vec != 0, smem);
}


// ---------------------------------------------------------------------------
// Block sort, two leaves per thread (keys).  Each of the NT threads holds
// E = 2L consecutive keys: two leaves of L keys, each sorted by the size-L
// network, then merged in registers by a bitonic merge.  The shared-memory
// levels then merge runs of w -> 2w: every thread finds its merge-path split
// and forms its E outputs as the lower half of a bitonic merge of the two
// E-key windows at the split (no dependent load chain).
//
// Shared layout: logical index i lives at i + 4*(i/32), which keeps the
// threads' 16-byte accesses to their own E keys free of bank conflicts.

HS_HD constexpr int pow2_at_least(int x) {
    int p = 1;
    while (p < x) p *= 2;
    return p;
}

// Padded shared index for the keys block sort: one pad word after every 8.
// Merge windows of neighbouring threads start about 8 keys apart; the pad
// puts their k-th words on different banks.
HS_DEV int pad4(int i) { return i + (i >> 3); }

template <int NT, int L>
struct BlockSort2 {
    static constexpr int E = 2 * L;
    static constexpr int P = pow2_at_least(E);
    static constexpr int T = NT * E;
    static constexpr int SZ = T + T / 8 + 64;  // padded tile (1 word per 8) + window slack
    static constexpr int SMEM_BYTES = SZ * 4;
};

// Full bitonic merge of two sorted runs of n <= P/2 keys held in x[0..n) and
// x[n..2n); the result (ascending) is written back to x[0..2n).
template <int N, int P>
HS_DEV void register_merge_two(int32_t *x) {
    int32_t lo[P / 2], hi[P / 2];
#pragma unroll
    for (int i = 0; i < P / 2; ++i) {
        const int32_t a = i < N ? x[i] : kKeyMax;
        const int j = P / 2 - 1 - i;  // reversed second run
        const int32_t b = j < N ? x[N + j] : kKeyMax;
        lo[i] = hs_min(a, b);
        hi[i] = hs_max(a, b);
    }
    bitonic_half_clean<P / 2>(lo);
    bitonic_half_clean<P / 2>(hi);
#pragma unroll
    for (int i = 0; i < 2 * N; ++i) x[i] = i < P / 2 ? lo[i] : hi[i - P / 2];
}

// A thread's own E keys at logical [my0, my0 + E): 16-byte accesses when E is
// a multiple of 4 (my0 is then a multiple of 4 and no group of 4 crosses a
// padding point).
template <int E>
HS_DEV void read_own(const int32_t *s, int my0, int32_t (&k)[E]) {
    if constexpr (false) {
#pragma unroll
        for (int q = 0; q < E / 4; ++q) {
            const int4 v = *reinterpret_cast<const int4 *>(s + pad4(my0 + 4 * q));
            k[4 * q] = v.x;
            k[4 * q + 1] = v.y;
            k[4 * q + 2] = v.z;
            k[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) k[j] = s[pad4(my0 + j)];
    }
}

template <int E>
HS_DEV void write_own(int32_t *s, int my0, const int32_t (&k)[E]) {
    if constexpr (false) {
#pragma unroll
        for (int q = 0; q < E / 4; ++q)
            *reinterpret_cast<int4 *>(s + pad4(my0 + 4 * q)) =
                make_int4(k[4 * q], k[4 * q + 1], k[4 * q + 2], k[4 * q + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) s[pad4(my0 + j)] = k[j];
    }
}

template <int NT, int L>
HS_DEV void block_sort_tile2(const int32_t *kin, int32_t *kout, int cnt, uint32_t netset,
                             bool vec, int32_t *s) {
    using C = BlockSort2<NT, L>;
    constexpr int E = C::E, P = C::P, T = C::T;

    // Load the tile (sentinels past cnt).
    if (vec && cnt == T) {
        const int4 *s4 = reinterpret_cast<const int4 *>(kin);
#pragma unroll 4
        for (int q = threadIdx.x; q < T / 4; q += NT) {
            const int4 v = ld_stream(s4 + q);
            const int i = pad4(4 * q);  // 4 consecutive keys never straddle a pad word
            s[i] = v.x;
            s[i + 1] = v.y;
            s[i + 2] = v.z;
            s[i + 3] = v.w;
        }
    } else {
        for (int i = threadIdx.x; i < T; i += NT) s[pad4(i)] = i < cnt ? kin[i] : kKeyMax;
    }
    __syncthreads();

    const int my0 = threadIdx.x * E;
    int32_t k[E];
    read_own<E>(s, my0, k);

    // Leaves ("ApplySortingNetwork" on each of the thread's two leaves).
    if constexpr (L > 1) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            KeyCE op{k + h * L};
            const int r = cnt - (my0 + h * L);
            if (r >= L) network<L>(op);
            else if (r > 0) network_dyn(ragged_net_size(r, netset), op);
        }
    }
    register_merge_two<L, P>(k);

    // Shared-memory merge levels (padded layout throughout).
    for (int w = E; w < T && w < cnt; w *= 2) {
        __syncthreads();
        write_own<E>(s, my0, k);
        __syncthreads();
        const int gs = ((E & (E - 1)) == 0) ? (my0 & ~(2 * w - 1)) : (my0 / (2 * w)) * (2 * w);
        const int diag = my0 - gs;
        int lo = diag > w ? diag - w : 0;
        int hi = diag < w ? diag : w;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s[pad4(gs + mid)] <= s[pad4(gs + w + diag - 1 - mid)]) lo = mid + 1;
            else hi = mid;
        }
        const int a0 = gs + lo, b0 = gs + w + diag - lo;
        const int ra = w - lo, rb = w - (diag - lo);
        int32_t o[P];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const int j = P - 1 - i;
            const int32_t a = (i < E && i < ra) ? s[pad4(a0 + i)] : kKeyMax;
            const int32_t b = (j < E && j < rb) ? s[pad4(b0 + j)] : kKeyMax;
            o[i] = hs_min(a, b);
        }
        bitonic_half_clean<P>(o);
#pragma unroll
        for (int j = 0; j < E; ++j) k[j] = o[j];
    }

    __syncthreads();
    write_own<E>(s, my0, k);
    __syncthreads();
    if (vec) {
        const int n4 = cnt >> 2;
        int4 *d4 = reinterpret_cast<int4 *>(kout);
        for (int q = threadIdx.x; q < n4; q += NT) {
            const int i = pad4(4 * q);
            st_stream(d4 + q, make_int4(s[i], s[i + 1], s[i + 2], s[i + 3]));
        }
        for (int i = 4 * n4 + threadIdx.x; i < cnt; i += NT) kout[i] = s[pad4(i)];
    } else {
        for (int i = threadIdx.x; i < cnt; i += NT) kout[i] = s[pad4(i)];
    }
}

template <int NT, int L>
__global__ void __launch_bounds__(NT)
    k_blocksort2(const int32_t *kin, int32_t *kout, int64_t n, uint32_t netset, int vec) {
    constexpr int T = BlockSort2<NT, L>::T;
    extern __shared__ __align__(16) int32_t smem[];
    const int64_t base = (int64_t)blockIdx.x * T;
    const int cnt = (int)((n - base) < T ? (n - base) : T);
    block_sort_tile2<NT, L>(kin + base, kout + base, cnt, netset, vec != 0, smem);
}

// ---------------------------------------------------------------------------
// Block sort, odd form (keys).  Each of the NT threads holds EO = 2L - 1
// consecutive keys as two leaves: one of L keys and one of L - 1 keys, each
// sorted by its network ("ApplySortingNetwork"; a leaf size that is not in
// the set is padded with +infinity sentinels up to the next size that is, the
// same rule as a ragged leaf), then merged in registers.  For the {6,7,8} set
// the leaves are 8 and 7 keys, both sizes in the set.
//
// The shared-memory levels merge runs of w -> 2w; every thread finds its
// merge-path split and forms its EO outputs as the lowest EO of the lower half
// of a P-wide bitonic merge of the two windows at the split.  Because EO is
// odd, neighbouring threads' windows and their own EO-key slots fall on
// different banks, so the tile is stored unpadded.

template <int NT, int L, int LEAVES = 2>
struct BlockSort3 {
    static_assert(LEAVES == 2 || LEAVES == 4, "two or four leaves per thread");
    static constexpr int EO = LEAVES * L - 1;
    static constexpr int P = pow2_at_least(EO);
    static constexpr int T = NT * EO;
    static constexpr int SZ = T + P + 32 + NT / 32 + 1;  // tile + window slack + warp splits
    static constexpr int SMEM_BYTES = SZ * 4;
};

// Sorts leaf x[0..N) in registers (N live keys at most; r of them real).
template <int N>
HS_DEV void sort_leaf(int32_t *x, int r, uint32_t netset) {
    if (r <= 1) return;
    const int m = ragged_net_size(r, netset);  // r if r is in the set, else the next size up
    if (m == N && r == N) {
        KeyCE op{x};
        network<N>(op);
        return;
    }
    // Pad to the network size with sentinels (never stored), sort, copy back.
    int32_t t[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) t[i] = (i < N && i < r) ? x[i < N ? i : 0] : kKeyMax;
    KeyCE op{t};
    network_dyn(m, op);
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = t[i];
}

// Bitonic merge of sorted x[0..N1) and x[N1..N1+N2) (N1, N2 <= P/2) in
// registers; the ascending result goes back to x[0..N1+N2).
template <int N1, int N2, int P>
HS_DEV void register_merge(int32_t *x) {
    int32_t lo[P / 2], hi[P / 2];
#pragma unroll
    for (int i = 0; i < P / 2; ++i) {
        const int32_t a = i < N1 ? x[i] : kKeyMax;
        const int j = P / 2 - 1 - i;  // second run, reversed
        const int32_t b = j < N2 ? x[N1 + (j < N2 ? j : 0)] : kKeyMax;
        lo[i] = hs_min(a, b);
        hi[i] = hs_max(a, b);
    }
    bitonic_half_clean<P / 2>(lo);
    bitonic_half_clean<P / 2>(hi);
#pragma unroll
    for (int i = 0; i < N1 + N2; ++i) x[i] = i < P / 2 ? lo[i] : hi[i - P / 2];
}

template <int NT, int L, int LEAVES = 2>
HS_DEV void block_sort_tile3(const int32_t *kin, int32_t *kout, int cnt, uint32_t netset,
                             bool vec, int32_t *s) {
    using C = BlockSort3<NT, L, LEAVES>;
    constexpr int EO = C::EO, P = C::P, T = C::T;
    int *wsplit = s + C::T + C::P + 32;  // one split per warp

    if (vec && cnt == T && (T % 4) == 0) {
        const int4 *s4 = reinterpret_cast<const int4 *>(kin);
#pragma unroll 4
        for (int q = threadIdx.x; q < T / 4; q += NT)
            *reinterpret_cast<int4 *>(s + 4 * q) = ld_stream(s4 + q);
    } else {
        for (int i = threadIdx.x; i < T; i += NT) s[i] = i < cnt ? kin[i] : kKeyMax;
    }
    __syncthreads();

    const int my0 = threadIdx.x * EO;
    int32_t k[EO];
#pragma unroll
    for (int j = 0; j < EO; ++j) k[j] = s[my0 + j];

    if constexpr (LEAVES == 2 && L > 1) {
        const int r0 = hs_min(hs_max(cnt - my0, 0), L);
        const int r1 = hs_min(hs_max(cnt - my0 - L, 0), L - 1);
        sort_leaf<L>(k, r0, netset);
        sort_leaf<L - 1>(k + L, r1, netset);
        register_merge<L, L - 1, P>(k);
    } else if constexpr (LEAVES == 4) {
        // Leaves of L, L, L and L - 1 keys (for L = 1: single keys, merged).
        if constexpr (L > 1) {
#pragma unroll
            for (int h = 0; h < 3; ++h)
                sort_leaf<L>(k + h * L, hs_min(hs_max(cnt - my0 - h * L, 0), L), netset);
            sort_leaf<L - 1>(k + 3 * L, hs_min(hs_max(cnt - my0 - 3 * L, 0), L - 1), netset);
        }
        register_merge<L, L, P / 2>(k);
        register_merge<L, L - 1, P / 2>(k + 2 * L);
        register_merge<2 * L, 2 * L - 1, P>(k);
    }

    for (int w = EO; w < T && w < cnt; w *= 2) {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < EO; ++j) s[my0 + j] = k[j];
        __syncthreads();
        const int gs = (my0 / (2 * w)) * (2 * w);
        const int diag = my0 - gs;
        const int32_t *A = s + gs, *B = s + gs + w;
        int lo = diag > w ? diag - w : 0;
        int hi = diag < w ? diag : w;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A[mid] <= B[diag - 1 - mid]) lo = mid + 1;
            else hi = mid;
        }
        // End split: the next lane's start inside the same group, all of A at
        // the group's end, or (the warp's last lane) the next warp's first
        // lane's start, passed through shared memory.
        int end = __shfl_down_sync(0xffffffffu, lo, 1);
        const int dend = diag + EO;  // 2w is a multiple of EO
        if (2 * w > 32 * EO) {  // groups span warps: exchange warp-boundary splits
            if ((threadIdx.x & 31) == 0) wsplit[threadIdx.x >> 5] = lo;
            __syncthreads();
            if ((threadIdx.x & 31) == 31 && dend != 2 * w) end = wsplit[(threadIdx.x >> 5) + 1];
        }
        if (dend == 2 * w) end = w;
        int32_t o[P];
        exact_window_merge<EO, P>(A, lo, B, diag - lo, end - lo, EO, o);
#pragma unroll
        for (int j = 0; j < EO; ++j) k[j] = o[j];
    }

    __syncthreads();
#pragma unroll
    for (int j = 0; j < EO; ++j) s[my0 + j] = k[j];
    __syncthreads();
    if (vec && (T % 4) == 0) {
        const int n4 = cnt >> 2;
        int4 *d4 = reinterpret_cast<int4 *>(kout);
        for (int q = threadIdx.x; q < n4; q += NT)
            st_stream(d4 + q, *reinterpret_cast<const int4 *>(s + 4 * q));
        for (int i = 4 * n4 + threadIdx.x; i < cnt; i += NT) kout[i] = s[i];
    } else {
        for (int i = threadIdx.x; i < cnt; i += NT) kout[i] = s[i];
    }
}

template <int NT, int L, int LEAVES = 2>
__global__ void __launch_bounds__(NT)
    k_blocksort3(const int32_t *kin, int32_t *kout, int64_t n, uint32_t netset, int vec) {
    constexpr int T = BlockSort3<NT, L, LEAVES>::T;
    extern __shared__ __align__(16) int32_t smem[];
    const int64_t base = (int64_t)blockIdx.x * T;
    const int cnt = (int)((n - base) < T ? (n - base) : T);
    block_sort_tile3<NT, L, LEAVES>(kin + base, kout + base, cnt, netset, vec != 0, smem);
}

// ---------------------------------------------------------------------------
// Global merge level.  Group g merges A = [g*2w, g*2w+w) with
// B = [g*2w+w, g*2w+2w) (both clipped to n).  Each group is cut into tpg
// output tiles of TO keys; block b = g*tpg + t writes tile t of group g.

struct MergeGeom {
    int64_t gs, alen, blen;
};

HS_DEV MergeGeom merge_geom(int64_t g, int64_t n, int64_t w) {
    MergeGeom m;
    m.gs = g * 2 * w;
    int64_t rest = n - m.gs;
    m.alen = rest < w ? rest : w;
    int64_t brest = rest - w;
    m.blen = brest <= 0 ? 0 : (brest < w ? brest : w);
    return m;
}

// part[b] = number of A elements before output tile b's first output.
static __global__ void k_merge_partition(const int32_t *in, int64_t n, int64_t w, int to, int tpg,
                                  int64_t nblocks, int64_t *part) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    int64_t g = b / tpg, t = b - g * tpg;
    MergeGeom m = merge_geom(g, n, w);
    int64_t diag = t * to;
    if (diag > m.alen + m.blen) diag = m.alen + m.blen;
    const int32_t *A = in + m.gs;
    const int32_t *B = in + m.gs + w;
    int64_t lo = diag > m.blen ? diag - m.blen : 0;
    int64_t hi = diag < m.alen ? diag : m.alen;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (A[mid] <= B[diag - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    part[b] = lo;
}

template <int NT, int E>
constexpr int merge_smem_words() {
    return NT * E + (NT * E) / 32 + 1;
}

template <int NT, int E, bool PAIRS>
__global__ void __launch_bounds__(NT)
    k_merge_pass(const int32_t *kin, int32_t *kout, const int32_t *vin, int32_t *vout,
                 int64_t n, int64_t w, const int64_t *part, int tpg, int vec) {
    constexpr int TO = NT * E;
    constexpr int SZ = merge_smem_words<NT, E>();
    extern __shared__ int32_t smem[];
    int32_t *sk = smem;
    int32_t *sv = smem + SZ;

    const int64_t g = blockIdx.x / tpg;
    const int t = blockIdx.x - (int)(g * tpg);
    const MergeGeom m = merge_geom(g, n, w);
    const int64_t glen = m.alen + m.blen;
    const int64_t o0 = (int64_t)t * TO;
    if (o0 >= glen) return;
    const int64_t o1 = (o0 + TO) < glen ? (o0 + TO) : glen;
    const int64_t a0 = part[blockIdx.x];
    const int64_t a1 = (o1 == glen) ? m.alen : part[blockIdx.x + 1];
    const int na = (int)(a1 - a0);
    const int tot = (int)(o1 - o0);
    const int64_t b0 = o0 - a0;

    // Stage A[a0, a1) then B[b0, b1) contiguously; all loads in flight first.
    {
        const int32_t *A = kin + m.gs + a0;
        const int32_t *B = kin + m.gs + w + b0 - na;  // B[i - na] for i >= na
        int32_t tk[E], tv[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            int i = threadIdx.x + j * NT;
            const int32_t *src = i < na ? A + i : B + i;
            if (i < tot) {
                tk[j] = ld_stream(src);
                if constexpr (PAIRS) tv[j] = ld_stream(src - kin + vin);
            }
        }
#pragma unroll
        for (int j = 0; j < E; ++j) {
            int i = threadIdx.x + j * NT;
            if (i < tot) {
                sk[i] = tk[j];
                if constexpr (PAIRS) sv[i] = tv[j];
            }
        }
    }
    __syncthreads();

    const int diag = threadIdx.x * E;
    int32_t k[E], v[E];
    if (diag < tot) {
        const int nb = tot - na;
        const int ai = merge_path<false>(sk, 0, na, na, nb, diag);
        serial_merge<E, false, PAIRS>(sk, sv, ai, na, na + diag - ai, tot, k, v);
    }
    __syncthreads();
    if (diag < tot) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            sk[pad32(diag + j)] = k[j];
            if constexpr (PAIRS) sv[pad32(diag + j)] = v[j];
        }
    }
    __syncthreads();
    store_tile_padded<NT>(kout + m.gs + o0, tot, sk, vec);
    if constexpr (PAIRS) store_tile_padded<NT>(vout + m.gs + o0, tot, sv, vec);
}

// ---------------------------------------------------------------------------
// Global merge level, tiled form (keys; 16-byte aligned buffers, n % 4 == 0).
//
// One CTA per output tile of TO = NT*EO keys (the partition pass gives its
// merge-path split), many CTAs per SM for latency hiding.  The tile's A and B
// ranges are staged in shared memory by 16-byte asynchronous copies
// (cp.async) of their 16-byte-aligned covers; each thread then forms its EO
// outputs from the lower half of a P-wide bitonic merge of its two windows
// and stores them directly.  EO is odd so that neighbouring threads' windows
// start on different banks.

HS_DEV void cp_async16(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}
HS_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

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
                 int tpg) {
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
    // Stage the outputs (odd stride EO: conflict-free) for coalesced stores.
    __syncthreads();
    if (diag < tot) {
#pragma unroll
        for (int k = 0; k < EO; ++k) sA[diag + k] = o[k];
    }
    __syncthreads();
    int32_t *dst = out + m.gs + o0;  // 16-byte aligned: gs and o0 are multiples of 4
    const int n4 = tot >> 2;
    for (int q = threadIdx.x; q < n4; q += NT)
        st_stream(reinterpret_cast<int4 *>(dst) + q, *reinterpret_cast<const int4 *>(sA + 4 * q));
    for (int i = 4 * n4 + threadIdx.x; i < tot; i += NT) st_stream(dst + i, sA[i]);
}

// ---------------------------------------------------------------------------
// Global merge level, tiled exact-window form (keys; 16-byte aligned buffers,
// n % 4 == 0).  Like k_merge_tile, but each thread merges exactly its own EO
// keys: its end split comes from the next lane (a shuffle), or from one extra
// search in the warp's last lane, so the windows read each key once.
template <int NT, int EO>
struct TileMerge2 {
    static constexpr int EOUT = EO;
    static constexpr int P = pow2_at_least(EO);
    static constexpr int TO = NT * EO;
    // A's and B's 16-byte aligned covers back to back: na + nb = TO keys plus
    // at most 3 extra keys at each end of each cover.
    static constexpr int REG = TO + 16;
    static constexpr int SMEM_BYTES = REG * 4;
};

template <int NT, int EO>
__global__ void __launch_bounds__(NT)
    k_merge_tile2(const int32_t *in, int32_t *out, int64_t n, int64_t w, const int64_t *part,
                  int tpg) {
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
    // End split: the next lane's start, or (the warp's last lane) the next
    // warp's first lane's start through shared memory; the tile end takes
    // all of A.
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
    const int n4 = tot >> 2;
    for (int q = threadIdx.x; q < n4; q += NT)
        st_stream(reinterpret_cast<int4 *>(dst) + q, *reinterpret_cast<const int4 *>(sA + 4 * q));
    for (int i = 4 * n4 + threadIdx.x; i < tot; i += NT) st_stream(dst + i, sA[i]);
}


}  // namespace hs
