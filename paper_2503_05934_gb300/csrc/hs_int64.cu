// Merge sort of int64 keys: Algorithm 1 with the same network leaves, block
// merge levels and global merge levels as the int32 path, on 8-byte keys.
//
//  * k_blocksort64: one CTA sorts a tile of NT*(4L-1) keys (leaves of L, L,
//    L and L-1 keys per thread, register merges, shared-memory merge levels).
//  * k_merge_partition_sampled64 + k_merge_tile64: one global level; every
//    pass also writes each 32nd key of its output, which the next level's
//    partition searches first.
// Loads and stores are plain coalesced 8-byte accesses, so any 8-byte
// aligned array works.
#include <algorithm>

#include "hs_bulk.cuh"
#include "hs_internal.h"
#include "hs_blocksort.cuh"

namespace hs {

using K64 = int64_t;

template <int NT, int L>
struct BlockSort64 {
    static constexpr int EO = 4 * L - 1;
    static constexpr int P = pow2_at_least(EO);
    static constexpr int T = NT * EO;
    static constexpr int W = T + P + 32 + NT / 32 + 1;  // tile + window slack + warp splits
    static constexpr int SMEM_BYTES = W * 8;
};

template <int NT, int L>
__global__ void __launch_bounds__(NT)
    k_blocksort64(const K64 *kin, K64 *kout, int64_t n, uint32_t netset, K64 *samp, int vec) {
    using C = BlockSort64<NT, L>;
    constexpr int EO = C::EO, P = C::P, T = C::T;
    static_assert(T % kSampleStride == 0, "tiles start on sample positions");
    extern __shared__ __align__(16) K64 s64[];
    int *wsplit = reinterpret_cast<int *>(s64 + T + P + 32);
    const int64_t base = (int64_t)blockIdx.x * T;
    const int cnt = (int)((n - base) < T ? (n - base) : T);
    const K64 *src = kin + base;
    if (vec && cnt == T) {  // T is even: 16-byte loads of two keys
        const int4 *s4 = reinterpret_cast<const int4 *>(src);
        for (int q = threadIdx.x; q < T / 2; q += NT) reinterpret_cast<int4 *>(s64)[q] = ld_stream(s4 + q);
    } else {
        for (int i = threadIdx.x; i < T; i += NT) s64[i] = i < cnt ? ld_stream(src + i) : word_max<K64>();
    }
    __syncthreads();
    const int my0 = threadIdx.x * EO;
    K64 k[EO];
#pragma unroll
    for (int j = 0; j < EO; ++j) k[j] = s64[my0 + j];
    sort_thread_leaves<L, 4, P>(k, cnt - my0, netset);
    block_merge_levels<NT, EO, P, false>(s64, wsplit, k, cnt);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < EO; ++j) s64[my0 + j] = k[j];
    __syncthreads();
    K64 *dst = kout + base;
    for (int i = threadIdx.x; i < cnt; i += NT) {
        st_stream(dst + i, s64[i]);
        if (samp && i % kSampleStride == 0) samp[(base + i) / kSampleStride] = s64[i];
    }
}

// Bulk-copy form for 16-byte aligned arrays: a full tile arrives by one bulk
// copy and leaves by one bulk store; each thread writes the samples among its
// own keys from registers.  A partial last tile takes k_blocksort64's plain
// path (the same code with vec = 0 below).  Same results as k_blocksort64.
template <int NT, int L>
__global__ void __launch_bounds__(NT)
    k_blocksort64_bulk(const K64 *kin, K64 *kout, int64_t n, uint32_t netset, K64 *samp,
                       unsigned *status) {
    using C = BlockSort64<NT, L>;
    constexpr int EO = C::EO, P = C::P, T = C::T;
    static_assert(T % kSampleStride == 0 && kSampleStride == 32, "tiles start on sample positions");
    static_assert(T % 2 == 0, "16-byte aligned tiles");
    extern __shared__ __align__(16) K64 s64[];
    __shared__ __align__(8) uint64_t bar;
    int *wsplit = reinterpret_cast<int *>(s64 + T + P + 32);
    const int64_t base = (int64_t)blockIdx.x * T;
    const int cnt = (int)((n - base) < T ? (n - base) : T);
    if (cnt < T) {  // uniform across the CTA: element-wise staging as in k_blocksort64
        for (int i = threadIdx.x; i < T; i += NT) s64[i] = i < cnt ? ld_stream(kin + base + i) : word_max<K64>();
        __syncthreads();
    } else {
        const uint64_t pol = l2_evict_first_policy();
        if (threadIdx.x == 0) mbar_init(&bar, 1);
        __syncthreads();
        const bool aligned16 = (smem_addr(s64) & 15u) == 0 &&
                               ((reinterpret_cast<uintptr_t>(kin + base) |
                                 reinterpret_cast<uintptr_t>(kout + base)) & 15u) == 0;
        if (!aligned16) {  // uniform across the CTA: nothing was issued
            if (threadIdx.x == 0) atomicOr(status, kStatusMisaligned);
            return;
        }
        if (threadIdx.x == 0) {
            mbar_arrive_expect_tx(&bar, (unsigned)T * 8u);
            bulk_load(s64, kin + base, (unsigned)T * 8u, &bar, pol);
        }
        const bool ok = mbar_wait(&bar, 0);
        if (__syncthreads_or(!ok)) {  // the copy never landed: report, drain, leave
            if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
            if (!ok) mbar_wait(&bar, 0);
            return;
        }
    }
    const int my0 = threadIdx.x * EO;
    K64 k[EO];
#pragma unroll
    for (int j = 0; j < EO; ++j) k[j] = s64[my0 + j];
    sort_thread_leaves<L, 4, P>(k, cnt - my0, netset);
    block_merge_levels<NT, EO, P, false>(s64, wsplit, k, cnt);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < EO; ++j) s64[my0 + j] = k[j];
    if (cnt < T) {
        __syncthreads();
        K64 *dst = kout + base;
        for (int i = threadIdx.x; i < cnt; i += NT) {
            st_stream(dst + i, s64[i]);
            if (samp && i % kSampleStride == 0) samp[(base + i) / kSampleStride] = s64[i];
        }
        return;
    }
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
        bulk_store(kout + base, s64, (unsigned)T * 8u, l2_evict_first_policy());
        bulk_wait_read();
    }
}

// Sampled merge-path partition (the int32 form's search on 8-byte keys).
static __global__ void k_merge_partition_sampled64(const K64 *in, const K64 *samp, int64_t n,
                                                   int64_t w, int to, int tpg, int64_t nblocks,
                                                   int64_t *part) {
    constexpr int64_t S = kSampleStride;
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    int64_t g = b / tpg, t = b - g * tpg;
    MergeGeom m = merge_geom(g, n, w);
    int64_t diag = t * to;
    if (diag > m.alen + m.blen) diag = m.alen + m.blen;
    const K64 *A = in + m.gs;
    const K64 *B = in + m.gs + w;
    int64_t lo = diag > m.blen ? diag - m.blen : 0;
    int64_t hi = diag < m.alen ? diag : m.alen;
    if (lo < hi) {
        const K64 *SA = samp + m.gs / S, *SB = samp + (m.gs + w) / S;
        const int64_t m0 = (lo + S - 1) / S, m1 = (hi - 1) / S;
        if (m0 <= m1) {
            int64_t fl = m0, fh = m1 + 1, tl = m0, th = m1 + 1;
            while (fl < fh || tl < th) {
                if (fl < fh) {
                    const int64_t fm = (fl + fh) >> 1;
                    const int64_t j = diag - 1 - fm * S;
                    if (SA[fm] <= SB[j / S]) fl = fm + 1;
                    else fh = fm;
                }
                if (tl < th) {
                    const int64_t tm = (tl + th) >> 1;
                    const int64_t j = diag - 1 - tm * S;
                    const int64_t ju = (j + S - 1) / S;
                    if (ju * S < m.blen && SA[tm] > SB[ju]) th = tm;
                    else tl = tm + 1;
                }
            }
            if (fl > m0) lo = hs_max(lo, (fl - 1) * S + 1);
            if (tl <= m1) hi = hs_min(hi, tl * S);
        }
    }
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (A[mid] <= B[diag - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    part[b] = lo;
}

// One global level: the tile's A and B ranges are staged back to back in
// shared memory, each thread merges exactly its own EO outputs (exact-window
// bitonic merge of 8-byte keys), and the outputs leave through shared memory.
template <int NT, int EO>
struct TileMerge64 {
    static constexpr int P = pow2_at_least(EO);
    static constexpr int TO = NT * EO;
    // A's and B's 16-byte covers back to back (at most one extra key at each
    // end of each) + the window slack.
    static constexpr int REG = TO + 4 + P;
    static constexpr int SMEM_BYTES = REG * 8;
};

// Thread-staged form (any 8-byte alignment, any n): the tile's A and B keys
// are loaded into shared memory by the threads and the outputs leave by
// plain stores.
template <int NT, int EO>
__global__ void __launch_bounds__(NT)
    k_merge_tile64(const K64 *in, K64 *out, int64_t n, int64_t w, const int64_t *part, int tpg,
                   K64 *samp) {
    using C = TileMerge64<NT, EO>;
    constexpr int TO = C::TO, P = C::P;
    extern __shared__ __align__(16) K64 s64[];
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
    const K64 *gA = in + m.gs + a0, *gB = in + m.gs + w + (o0 - a0);
    for (int q = threadIdx.x; q < tot; q += NT) s64[q] = ld_stream(q < na ? gA + q : gB + (q - na));
    __syncthreads();
    const K64 *A = s64, *B = s64 + na;

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
    K64 x[P];
    const int cnt = dend - dcl;
    if (cnt > 0) exact_window_merge<EO, P>(A, lo, B, dcl - lo, end - lo, cnt, x);
    __syncthreads();
    if (cnt > 0) {
#pragma unroll
        for (int k = 0; k < EO; ++k)
            if (k < cnt) s64[diag + k] = x[k];
    }
    __syncthreads();
    K64 *dst = out + m.gs + o0;
    for (int i = threadIdx.x; i < tot; i += NT) {
        st_stream(dst + i, s64[i]);
        if (samp && i % kSampleStride == 0) samp[(m.gs + o0 + i) / kSampleStride] = s64[i];
    }
}

// Bulk-copy form for 16-byte aligned buffers with n even: one thread issues
// the two cover copies (cp.async.bulk, completion counted on an mbarrier)
// and, once the tile is merged, one bulk store of the output tile; each
// thread writes the samples among its own outputs from registers.  Same
// merge and results as k_merge_tile64.
template <int NT, int EO>
__global__ void __launch_bounds__(NT)
    k_merge_tile64_bulk(const K64 *in, K64 *out, int64_t n, int64_t w, const int64_t *part,
                        int tpg, K64 *samp, unsigned *status) {
    using C = TileMerge64<NT, EO>;
    constexpr int TO = C::TO, P = C::P;
    static_assert(kSampleStride == 32, "sample positions are multiples of 32");
    extern __shared__ __align__(16) K64 s64[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int wsplit[NT / 32 + 1];
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
    const int64_t ca = ga & ~int64_t(1), cb = gb & ~int64_t(1);
    const int nca = (int)(((ga + na + 1) & ~int64_t(1)) - ca) / 2;  // 16-byte words
    const int ncb = (int)(((gb + nb + 1) & ~int64_t(1)) - cb) / 2;
    const uint64_t pol = l2_evict_first_policy();
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    const bool aligned16 = (smem_addr(s64) & 15u) == 0 &&
                           ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
    if (!aligned16) {  // uniform across the CTA: nothing was issued
        if (threadIdx.x == 0) atomicOr(status, kStatusMisaligned);
        return;
    }
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, (unsigned)(nca + ncb) * 16u);
        if (nca > 0) bulk_load(s64, in + ca, (unsigned)nca * 16u, &bar, pol);
        if (ncb > 0) bulk_load(s64 + 2 * nca, in + cb, (unsigned)ncb * 16u, &bar, pol);
    }
    const bool ok = mbar_wait(&bar, 0);
    if (__syncthreads_or(!ok)) {  // a copy never landed: report, drain, leave
        if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
        if (!ok) mbar_wait(&bar, 0);
        return;
    }
    const K64 *A = s64 + (int)(ga - ca);
    const K64 *B = s64 + 2 * nca + (int)(gb - cb);

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
    K64 x[P];
    const int cnt = dend - dcl;
    if (cnt > 0) exact_window_merge<EO, P>(A, lo, B, dcl - lo, end - lo, cnt, x);
    __syncthreads();
    if (cnt > 0) {
#pragma unroll
        for (int k = 0; k < EO; ++k)
            if (k < cnt) s64[diag + k] = x[k];
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
        // 16-byte aligned: m.gs + o0 and tot are even.
        bulk_store(out + m.gs + o0, s64, (unsigned)tot * 8u, pol);
        bulk_wait_read();
    }
}

// ---------------------------------------------------------------- planner

// Block sort: 256 threads x four leaves (7936 keys for {6,7,8}).  A 288-thread
// tile (8928 keys) would save a global level at powers of two, as it does for
// int32 keys, but on 8-byte keys its block sort costs more than that level:
// 3.05 against 2.37 ms at 2^27 keys, 8.63 against 8.35 ms for the whole sort.
constexpr int B64_NT = 256;
constexpr int M64_NT = 96, M64_EO = 31;      // merge level: 96 threads x 31 keys

int64_t tile64(int L, int64_t) { return (int64_t)B64_NT * (4 * L - 1); }

// Tile copies: the bulk-copy forms (k_blocksort64_bulk for 16-byte aligned
// arrays, k_merge_tile64_bulk when the buffers are 16-byte aligned and n is
// even), else the thread-staged block sort and levels.

size_t merge_workspace_bytes_i64(size_t n) {
    return ws_align(n * sizeof(K64)) + merge_ws_part_bytes(n) + ws_align((n / 32 + 8) * sizeof(K64));
}

template <int L>
static hs_status launch_blocksort64_t(const K64 *kin, K64 *kout, int64_t n, hs_netset s, K64 *samp,
                                      cudaStream_t st) {
    const int vec = aligned(kin, 16) ? 1 : 0;
    using C = BlockSort64<B64_NT, L>;
    const unsigned grid = (unsigned)((n + C::T - 1) / C::T);
    hs_status r;
    if (vec && aligned(kout, 16)) {
        unsigned *status = nullptr;
        if ((r = device_status(&status)) != HS_OK) return r;
        auto kern = k_blocksort64_bulk<B64_NT, L>;
        if ((r = ensure_smem((const void *)kern, C::SMEM_BYTES)) != HS_OK) return r;
        LaunchToken t = launch_begin(K_BLOCKSORT_KEYS, st);
        kern<<<grid, B64_NT, C::SMEM_BYTES, st>>>(kin, kout, n, s, samp, status);
        return launch_end(t);
    }
    auto kern = k_blocksort64<B64_NT, L>;
    if ((r = ensure_smem((const void *)kern, C::SMEM_BYTES)) != HS_OK) return r;
    LaunchToken t = launch_begin(K_BLOCKSORT_KEYS, st);
    kern<<<grid, B64_NT, C::SMEM_BYTES, st>>>(kin, kout, n, s, samp, vec);
    return launch_end(t);
}

static hs_status launch_blocksort64(int L, const K64 *kin, K64 *kout, int64_t n, hs_netset s,
                                    K64 *samp, cudaStream_t st) {
    switch (L) {
        case 1: return launch_blocksort64_t<1>(kin, kout, n, s, samp, st);
        case 3: return launch_blocksort64_t<3>(kin, kout, n, s, samp, st);
        case 4: return launch_blocksort64_t<4>(kin, kout, n, s, samp, st);
        case 5: return launch_blocksort64_t<5>(kin, kout, n, s, samp, st);
        case 6: return launch_blocksort64_t<6>(kin, kout, n, s, samp, st);
        case 7: return launch_blocksort64_t<7>(kin, kout, n, s, samp, st);
        case 8: return launch_blocksort64_t<8>(kin, kout, n, s, samp, st);
    }
    return fail(HS_ERR_INVALID_ARG, "leaf size outside 1, 3..8");
}

hs_status merge_sort_i64(int64_t *d_keys, size_t n_, hs_netset s, void *d_ws, size_t ws_bytes,
                         cudaStream_t st) {
    const int64_t n = (int64_t)n_;
    const int L = leaf_size(s);
    const int64_t T = tile64(L, n);
    int passes = 0;
    for (int64_t w = T; w < n; w *= 2) ++passes;

    K64 *kbuf = nullptr, *samp = nullptr;
    int64_t *part = nullptr;
    if (passes > 0) {
        if (!d_ws || ws_bytes < merge_workspace_bytes_i64(n_))
            return fail(HS_ERR_INVALID_ARG, "int64 sort: workspace smaller than hs_sort_i64_workspace_bytes");
        if (!aligned(d_ws, 16)) return fail(HS_ERR_INVALID_ARG, "int64 sort: workspace not 16-byte aligned");
        char *p = static_cast<char *>(d_ws);
        kbuf = reinterpret_cast<K64 *>(p);
        part = reinterpret_cast<int64_t *>(p + ws_align(n_ * sizeof(K64)));
        samp = reinterpret_cast<K64 *>(p + ws_align(n_ * sizeof(K64)) + merge_ws_part_bytes(n_));
    }
    // Land the last level in the caller's array.
    K64 *kcur = (passes % 2 == 0) ? d_keys : kbuf;
    K64 *kalt = (kcur == d_keys) ? kbuf : d_keys;
    hs_status r = launch_blocksort64(L, d_keys, kcur, n, s, samp, st);
    if (r != HS_OK) return r;
    using C = TileMerge64<M64_NT, M64_EO>;
    static_assert(C::TO % kSampleStride == 0, "output tiles start on sample positions");
    const bool vec = aligned(d_keys, 16) && (!kbuf || aligned(kbuf, 16)) && (n % 2) == 0;
    const bool bulk = vec;
    auto kern = k_merge_tile64<M64_NT, M64_EO>;
    auto kern_bulk = k_merge_tile64_bulk<M64_NT, M64_EO>;
    unsigned *status = nullptr;
    if (bulk && passes > 0 && (r = device_status(&status)) != HS_OK) return r;
    for (int64_t w = T; w < n; w *= 2) {
        const LevelTiles lt = level_tiles(n, w, C::TO);
        LaunchToken t = launch_begin(K_MERGE_PARTITION, st);
        k_merge_partition_sampled64<<<(unsigned)((lt.nblocks + 255) / 256), 256, 0, st>>>(
            kcur, samp, n, w, C::TO, (int)lt.tpg, lt.nblocks, part);
        if ((r = launch_end(t)) != HS_OK) return r;
        if ((r = ensure_smem(bulk ? (const void *)kern_bulk : (const void *)kern, C::SMEM_BYTES)) != HS_OK)
            return r;
        t = launch_begin(K_MERGE_KEYS, st);
        if (bulk)
            kern_bulk<<<(unsigned)lt.nblocks, M64_NT, C::SMEM_BYTES, st>>>(kcur, kalt, n, w, part,
                                                                           (int)lt.tpg, samp, status);
        else
            kern<<<(unsigned)lt.nblocks, M64_NT, C::SMEM_BYTES, st>>>(kcur, kalt, n, w, part,
                                                                      (int)lt.tpg, samp);
        if ((r = launch_end(t)) != HS_OK) return r;
        std::swap(kcur, kalt);
    }
    return HS_OK;
}

}  // namespace hs
