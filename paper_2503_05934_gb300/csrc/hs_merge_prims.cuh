// Merge primitives shared by the merge-sort kernels (Algorithm 1, "Merge"):
// bitonic merging networks on register arrays, merge-path splits, the
// exact-window merge of one thread's outputs, the global-level geometry and
// its partition pass, and the generic (any alignment, keys or pairs) merge
// pass.
//
// Stability (pairs): every merge takes the left run's element on ties, which
// keeps equal keys in input order.
#pragma once

#include "hs_common.cuh"

namespace hs {

HS_HD constexpr int pow2_at_least(int x) {
    int p = 1;
    while (p < x) p *= 2;
    return p;
}

// Largest value of a sort word: +infinity sentinel of padded slots.
template <class K>
HS_HD constexpr K word_max();
template <>
HS_HD constexpr int32_t word_max<int32_t>() { return INT32_MAX; }
template <>
HS_HD constexpr int64_t word_max<int64_t>() { return INT64_MAX; }

// A pair sort word: the key in the high half and a tie-break tag (a position)
// in the low half, so that the signed 64-bit order is the (key, tag) order.
HS_HD int64_t pack_word(int32_t key, uint32_t tag) {
    return (int64_t)(((uint64_t)(uint32_t)key << 32) | tag);
}
HS_HD int32_t word_key(int64_t w) { return (int32_t)(w >> 32); }
HS_HD uint32_t word_tag(int64_t w) { return (uint32_t)(uint64_t)w; }

// Sorts a bitonic sequence x[0..E) ascending (half-cleaners of decreasing
// distance, Batcher 1968).
template <int E, class K>
HS_DEV void bitonic_half_clean(K (&x)[E]) {
#pragma unroll
    for (int d = E / 2; d > 0; d >>= 1) {
#pragma unroll
        for (int i = 0; i < E; ++i) {
            if ((i & d) == 0) {
                K lo = hs_min(x[i], x[i + d]);
                K hi = hs_max(x[i], x[i + d]);
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

// Merge-path split of two separate sorted arrays (keys or unique words).
template <class K>
HS_DEV int merge_path2(const K *A, int na, const K *B, int nb, int diag) {
    int lo = diag > nb ? diag - nb : 0;
    int hi = diag < na ? diag : na;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (A[mid] <= B[diag - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The cnt (<= EO) outputs of one thread as a sorted run: its merge-path split
// (ai, bi) and end split (ai + na) are known, so it reads exactly its na keys
// of A (ascending) and cnt - na keys of B (descending), with +infinity padding
// between them, which is one bitonic sequence of P keys; a P-wide bitonic
// merge sorts it.  Only ties between equal keys can land in either order,
// which keys alone cannot show.  Works on keys or on unique sort words.
//
// Every slot issues one load at a constant offset from A + ai or from
// B + bi + P - 1, and the +infinity slots discard theirs: those loads reach
// up to P - 1 words past the thread's last B key, so every buffer read this
// way keeps P words of slack after its B runs.
template <int EO, int P, class K>
HS_DEV void exact_window_merge(const K *A, int ai, const K *B, int bi, int na, int cnt,
                               K (&x)[P]) {
    const int tb = P - (cnt - na);  // first slot of the descending B part
    const K *pa = A + ai, *pb = B + bi + (P - 1);
#pragma unroll
    for (int i = 0; i < P; ++i) {
        const K v = (i < na) ? pa[i] : pb[-i];
        x[i] = (i < na || i >= tb) ? v : word_max<K>();
    }
    bitonic_half_clean<P>(x);
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

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned).
HS_DEV void cp_async16(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}
// Four-byte asynchronous copy (any 4-byte aligned address): a loop of these
// keeps every load of a staged tile in flight at once, where a loop of plain
// load-then-store waits out one memory latency per iteration.
HS_DEV void cp_async4(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}
HS_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Global merge level.  Group g merges A = [g*2w, g*2w+w) with
// B = [g*2w+w, g*2w+2w) (both clipped to n).  Each group is cut into tpg
// output tiles of TO keys; block b = g*tpg + t writes tile t of group g.

struct MergeGeom {
    int64_t gs, alen, blen;
};

HS_HD MergeGeom merge_geom(int64_t g, int64_t n, int64_t w) {
    MergeGeom m;
    m.gs = g * 2 * w;
    int64_t rest = n - m.gs;
    m.alen = rest < w ? rest : w;
    int64_t brest = rest - w;
    m.blen = brest <= 0 ? 0 : (brest < w ? brest : w);
    return m;
}

// Output tiles of one global level: groups of 2w keys cut into tiles of TO.
struct LevelTiles {
    int64_t tpg, nblocks;
};
HS_HD LevelTiles level_tiles(int64_t n, int64_t w, int64_t to) {
    const int64_t span = 2 * w;
    const int64_t ngroups = (n + span - 1) / span;
    const int64_t last = n - (ngroups - 1) * span;
    LevelTiles t;
    t.tpg = (span + to - 1) / to;
    t.nblocks = (ngroups - 1) * t.tpg + (last + to - 1) / to;
    return t;
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

// Sampled form for arrays whose runs start at multiples of kSampleStride:
// samp[j] = in[j * kSampleStride] (written by the kernel that produced `in`,
// and small enough to stay in L2).  Two interleaved binary searches over the
// samples narrow [lo, hi] from both sides with conclusions that hold for the
// unsampled keys too; the exact search then finishes in the array.  At a
// candidate split i = m*S (S = kSampleStride), with j = diag - 1 - i:
//   A[i] <= Bs[floor(j/S)] <= B[j]   proves A[i] <= B[j]  (split above i),
//   A[i] >  Bs[ceil(j/S)]  >= B[j]   proves A[i] >  B[j]  (split at most i),
// and both tests are monotone in m.  Same result as k_merge_partition.
constexpr int kSampleStride = 32;

// Merge-path split by one warp (32-ary search): the smallest i in [lo, hi]
// with A[i] > B[diag - 1 - i] (hi when there is none), the number of A
// elements among the first diag outputs of the stable merge.  Each round the
// lanes test 32 evenly spaced candidates (two independent loads each) and the
// range shrinks 32-fold, so a 65536-key range takes about four dependent load
// rounds instead of sixteen.  The final round starts with fewer than 32
// candidates left, so the last lane always tests a position >= hi and the
// ballot is never empty.  Every lane returns the result.
HS_DEV int64_t warp_merge_path(const int32_t *A, const int32_t *B, int64_t diag, int64_t lo,
                               int64_t hi, int lane) {
    while (hi - lo >= 32) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t q = lo + (int64_t)(lane + 1) * step;  // candidate; q >= hi counts as true
        const bool t = q >= hi || A[q] > B[diag - 1 - q];
        const unsigned m = __ballot_sync(0xffffffffu, t);
        const int f = __ffs(m) - 1;  // some lane holds q >= hi, so m != 0
        const int64_t nlo = f == 0 ? lo : lo + (int64_t)f * step + 1;
        hi = hs_min(hi, lo + (int64_t)(f + 1) * step);
        lo = nlo;
    }
    const int64_t q = lo + lane;
    const bool t = q >= hi || A[q] > B[diag - 1 - q];
    const unsigned m = __ballot_sync(0xffffffffu, t);
    return lo + (__ffs(m) - 1);
}

// Levels of at most this many output tiles (about 17.8M keys: both buffers
// of such a level fit the 129 MB L2) search their splits inside the merge
// tiles (SELF_SPLIT) instead of a partition pass.  Measured per sort, with /
// without: 25K keys 40.6 / 47 us, 100K 50 / 71 us, 1M 68.7 / 117.6 us, 4M 146
// / 219 us, 16M 0.497 / 0.513 ms; past L2 the searches go to DRAM and lose:
// 64M keys (16,900 tiles) 1.963 / 1.697 ms.  Stable pairs (the same
// 3968-pair tiles): 100K 67 / 88 us, 1M 99 / 154 us, 4M 249 / 323 us, 16M
// 937 / 980 us.
constexpr int64_t kSelfSplitMaxTiles = 4500;

// A merge tile's own two splits (the number of A keys before its first and
// after its last output), found by warps 0 and 1, one boundary each, with
// 32-ary searches: o0 and o1 are the tile's output range in its group of
// runs A (alen keys at keys + gs) and B (blen keys at keys + gs + w), and a
// tile that ends its group takes all of A.  Every thread of the CTA calls it
// (it holds a barrier); the CTA needs at least two warps.
HS_DEV void tile_self_split(const int32_t *keys, int64_t gs, int64_t w, int64_t alen, int64_t blen,
                            int64_t o0, int64_t o1, int64_t *a0, int64_t *a1) {
    __shared__ int64_t s_split[2];
    const int wp = (int)(threadIdx.x >> 5);
    if (wp < 2) {
        const int64_t diag = wp == 0 ? o0 : o1;
        const int64_t lo = diag > blen ? diag - blen : 0;
        const int64_t hi = diag < alen ? diag : alen;
        const int64_t r = (wp == 1 && o1 == alen + blen)
                              ? alen
                              : warp_merge_path(keys + gs, keys + gs + w, diag, lo, hi,
                                                (int)(threadIdx.x & 31));
        if ((threadIdx.x & 31) == 0) s_split[wp] = r;
    }
    __syncthreads();
    *a0 = s_split[0];
    *a1 = s_split[1];
}

static __global__ void k_merge_partition_sampled(const int32_t *in, const int32_t *samp,
                                                 int64_t n, int64_t w, int to, int tpg,
                                                 int64_t nblocks, int64_t *part) {
    constexpr int64_t S = kSampleStride;
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
    if (lo < hi) {
        const int32_t *SA = samp + m.gs / S, *SB = samp + (m.gs + w) / S;
        const int64_t m0 = (lo + S - 1) / S, m1 = (hi - 1) / S;  // candidates m*S in [lo, hi - 1]
        if (m0 <= m1) {
            int64_t fl = m0, fh = m1 + 1;  // first m whose lower-bound test fails
            int64_t tl = m0, th = m1 + 1;  // first m whose upper-bound test holds
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

// Stores a tile staged in shared memory, s[0, cnt), to dst (16-byte aligned)
// as 16-byte streaming stores.  With samp, also writes the tile's samples
// samp[(base + q) / S] = s[q] for q % S == 0 (base % S == 0), taken from the
// lanes whose 16-byte word starts on a sample, so no extra shared-memory
// reads (which would all fall on one bank).
template <int NT>
HS_DEV void store_tile_out(int32_t *dst, const int32_t *s, int cnt, int32_t *samp, int64_t base) {
    constexpr int Q = kSampleStride / 4;  // 16-byte words per sample
    const int n4 = cnt >> 2;
    int32_t *sp = samp ? samp + base / kSampleStride : nullptr;
    for (int q = threadIdx.x; q < n4; q += NT) {
        const int4 v = *reinterpret_cast<const int4 *>(s + 4 * q);
        st_stream(reinterpret_cast<int4 *>(dst) + q, v);
        if (sp && q % Q == 0) sp[q / Q] = v.x;
    }
    for (int i = 4 * n4 + threadIdx.x; i < cnt; i += NT) {
        st_stream(dst + i, s[i]);
        if (sp && i % kSampleStride == 0) sp[i / kSampleStride] = s[i];
    }
}

// ---------------------------------------------------------------------------
// Generic global merge level (any alignment; keys, or pairs with PAIRS): one
// CTA per output tile of NT*E keys, staged in padded shared memory and merged
// by per-thread serial merges from their merge-path splits.

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

}  // namespace hs
