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

}  // namespace hs
