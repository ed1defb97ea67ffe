// Host planner of the merge path (Algorithm 1 on the GPU): one block-sort
// launch, then per global level a partition launch and a merge launch,
// ping-ponging between the caller's array and the workspace so that the last
// level lands in the caller's array.
#include <algorithm>
#include <mutex>

#include "hs_internal.h"
#include "hs_merge_kernels.cuh"

namespace hs {


// Block sort: 1024 threads, one leaf of L keys each -> tiles of 1024*L keys
// (8192 for the {6,7,8} set).  Merge levels: 256 threads x 16 keys (keys) or
// 256 x 8 (pairs) per output tile.
constexpr int BS_NT = 1024;
constexpr int MK_NT = 256, MK_E = 16;
constexpr int MP_NT = 256, MP_E = 8;

// Output tiles per pass are at most n/TO + n/(2T) + 1 <= n/1024 + 2 for the
// smallest TO (2048) and tile (1024); one more entry closes the last tile.
static size_t partition_entries(size_t n) { return n / 1024 + 8; }

size_t merge_workspace_bytes(size_t n, int with_values) {
    size_t kb = align_up(n * sizeof(int32_t), 256);
    return kb + (with_values ? kb : 0) + align_up(partition_entries(n) * sizeof(int64_t), 256);
}

template <int L, bool PAIRS>
static hs_status launch_blocksort_t(const int32_t *kin, int32_t *kout, const int32_t *vin,
                                    int32_t *vout, int64_t n, hs_netset s, int vec,
                                    cudaStream_t st) {
    constexpr int T = BS_NT * L;
    const int smem = blocksort_smem_words<BS_NT, L>() * (int)sizeof(int32_t) * (PAIRS ? 2 : 1);
    auto kern = k_blocksort<BS_NT, L, PAIRS>;
    hs_status r = ensure_smem((const void *)kern, smem);
    if (r != HS_OK) return r;
    const int64_t grid = (n + T - 1) / T;
    LaunchToken t = launch_begin(PAIRS ? K_BLOCKSORT_PAIRS : K_BLOCKSORT_KEYS, st);
    kern<<<(unsigned)grid, BS_NT, smem, st>>>(kin, kout, vin, vout, n, s, vec);
    return launch_end(t);
}

// Keys: block_sort_tile3 with two leaves (L, L-1) or four leaves (L, L, L,
// L-1) per thread.  Shapes (option "blocksort_shape"):
//   0: 512 threads x 2 leaves   1: 1024 x 2   2: 256 x 4 (default)   3: 512 x 4
static int g_bs_shape = 2;

static int bs_threads() { return (g_bs_shape == 1) ? 1024 : (g_bs_shape == 2) ? 256 : 512; }
static int bs_leaves() { return g_bs_shape >= 2 ? 4 : 2; }

int64_t keys_tile(int L) { return (int64_t)bs_threads() * (bs_leaves() * L - 1); }

void merge_set_blocksort_threads(int nt) { g_bs_shape = (nt == 1024) ? 1 : 0; }
void merge_set_blocksort_shape(int v) { g_bs_shape = v; }

template <int NT, int L, int LEAVES>
static hs_status launch_blocksort2_t(const int32_t *kin, int32_t *kout, int64_t n, hs_netset s,
                                     int vec, cudaStream_t st) {
    using C = BlockSort3<NT, L, LEAVES>;
    auto kern = k_blocksort3<NT, L, LEAVES>;
    hs_status r = ensure_smem((const void *)kern, C::SMEM_BYTES);
    if (r != HS_OK) return r;
    const int64_t grid = (n + C::T - 1) / C::T;
    LaunchToken t = launch_begin(K_BLOCKSORT_KEYS, st);
    kern<<<(unsigned)grid, NT, C::SMEM_BYTES, st>>>(kin, kout, n, s, vec);
    return launch_end(t);
}

template <int NT, int LEAVES>
static hs_status launch_blocksort2_nt(int L, const int32_t *kin, int32_t *kout, int64_t n,
                                      hs_netset s, int vec, cudaStream_t st) {
    switch (L) {
        case 1: return launch_blocksort2_t<NT, 1, LEAVES>(kin, kout, n, s, vec, st);
        case 3: return launch_blocksort2_t<NT, 3, LEAVES>(kin, kout, n, s, vec, st);
        case 4: return launch_blocksort2_t<NT, 4, LEAVES>(kin, kout, n, s, vec, st);
        case 5: return launch_blocksort2_t<NT, 5, LEAVES>(kin, kout, n, s, vec, st);
        case 6: return launch_blocksort2_t<NT, 6, LEAVES>(kin, kout, n, s, vec, st);
        case 7: return launch_blocksort2_t<NT, 7, LEAVES>(kin, kout, n, s, vec, st);
        case 8: return launch_blocksort2_t<NT, 8, LEAVES>(kin, kout, n, s, vec, st);
    }
    return fail(HS_ERR_INVALID_ARG, "leaf size outside 1, 3..8");
}

template <bool PAIRS>
static hs_status launch_blocksort(int L, const int32_t *kin, int32_t *kout, const int32_t *vin,
                                  int32_t *vout, int64_t n, hs_netset s, int vec, cudaStream_t st) {
    if constexpr (!PAIRS) {
        switch (g_bs_shape) {
            case 1: return launch_blocksort2_nt<1024, 2>(L, kin, kout, n, s, vec, st);
            case 2: return launch_blocksort2_nt<256, 4>(L, kin, kout, n, s, vec, st);
            case 3: return launch_blocksort2_nt<512, 4>(L, kin, kout, n, s, vec, st);
            default: return launch_blocksort2_nt<512, 2>(L, kin, kout, n, s, vec, st);
        }
    }
    switch (L) {
        case 1: return launch_blocksort_t<1, PAIRS>(kin, kout, vin, vout, n, s, vec, st);
        case 3: return launch_blocksort_t<3, PAIRS>(kin, kout, vin, vout, n, s, vec, st);
        case 4: return launch_blocksort_t<4, PAIRS>(kin, kout, vin, vout, n, s, vec, st);
        case 5: return launch_blocksort_t<5, PAIRS>(kin, kout, vin, vout, n, s, vec, st);
        case 6: return launch_blocksort_t<6, PAIRS>(kin, kout, vin, vout, n, s, vec, st);
        case 7: return launch_blocksort_t<7, PAIRS>(kin, kout, vin, vout, n, s, vec, st);
        case 8: return launch_blocksort_t<8, PAIRS>(kin, kout, vin, vout, n, s, vec, st);
    }
    return fail(HS_ERR_INVALID_ARG, "leaf size outside 1, 3..8");
}

hs_status blocksort_launch(int L, const int32_t *kin, int32_t *kout, int64_t n, hs_netset s,
                           int vec, cudaStream_t st) {
    return launch_blocksort<false>(L, kin, kout, nullptr, nullptr, n, s, vec, st);
}

// Keys with 16-byte aligned buffers and n % 4 == 0: the streaming bulk-copy
// merge kernel (option "merge_kernel" 1, the default); otherwise, or with
// option 0, the staged-load kernel with a partition pass.
static int g_merge_tile = 2;

void merge_set_tile(int v) { g_merge_tile = v; }

// Partition pass + one tiled merge launch for one level (keys).
template <auto KERN, class C>
static hs_status launch_tile(const int32_t *kin, int32_t *kout, int64_t n, int64_t w,
                             int64_t *part, cudaStream_t st) {
    constexpr int TTO = C::TO;
    const int64_t span = 2 * w;
    const int64_t ngroups = (n + span - 1) / span;
    const int64_t last = n - (ngroups - 1) * span;
    const int64_t ttpg = (span + TTO - 1) / TTO;
    const int64_t tnb = (ngroups - 1) * ttpg + (last + TTO - 1) / TTO;
    LaunchToken t = launch_begin(K_MERGE_PARTITION, st);
    k_merge_partition<<<(unsigned)((tnb + 255) / 256), 256, 0, st>>>(kin, n, w, TTO, (int)ttpg, tnb,
                                                                     part);
    hs_status r = launch_end(t);
    if (r != HS_OK) return r;
    if ((r = ensure_smem((const void *)KERN, C::SMEM_BYTES)) != HS_OK) return r;
    constexpr int NTH = C::TO / C::EOUT;
    t = launch_begin(K_MERGE_KEYS, st);
    KERN<<<(unsigned)tnb, NTH, C::SMEM_BYTES, st>>>(kin, kout, n, w, part, (int)ttpg);
    return launch_end(t);
}
static int g_merge_kernel = 1;

void merge_set_kernel(int k) { g_merge_kernel = k; }

template <int NT, int E, bool PAIRS>
static hs_status launch_merge_level(const int32_t *kin, int32_t *kout, const int32_t *vin,
                                    int32_t *vout, int64_t n, int64_t w, int64_t *part, int vec,
                                    cudaStream_t st) {
    constexpr int TO = NT * E;
    const int64_t span = 2 * w;
    const int64_t ngroups = (n + span - 1) / span;
    const int64_t tpg = (span + TO - 1) / TO;
    const int64_t last = n - (ngroups - 1) * span;
    const int64_t nblocks = (ngroups - 1) * tpg + (last + TO - 1) / TO;

    hs_status r = HS_OK;
    LaunchToken t;
    if (!PAIRS && vec && g_merge_kernel == 1 && (n % 4) == 0) {
        switch (g_merge_tile) {
            case 0: return launch_tile<k_merge_tile<256, 15>, TileMerge<256, 15>>(kin, kout, n, w, part, st);
            case 1: return launch_tile<k_merge_tile2<64, 31>, TileMerge2<64, 31>>(kin, kout, n, w, part, st);
            case 2: return launch_tile<k_merge_tile2<128, 31>, TileMerge2<128, 31>>(kin, kout, n, w, part, st);
            case 3: return launch_tile<k_merge_tile2<64, 63>, TileMerge2<64, 63>>(kin, kout, n, w, part, st);
            case 4: return launch_tile<k_merge_tile2<128, 23>, TileMerge2<128, 23>>(kin, kout, n, w, part, st);
            case 5: return launch_tile<k_merge_tile2<96, 31>, TileMerge2<96, 31>>(kin, kout, n, w, part, st);
            default: return launch_tile<k_merge_tile2<192, 31>, TileMerge2<192, 31>>(kin, kout, n, w, part, st);
        }
    }
    t = launch_begin(K_MERGE_PARTITION, st);
    k_merge_partition<<<(unsigned)((nblocks + 255) / 256), 256, 0, st>>>(kin, n, w, TO, (int)tpg,
                                                                         nblocks, part);
    r = launch_end(t);
    if (r != HS_OK) return r;

    const int smem = merge_smem_words<NT, E>() * (int)sizeof(int32_t) * (PAIRS ? 2 : 1);
    auto kern = k_merge_pass<NT, E, PAIRS>;
    r = ensure_smem((const void *)kern, smem);
    if (r != HS_OK) return r;
    t = launch_begin(PAIRS ? K_MERGE_PAIRS : K_MERGE_KEYS, st);
    kern<<<(unsigned)nblocks, NT, smem, st>>>(kin, kout, vin, vout, n, w, part, (int)tpg, vec);
    return launch_end(t);
}

hs_status merge_sort(int32_t *d_keys, int32_t *d_vals, size_t n_, hs_netset s, void *d_ws,
                     size_t ws_bytes, cudaStream_t st) {
    const bool pairs = d_vals != nullptr;
    const int64_t n = (int64_t)n_;
    const int L = leaf_size(s);
    const int64_t T = pairs ? (int64_t)BS_NT * L : keys_tile(L);
    int passes = 0;
    for (int64_t w = T; w < n; w *= 2) ++passes;

    int32_t *kbuf = nullptr, *vbuf = nullptr;
    int64_t *part = nullptr;
    if (passes > 0) {
        if (!d_ws || ws_bytes < merge_workspace_bytes(n_, pairs))
            return fail(HS_ERR_INVALID_ARG, "merge sort: workspace smaller than hs_sort_workspace_bytes");
        if (!aligned(d_ws, 16)) return fail(HS_ERR_INVALID_ARG, "merge sort: workspace not 16-byte aligned");
        char *p = static_cast<char *>(d_ws);
        size_t kb = align_up(n_ * sizeof(int32_t), 256);
        kbuf = reinterpret_cast<int32_t *>(p);
        p += kb;
        if (pairs) {
            vbuf = reinterpret_cast<int32_t *>(p);
            p += kb;
        }
        part = reinterpret_cast<int64_t *>(p);
    }
    const int vec = aligned(d_keys, 16) && (!pairs || aligned(d_vals, 16)) ? 1 : 0;

    // Land the last level in the caller's array: with an even number of
    // global levels the block sort writes in place.
    int32_t *kcur = (passes % 2 == 0) ? d_keys : kbuf;
    int32_t *vcur = pairs ? ((passes % 2 == 0) ? d_vals : vbuf) : nullptr;
    int32_t *kalt = (kcur == d_keys) ? kbuf : d_keys;
    int32_t *valt = pairs ? ((vcur == d_vals) ? vbuf : d_vals) : nullptr;

    hs_status r = pairs ? launch_blocksort<true>(L, d_keys, kcur, d_vals, vcur, n, s, vec, st)
                        : launch_blocksort<false>(L, d_keys, kcur, nullptr, nullptr, n, s, vec, st);
    if (r != HS_OK) return r;

    for (int64_t w = T; w < n; w *= 2) {
        r = pairs ? launch_merge_level<MP_NT, MP_E, true>(kcur, kalt, vcur, valt, n, w, part, vec, st)
                  : launch_merge_level<MK_NT, MK_E, false>(kcur, kalt, nullptr, nullptr, n, w, part,
                                                           vec, st);
        if (r != HS_OK) return r;
        std::swap(kcur, kalt);
        std::swap(vcur, valt);
    }
    return HS_OK;
}

}  // namespace hs
