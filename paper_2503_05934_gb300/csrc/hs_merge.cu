// Host planner of the merge path (Algorithm 1 on the GPU): one block-sort
// launch, then per global level a partition launch and a merge launch,
// ping-ponging between the caller's array and the workspace so that the last
// level lands in the caller's array.
#include <algorithm>

#include "hs_internal.h"
#include "hs_blocksort.cuh"
#include "hs_merge_tile.cuh"
#include "hs_merge4.cuh"

namespace hs {

size_t merge_workspace_bytes(size_t n, int with_values) { return merge_workspace_size(n, with_values); }

// Keys block sort: four leaves (L, L, L, L-1 keys) per thread, in one of two
// shapes (option "blocksort_shape"):
//   2: 256 threads (tiles of 256 * (4L - 1) keys: 7936 for the {6,7,8} set)
//   4: 288 threads (8928 keys for the {6,7,8} set)
//  -1 (default): per n, shape 4 when its larger tile needs fewer global
//      levels than shape 2's (e.g. every power of two from 2^14 up), else 2.
static int g_bs_shape = -1;

static int shape_threads(int shape) { return shape == 4 ? 288 : 256; }
static int64_t shape_tile(int shape, int L) { return (int64_t)shape_threads(shape) * (4 * L - 1); }
static int global_levels(int64_t n, int64_t tile) {
    int p = 0;
    for (int64_t w = tile; w < n; w *= 2) ++p;
    return p;
}
static int shape_for(int64_t n, int L) {
    if (g_bs_shape >= 0) return g_bs_shape;
    return global_levels(n, shape_tile(4, L)) < global_levels(n, shape_tile(2, L)) ? 4 : 2;
}

int64_t keys_tile(int L, int64_t n) { return shape_tile(shape_for(n, L), L); }

void merge_set_blocksort_shape(int v) { g_bs_shape = v; }

// 16-byte aligned arrays (vec) use the bulk-copy form (k_blocksort3_bulk:
// each full tile in and out by one bulk copy); others the thread-staged form.
template <int NT, int L>
static hs_status launch_blocksort_t(const int32_t *kin, int32_t *kout, int64_t n, hs_netset s,
                                    int vec, int32_t *samp, cudaStream_t st) {
    using C = BlockSort3<NT, L, 4>;
    const int64_t grid = (n + C::T - 1) / C::T;
    hs_status r;
    if (vec) {
        unsigned *status = nullptr;
        if ((r = device_status(&status)) != HS_OK) return r;
        auto kern = k_blocksort3_bulk<NT, L, 4>;
        if ((r = ensure_smem((const void *)kern, C::SMEM_BYTES)) != HS_OK) return r;
        LaunchToken t = launch_begin(K_BLOCKSORT_KEYS, st);
        kern<<<(unsigned)grid, NT, C::SMEM_BYTES, st>>>(kin, kout, n, s, samp, status);
        return launch_end(t);
    }
    auto kern = k_blocksort3<NT, L, 4>;
    if ((r = ensure_smem((const void *)kern, C::SMEM_BYTES)) != HS_OK) return r;
    LaunchToken t = launch_begin(K_BLOCKSORT_KEYS, st);
    kern<<<(unsigned)grid, NT, C::SMEM_BYTES, st>>>(kin, kout, n, s, vec, samp);
    return launch_end(t);
}

template <int NT>
static hs_status launch_blocksort_nt(int L, const int32_t *kin, int32_t *kout, int64_t n,
                                     hs_netset s, int vec, int32_t *samp, cudaStream_t st) {
    switch (L) {
        case 1: return launch_blocksort_t<NT, 1>(kin, kout, n, s, vec, samp, st);
        case 3: return launch_blocksort_t<NT, 3>(kin, kout, n, s, vec, samp, st);
        case 4: return launch_blocksort_t<NT, 4>(kin, kout, n, s, vec, samp, st);
        case 5: return launch_blocksort_t<NT, 5>(kin, kout, n, s, vec, samp, st);
        case 6: return launch_blocksort_t<NT, 6>(kin, kout, n, s, vec, samp, st);
        case 7: return launch_blocksort_t<NT, 7>(kin, kout, n, s, vec, samp, st);
        case 8: return launch_blocksort_t<NT, 8>(kin, kout, n, s, vec, samp, st);
    }
    return fail(HS_ERR_INVALID_ARG, "leaf size outside 1, 3..8");
}

static hs_status blocksort_launch_shape(int shape, int L, const int32_t *kin, int32_t *kout,
                                        int64_t n, hs_netset s, int vec, cudaStream_t st,
                                        int32_t *samp) {
    if (shape == 4) return launch_blocksort_nt<288>(L, kin, kout, n, s, vec, samp, st);
    return launch_blocksort_nt<256>(L, kin, kout, n, s, vec, samp, st);
}

hs_status blocksort_launch(int L, const int32_t *kin, int32_t *kout, int64_t n, hs_netset s,
                           int vec, cudaStream_t st, int32_t *samp) {
    return blocksort_launch_shape(shape_for(n, L), L, kin, kout, n, s, vec, st, samp);
}

// Global levels: the tiled kernels (bulk-copy tiles, sampled partition
// searches) for 16-byte aligned buffers with n % 4 == 0; otherwise the
// generic serial-merge pass, which takes any 4-byte alignment.
constexpr int MG_NT = 256, MG_E = 16;  // generic keys level

static bool tiled_levels(int64_t n, int vec) { return vec && (n % 4) == 0; }

static hs_status launch_keys_level(const int32_t *kin, int32_t *kout, int64_t n, int64_t w,
                                   int64_t *part, int32_t *samp, int vec, cudaStream_t st) {
    if (tiled_levels(n, vec))
        return launch_keys_tile_level(kin, kout, n, w, part, samp, st);
    const LevelTiles lt = level_tiles(n, w, MG_NT * MG_E);
    LaunchToken t = launch_begin(K_MERGE_PARTITION, st);
    k_merge_partition<<<(unsigned)((lt.nblocks + 255) / 256), 256, 0, st>>>(
        kin, n, w, MG_NT * MG_E, (int)lt.tpg, lt.nblocks, part);
    hs_status r = launch_end(t);
    if (r != HS_OK) return r;
    const int smem = merge_smem_words<MG_NT, MG_E>() * (int)sizeof(int32_t);
    auto kern = k_merge_pass<MG_NT, MG_E, false>;
    if ((r = ensure_smem((const void *)kern, smem)) != HS_OK) return r;
    t = launch_begin(K_MERGE_KEYS, st);
    kern<<<(unsigned)lt.nblocks, MG_NT, smem, st>>>(kin, kout, nullptr, nullptr, n, w, part,
                                                     (int)lt.tpg, vec);
    return launch_end(t);
}

// Option "merge_fanin": 4 (default) the tiled keys levels merge four runs
// per pass (two binary levels of Algorithm 1's Merge in one read and one
// write of every key; a binary level first when the number of doublings is
// odd); 2 binary levels only.
static int g_merge_fanin = 4;
void merge_set_fanin(int v) { g_merge_fanin = v; }

constexpr int M4_NT = kMerge4Threads, M4_EO = kMerge4Keys;

// One four-way keys level: its partition (four splits per tile boundary,
// part_cap int64 entries available) and its merge.
static hs_status launch_keys_level4(const int32_t *kin, int32_t *kout, int64_t n, int64_t w,
                                    int64_t *part, int64_t part_cap, int32_t *samp,
                                    cudaStream_t st) {
    using C = TileMerge4<M4_NT, M4_EO>;
    static_assert(C::TO % kSampleStride == 0, "output tiles start on sample positions");
    unsigned *status = nullptr;
    hs_status r = device_status(&status);
    if (r != HS_OK) return r;
    const LevelTiles lt = level_tiles_span(n, 4 * w, C::TO);
    if (4 * (lt.nblocks + 1) > part_cap)
        return fail(HS_ERR_INVALID_ARG, "merge sort: workspace too small for the four-way partitions");
    LaunchToken t = launch_begin(K_MERGE_PARTITION, st);
    k_merge4_partition<4><<<(unsigned)((lt.nblocks + 127) / 128), 128, 0, st>>>(
        kin, samp, n, w, C::TO, lt.tpg, lt.nblocks, part);
    if ((r = launch_end(t)) != HS_OK) return r;
    auto kern = k_merge4_tile_bulk<M4_NT, M4_EO>;
    if ((r = ensure_smem((const void *)kern, C::SMEM_BYTES)) != HS_OK) return r;
    t = launch_begin(K_MERGE4_KEYS, st);
    kern<<<(unsigned)lt.nblocks, M4_NT, C::SMEM_BYTES, st>>>(kin, kout, n, w, part, lt.tpg, samp,
                                                             status);
    return launch_end(t);
}

// Whether the global levels over an n-key array merge four runs per pass.
static bool four_way_levels(int64_t n, int vec) { return g_merge_fanin == 4 && tiled_levels(n, vec); }

// Launches of the global levels that double the runs d times.
static int level_launches(int d, bool four) { return four ? d / 2 + d % 2 : d; }

// Runs the global levels that take sorted runs of w keys through d
// doublings (one launch pair per binary or four-way level), ping-ponging
// kcur/kalt; on return kcur holds the result.
static hs_status run_levels(int32_t *&kcur, int32_t *&kalt, int64_t n, int64_t w, int d,
                            bool four, int64_t *part, int64_t part_cap, int32_t *samp, int vec,
                            cudaStream_t st) {
    hs_status r = HS_OK;
    while (d > 0 && r == HS_OK) {
        if (four && d % 2 == 0) {
            r = launch_keys_level4(kcur, kalt, n, w, part, part_cap, samp, st);
            w *= 4;
            d -= 2;
        } else {
            r = launch_keys_level(kcur, kalt, n, w, part, samp, vec, st);
            w *= 2;
            d -= 1;
        }
        std::swap(kcur, kalt);
    }
    return r;
}

// Sorts d_keys[0, n) with explicit scratch: kbuf (n keys), part (part_cap
// partition entries) and samp (every 32nd key of n keys, or null for plain
// partition searches).  The result lands in d_keys.
static hs_status merge_sort_with(int32_t *d_keys, int64_t n, hs_netset s, int32_t *kbuf,
                                 int64_t *part, int64_t part_cap, int32_t *samp,
                                 cudaStream_t st) {
    const int L = leaf_size(s);
    const int64_t T = keys_tile(L, n);
    const int d = global_levels(n, T);
    const int vec = aligned(d_keys, 16) ? 1 : 0;
    if (!tiled_levels(n, vec)) samp = nullptr;
    const bool four = four_way_levels(n, vec);
    // Land the last level in the caller's array: with an even number of
    // launched levels the block sort writes in place.
    int32_t *kcur = (level_launches(d, four) % 2 == 0) ? d_keys : kbuf;
    int32_t *kalt = (kcur == d_keys) ? kbuf : d_keys;
    hs_status r = blocksort_launch(L, d_keys, kcur, n, s, vec, st, samp);
    if (r != HS_OK) return r;
    return run_levels(kcur, kalt, n, T, d, four, part, part_cap, samp, vec, st);
}

struct MergeScratch {
    int32_t *kbuf, *samp;
    int64_t *part;
};

static MergeScratch carve_merge_workspace(void *d_ws, size_t n) {
    char *p = static_cast<char *>(d_ws);
    MergeScratch m;
    m.kbuf = reinterpret_cast<int32_t *>(p);
    m.part = reinterpret_cast<int64_t *>(p + merge_ws_keys_bytes(n));
    m.samp = reinterpret_cast<int32_t *>(p + merge_ws_keys_bytes(n) + merge_ws_part_bytes(n));
    return m;
}

hs_status merge_sort(int32_t *d_keys, int32_t *d_vals, size_t n_, hs_netset s, void *d_ws,
                     size_t ws_bytes, cudaStream_t st) {
    if (d_vals) return pairs_sort(d_keys, d_vals, n_, s, d_ws, ws_bytes, st);
    const int64_t n = (int64_t)n_;
    const int L = leaf_size(s);
    if (n <= keys_tile(L, n)) return blocksort_launch(L, d_keys, d_keys, n, s, aligned(d_keys, 16) ? 1 : 0, st);
    if (!d_ws || ws_bytes < merge_workspace_bytes(n_, 0))
        return fail(HS_ERR_INVALID_ARG, "merge sort: workspace smaller than hs_sort_workspace_bytes");
    if (!aligned(d_ws, 16)) return fail(HS_ERR_INVALID_ARG, "merge sort: workspace not 16-byte aligned");
    const MergeScratch m = carve_merge_workspace(d_ws, n_);
    return merge_sort_with(d_keys, n, s, m.kbuf, m.part, (int64_t)merge_ws_part_entries(n_), m.samp, st);
}

// Chunk-local merge levels of the host-buffer sort: the most that keep one
// chunk's sort (block sort + k levels) within the time its copy in takes, so
// that sorting keeps pace with the copies.  Planning rates, measured on
// GB300: host link 200 GB/s, block sort 130 Gkeys/s, a merge level 8 B/key at
// 6.5 TB/s plus 30 us of partition and launch latency.
static int host_local_levels(int64_t chunk, int max_levels) {
    const double copy_s = 4.0 * chunk / 200e9;
    const double sort_s = chunk / 130e9;
    const double level_s = 8.0 * chunk / 6.5e12 + 30e-6;
    int k = 0;
    while (k < max_levels && sort_s + (k + 1) * level_s <= copy_s) ++k;
    return k;
}

// Host-buffer merge sort.  The keys are copied in as about eight chunks on a
// second stream; as each chunk lands it is block sorted and merged k levels
// deep into runs of W = T << k keys (chunks are whole multiples of W, so these
// are exactly the first k levels of the whole sort).  The remaining levels run
// over the whole array, and the result is copied out.  d_keys is device
// memory for n keys; d_ws the merge workspace for n keys.
hs_status merge_sort_host_chunked(int32_t *h_keys, int32_t *d_keys, size_t n_, hs_netset s,
                                  void *d_ws, cudaStream_t st) {
    constexpr int kChunks = 8;
    const int64_t n = (int64_t)n_;
    const int L = leaf_size(s);
    const int shape = shape_for(n, L);
    const int64_t T = shape_tile(shape, L);
    const int levels = global_levels(n, T);
    const int k = host_local_levels((n + kChunks - 1) / kChunks, levels > 0 ? levels - 1 : 0);
    const int64_t W = T << k;
    // Chunk length: whole runs of W keys, so chunk starts are multiples of
    // T (16-byte aligned, sample positions at multiples of 32).
    const int64_t C = W * std::max<int64_t>(1, (n + kChunks * W - 1) / (kChunks * W));
    const int nch = (int)((n + C - 1) / C);
    const MergeScratch m = carve_merge_workspace(d_ws, n_);
    const int vec = aligned(d_keys, 16) ? 1 : 0;
    int32_t *samp = tiled_levels(n, vec) ? m.samp : nullptr;
    // Decided once for the whole array, so that every chunk runs the same
    // number of launches (the parity that places its block sort).
    const bool four = four_way_levels(n, vec);
    const int64_t part_cap = (int64_t)merge_ws_part_entries(n_);

    cudaStream_t cs = nullptr;
    cudaEvent_t ev[kChunks] = {};
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    hs_status r = HS_OK;
    for (int c = 0; c < nch && e == cudaSuccess; ++c) e = cudaEventCreateWithFlags(&ev[c], cudaEventDisableTiming);
    for (int c = 0; c < nch && e == cudaSuccess; ++c) {
        const int64_t b = c * C, len = std::min<int64_t>(C, n - b);
        e = cudaMemcpyAsync(d_keys + b, h_keys + b, (size_t)len * sizeof(int32_t), cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev[c], cs);
    }
    if (e != cudaSuccess) r = fail_cuda(e, "host sort: chunked copy in");
    for (int c = 0; c < nch && r == HS_OK; ++c) {
        const int64_t b = c * C, len = std::min<int64_t>(C, n - b);
        if ((e = cudaStreamWaitEvent(st, ev[c], 0)) != cudaSuccess) {
            r = fail_cuda(e, "host sort: wait for a chunk");
            break;
        }
        // The block sort writes where the chunk's ping-pong levels end in d_keys.
        const bool even = level_launches(k, four) % 2 == 0;
        int32_t *cur = even ? d_keys + b : m.kbuf + b;
        int32_t *alt = even ? m.kbuf + b : d_keys + b;
        int32_t *csamp = samp ? samp + b / kSampleStride : nullptr;
        r = blocksort_launch_shape(shape, L, d_keys + b, cur, len, s, vec, st, csamp);
        if (r == HS_OK) r = run_levels(cur, alt, len, T, k, four, m.part, part_cap, csamp, vec, st);
    }
    int32_t *kcur = d_keys, *kalt = m.kbuf;
    if (r == HS_OK) r = run_levels(kcur, kalt, n, W, levels - k, four, m.part, part_cap, samp, vec, st);
    if (r == HS_OK && (e = cudaMemcpyAsync(h_keys, kcur, n_ * sizeof(int32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        r = fail_cuda(e, "host sort: copy out");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess && r == HS_OK) r = fail_cuda(e, "host sort: synchronize");
    if (cs && (e = cudaStreamSynchronize(cs)) != cudaSuccess && r == HS_OK) r = fail_cuda(e, "host sort: copy stream");
    for (int c = 0; c < nch; ++c)
        if (ev[c]) cudaEventDestroy(ev[c]);
    if (cs) cudaStreamDestroy(cs);
    return r;
}

}  // namespace hs
