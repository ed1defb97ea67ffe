// Host planner of the merge path (Algorithm 1 on the GPU): one block-sort
// launch, then per global level a partition launch and a merge launch,
// ping-ponging between the caller's array and the workspace so that the last
// level lands in the caller's array.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <new>
#include <vector>

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
// ---------------------------------------------------------------------------
// Launch plans of the single-array merge path: block-sort shape and merge
// fan-in.  Decided, in this order, by a plan forced on this thread (while
// the autotuner times candidates), by the options when they are not at
// their automatic values, by a plan the autotuner cached for this device,
// array size (log2 bucket) and leaf size, and otherwise by the built-in
// rules (shape_rule, the fan-in's size rule).
static thread_local const SortPlan *t_forced_plan = nullptr;
void sort_plan_force(const SortPlan *p) { t_forced_plan = p; }

struct SortPlanEntry {
    std::string device;
    int n_bucket, leaf;
    SortPlan plan;
    double ms;
};
static std::mutex g_plan_mu;
static std::vector<SortPlanEntry> g_plans;
static std::atomic<int> g_plans_count{0};  // entries cached (a lock-free "none" test)

int size_bucket(int64_t n) {
    int b = 0;
    while (b < 62 && (int64_t(2) << b) <= n) ++b;
    return b;  // floor(log2 n) for n >= 1
}

// Name of device `dev`, looked up once per ordinal.
static const std::string *device_name_cached(int dev) {
    static std::mutex mu;
    static std::string names[64];
    static bool have[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!have[dev]) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        names[dev] = prop.name;
        have[dev] = true;
    }
    return &names[dev];
}

hs_status current_device_name(std::string *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
    const std::string *nm = device_name_cached(dev);
    if (!nm) return fail(HS_ERR_CUDA, "cudaGetDeviceProperties failed");
    *out = *nm;
    return HS_OK;
}

void sort_plan_cache_put(const std::string &device, int n_bucket, int leaf, const SortPlan &p,
                         double ms) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (SortPlanEntry &e : g_plans)
        if (e.device == device && e.n_bucket == n_bucket && e.leaf == leaf) {
            e.plan = p;
            e.ms = ms;
            bump_config_generation();
            return;
        }
    g_plans.push_back(SortPlanEntry{device, n_bucket, leaf, p, ms});
    g_plans_count.store((int)g_plans.size());
    bump_config_generation();
}

bool sort_plan_cache_get(const std::string &device, int n_bucket, int leaf, SortPlan *p,
                         double *ms) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (const SortPlanEntry &e : g_plans)
        if (e.device == device && e.n_bucket == n_bucket && e.leaf == leaf) {
            *p = e.plan;
            if (ms) *ms = e.ms;
            return true;
        }
    return false;
}

void sort_plan_cache_clear() {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans.clear();
    g_plans_count.store(0);
    bump_config_generation();
}

void sort_plan_cache_each(void (*fn)(void *, const std::string &, int, int, const SortPlan &, double),
                          void *ctx) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (const SortPlanEntry &e : g_plans) fn(ctx, e.device, e.n_bucket, e.leaf, e.plan, e.ms);
}

// The cached plan for an n-key array of leaf size L on the current device.
static bool tuned_plan(int64_t n, int L, SortPlan *p) {
    if (g_plans_count.load() == 0) return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const std::string *nm = device_name_cached(dev);
    return nm && sort_plan_cache_get(*nm, size_bucket(n), L, p, nullptr);
}

static int shape_rule(int64_t n, int L) {
    return global_levels(n, shape_tile(4, L)) < global_levels(n, shape_tile(2, L)) ? 4 : 2;
}

static int shape_for(int64_t n, int L) {
    if (t_forced_plan) return t_forced_plan->shape;
    if (g_bs_shape >= 0) return g_bs_shape;
    SortPlan p;
    if (tuned_plan(n, L, &p)) return p.shape;
    return shape_rule(n, L);
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

// Option "merge_fanin": the tiled keys levels of an array merge four runs
// per pass (two binary levels of Algorithm 1's Merge in one read and one
// write of every key; a binary level first when the number of doublings is
// odd) with 4, binary levels only with 2, and with 0 (the default) four-way
// levels for arrays of at least kFourWayMinKeys keys.  A four-way level
// saves a pass over the keys but its partition is a latency-bound chain of
// 15 to 27 rounds (0.04 to 0.1 ms), so it pays off only on large arrays:
// whole sorts measured on GB300 with four-way against binary levels took
// 0.17 / 0.11 ms at 2^18 keys, 0.39 / 0.26 at 2^22, 1.10 / 0.95 at 2^25,
// 1.84 / 1.74 at 2^26, 3.37 / 3.38 at 2^27 and 6.54 / 6.90 ms at 2^28.
constexpr int64_t kFourWayMinKeys = int64_t(1) << 27;
static int g_merge_fanin = 0;
void merge_set_fanin(int v) { g_merge_fanin = v; }
int merge_fanin() { return g_merge_fanin; }

constexpr int M4_NT = kMerge4Threads, M4_EO = kMerge4Keys;

// One four-way keys level: its partition (four splits per tile boundary,
// part_cap int64 entries available) and its merge.  With parts > 1 the merge
// is launched as `parts` launches over consecutive ranges of output tiles,
// and part_done[p] is recorded on st after launch p, whose outputs end at
// part_end[p] (for a level of one group, every last level: outputs
// [part_end[p - 1], part_end[p]) of the array).
static hs_status launch_keys_level4(const int32_t *kin, int32_t *kout, int64_t n, int64_t w,
                                    int64_t *part, int64_t part_cap, int32_t *samp,
                                    cudaStream_t st, int parts = 1,
                                    cudaEvent_t *part_done = nullptr,
                                    int64_t *part_end = nullptr) {
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
    if (parts < 1 || !part_done) parts = 1;
    for (int p = 0; p < parts; ++p) {
        const int64_t b0 = lt.nblocks * p / parts, b1 = lt.nblocks * (p + 1) / parts;
        if (b1 > b0) {
            t = launch_begin(K_MERGE4_KEYS, st);
            kern<<<(unsigned)(b1 - b0), M4_NT, C::SMEM_BYTES, st>>>(kin, kout, n, w, part, lt.tpg,
                                                                    samp, status, b0);
            if ((r = launch_end(t)) != HS_OK) return r;
        }
        if (part_done) {
            if (part_end) part_end[p] = std::min<int64_t>(b1 * C::TO, n);
            const cudaError_t e = cudaEventRecord(part_done[p], st);
            if (e != cudaSuccess) return fail_cuda(e, "merge sort: record a level part");
        }
    }
    return HS_OK;
}

// Whether the global levels over an n-key array (leaf size L) merge four
// runs per pass.
bool merge_four_way_possible(const int32_t *d_keys, int64_t n) {
    return tiled_levels(n, aligned(d_keys, 16) ? 1 : 0);
}
static bool four_way_levels(int64_t n, int vec, int L) {
    if (!tiled_levels(n, vec)) return false;
    if (t_forced_plan) return t_forced_plan->fanin == 4;
    if (g_merge_fanin != 0) return g_merge_fanin == 4;
    SortPlan p;
    if (tuned_plan(n, L, &p)) return p.fanin == 4;
    return n >= kFourWayMinKeys;
}

SortPlan merge_plan_for(const int32_t *d_keys, int64_t n, int L) {
    return SortPlan{shape_for(n, L), four_way_levels(n, aligned(d_keys, 16) ? 1 : 0, L) ? 4 : 2};
}

// Launches of the global levels that double the runs d times.
static int level_launches(int d, bool four) { return four ? d / 2 + d % 2 : d; }

// Runs the global levels that take sorted runs of w keys through d
// doublings (one launch pair per binary or four-way level), ping-ponging
// kcur/kalt; on return kcur holds the result.  With last_parts > 1 a
// four-way last level is launched in that many parts (see
// launch_keys_level4), recording part_done[p] after each.
static hs_status run_levels(int32_t *&kcur, int32_t *&kalt, int64_t n, int64_t w, int d,
                            bool four, int64_t *part, int64_t part_cap, int32_t *samp, int vec,
                            cudaStream_t st, int last_parts = 1, cudaEvent_t *part_done = nullptr,
                            int64_t *part_end = nullptr) {
    hs_status r = HS_OK;
    while (d > 0 && r == HS_OK) {
        if (four && d % 2 == 0) {
            const bool last = d == 2;
            r = launch_keys_level4(kcur, kalt, n, w, part, part_cap, samp, st,
                                   last ? last_parts : 1, last ? part_done : nullptr,
                                   last ? part_end : nullptr);
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
    const bool four = four_way_levels(n, vec, L);
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

// Small arrays: one CTA of SMALL_NT threads sorts the whole array in one
// launch (leaves and all merge levels in shared memory, work past the live
// keys skipped; no workspace), for n up to its tile of
// SMALL_NT * (SMALL_LEAVES * L - 1) keys (15,360 for the {6,7,8} set).
// Measured at 10,000 uniform keys ({6,7,8}): 28.5 us, against 30.6 us for
// the block sort of two tiles plus one merge level; with four leaves per
// thread (31,744-key tile) 31.0 us, and 53 us against 42 us at 25,000 keys.
// One SM's latency through about ten merge levels bounds these sizes.
constexpr int SMALL_NT = 1024, SMALL_LEAVES = 2;

static int64_t small_tile(int L) { return (int64_t)SMALL_NT * (L == 1 ? 3 : SMALL_LEAVES * L - 1); }

template <int L, int LV>
static hs_status launch_small_t(int32_t *keys, int64_t n, hs_netset s, int vec, cudaStream_t st) {
    using C = BlockSort3<SMALL_NT, L, LV>;
    auto kern = k_blocksort_small<SMALL_NT, L, LV>;
    hs_status r = ensure_smem((const void *)kern, C::SMEM_BYTES);
    if (r != HS_OK) return r;
    LaunchToken t = launch_begin(K_BLOCKSORT_KEYS, st);
    kern<<<1, SMALL_NT, C::SMEM_BYTES, st>>>(keys, keys, (int)n, s, vec);
    return launch_end(t);
}

static hs_status small_sort_launch(int32_t *keys, int64_t n, hs_netset s, cudaStream_t st) {
    const int vec = aligned(keys, 16) ? 1 : 0;
    switch (leaf_size(s)) {
        case 1: return launch_small_t<1, 4>(keys, n, s, vec, st);
        case 3: return launch_small_t<3, SMALL_LEAVES>(keys, n, s, vec, st);
        case 4: return launch_small_t<4, SMALL_LEAVES>(keys, n, s, vec, st);
        case 5: return launch_small_t<5, SMALL_LEAVES>(keys, n, s, vec, st);
        case 6: return launch_small_t<6, SMALL_LEAVES>(keys, n, s, vec, st);
        case 7: return launch_small_t<7, SMALL_LEAVES>(keys, n, s, vec, st);
        case 8: return launch_small_t<8, SMALL_LEAVES>(keys, n, s, vec, st);
    }
    return fail(HS_ERR_INVALID_ARG, "leaf size outside 1, 3..8");
}

int64_t small_sort_max(int L) { return small_tile(L); }
hs_status small_sort(int32_t *keys, int64_t n, hs_netset s, cudaStream_t st) {
    return small_sort_launch(keys, n, s, st);
}

hs_status merge_sort(int32_t *d_keys, int32_t *d_vals, size_t n_, hs_netset s, void *d_ws,
                     size_t ws_bytes, cudaStream_t st) {
    if (d_vals) return pairs_sort(d_keys, d_vals, n_, s, d_ws, ws_bytes, st);
    const int64_t n = (int64_t)n_;
    const int L = leaf_size(s);
    if (n <= small_tile(L)) return small_sort_launch(d_keys, n, s, st);
    if (n <= keys_tile(L, n)) return blocksort_launch(L, d_keys, d_keys, n, s, aligned(d_keys, 16) ? 1 : 0, st);
    if (!d_ws || ws_bytes < merge_workspace_bytes(n_, 0))
        return fail(HS_ERR_INVALID_ARG, "merge sort: workspace smaller than hs_sort_workspace_bytes");
    if (!aligned(d_ws, 16)) return fail(HS_ERR_INVALID_ARG, "merge sort: workspace not 16-byte aligned");
    const MergeScratch m = carve_merge_workspace(d_ws, n_);
    return merge_sort_with(d_keys, n, s, m.kbuf, m.part, (int64_t)merge_ws_part_entries(n_), m.samp, st);
}

// Host-buffer merge sort, for n of at least a few chunks' worth of keys.
//
//  * The keys are copied in as at most kHostChunks chunks on a copy stream.
//    A chunk holds C = T * 2^k keys (T the block-sort tile, C the smallest
//    such length with at most kHostChunks chunks), so every chunk is a whole
//    run of the merge sort's level of width C.
//  * As each chunk lands it is sorted completely (block sort and its own
//    merge levels) on one of kHostSideStreams side streams; chunks overlap
//    one another and the copy of the next ones.  Each chunk uses its own
//    slice of partition entries (hs_host_part_entries per chunk).
//  * On the caller's stream the merge levels over the sorted chunks finish
//    the sort.  The last (four-way) level runs as kHostOutParts launches
//    over consecutive ranges of output tiles, and each part's keys are
//    copied out as soon as it is done, while the next parts still merge.
//
// d_keys is device memory for n keys; d_ws the merge workspace for n keys;
// d_part the chunks' partition slices (host_part_entries(n) int64).
// Measured at 2^28 keys (median call): 8 chunks with 2 / 3 / 4 side streams
// 13.53 / 13.33 / 13.18 ms, 16 chunks with 3 / 4 13.34 / 13.31 ms, 4 chunks
// with 2 13.93 ms; the two copies alone take 10.66 ms on that box.
constexpr int kHostChunks = 8, kHostSideStreams = 4, kHostOutParts = 8;

static int64_t host_chunk_keys(int64_t n, int64_t T) {
    int64_t C = T;
    while (C * kHostChunks < n) C *= 2;
    return C;
}
// Partition entries one chunk of C keys needs at most (four per tile
// boundary of 3936-key tiles over groups of four runs of at least one
// block-sort tile, or one per 3968-key tile of a binary level), with room.
static int64_t chunk_part_entries(int64_t C) { return C / 512 + 64; }

size_t host_part_entries(size_t n) {
    // C < 2n / kHostChunks + 2T (T <= 8928), and at most kHostChunks chunks.
    return (size_t)kHostChunks *
               (size_t)chunk_part_entries((int64_t)(2 * n / kHostChunks + 2 * 8928)) + 64;
}

// Streams and events of the host-buffer pipeline, created on first use per
// host thread and device and kept for the life of the process (creating them
// per call costs host time on every call).
struct HostPipe {
    int device = -1;
    cudaStream_t cs = nullptr, side[kHostSideStreams] = {};
    cudaEvent_t ev_start = nullptr, ev_in[kHostChunks] = {}, ev_done[kHostChunks] = {},
                ev_part[kHostOutParts] = {};
};

static hs_status host_pipe(HostPipe **out) {
    static thread_local std::vector<HostPipe *> pipes;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "host sort: current device");
    for (HostPipe *p : pipes)
        if (p->device == dev) {
            *out = p;
            return HS_OK;
        }
    HostPipe *p = new (std::nothrow) HostPipe();
    if (!p) return fail(HS_ERR_NO_MEMORY, "host sort: pipeline state");
    p->device = dev;
    e = cudaStreamCreateWithFlags(&p->cs, cudaStreamNonBlocking);
    for (int i = 0; i < kHostSideStreams && e == cudaSuccess; ++i)
        e = cudaStreamCreateWithFlags(&p->side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming);
    for (int c = 0; c < kHostChunks && e == cudaSuccess; ++c) {
        e = cudaEventCreateWithFlags(&p->ev_in[c], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_done[c], cudaEventDisableTiming);
    }
    for (int q = 0; q < kHostOutParts && e == cudaSuccess; ++q)
        e = cudaEventCreateWithFlags(&p->ev_part[q], cudaEventDisableTiming);
    if (e != cudaSuccess) {  // release what was made; the next call retries
        for (int c = 0; c < kHostChunks; ++c) {
            if (p->ev_in[c]) cudaEventDestroy(p->ev_in[c]);
            if (p->ev_done[c]) cudaEventDestroy(p->ev_done[c]);
        }
        for (int q = 0; q < kHostOutParts; ++q)
            if (p->ev_part[q]) cudaEventDestroy(p->ev_part[q]);
        if (p->ev_start) cudaEventDestroy(p->ev_start);
        for (int i = 0; i < kHostSideStreams; ++i)
            if (p->side[i]) cudaStreamDestroy(p->side[i]);
        if (p->cs) cudaStreamDestroy(p->cs);
        delete p;
        return fail_cuda(e, "host sort: streams and events");
    }
    pipes.push_back(p);
    *out = p;
    return HS_OK;
}

hs_status merge_sort_host_chunked(int32_t *h_keys, int32_t *d_keys, size_t n_, hs_netset s,
                                  void *d_ws, int64_t *d_part, cudaStream_t st) {
    const int64_t n = (int64_t)n_;
    const int L = leaf_size(s);
    const int shape = shape_for(n, L);
    const int64_t T = shape_tile(shape, L);
    const int64_t C = host_chunk_keys(n, T);
    const int nch = (int)((n + C - 1) / C);
    const int64_t PC = chunk_part_entries(C);
    if ((size_t)(nch * PC) > host_part_entries(n_))
        return fail(HS_ERR_INVALID_ARG, "host sort: partition slices exceed their workspace");
    const MergeScratch m = carve_merge_workspace(d_ws, n_);
    const int vec = aligned(d_keys, 16) ? 1 : 0;
    int32_t *samp = tiled_levels(n, vec) ? m.samp : nullptr;
    // The levels over the whole array are four-way by its size; a chunk's own
    // levels by the chunk's (the parity of its launches places its block
    // sort), and only when the whole array takes tiled levels.
    const bool four = four_way_levels(n, vec, L);
    const int64_t part_cap = (int64_t)merge_ws_part_entries(n_);

    HostPipe *pp = nullptr;
    hs_status r = host_pipe(&pp);
    if (r != HS_OK) return r;
    cudaStream_t cs = pp->cs;
    cudaStream_t *side = pp->side;
    cudaEvent_t *ev_in = pp->ev_in, *ev_done = pp->ev_done, *ev_part = pp->ev_part;
    cudaEvent_t ev_start = pp->ev_start;
    int64_t part_end[kHostOutParts] = {};
    // The copy stream and the side streams start after what the caller's
    // stream has queued so far (the workspace may still be in use there).
    cudaError_t e = cudaEventRecord(ev_start, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_start, 0);
    for (int i = 0; i < kHostSideStreams && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(side[i], ev_start, 0);
    if (e != cudaSuccess) r = fail_cuda(e, "host sort: order the streams");
    for (int c = 0; c < nch && r == HS_OK; ++c) {
        const int64_t b = c * C, len = std::min<int64_t>(C, n - b);
        e = cudaMemcpyAsync(d_keys + b, h_keys + b, (size_t)len * sizeof(int32_t), cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev_in[c], cs);
        if (e != cudaSuccess) r = fail_cuda(e, "host sort: chunked copy in");
    }
    for (int c = 0; c < nch && r == HS_OK; ++c) {
        const int64_t b = c * C, len = std::min<int64_t>(C, n - b);
        cudaStream_t ss = side[c % kHostSideStreams];
        if ((e = cudaStreamWaitEvent(ss, ev_in[c], 0)) != cudaSuccess) {
            r = fail_cuda(e, "host sort: wait for a chunk");
            break;
        }
        // The block sort writes where the chunk's ping-pong levels end in d_keys.
        const int d = global_levels(len, T);
        const bool four_c = tiled_levels(n, vec) && four_way_levels(len, vec, L);
        const bool even = level_launches(d, four_c) % 2 == 0;
        int32_t *cur = even ? d_keys + b : m.kbuf + b;
        int32_t *alt = even ? m.kbuf + b : d_keys + b;
        int32_t *csamp = samp ? samp + b / kSampleStride : nullptr;
        r = blocksort_launch_shape(shape, L, d_keys + b, cur, len, s, vec, ss, csamp);
        if (r == HS_OK) r = run_levels(cur, alt, len, T, d, four_c, d_part + c * PC, PC, csamp, vec, ss);
        if (r == HS_OK && (e = cudaEventRecord(ev_done[c], ss)) != cudaSuccess)
            r = fail_cuda(e, "host sort: chunk done");
        if (r == HS_OK && (e = cudaStreamWaitEvent(st, ev_done[c], 0)) != cudaSuccess)
            r = fail_cuda(e, "host sort: join a chunk");
    }
    int32_t *kcur = d_keys, *kalt = m.kbuf;
    const int d_final = global_levels(n, C);
    // The last level in parts, each copied out as soon as it is done (a
    // four-way last level; otherwise one copy after the last level).
    const bool split = four && d_final >= 2;
    if (r == HS_OK)
        r = run_levels(kcur, kalt, n, C, d_final, four, m.part, part_cap, samp, vec, st,
                       split ? kHostOutParts : 1, split ? ev_part : nullptr, split ? part_end : nullptr);
    if (r == HS_OK) {
        if (split) {
            int64_t lo = 0;
            for (int p = 0; p < kHostOutParts && e == cudaSuccess; ++p) {
                const int64_t hi = part_end[p];
                e = cudaStreamWaitEvent(cs, ev_part[p], 0);
                if (e == cudaSuccess && hi > lo)
                    e = cudaMemcpyAsync(h_keys + lo, kcur + lo, (size_t)(hi - lo) * sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, cs);
                lo = hi;
            }
        } else {
            e = cudaEventRecord(ev_start, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_start, 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_keys, kcur, n_ * sizeof(int32_t), cudaMemcpyDeviceToHost, cs);
        }
        if (e != cudaSuccess) r = fail_cuda(e, "host sort: copy out");
    }
    // Wait for everything queued, on every stream: the call is synchronous,
    // and the cached streams start the next call idle.
    for (int i = 0; i < kHostSideStreams; ++i)
        if ((e = cudaStreamSynchronize(side[i])) != cudaSuccess && r == HS_OK)
            r = fail_cuda(e, "host sort: side stream");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess && r == HS_OK) r = fail_cuda(e, "host sort: synchronize");
    if ((e = cudaStreamSynchronize(cs)) != cudaSuccess && r == HS_OK) r = fail_cuda(e, "host sort: copy stream");
    return r;
}

}  // namespace hs
