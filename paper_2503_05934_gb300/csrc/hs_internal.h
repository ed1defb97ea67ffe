// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/hsort.h"

namespace hs {

// Kernel ids for launch counting and the optional per-kernel event timing.
enum KernelId {
    K_BLOCKSORT_KEYS = 0,
    K_BLOCKSORT_PAIRS,
    K_MERGE_PARTITION,
    K_MERGE_KEYS,
    K_MERGE_PAIRS,
    K_QS_PLAN,
    K_QS_PARTITION,
    K_QS_LEAVES,
    K_SEG_CLASSIFY,
    K_SEG_SORT,
    K_SELFTEST,
    K_MERGE4_KEYS,
    K_COUNT
};
const char *kernel_name(int id);

// Sets the thread-local error message and returns st.
hs_status fail(hs_status st, const std::string &msg);
hs_status fail_cuda(cudaError_t e, const char *what);
void clear_error();

// An NVTX range over one public call (pushed on construction, popped on
// destruction), for profilers that select work by range.
struct ApiRange {
    explicit ApiRange(const char *name);
    ~ApiRange();
    ApiRange(const ApiRange &) = delete;
    ApiRange &operator=(const ApiRange &) = delete;
};

// Brackets one launch: counts it, marks it with an NVTX range named for the
// kernel and, when timing is on, records events on `stream` around it.  Usage: auto t = launch_begin(id, s); <<<...>>>;
// st = launch_end(t).
struct LaunchToken {
    int id;
    cudaStream_t stream;
    cudaEvent_t ev_a, ev_b;  // non-null while per-kernel timing is on
};
LaunchToken launch_begin(int id, cudaStream_t stream);
// Adds k kernels launched indirectly (graph replays) to the launch count.
void count_launches(uint64_t k);
hs_status launch_end(const LaunchToken &t);
// While this thread captures a sort into a graph, launches are counted into
// *counter instead of the global count (replays add them); null ends it.
void capture_launches_into(uint64_t *counter);
// Whether per-kernel event timing is on (graph replays are then not used).
bool prof_enabled();

// Generation of everything that decides a merge sort's launches (options,
// tuned plans): bumped on every change, so cached graphs of older
// generations are not replayed.
uint64_t config_generation();
void bump_config_generation();
// Replays a captured graph of an earlier merge sort with the same
// arguments, or captures one on the second call (hs_sort_i32's merge path).
hs_status merge_sort_graphed(int32_t *d_keys, int32_t *d_vals, size_t n, hs_netset s, void *d_ws,
                             size_t ws_bytes, cudaStream_t st);
hs_status merge_sort_i64_graphed(int64_t *d_keys, size_t n, hs_netset s, void *d_ws,
                                 size_t ws_bytes, cudaStream_t st);
void sort_graphs_enable(int on);

// Validation shared by the entry points.
inline bool netset_ok(hs_netset s) {
    if (s & HS_NETS_VARSORT) {  // VarSortk: the flag and exactly one size bit k in 3..8
        const hs_netset k = s & ~HS_NETS_VARSORT;
        return k != 0 && (k & ~0x1F8u) == 0 && (k & (k - 1)) == 0;
    }
    return (s & ~0x1F8u) == 0;
}
inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Opt a kernel into more than 48 KB of dynamic shared memory, once per
// device (the attribute is per function and device).
hs_status ensure_smem(const void *func, int bytes);

// Merge path internals exposed to the other translation units.  merge_sort
// sorts keys, or stable pairs when d_vals is non-null (pairs_sort).
//
// Workspace layout (each part 256-byte aligned): the keys ping-pong copy,
// the values copy (pairs), the merge partition indices (n/256 + 64 int64:
// one per output tile of a binary level, whose tiles hold at least 1984
// keys, or four per tile boundary of a four-way level, whose tiles hold 3936
// keys over groups of at least four block-sort tiles of 768 keys), and the
// keys' samples (every 32nd key, n/32 + 8 int32).
constexpr size_t ws_align(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t merge_ws_keys_bytes(size_t n) { return ws_align(n * sizeof(int32_t)); }
constexpr size_t merge_ws_part_entries(size_t n) { return n / 256 + 64; }
constexpr size_t merge_ws_part_bytes(size_t n) { return ws_align(merge_ws_part_entries(n) * sizeof(int64_t)); }
constexpr size_t merge_ws_samp_bytes(size_t n) { return ws_align((n / 32 + 8) * sizeof(int32_t)); }
constexpr size_t merge_workspace_size(size_t n, int with_values) {
    return merge_ws_keys_bytes(n) * (with_values ? 2 : 1) + merge_ws_part_bytes(n) +
           merge_ws_samp_bytes(n);
}
size_t merge_workspace_bytes(size_t n, int with_values);
hs_status merge_sort(int32_t *d_keys, int32_t *d_vals, size_t n, hs_netset s, void *d_ws,
                     size_t ws_bytes, cudaStream_t st);
hs_status pairs_sort(int32_t *d_keys, int32_t *d_vals, size_t n, hs_netset s, void *d_ws,
                     size_t ws_bytes, cudaStream_t st);
// Host keys in and out, input copy overlapped with per-chunk sorts and the
// copy out with the last level (merge path; synchronous).  d_keys: device
// space for n keys; d_ws: merge workspace; d_part: host_part_entries(n)
// int64 partition entries for the chunks' own levels.
size_t host_part_entries(size_t n);
hs_status merge_sort_host_chunked(int32_t *h_keys, int32_t *d_keys, size_t n, hs_netset s,
                                  void *d_ws, int64_t *d_part, cudaStream_t st);
int64_t pairs_tile(int L);
size_t merge_workspace_bytes_i64(size_t n);
int64_t tile64(int L, int64_t n);  // int64 block-sort tile for n keys
hs_status merge_sort_i64(int64_t *d_keys, size_t n, hs_netset s, void *d_ws, size_t ws_bytes,
                         cudaStream_t st);

// Tile of the keys block sort of an n-key array for leaf size L, and its
// shape options.
int64_t keys_tile(int L, int64_t n);
// One CTA sorts a whole array of up to small_sort_max(L) keys in one launch
// (no workspace).
int64_t small_sort_max(int L);
hs_status small_sort(int32_t *keys, int64_t n, hs_netset s, cudaStream_t st);
void merge_set_blocksort_shape(int v);
void merge_set_fanin(int v);

// Launch plan of the single-array merge path (see hs_sort_plan).
struct SortPlan {
    int shape;  // block-sort shape: 2 (256 threads) or 4 (288 threads)
    int fanin;  // merge fan-in of the tiled keys levels: 2 or 4
};
void sort_plan_force(const SortPlan *p);  // this thread's override (null clears)
// Whether the merge levels over these keys can run four-way (16-byte
// aligned keys, n a multiple of 4); otherwise the fan-in is always 2.
bool merge_four_way_possible(const int32_t *d_keys, int64_t n);
// The plan the merge path takes for these keys now (forced, options, cache, rules).
SortPlan merge_plan_for(const int32_t *d_keys, int64_t n, int L);
int size_bucket(int64_t n);               // floor(log2 n)
hs_status current_device_name(std::string *out);
void sort_plan_cache_put(const std::string &device, int n_bucket, int leaf, const SortPlan &p,
                         double ms);
bool sort_plan_cache_get(const std::string &device, int n_bucket, int leaf, SortPlan *p,
                         double *ms);
void sort_plan_cache_clear();
void sort_plan_cache_each(void (*fn)(void *, const std::string &, int, int, const SortPlan &, double),
                          void *ctx);
int merge_fanin();  // the option's value: 0 (by size), 2 or 4

// Block sort of [0, n) in tiles of keys_tile(L) keys (the merge path's first pass;
// the whole sort when n fits one tile).
hs_status blocksort_launch(int L, const int32_t *kin, int32_t *kout, int64_t n, hs_netset s,
                           int vec, cudaStream_t st, int32_t *samp = nullptr);

// Device address of the current device's status word (kernels OR status bits
// into it), and the check that waits for `st`, then reads and clears it.
hs_status device_status(unsigned **out);
hs_status device_check(cudaStream_t st);

size_t quick_workspace_bytes(size_t n);
void quick_set_max_levels(int64_t v);
void quick_set_two_way(int v);
hs_status quick_sort(int32_t *d_keys, size_t n, hs_netset s, void *d_ws, size_t ws_bytes,
                     cudaStream_t st);

}  // namespace hs
