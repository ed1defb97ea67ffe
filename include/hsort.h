/*
 * hsort: hybrid network-leaf sorting of int32 keys on one GB300 (sm_103a).
 *
 * The method is that of Aly, Jensen and ElAarag, "Improving Merge Sort and
 * Quick Sort Performance by Utilizing AlphaDev's Sorting Networks as Base
 * Cases" (ACMSE 2025):
 *   - Algorithm 1 (Optimized Merge Sort with Sorting Networks): subarrays whose
 *     size has a fixed sorting network are sorted by that network; everything
 *     above them is sorted by Merge.
 *   - Algorithm 2 (Optimized Quick Sort with Sorting Networks): the same leaves
 *     under median-of-three partitioning.
 *   - Table 3 (Sorting Network Configurations): which network sizes (3..8) a
 *     configuration may use; see hs_netset below.
 * On the GPU a leaf is a thread's register tile sorted by a branch-free
 * network; merge-path partitioned merges (or 3-way partitions) do the rest.
 *
 * Conventions for every call:
 *   - Device pointers come from cudaMalloc (or any allocation the device can
 *     address); the caller owns every buffer.  Sorting is in place.
 *   - Workspace is caller-provided: query its size first.  No call below
 *     allocates device memory on the sorting path.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream) unless stated otherwise.  Argument errors are detected
 *     on the host before any launch and return synchronously.
 *   - Keys use the signed int32 order.  No C++ exception crosses this ABI.
 *   - A failing call returns a status; hs_last_error() (thread-local) then
 *     holds a one-line message.
 */
#ifndef HSORT_H
#define HSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define HS_API __attribute__((visibility("default")))
#else
#define HS_API
#endif

typedef void *hs_stream_t; /* a cudaStream_t */

typedef enum {
    HS_OK = 0,
    HS_ERR_INVALID_ARG = 1, /* bad pointer, size, netset, algo or workspace */
    HS_ERR_UNSUPPORTED = 2, /* valid request the library does not serve */
    HS_ERR_NO_MEMORY = 3,   /* a host-side allocation failed */
    HS_ERR_CUDA = 4,        /* a CUDA runtime call or launch failed */
    HS_ERR_TIMEOUT = 5,     /* a bounded device or host wait gave up */
    HS_ERR_OVER_BUDGET = 6  /* request larger than a server's memory budget */
} hs_status;

typedef enum {
    HS_ALGO_MERGE = 0, /* Algorithm 1: network leaves + merge passes */
    HS_ALGO_QUICK = 1  /* Algorithm 2: network leaves + 3-way partitions */
} hs_algo;

/* Network set (Table 3): bit k set <=> the size-k network may be used,
 * k in 3..8.  0 is the classical algorithm (no networks).  HS_NETS_VARSORT
 * with exactly one size bit k is VarSortk (Table 3's VarSort3/4/5, a
 * "dynamic sorting network" for any input of up to k elements): every leaf
 * of up to k keys is sorted by the size-k network on +infinity-padded input.
 * Any other bit pattern is HS_ERR_INVALID_ARG.  The GPU leaf is the largest
 * size in the set; a ragged last leaf of r keys uses the size-r network when
 * the set has it, else the next larger size in the set padded with +infinity
 * sentinels (so on the GPU VarSortk and the set {k} run the same networks). */
typedef uint32_t hs_netset;
#define HS_NETS_NONE 0x000u
#define HS_NETS_3 0x008u        /* {3} */
#define HS_NETS_3TO4 0x018u     /* {3,4} */
#define HS_NETS_3TO5 0x038u     /* {3,4,5} */
#define HS_NETS_6TO8 0x1C0u     /* {6,7,8} */
#define HS_NETS_3TO8 0x1F8u     /* {3,...,8} */
#define HS_NETS_POWEROF2 0x110u /* {4,8} */
#define HS_NETS_EVEN 0x150u     /* {4,6,8} */
#define HS_NETS_ODD 0x0A8u      /* {3,5,7} */
#define HS_NETS_VARSORT 0x10000u
#define HS_NETS_VARSORT3 0x10008u /* VarSort3 */
#define HS_NETS_VARSORT4 0x10010u /* VarSort4 */
#define HS_NETS_VARSORT5 0x10020u /* VarSort5 */

/* ---------------------------------------------------------------- sorting */

/* Workspace bytes for sorting n keys (with_values != 0: key/value pairs) with
 * algorithm a.  Valid for every network set.  The workspace must be 16-byte
 * aligned; it holds a ping-pong copy of the keys (and values) plus
 * partition indices. */
HS_API size_t hs_sort_workspace_bytes(size_t n, int with_values, hs_algo a);

/* Sorts d_keys[0..n-1] ascending in place (Algorithm 1 for HS_ALGO_MERGE,
 * Algorithm 2 for HS_ALGO_QUICK) with the network set s.
 *   d_keys   device pointer, 4-byte aligned (16-byte alignment enables the
 *            vectorised paths); may be NULL only when n == 0.
 *   n        number of keys; 0 and 1 are no-ops.
 *   d_ws     device workspace of ws_bytes >= hs_sort_workspace_bytes(n, 0, a).
 * MERGE is fully asynchronous, and a caller may capture it into its own CUDA
 * graph.  A merge sort of more than one tile called again with the same
 * keys and workspace addresses, n and s (on any stream, from the same host
 * thread) is captured into a library graph on its second call and replayed
 * from then on: the same kernels, with one graph launch instead of one
 * launch per kernel (option "sort_graphs").  The graphs belong to the CUDA
 * context they were captured in and are kept for the life of the process:
 * with "sort_graphs" on, do not sort across a cudaDeviceReset of a device the
 * library has sorted on (a later call could replay or free a graph of the old
 * context).  QUICK learns each partition level's
 * counters through mapped host memory and waits for the level two behind the
 * one it launches, so the call returns only when all but the last levels have
 * run, and it cannot be captured in a CUDA graph.  It also runs each level's
 * leaf sorts on a library-owned second stream (one per host thread and
 * device), joined back into `stream` before it returns; its work is complete
 * when `stream` reaches that point.
 * Errors: HS_ERR_INVALID_ARG for a NULL/unaligned pointer with n > 0, an
 * unknown algo, netset bits outside 3..8 or a short workspace;
 * HS_ERR_CUDA if a launch fails. */
HS_API hs_status hs_sort_i32(int32_t *d_keys, size_t n, hs_algo a, hs_netset s, void *d_ws,
                      size_t ws_bytes, hs_stream_t stream);

/* Stable key/value sort: d_keys and d_vals (n each) are permuted together so
 * that keys ascend and equal keys keep their input order.  Networks compare
 * (key, input position); merges take the left run on ties.
 *   a must be HS_ALGO_MERGE: QUICK is not stable -> HS_ERR_UNSUPPORTED.
 *   d_ws: ws_bytes >= hs_sort_workspace_bytes(n, 1, HS_ALGO_MERGE).
 * Other conventions and errors as hs_sort_i32 (graph replay of repeated calls
 * included: the signature also holds d_vals). */
HS_API hs_status hs_sort_pairs_i32(int32_t *d_keys, int32_t *d_vals, size_t n, hs_algo a,
                            hs_netset s, void *d_ws, size_t ws_bytes, hs_stream_t stream);

/* int64 keys (Algorithm 1 on 8-byte keys, the same network leaves and merge
 * levels as hs_sort_i32): sorts d_keys[0..n) (signed order) in place.  Merge
 * path only: HS_ALGO_QUICK returns HS_ERR_UNSUPPORTED.  d_keys must be 8-byte
 * aligned; the workspace (hs_sort_i64_workspace_bytes, 16-byte aligned,
 * owned by the caller) holds a keys copy, the merge partitions and every
 * 32nd key.  Errors as hs_sort_i32.  Asynchronous on stream; repeated calls
 * replay a captured graph as hs_sort_i32's merge path does. */
HS_API size_t hs_sort_i64_workspace_bytes(size_t n);
HS_API hs_status hs_sort_i64(int64_t *d_keys, size_t n, hs_algo a, hs_netset s, void *d_ws,
                             size_t ws_bytes, hs_stream_t stream);

/* Host-buffer form, for callers whose keys live in host memory: copies
 * h_keys to the device, sorts them as hs_sort_i32 does, copies the result
 * back into h_keys and waits for `stream` before returning (synchronous).
 * For merge sorts of 2^22 keys or more the copy in travels in at most 8
 * chunks on a library-created copy stream; each chunk is sorted completely on
 * one of four library-created side streams as soon as it has arrived (the
 * chunks' sorts overlap one another and the copy of the next chunks); merge
 * levels over the sorted chunks on `stream` finish the sort, and the last
 * one runs in eight parts whose keys are copied out as soon as each is done.
 * The copy and side streams and their events are created by the first such
 * call per host thread and device and kept for the life of the process.
 * Pinned host memory makes the copies faster; pageable memory also works.
 *   d_ws: ws_bytes >= hs_sort_host_workspace_bytes(n, a); it holds the
 *   device copy of the keys, the sort workspace and (merge) the chunks'
 *   partition entries. */
HS_API size_t hs_sort_host_workspace_bytes(size_t n, hs_algo a);
HS_API hs_status hs_sort_i32_host(int32_t *h_keys, size_t n, hs_algo a, hs_netset s, void *d_ws,
                           size_t ws_bytes, hs_stream_t stream);

/* Allocation-free merge sort, for callers that cannot allocate device memory:
 * for example a plugin whose host application owns every device allocation
 * and forbids side allocations, code that runs under a device-memory budget
 * fixed at start-up, or a latency-critical path where cudaMalloc may
 * synchronise the device and stall.  The paper has no counterpart; this is a
 * library convenience around the HS_ALGO_MERGE path of hs_sort_i32.
 *   d_keys, n, s, stream   as hs_sort_i32; no workspace argument.
 *   Scratch: a fixed __device__ array of 17,433,344 bytes (16.6 MiB) inside
 *     the library (keys copy, partition entries and samples for
 *     HS_NOALLOC_MAX_KEYS keys).  Every GPU where the library's code is loaded
 *     holds it until the process exits.
 *   Limit: n <= HS_NOALLOC_MAX_KEYS (2^22 = 4,194,304 keys); a larger n returns
 *     HS_ERR_INVALID_ARG before any launch.
 *   Set-up: the first call on a device, with that device current, looks up the
 *     scratch array's device address (cudaGetSymbolAddress) and caches it for
 *     the life of the process; make that first call before any stream capture.
 *     The current device must be the one that owns d_keys and stream.  Do not
 *     use this entry point across a cudaDeviceReset of a device it has run on:
 *     the cached address belongs to the context that the reset destroyed.
 *   Sharing: every call uses the same scratch array, which keeps the previous
 *     call's contents (nothing in it needs to start at zero).  Calls whose GPU
 *     work overlaps (other streams, other host threads) race on it: serialise
 *     them.
 *   Calls no cudaMalloc, cudaFree or other allocating routine.  Asynchronous
 *   on stream; other errors as hs_sort_i32. */
#define HS_NOALLOC_MAX_KEYS 4194304u
HS_API hs_status hs_sort_i32_noalloc(int32_t *d_keys, size_t n, hs_netset s, hs_stream_t stream);

/* ------------------------------------------------ single-array launch plan */

/* Launch plan of the single-array merge path (hs_sort_i32 with
 * HS_ALGO_MERGE, its host-buffer form and the server's sorts).  Both fields
 * change only the time, never the result.  The path decides each of them, in
 * this order: the options "blocksort_shape" / "merge_fanin" when set to a
 * value other than their automatic one; a plan hs_sort_autotune (or
 * hs_tune_cache_load) cached for this device, this array size's log2
 * bucket and this leaf size; the built-in rules (the larger block-sort tile
 * when it saves a merge level; four-way levels from 2^27 keys). */
typedef struct {
    int32_t blocksort_threads; /* block-sort CTA: 256 (tile 256 x (4L - 1) keys)
                                  or 288 (288 x (4L - 1) keys); L = leaf size */
    int32_t merge_fanin;       /* runs merged per pass of the global levels: 2 or
                                  4 (four applies only to 16-byte aligned keys
                                  with n % 4 == 0; other arrays merge two-way) */
    int32_t reserved[2];       /* 0 */
} hs_sort_plan;

/* Autotuner of the single-array merge path: times every candidate plan
 * (blocksort_threads 256 / 288 x merge_fanin 2 / 4 where four-way applies),
 * one warm-up and two timed sorts each with CUDA events on `stream`, on the
 * caller's keys with network set s, and returns the fastest in *best (its
 * time, the smaller of the two, in *best_ms if non-NULL).  The keys are
 * restored to their input order afterwards.  The winner is cached
 * in-process by device name, floor(log2 n) and leaf size, and from then on
 * the merge path uses it for every array in that bucket (unless an option
 * overrides it); a cached entry is returned without timing.  The cache is
 * saved and loaded with the batched form's (hs_tune_cache_save / _load,
 * entries of kind "sort").  n <= 1 returns {256, 2} without timing.
 * Synchronous.
 *   d_keys  device keys, 4-byte aligned.
 *   d_ws    ws_bytes >= hs_sort_autotune_workspace_bytes(n), 16-byte
 *           aligned (the merge workspace plus a copy of the keys).
 * Errors: HS_ERR_INVALID_ARG for NULL/unaligned pointers, a bad netset or a
 * short workspace; HS_ERR_CUDA if a copy, launch or event fails (the keys are
 * still restored when the restoring copy itself succeeds). */
HS_API size_t hs_sort_autotune_workspace_bytes(size_t n);
HS_API hs_status hs_sort_autotune(int32_t *d_keys, size_t n, hs_netset s, void *d_ws,
                                  size_t ws_bytes, hs_stream_t stream, hs_sort_plan *best,
                                  double *best_ms);
/* The plan the merge path would take now for n keys at address d_keys
 * (only its 16-byte alignment is read; NULL reads as aligned) with network
 * set s: options, cached plan or rules, as above.  Host only; launches
 * nothing.  HS_ERR_INVALID_ARG for a NULL result or a bad netset. */
HS_API hs_status hs_sort_plan_for(const int32_t *d_keys, size_t n, hs_netset s,
                                  hs_sort_plan *out);

/* ----------------------------------------------------------- batched form */

/* Launch plan of the batched form: which network set forms the leaves and
 * how the persistent kernel is shaped.  hs_segsort_autotune picks one by
 * timing candidates on the caller's data. */
typedef struct {
    hs_netset netset;      /* leaf networks (Table 3 set; leaf = largest size) */
    int32_t block_threads; /* 256 (four leaves per thread) or 512 (two leaves per
                              thread); a tile holds (leaves*leaf - 1)*block_threads keys */
    int32_t ctas_per_sm;   /* persistent CTAs per SM, 1..8; 0 = as many as fit */
    int32_t reserved;      /* must be 0 */
} hs_plan;

/* Workspace for hs_segsort_i32 over n_keys keys in num_segs segments:
 * scratch for every key plus one descriptor per segment. */
HS_API size_t hs_segsort_workspace_bytes(size_t n_keys, size_t num_segs);

/* Sorts every segment d_keys[off[i] .. off[i+1]) (i < num_segs) independently,
 * each ascending, in one persistent launch: one CTA per segment at a time,
 * network leaves and merge levels as in Algorithm 1; segments longer than a
 * tile merge through their own scratch range.
 *   d_offsets  device int64[num_segs + 1], non-decreasing, within [0, n_keys].
 *              Malformed offsets are detected on the device: the segment is
 *              skipped and hs_device_check reports HS_ERR_INVALID_ARG.
 *   a          HS_ALGO_MERGE (QUICK -> HS_ERR_UNSUPPORTED).
 *   s, plan    plan == NULL: the plan hs_segsort_autotune cached for this
 *              device and these size buckets when its network set is s, else
 *              network set s with the default shape; otherwise the plan (its
 *              netset replaces s).
 *   d_ws       ws_bytes >= hs_segsort_workspace_bytes(n_keys, num_segs).
 * No host synchronisation: the call can be captured (see hs_segsort_capture).
 * Designed for segments up to about 2^20 keys (larger ones work but are
 * sorted by a single CTA; use hs_sort_i32 for those). */
HS_API hs_status hs_segsort_i32(int32_t *d_keys, size_t n_keys, const int64_t *d_offsets,
                                size_t num_segs, hs_algo a, hs_netset s, const hs_plan *plan,
                                void *d_ws, size_t ws_bytes, hs_stream_t stream);

/* The same result with one hs_sort_i32 call per segment (the per-array plain
 * launches the batched form is measured against).  h_offsets is a HOST array
 * of num_segs + 1 offsets; d_ws must satisfy hs_sort_workspace_bytes for the
 * longest segment.  Asynchronous on `stream`; stops at the first error. */
HS_API hs_status hs_sort_i32_many(int32_t *d_keys, size_t n_keys, const int64_t *h_offsets,
                                  size_t num_segs, hs_algo a, hs_netset s, void *d_ws,
                                  size_t ws_bytes, hs_stream_t stream);

/* CUDA-graph form: captures the whole hs_segsort_i32 sequence (queue reset,
 * descriptor build, persistent sort) for these exact buffers into a graph;
 * hs_graph_launch replays it on any stream.  The buffers must outlive the
 * graph.  hs_graph_destroy(NULL) is a no-op. */
typedef struct hs_graph hs_graph;
HS_API hs_status hs_segsort_capture(int32_t *d_keys, size_t n_keys, const int64_t *d_offsets,
                                    size_t num_segs, const hs_plan *plan, void *d_ws,
                                    size_t ws_bytes, hs_graph **out);
HS_API hs_status hs_graph_launch(hs_graph *g, hs_stream_t stream);
HS_API void hs_graph_destroy(hs_graph *g);

/* Autotuner: times candidate plans (leaf network set x CTA size x CTAs per
 * SM) on the caller's segments and returns the fastest in *best (and its
 * time in *best_ms).  The keys are restored to their input order afterwards.
 * Results are cached in-process, keyed by device name and size buckets
 * (log2 of n_keys, of num_segs and of the mean segment); a cached entry is
 * returned without timing.  Synchronous.
 *   d_ws: ws_bytes >= hs_segsort_autotune_workspace_bytes(n_keys, num_segs)
 *   (the segsort workspace plus a copy of the keys). */
HS_API size_t hs_segsort_autotune_workspace_bytes(size_t n_keys, size_t num_segs);
/* The plan hs_segsort_i32 takes for plan == NULL with these sizes and network
 * set s (see there); host only, launches nothing.  HS_ERR_INVALID_ARG for a
 * NULL result or a bad netset. */
HS_API hs_status hs_segsort_plan_for(size_t n_keys, size_t num_segs, hs_netset s, hs_plan *out);
HS_API hs_status hs_segsort_autotune(int32_t *d_keys, size_t n_keys, const int64_t *d_offsets,
                                     size_t num_segs, void *d_ws, size_t ws_bytes,
                                     hs_stream_t stream, hs_plan *best, double *best_ms);
/* The autotuners' cache as a JSON file: an array of objects, one per entry,
 * of kind "batched" (hs_segsort_autotune; objects without a kind read as
 * batched) or "sort" (hs_sort_autotune).  Save writes every entry; load
 * merges the file's entries into the in-process cache, all or none
 * (HS_ERR_INVALID_ARG if the file cannot be read or parsed, or an entry
 * holds an invalid plan). */
HS_API hs_status hs_tune_cache_save(const char *path);
HS_API hs_status hs_tune_cache_load(const char *path);
/* Empties both autotuners' in-process caches: the merge path goes back to
 * its built-in rules and the next autotune call times again. */
HS_API void hs_tune_cache_clear(void);

/* ---------------------------------------------------------------- serving */

/* Continuous-batching sort server for one device (the device current at
 * creation).  Requests are device arrays sorted in place with the merge path;
 * a worker thread admits them in arrival order while the memory budget fits
 * (a request counts its keys plus the workspace the server reserves for it),
 * batches everything admitted into one launch per free stream slot (requests
 * of up to 65,536 keys share one persistent batched launch; longer ones run
 * the multi-CTA merge path in the same slot), and keeps up to four slots in
 * flight, so newly admitted work overlaps with running work.  A request's
 * result is the same as hs_sort_i32's on its own.
 *   hs_server_create: budget_bytes >= 1 MiB; the server allocates a workspace
 *     pool of budget_bytes once, plus four streams.
 *   hs_server_submit: returns at once with a ticket; HS_ERR_OVER_BUDGET if the
 *     request alone exceeds the budget; HS_ERR_UNSUPPORTED for HS_ALGO_QUICK.
 *     d_keys must hold its final contents when submit is called: the server's
 *     streams wait on no stream of the caller, so keys written asynchronously
 *     must be complete first (for example, synchronise the stream that wrote
 *     them).  The caller must not touch d_keys until hs_server_wait returns.
 *   hs_server_wait: blocks until the request finished; *result is its status,
 *     *latency_s the seconds from submit to completion.  Each ticket is waited
 *     for once.
 *   hs_server_replay: load generator: submits count requests at arrival_s[i]
 *     seconds after the call (busy-waiting on the host clock), waits for all,
 *     and returns each latency and the total makespan.
 *   hs_server_destroy: finishes all submitted work, then frees everything. */
typedef struct hs_server hs_server;
HS_API hs_status hs_server_create(size_t budget_bytes, hs_server **out);
HS_API hs_status hs_server_submit(hs_server *srv, int32_t *d_keys, size_t n, hs_algo a,
                                  hs_netset s, uint64_t *ticket);
HS_API hs_status hs_server_wait(hs_server *srv, uint64_t ticket, hs_status *result,
                                double *latency_s);
HS_API hs_status hs_server_stats(hs_server *srv, uint64_t *batches, uint64_t *batched_requests,
                                 size_t *bytes_in_use);
HS_API hs_status hs_server_replay(hs_server *srv, const double *arrival_s,
                                  int32_t *const *d_keys, const size_t *n, size_t count,
                                  hs_netset s, double *latency_s, double *makespan_s);
HS_API void hs_server_destroy(hs_server *srv);

/* ------------------------------------------------------- errors, counters */

HS_API const char *hs_status_str(hs_status st);
/* Message of the last failing call on this thread ("" if none). */
HS_API const char *hs_last_error(void);
/* Library version string. */
HS_API const char *hs_version(void);

/* Number of kernels this library has launched in this process. */
HS_API uint64_t hs_launch_count(void);

/* Per-kernel timing with CUDA events recorded on the launching stream around
 * each launch while enabled (off by default; it adds two event records per
 * launch).  hs_prof_read waits for the recorded events, then returns the
 * launches and summed milliseconds of the kernel named `kernel` since the
 * last reset; unknown names give 0 launches.  Names: "blocksort_keys",
 * "blocksort_pairs", "merge_partition" (binary and four-way partitions),
 * "merge_keys" (binary keys levels, and int64 levels), "merge4_keys"
 * (four-way keys levels), "merge_pairs", "qs_plan", "qs_partition",
 * "qs_leaves", "seg_classify", "seg_sort", "selftest". */
HS_API void hs_prof_enable(int on);
/* Restricts the timing to launches of the kernel named `kernel` (the names
 * hs_prof_read accepts), so that the other launches carry no extra events;
 * NULL times every kernel again.  Unknown names return HS_ERR_INVALID_ARG. */
HS_API hs_status hs_prof_select(const char *kernel);
HS_API void hs_prof_reset(void);
HS_API hs_status hs_prof_read(const char *kernel, uint64_t *launches, double *total_ms);

/* Waits for `stream`, then reads and clears the current device's kernel
 * status word.  Kernels never trap: a kernel that meets invalid device-side
 * input (segment offsets that decrease or run past the key count) raises
 * this word and skips that work.  Returns HS_ERR_INVALID_ARG for such input,
 * HS_ERR_TIMEOUT if a bounded device-side wait gave up (such as a merge
 * level's wait for its bulk tile copy), HS_ERR_CUDA on a CUDA error, when a
 * kernel found bulk-copy addresses that are not 16-byte aligned (it then
 * skipped its copies) or when the batched form found merge splits that would
 * stage outside its buffer (it then dropped that segment), else HS_OK.
 * Synchronous. */
HS_API hs_status hs_device_check(hs_stream_t stream);

/* Diagnostic of the bounded waits (no counterpart in the paper: the paper's
 * sorts run on one CPU thread).  The bulk-copy kernels wait on an mbarrier
 * for their tile copies with a limit of 2^22 polls, after which they raise
 * the status word and return instead of hanging.  This call launches one
 * CTA on `stream` that arms such a barrier for 16 bytes, issues no copy and
 * waits with a limit of `polls` polls, so its wait always gives up; a
 * following hs_device_check(stream) returns HS_ERR_TIMEOUT (and clears the
 * word).  Nothing is left in flight and the context stays usable.
 *   polls  1 .. 4194304, else HS_ERR_INVALID_ARG (no launch).
 * Asynchronous; HS_ERR_CUDA if the launch fails. */
HS_API hs_status hs_bulk_wait_selftest(uint32_t polls, hs_stream_t stream);

/* Process-wide tuning knobs (set them while no sort is in flight).
 *   "quick_max_levels": partition levels the quick path runs before its depth
 *     guard merge-sorts the segments still open (default -1 = automatic,
 *     4*ceil(log2 n) + 16).
 *   "quick_partition": 3 (default) 3-way partitions (< / = / > pivot); 2 the
 *     2-way form of Algorithm 2 (left <= pivot <= right, keys equal to the
 *     pivot alternating sides by their rank among the equal keys).
 *   "blocksort_shape": keys block-sort shape, 2: 256 threads, 4: 288 threads,
 *     -1 (default): per array, 4 when its larger tile saves a global level
 *     over 2, else 2.  A thread holds four leaves of leaf, leaf, leaf and
 *     leaf-1 keys, so a tile holds (4 * leaf - 1) * threads keys.
 *   "merge_fanin": 4 the tiled keys levels merge four runs per pass: a
 *     four-way merge-path split per output tile, then two stages of binary
 *     merges in shared memory, one read and one write of every key for two
 *     of Algorithm 1's merge levels (a binary level first when the number of
 *     levels is odd); 2 binary levels only; 0 (default) four-way levels for
 *     arrays of at least 2^27 keys, binary below (the four-way partition's
 *     latency outweighs the saved pass on smaller arrays).
 *   "sort_graphs": 1 (default) hs_sort_i32's merge path replays a captured
 *     graph for repeated calls with the same arguments (see hs_sort_i32); 0
 *     always launches kernel by kernel.  Changing any option, or the tuned
 *     plans, retires the graphs captured before.
 * Tiled levels (bulk-copied tiles, sampled partition searches) serve 16-byte
 * aligned buffers whose length is a multiple of 4 keys (of 2 for int64);
 * other buffers take thread-staged generic forms.  Every option gives
 * identical results.  Unknown names or values return HS_ERR_INVALID_ARG. */
HS_API hs_status hs_set_option(const char *name, int64_t value);

/* Keys per block-sort tile of the merge path for an n-key array and network
 * set s under the current options (the global merge levels above it number
 * ceil(log2(n / tile))); 0 for an invalid set. */
HS_API size_t hs_keys_tile(hs_netset s, size_t n);

/* Pairs per block-sort tile of the stable pair sort for network set s under
 * the current options; 0 for an invalid set. */
HS_API size_t hs_pairs_tile(hs_netset s);

/* Keys per block-sort tile of hs_sort_i64 for an n-key array and network set
 * s (the global merge levels above it number ceil(log2(n / tile))); 0 for an
 * invalid set. */
HS_API size_t hs_i64_tile(hs_netset s, size_t n);

/* --------------------------------------------------------- host checking */

/* The device networks compiled for the host, for exhaustive CPU checks of
 * the comparator lists the kernels use.  hs_network_pairs writes up to cap
 * (lo, hi) pairs of the size-m network and returns its comparator count
 * (-1 if m is outside 2..8); hs_network_apply sorts a[0..m-1] with it. */
HS_API int hs_network_pairs(int m, int *pairs, int cap);
HS_API int hs_network_apply(int m, int32_t *a);

/* The K-way merge-path split of the four-way merge levels (two levels of
 * Algorithm 1's Merge per pass), compiled for the host.  Run i is
 * keys[starts[i] .. starts[i] + lens[i]), sorted ascending; the runs are
 * merged stably (equal keys in run order, run 0 first).  For output rank
 * `rank` (0 <= rank <= sum of lens), a[i] receives the number of elements of
 * run i among the first `rank` outputs of that merge.  samp, when not NULL,
 * holds keys[32 j] at samp[j] (the merge levels' sample array) and every start
 * must be a multiple of 32; the search then reads positions that are
 * multiples of 32 from it.  k_runs is 2, 4 or 8.  Returns 0, or -1 for
 * invalid arguments (nothing written).  Host memory only; no GPU needed. */
HS_API int hs_merge_split(const int32_t *keys, const int32_t *samp, const int64_t *starts,
                          const int64_t *lens, int k_runs, int64_t rank, int64_t *a);

#ifdef __cplusplus
}
#endif
#endif /* HSORT_H */
