// Library runtime: error strings, launch counting, optional per-kernel event
// timing, the top-level entry points and the host build of the networks.
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hs_internal.h"
#include "hs_bulk.cuh"
#include "hs_common.cuh"
#include "hs_networks.cuh"
#include "hs_merge4.cuh"

namespace hs {

// NVTX range names of the launches ("hs:" + the kernel name), so that a
// profiler can select one kernel's launches (ncu --nvtx --nvtx-include).
static const char *const kRangeNames[K_COUNT] = {
    "hs:blocksort_keys", "hs:blocksort_pairs", "hs:merge_partition", "hs:merge_keys",
    "hs:merge_pairs",    "hs:qs_plan",         "hs:qs_partition",    "hs:qs_leaves",
    "hs:seg_classify",   "hs:seg_sort",        "hs:selftest",        "hs:merge4_keys"};

static const char *const kKernelNames[K_COUNT] = {
    "blocksort_keys", "blocksort_pairs", "merge_partition", "merge_keys",
    "merge_pairs",    "qs_plan",         "qs_partition",
    "qs_leaves",      "seg_classify",    "seg_sort",
    "selftest",       "merge4_keys"};

const char *kernel_name(int id) { return (id >= 0 && id < K_COUNT) ? kKernelNames[id] : "?"; }

static thread_local std::string t_last_error;

hs_status fail(hs_status st, const std::string &msg) {
    t_last_error = msg;
    return st;
}

hs_status fail_cuda(cudaError_t e, const char *what) {
    t_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) +
                   ")";
    return HS_ERR_CUDA;
}

void clear_error() { t_last_error.clear(); }

// ------------------------------------------------------------ launch stats
static std::atomic<uint64_t> g_launches{0};
static std::atomic<int> g_prof_on{0};
static std::atomic<int> g_prof_only{-1};  // kernel id timed alone, or -1 for all

struct ProfSlot {
    int id;
    cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static std::vector<ProfSlot> g_prof_pending;
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_event_pool;
static uint64_t g_prof_count[K_COUNT];
static double g_prof_ms[K_COUNT];

ApiRange::ApiRange(const char *name) { nvtxRangePushA(name); }
ApiRange::~ApiRange() { nvtxRangePop(); }

static thread_local uint64_t *t_capture_counter = nullptr;
void capture_launches_into(uint64_t *counter) { t_capture_counter = counter; }

LaunchToken launch_begin(int id, cudaStream_t stream) {
    nvtxRangePushA(kRangeNames[id]);  // popped by launch_end
    LaunchToken t{id, stream, nullptr, nullptr};
    const int only = g_prof_only.load(std::memory_order_relaxed);
    if (g_prof_on.load(std::memory_order_relaxed) && (only < 0 || only == id)) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
        if (!g_event_pool.empty()) {
            ev = g_event_pool.back();
            g_event_pool.pop_back();
        } else if (cudaEventCreate(&ev.first) != cudaSuccess ||
                   cudaEventCreate(&ev.second) != cudaSuccess) {
            cudaGetLastError();
            return t;
        }
        cudaEventRecord(ev.first, stream);
        t.ev_a = ev.first;
        t.ev_b = ev.second;
    }
    return t;
}

hs_status launch_end(const LaunchToken &t) {
    nvtxRangePop();
    cudaError_t e = cudaGetLastError();
    if (t_capture_counter) *t_capture_counter += 1;
    else g_launches.fetch_add(1, std::memory_order_relaxed);
    if (t.ev_a) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        cudaEventRecord(t.ev_b, t.stream);
        g_prof_pending.push_back({t.id, t.ev_a, t.ev_b});
    }
    if (e != cudaSuccess) return fail_cuda(e, kernel_name(t.id));
    return HS_OK;
}

void count_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

bool prof_enabled() { return g_prof_on.load(std::memory_order_relaxed) != 0; }

static std::atomic<uint64_t> g_config_gen{1};
uint64_t config_generation() { return g_config_gen.load(); }
void bump_config_generation() { g_config_gen.fetch_add(1); }

static void prof_drain_locked() {
    for (auto &s : g_prof_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(s.b) == cudaSuccess && cudaEventElapsedTime(&ms, s.a, s.b) == cudaSuccess) {
            g_prof_count[s.id] += 1;
            g_prof_ms[s.id] += ms;
        } else {
            cudaGetLastError();
        }
        g_event_pool.push_back({s.a, s.b});
    }
    g_prof_pending.clear();
}

// Device status word raised by kernels instead of trapping (bounded waits
// that gave up, malformed offsets); one copy per device.
static __device__ unsigned g_status;

hs_status device_status(unsigned **out) {
    static std::mutex mu;
    static unsigned *addr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(HS_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, g_status)) != cudaSuccess)
            return fail_cuda(e, "cudaGetSymbolAddress(status)");
        addr[dev] = static_cast<unsigned *>(p);
    }
    *out = addr[dev];
    return HS_OK;
}

// Diagnostic kernel of hs_bulk_wait_selftest: one CTA arms an mbarrier for
// 16 bytes of bulk-copy transactions, issues no copy, and waits as the
// bulk-copy kernels do, with `polls` polls.  The wait gives up, the CTA
// raises the status word and returns; nothing is left in flight.
static __global__ void k_bulk_wait_selftest(long polls, unsigned *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16u);
    const bool ok = mbar_wait(&bar, 0, polls);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
        return;
    }
}

hs_status device_check(cudaStream_t st) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(e, "hs_device_check: stream synchronize");
    unsigned *p = nullptr;
    hs_status r = device_status(&p);
    if (r != HS_OK) return r;
    unsigned v = 0;
    if ((e = cudaMemcpy(&v, p, sizeof v, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail_cuda(e, "hs_device_check: read status");
    if (v) {
        const unsigned zero = 0;
        if ((e = cudaMemcpy(p, &zero, sizeof zero, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail_cuda(e, "hs_device_check: clear status");
        if (v & kStatusTimeout)
            return fail(HS_ERR_TIMEOUT, "a kernel gave up on a bounded wait");
        if (v & kStatusMisaligned)
            return fail(HS_ERR_CUDA, "a kernel found bulk-copy addresses that are not 16-byte aligned");
        if (v & kStatusInconsistent)
            return fail(HS_ERR_CUDA, "a kernel found merge splits that would stage outside its buffer");
        return fail(HS_ERR_INVALID_ARG, "a kernel found malformed segment offsets");
    }
    return HS_OK;
}

hs_status ensure_smem(const void *func, int bytes) {
    if (bytes <= 48 * 1024) return HS_OK;
    // One flag per (function, device): the attribute is set per device.
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(mu);
    for (auto &d : done)
        if (d.first == func && d.second == dev) return HS_OK;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return fail_cuda(e, "cudaFuncSetAttribute");
    done.push_back({func, dev});
    return HS_OK;
}

template <int K>
static void merge_split_k(const int32_t *keys, const int32_t *samp, const int64_t *starts,
                          const int64_t *lens, int64_t rank, int64_t *a) {
    KwayRuns<K> R;
    R.keys = keys;
    R.samp = samp;
    for (int i = 0; i < K; ++i) {
        R.start[i] = starts[i];
        R.len[i] = lens[i];
    }
    int64_t out[K];
    kway_split<K>(R, rank, out);
    for (int i = 0; i < K; ++i) a[i] = out[i];
}

}  // namespace hs

using namespace hs;

extern "C" {

const char *hs_status_str(hs_status st) {
    switch (st) {
        case HS_OK: return "HS_OK";
        case HS_ERR_INVALID_ARG: return "HS_ERR_INVALID_ARG";
        case HS_ERR_UNSUPPORTED: return "HS_ERR_UNSUPPORTED";
        case HS_ERR_NO_MEMORY: return "HS_ERR_NO_MEMORY";
        case HS_ERR_CUDA: return "HS_ERR_CUDA";
        case HS_ERR_TIMEOUT: return "HS_ERR_TIMEOUT";
        case HS_ERR_OVER_BUDGET: return "HS_ERR_OVER_BUDGET";
    }
    return "HS_ERR_UNKNOWN";
}

const char *hs_last_error(void) { return t_last_error.c_str(); }

const char *hs_version(void) { return "hsort 0.1 (sm_103a)"; }

uint64_t hs_launch_count(void) { return g_launches.load(); }

void hs_prof_enable(int on) { g_prof_on.store(on ? 1 : 0); }

hs_status hs_prof_select(const char *kernel) {
    clear_error();
    if (!kernel) {
        g_prof_only.store(-1);
        return HS_OK;
    }
    for (int i = 0; i < K_COUNT; ++i)
        if (std::strcmp(kernel, kKernelNames[i]) == 0) {
            g_prof_only.store(i);
            return HS_OK;
        }
    return fail(HS_ERR_INVALID_ARG, std::string("hs_prof_select: unknown kernel ") + kernel);
}

void hs_prof_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain_locked();
    for (int i = 0; i < K_COUNT; ++i) {
        g_prof_count[i] = 0;
        g_prof_ms[i] = 0.0;
    }
}

hs_status hs_prof_read(const char *kernel, uint64_t *launches, double *total_ms) {
    if (!kernel || !launches || !total_ms) return fail(HS_ERR_INVALID_ARG, "hs_prof_read: NULL argument");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain_locked();
    *launches = 0;
    *total_ms = 0.0;
    for (int i = 0; i < K_COUNT; ++i)
        if (std::strcmp(kernel, kKernelNames[i]) == 0) {
            *launches = g_prof_count[i];
            *total_ms = g_prof_ms[i];
        }
    return HS_OK;
}

size_t hs_sort_workspace_bytes(size_t n, int with_values, hs_algo a) {
    if (a == HS_ALGO_QUICK) return quick_workspace_bytes(n);
    return merge_workspace_bytes(n, with_values);
}

static hs_status check_common(const void *d_keys, size_t n, hs_algo a, hs_netset s, const char *fn) {
    if (a != HS_ALGO_MERGE && a != HS_ALGO_QUICK)
        return fail(HS_ERR_INVALID_ARG, std::string(fn) + ": unknown algo");
    if (!netset_ok(s))
        return fail(HS_ERR_INVALID_ARG, std::string(fn) + ": netset is neither a set of sizes 3..8 nor a VarSort configuration");
    if (n > 0 && !d_keys) return fail(HS_ERR_INVALID_ARG, std::string(fn) + ": NULL keys with n > 0");
    if (n > 0 && !aligned(d_keys, 4)) return fail(HS_ERR_INVALID_ARG, std::string(fn) + ": keys not 4-byte aligned");
    if (n > (size_t)INT64_MAX / 16) return fail(HS_ERR_INVALID_ARG, std::string(fn) + ": n too large");
    return HS_OK;
}

hs_status hs_sort_i32(int32_t *d_keys, size_t n, hs_algo a, hs_netset s, void *d_ws,
                      size_t ws_bytes, hs_stream_t stream) {
    const ApiRange range("hs_sort_i32");
    clear_error();
    hs_status st = check_common(d_keys, n, a, s, "hs_sort_i32");
    if (st != HS_OK) return st;
    if (n <= 1) return HS_OK;
    if (a == HS_ALGO_QUICK) return quick_sort(d_keys, n, s, d_ws, ws_bytes, (cudaStream_t)stream);
    return merge_sort_graphed(d_keys, nullptr, n, s, d_ws, ws_bytes, (cudaStream_t)stream);
}

hs_status hs_sort_pairs_i32(int32_t *d_keys, int32_t *d_vals, size_t n, hs_algo a, hs_netset s,
                            void *d_ws, size_t ws_bytes, hs_stream_t stream) {
    const ApiRange range("hs_sort_pairs_i32");
    clear_error();
    hs_status st = check_common(d_keys, n, a, s, "hs_sort_pairs_i32");
    if (st != HS_OK) return st;
    if (n > 0 && (!d_vals || !aligned(d_vals, 4)))
        return fail(HS_ERR_INVALID_ARG, "hs_sort_pairs_i32: NULL or unaligned values with n > 0");
    if (a == HS_ALGO_QUICK)
        return fail(HS_ERR_UNSUPPORTED, "hs_sort_pairs_i32: quick sort is not stable; use HS_ALGO_MERGE");
    if (n <= 1) return HS_OK;
    return merge_sort_graphed(d_keys, d_vals, n, s, d_ws, ws_bytes, (cudaStream_t)stream);
}

size_t hs_sort_i64_workspace_bytes(size_t n) { return merge_workspace_bytes_i64(n); }

hs_status hs_sort_i64(int64_t *d_keys, size_t n, hs_algo a, hs_netset s, void *d_ws,
                      size_t ws_bytes, hs_stream_t stream) {
    const ApiRange range("hs_sort_i64");
    clear_error();
    if (a != HS_ALGO_MERGE && a != HS_ALGO_QUICK)
        return fail(HS_ERR_INVALID_ARG, "hs_sort_i64: unknown algorithm");
    if (!netset_ok(s))
        return fail(HS_ERR_INVALID_ARG, "hs_sort_i64: netset is neither a set of sizes 3..8 nor a VarSort configuration");
    if (n > 0 && !d_keys) return fail(HS_ERR_INVALID_ARG, "hs_sort_i64: NULL keys with n > 0");
    if (n > 0 && !aligned(d_keys, 8)) return fail(HS_ERR_INVALID_ARG, "hs_sort_i64: keys not 8-byte aligned");
    if (n > (size_t)INT64_MAX / 16) return fail(HS_ERR_INVALID_ARG, "hs_sort_i64: n too large");
    if (a == HS_ALGO_QUICK)
        return fail(HS_ERR_UNSUPPORTED, "hs_sort_i64: int64 keys use the merge path");
    if (n <= 1) return HS_OK;
    return merge_sort_i64_graphed(d_keys, n, s, d_ws, ws_bytes, (cudaStream_t)stream);
}

size_t hs_sort_host_workspace_bytes(size_t n, hs_algo a) {
    // [device keys][sort workspace][partition entries of the chunks' levels]
    return align_up(n * sizeof(int32_t), 256) + align_up(hs_sort_workspace_bytes(n, 0, a), 256) +
           (a == HS_ALGO_MERGE ? align_up(host_part_entries(n) * sizeof(int64_t), 256) : 0);
}

hs_status hs_sort_i32_host(int32_t *h_keys, size_t n, hs_algo a, hs_netset s, void *d_ws,
                           size_t ws_bytes, hs_stream_t stream) {
    const ApiRange range("hs_sort_i32_host");
    clear_error();
    hs_status st = check_common(h_keys, n, a, s, "hs_sort_i32_host");
    if (st != HS_OK) return st;
    if (n <= 1) return HS_OK;
    size_t need = hs_sort_host_workspace_bytes(n, a);
    if (!d_ws || ws_bytes < need)
        return fail(HS_ERR_INVALID_ARG, "hs_sort_i32_host: workspace smaller than hs_sort_host_workspace_bytes");
    if (!aligned(d_ws, 16)) return fail(HS_ERR_INVALID_ARG, "hs_sort_i32_host: workspace not 16-byte aligned");
    cudaStream_t cs = (cudaStream_t)stream;
    int32_t *d_keys = static_cast<int32_t *>(d_ws);
    size_t kb = align_up(n * sizeof(int32_t), 256);
    // Large merge sorts overlap the copy in with per-chunk sorts.
    if (a == HS_ALGO_MERGE && n >= ((size_t)1 << 22)) {
        const size_t wb = align_up(hs_sort_workspace_bytes(n, 0, a), 256);
        return merge_sort_host_chunked(h_keys, d_keys, n, s, static_cast<char *>(d_ws) + kb,
                                       reinterpret_cast<int64_t *>(static_cast<char *>(d_ws) + kb + wb), cs);
    }
    cudaError_t e = cudaMemcpyAsync(d_keys, h_keys, n * sizeof(int32_t), cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return fail_cuda(e, "hs_sort_i32_host: host-to-device copy");
    st = hs_sort_i32(d_keys, n, a, s, static_cast<char *>(d_ws) + kb, ws_bytes - kb, stream);
    if (st != HS_OK) return st;
    e = cudaMemcpyAsync(h_keys, d_keys, n * sizeof(int32_t), cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess) return fail_cuda(e, "hs_sort_i32_host: device-to-host copy");
    e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return fail_cuda(e, "hs_sort_i32_host: stream synchronize");
    return HS_OK;
}

hs_status hs_bulk_wait_selftest(uint32_t polls, hs_stream_t stream) {
    clear_error();
    if (polls < 1 || polls > (uint32_t)kBulkSpinLimit)
        return fail(HS_ERR_INVALID_ARG, "hs_bulk_wait_selftest: polls must be in [1, 2^22]");
    unsigned *status = nullptr;
    hs_status r = device_status(&status);
    if (r != HS_OK) return r;
    LaunchToken t = launch_begin(K_SELFTEST, (cudaStream_t)stream);
    k_bulk_wait_selftest<<<1, 64, 0, (cudaStream_t)stream>>>((long)polls, status);
    return launch_end(t);
}

hs_status hs_device_check(hs_stream_t stream) {
    clear_error();
    return device_check((cudaStream_t)stream);
}

hs_status hs_set_option(const char *name, int64_t value) {
    clear_error();
    if (!name) return fail(HS_ERR_INVALID_ARG, "hs_set_option: NULL name");
    bump_config_generation();
    if (std::strcmp(name, "sort_graphs") == 0) {
        if (value != 0 && value != 1)
            return fail(HS_ERR_INVALID_ARG, "hs_set_option: sort_graphs must be 0 or 1");
        sort_graphs_enable((int)value);
        return HS_OK;
    }
    if (std::strcmp(name, "quick_max_levels") == 0) {
        quick_set_max_levels(value);
        return HS_OK;
    }
    if (std::strcmp(name, "quick_partition") == 0) {
        if (value != 2 && value != 3)
            return fail(HS_ERR_INVALID_ARG, "hs_set_option: quick_partition must be 2 or 3");
        quick_set_two_way(value == 2 ? 1 : 0);
        return HS_OK;
    }
    if (std::strcmp(name, "blocksort_shape") == 0) {
        if (value != -1 && value != 2 && value != 4)
            return fail(HS_ERR_INVALID_ARG, "hs_set_option: blocksort_shape must be -1, 2 or 4");
        merge_set_blocksort_shape((int)value);
        return HS_OK;
    }
    if (std::strcmp(name, "merge_fanin") == 0) {
        if (value != 0 && value != 2 && value != 4)
            return fail(HS_ERR_INVALID_ARG, "hs_set_option: merge_fanin must be 0, 2 or 4");
        merge_set_fanin((int)value);
        return HS_OK;
    }
    return fail(HS_ERR_INVALID_ARG, std::string("hs_set_option: unknown option ") + name);
}

size_t hs_keys_tile(hs_netset s, size_t n) {
    if (!netset_ok(s)) return 0;
    return (size_t)keys_tile(leaf_size(s), (int64_t)n);
}

size_t hs_i64_tile(hs_netset s, size_t n) {
    if (!netset_ok(s)) return 0;
    return (size_t)tile64(leaf_size(s), (int64_t)n);
}

size_t hs_pairs_tile(hs_netset s) {
    if (!netset_ok(s)) return 0;
    return (size_t)pairs_tile(leaf_size(s));
}

int hs_network_pairs(int m, int *pairs, int cap) {
    if (m < 2 || m > 8) return -1;
    CountCE op;
    op.pairs = pairs;
    op.cap = cap;
    network_dyn(m, op);
    return op.n;
}

int hs_merge_split(const int32_t *keys, const int32_t *samp, const int64_t *starts,
                   const int64_t *lens, int k_runs, int64_t rank, int64_t *a) {
    if (!starts || !lens || !a || (k_runs != 2 && k_runs != 4 && k_runs != 8)) return -1;
    int64_t total = 0;
    for (int i = 0; i < k_runs; ++i) {
        if (lens[i] < 0 || starts[i] < 0) return -1;
        if (lens[i] > 0 && !keys) return -1;
        if (samp && starts[i] % kSampleStride != 0) return -1;
        total += lens[i];
    }
    if (rank < 0 || rank > total) return -1;
    switch (k_runs) {
        case 2: merge_split_k<2>(keys, samp, starts, lens, rank, a); break;
        case 4: merge_split_k<4>(keys, samp, starts, lens, rank, a); break;
        default: merge_split_k<8>(keys, samp, starts, lens, rank, a); break;
    }
    return 0;
}

int hs_network_apply(int m, int32_t *a) {
    if (m < 2 || m > 8 || !a) return -1;
    KeyCE op{a};
    switch (m) {  // a[] is a caller array of exactly m keys
        case 2: network<2>(op); break;
        case 3: network<3>(op); break;
        case 4: network<4>(op); break;
        case 5: network<5>(op); break;
        case 6: network<6>(op); break;
        case 7: network<7>(op); break;
        case 8: network<8>(op); break;
    }
    return 0;
}

}  // extern "C"
