// CUDA-graph replay of repeated merge sorts (hs_sort_i32 with HS_ALGO_MERGE,
// hs_sort_pairs_i32, hs_sort_i64).
//
// A merge sort of more than one tile is a fixed sequence of launches whose
// parameters depend only on the arguments (keys, values and workspace
// addresses, n, network set) and on the library's configuration (options,
// tuned plans).
// At the paper's sizes (10^4 to 10^6 keys) the launches, not the kernels,
// take most of the time, and callers that sort the same buffers again and
// again pay that launch cost on every call.  So:
//   * the first call with a given signature runs directly and is remembered;
//   * the second captures the sort on a private stream into a graph
//     (thread-local capture mode), instantiates it and launches it on the
//     caller's stream;
//   * later calls launch the instantiated graph: the same kernels with the
//     same parameters, in the same order, on the caller's stream.
// Entries carry the configuration generation they were captured under and
// are not replayed after an option or a tuned plan changed.  Graphs are not
// used while per-kernel timing is on or when the caller's stream is itself
// being captured (the launches then go into the caller's graph), and the
// option "sort_graphs" = 0 turns them off.  Caches are per host thread: at
// most kGraphs graphs and kSeen remembered signatures, least recently used
// first out.
#include <atomic>
#include <vector>

#include "hs_internal.h"
#include "hs_networks.cuh"

namespace hs {

namespace {

struct Signature {
    int device;
    int kind;  // 0 keys, 1 pairs, 2 int64 keys
    const void *keys, *vals;
    size_t n;
    hs_netset s;
    const void *ws;
    size_t ws_bytes;
    uint64_t gen;
    bool operator==(const Signature &o) const {
        return device == o.device && kind == o.kind && keys == o.keys && vals == o.vals &&
               n == o.n && s == o.s && ws == o.ws && ws_bytes == o.ws_bytes && gen == o.gen;
    }
};

struct Entry {
    Signature sig;
    cudaGraphExec_t exec;
    uint64_t launches;  // kernels in the graph
    uint64_t last_use;
};

constexpr size_t kGraphs = 8, kSeen = 16;

struct ThreadCache {
    std::vector<Entry> graphs;
    std::vector<Signature> seen;
    uint64_t clock = 0;
    int capture_device = -1;
    cudaStream_t capture_stream = nullptr;
};

// Per host thread; never destroyed (graph objects may not outlive the
// context at process exit, so they are left to the driver).
ThreadCache &cache() {
    static thread_local ThreadCache *c = new ThreadCache();
    return *c;
}

}  // namespace

static std::atomic<int> g_sort_graphs{1};
void sort_graphs_enable(int on) { g_sort_graphs.store(on); }

// Runs sort(stream) for signature sig: directly, by capture, or by replay.
// `multi`: the sort makes more than one launch (else a graph gains nothing).
template <class Sort>
static hs_status graphed(Signature sig, bool multi, cudaStream_t st, const Sort &sort) {
    if (!g_sort_graphs.load() || prof_enabled() || !multi) return sort(st);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return sort(st);
    }
    if (cap != cudaStreamCaptureStatusNone) return sort(st);  // the caller is capturing
    cudaError_t e = cudaGetDevice(&sig.device);
    if (e != cudaSuccess) return fail_cuda(e, "sort graphs: current device");
    sig.gen = config_generation();
    ThreadCache &c = cache();
    ++c.clock;
    for (Entry &g : c.graphs)
        if (g.sig == sig) {
            g.last_use = c.clock;
            e = cudaGraphLaunch(g.exec, st);
            if (e != cudaSuccess) return fail_cuda(e, "sort graphs: replay");
            count_launches(g.launches);
            return HS_OK;
        }
    bool seen = false;
    for (size_t i = 0; i < c.seen.size(); ++i)
        if (c.seen[i] == sig) {
            seen = true;
            c.seen.erase(c.seen.begin() + (long)i);
            break;
        }
    if (!seen) {
        if (c.seen.size() >= kSeen) c.seen.erase(c.seen.begin());
        c.seen.push_back(sig);
        return sort(st);
    }
    // Second call with this signature: capture it.
    if (c.capture_device != sig.device) {
        if (c.capture_stream) cudaStreamDestroy(c.capture_stream);
        c.capture_stream = nullptr;
        e = cudaStreamCreateWithFlags(&c.capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            c.capture_stream = nullptr;
            return fail_cuda(e, "sort graphs: capture stream");
        }
        c.capture_device = sig.device;
    }
    e = cudaStreamBeginCapture(c.capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail_cuda(e, "sort graphs: begin capture");
    uint64_t launches = 0;
    capture_launches_into(&launches);
    hs_status r = sort(c.capture_stream);
    capture_launches_into(nullptr);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(c.capture_stream, &graph);
    cudaGraphExec_t exec = nullptr;
    if (r == HS_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (r != HS_OK) return r;
    if (e != cudaSuccess) {
        // Capture is an optimisation: on failure the sort runs directly.
        cudaGetLastError();
        return sort(st);
    }
    if (c.graphs.size() >= kGraphs) {
        size_t old = 0;
        for (size_t i = 1; i < c.graphs.size(); ++i)
            if (c.graphs[i].last_use < c.graphs[old].last_use) old = i;
        cudaGraphExecDestroy(c.graphs[old].exec);
        c.graphs.erase(c.graphs.begin() + (long)old);
    }
    c.graphs.push_back(Entry{sig, exec, launches, c.clock});
    e = cudaGraphLaunch(exec, st);
    if (e != cudaSuccess) return fail_cuda(e, "sort graphs: launch");
    count_launches(launches);
    return HS_OK;
}

hs_status merge_sort_graphed(int32_t *d_keys, int32_t *d_vals, size_t n, hs_netset s, void *d_ws,
                             size_t ws_bytes, cudaStream_t st) {
    const int L = leaf_size(s);
    const bool multi = d_vals ? (int64_t)n > pairs_tile(L) : (int64_t)n > keys_tile(L, (int64_t)n);
    return graphed(Signature{0, d_vals ? 1 : 0, d_keys, d_vals, n, s, d_ws, ws_bytes, 0}, multi, st,
                   [&](cudaStream_t x) { return merge_sort(d_keys, d_vals, n, s, d_ws, ws_bytes, x); });
}

hs_status merge_sort_i64_graphed(int64_t *d_keys, size_t n, hs_netset s, void *d_ws,
                                 size_t ws_bytes, cudaStream_t st) {
    const int L = leaf_size(s);
    return graphed(Signature{0, 2, d_keys, nullptr, n, s, d_ws, ws_bytes, 0},
                   (int64_t)n > tile64(L, (int64_t)n), st,
                   [&](cudaStream_t x) { return merge_sort_i64(d_keys, n, s, d_ws, ws_bytes, x); });
}

}  // namespace hs
