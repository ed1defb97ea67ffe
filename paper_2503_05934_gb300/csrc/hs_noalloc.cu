// hs_sort_i32_noalloc: the merge sort of hs_sort_i32 for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc (or have anyone call it for them): a
// plugin whose host application owns every device allocation through its own
// allocator and forbids side allocations, code that runs under a device-memory
// budget fixed at start-up, or a latency-critical path where cudaMalloc may
// synchronise the device and stall for an unpredictable time.  Such a caller
// cannot provide the ping-pong workspace that hs_sort_i32 asks for.
//
// This entry point uses a fixed scratch area in a file-scope __device__ array
// instead.  The array exists on every GPU where this library's code is loaded
// and stays there until the process exits.  Its size caps the input length at
// HS_NOALLOC_MAX_KEYS.
#include <mutex>

#include "hs_internal.h"

namespace hs {

constexpr size_t kNoallocMaxKeys = HS_NOALLOC_MAX_KEYS;
// The merge path's keys workspace for the largest accepted input, by the same
// formula as hs_sort_workspace_bytes (the layout grows monotonically in n, so
// every shorter input fits).
constexpr size_t kNoallocBytes = merge_workspace_size(kNoallocMaxKeys, 0);
// 17,433,344 bytes (16.6 MiB): 16 MiB of keys, 131,584 bytes of partition
// entries and 524,544 bytes of samples.  The header states this figure.
static_assert(kNoallocBytes == 17433344, "the scratch size the header documents changed");

// The scratch area.  In host code this name is only a host-side stand-in for
// the device symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[kMaxDevices] = {};

// Set-up, once per device, with that device current: look up the device
// address of the scratch array.
static hs_status noalloc_scratch(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "hs_sort_i32_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(HS_ERR_UNSUPPORTED, "hs_sort_i32_noalloc: device ordinal above 63");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fail_cuda(e, "hs_sort_i32_noalloc: cudaGetSymbolAddress");
        if (!p) return fail(HS_ERR_CUDA, "hs_sort_i32_noalloc: scratch symbol has no device address");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return HS_OK;
}

}  // namespace hs

using namespace hs;

extern "C" hs_status hs_sort_i32_noalloc(int32_t *d_keys, size_t n, hs_netset s,
                                         hs_stream_t stream) {
    const ApiRange range("hs_sort_i32_noalloc");
    clear_error();
    if (!netset_ok(s))
        return fail(HS_ERR_INVALID_ARG, "hs_sort_i32_noalloc: netset is neither a set of sizes 3..8 nor a VarSort configuration");
    if (n > 0 && !d_keys) return fail(HS_ERR_INVALID_ARG, "hs_sort_i32_noalloc: NULL keys with n > 0");
    if (n > 0 && !aligned(d_keys, 4))
        return fail(HS_ERR_INVALID_ARG, "hs_sort_i32_noalloc: keys not 4-byte aligned");
    if (n > kNoallocMaxKeys)
        return fail(HS_ERR_INVALID_ARG,
                    "hs_sort_i32_noalloc: n exceeds HS_NOALLOC_MAX_KEYS (4194304 keys); "
                    "use hs_sort_i32 with a caller-provided workspace");
    if (n <= 1) return HS_OK;
    void *scratch = nullptr;
    hs_status st = noalloc_scratch(&scratch);
    if (st != HS_OK) return st;
    // Nothing in the scratch has to start at zero: the merge path writes every
    // word it reads (keys copy, partition indices, samples) earlier in the
    // same call.
    return merge_sort(d_keys, nullptr, n, s, scratch, kNoallocBytes, (cudaStream_t)stream);
}
