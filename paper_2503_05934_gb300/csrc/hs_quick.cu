// Quick path (Algorithm 2 on the GPU).  Placeholder until the 3-way
// partition kernels land: reports the request as unsupported.
#include "hs_internal.h"

namespace hs {

size_t quick_workspace_bytes(size_t n) { return merge_workspace_bytes(n, 0); }

hs_status quick_sort(int32_t *, size_t, hs_netset, void *, size_t, cudaStream_t) {
    return fail(HS_ERR_UNSUPPORTED, "hs_sort_i32: HS_ALGO_QUICK is not built yet");
}

}  // namespace hs
