// Internals of the batched (segmented) form, shared with the serving loop.
#pragma once

#include "hs_internal.h"

namespace hs {

// One array to sort: n keys at `keys`, with n words of scratch at `scratch`
// (used only when n exceeds one block-sort tile).
struct SegDesc {
    int32_t *keys;
    int32_t *scratch;
    int64_t n;
    int64_t reserved;
};

hs_plan default_seg_plan(hs_netset s);
hs_status check_plan(const hs_plan &p);

// Sorts ndesc arrays described by device descriptors: a classify launch
// files them into d_cdesc (ndesc entries; large segments from the front,
// warp-sized ones from the back), then one persistent launch sorts them.
// d_ctrl holds the launch's four queue counters (32 bytes, reset first).
hs_status seg_launch_descs(const SegDesc *d_descs, int64_t ndesc, SegDesc *d_cdesc,
                           unsigned long long *d_ctrl, const hs_plan &plan, cudaStream_t st);

size_t segsort_workspace_bytes(size_t n_keys, size_t num_segs);
hs_status segsort(int32_t *d_keys, size_t n_keys, const int64_t *d_offsets, size_t num_segs,
                  const hs_plan &plan, void *d_ws, size_t ws_bytes, cudaStream_t st);

hs_status segsort_capture(int32_t *d_keys, size_t n_keys, const int64_t *d_offsets,
                          size_t num_segs, const hs_plan &plan, void *d_ws, size_t ws_bytes,
                          void **out);
hs_status graph_launch(void *handle, cudaStream_t st);
void graph_destroy(void *handle);

}  // namespace hs
