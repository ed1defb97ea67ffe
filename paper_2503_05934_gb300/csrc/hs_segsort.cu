// Batched form: many independent arrays sorted by one persistent launch.
//
// Every array ("segment") is sorted by a single CTA, as Algorithm 1 would sort
// it: network leaves and shared-memory merge levels (block_sort_tile3) for a
// segment of at most one tile; for a longer segment, tile-sized pieces first,
// then CTA-local merge levels through the segment's scratch area, which stays
// in L2 at the sizes this form targets (up to 64K keys).  Persistent CTAs take
// segments from an atomic queue, so uneven sizes balance themselves.
//
// The same kernel serves two front ends: an offsets array over one key buffer
// (hs_segsort_i32) and a list of separate arrays (the serving loop).  The
// launch sequence (queue reset, descriptor build, sort) has no host
// synchronisation, so it can be captured in a CUDA graph (hs_segsort_capture).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hs_internal.h"
#include "hs_blocksort.cuh"
#include "hs_segsort.h"

namespace hs {

constexpr int SPLIT_CAP = 256;  // merge-level chunk boundaries searched per batch

HS_DEV bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Merge-path split by one warp (32-ary search): the smallest i in [lo, hi]
// with A[i] > B[diag - 1 - i] (hi when there is none), the number of A
// elements among the first diag outputs of the stable merge.  Each round the
// lanes test 32 evenly spaced candidates (two independent loads each) and the
// range shrinks 32-fold, so a 65536-key range takes about four dependent load
// rounds instead of sixteen.  The final round starts with fewer than 32
// candidates left, so the last lane always tests a position >= hi and the
// ballot is never empty.  Every lane returns the result.
HS_DEV int64_t warp_merge_path(const int32_t *A, const int32_t *B, int64_t diag, int64_t lo,
                               int64_t hi, int lane) {
    while (hi - lo >= 32) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t q = lo + (int64_t)(lane + 1) * step;  // candidate; q >= hi counts as true
        const bool t = q >= hi || A[q] > B[diag - 1 - q];
        const unsigned m = __ballot_sync(0xffffffffu, t);
        const int f = __ffs(m) - 1;  // some lane holds q >= hi, so m != 0
        const int64_t nlo = f == 0 ? lo : lo + (int64_t)f * step + 1;
        hi = hs_min(hi, lo + (int64_t)(f + 1) * step);
        lo = nlo;
    }
    const int64_t q = lo + lane;
    const bool t = q >= hi || A[q] > B[diag - 1 - q];
    const unsigned m = __ballot_sync(0xffffffffu, t);
    return lo + (__ffs(m) - 1);
}

// One merge level over a single segment by one CTA: runs of w in src are
// merged into runs of 2w in dst.  Output chunks of T keys: their merge-path
// splits are found by one warp per chunk boundary; each chunk is then staged
// in shared memory, each thread merges exactly its own EO outputs (exact
// window, end split from the next lane), and the outputs leave through shared
// memory as coalesced stores.
template <int NT, int L, int LV>
HS_DEV void cta_merge_level(const int32_t *src, int32_t *dst, int64_t n, int64_t w, int32_t *s,
                            int64_t *split) {
    using C = BlockSort3<NT, L, LV>;
    constexpr int T = C::T, EO = C::EO, P = C::P;
    const int64_t span = 2 * w;
    const int64_t ngroups = (n + span - 1) / span;
    const int64_t tpg = (span + T - 1) / T;
    const int64_t last = n - (ngroups - 1) * span;
    const int64_t nchunks = (ngroups - 1) * tpg + (last + T - 1) / T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int *wsplit = s + C::T + C::P + 32;
    for (int64_t c0 = 0; c0 < nchunks; c0 += SPLIT_CAP) {
        const int64_t c1 = std::min<int64_t>(nchunks, c0 + SPLIT_CAP);
        // Splits of boundaries c0 .. c1 (c1 may open the next batch).
        for (int64_t c = c0 + warp; c <= c1 && c < nchunks; c += NT / 32) {
            const int64_t g = c / tpg, t = c - g * tpg;
            const MergeGeom m = merge_geom(g, n, w);
            int64_t diag = t * T;
            if (diag > m.alen + m.blen) diag = m.alen + m.blen;
            const int64_t lo = diag > m.blen ? diag - m.blen : 0;
            const int64_t hi = diag < m.alen ? diag : m.alen;
            const int64_t r = warp_merge_path(src + m.gs, src + m.gs + w, diag, lo, hi, lane);
            if (lane == 0) split[c - c0] = r;
        }
        __syncthreads();
        for (int64_t c = c0; c < c1; ++c) {
            const int64_t g = c / tpg, t = c - g * tpg;
            const MergeGeom m = merge_geom(g, n, w);
            const int64_t glen = m.alen + m.blen;
            const int64_t o0 = t * T;
            const int64_t o1 = std::min<int64_t>(o0 + T, glen);
            const int64_t a0 = split[c - c0];
            const int64_t a1 = (o1 == glen) ? m.alen : split[c + 1 - c0];
            const int na = (int)(a1 - a0);
            const int tot = (int)(o1 - o0);
            const int nb = tot - na;
            const int32_t *gA = src + m.gs + a0, *gB = src + m.gs + w + (o0 - a0);
            for (int i = threadIdx.x; i < tot; i += NT) cp_async4(s + i, i < na ? gA + i : gB + (i - na));
            cp_async_wait_all();
            __syncthreads();
            const int32_t *A = s, *B = s + na;
            const int diag = threadIdx.x * EO;
            const int dcl = diag < tot ? diag : tot;
            int lo = dcl > nb ? dcl - nb : 0, hi = dcl < na ? dcl : na;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (A[mid] <= B[dcl - 1 - mid]) lo = mid + 1;
                else hi = mid;
            }
            int end = __shfl_down_sync(0xffffffffu, lo, 1);
            if (lane == 0) wsplit[warp] = lo;
            if (threadIdx.x == 0) wsplit[NT / 32] = na;
            __syncthreads();
            const int dend = (diag + EO) < tot ? (diag + EO) : tot;
            if (lane == 31) end = wsplit[warp + 1];
            if (dend == tot) end = na;
            const int cnt = dend - dcl;
            int32_t x[P];
            if (cnt > 0) exact_window_merge<EO, P>(A, lo, B, dcl - lo, end - lo, cnt, x);
            __syncthreads();
            if (cnt > 0) {
#pragma unroll
                for (int k = 0; k < EO; ++k)
                    if (k < cnt) s[diag + k] = x[k];
            }
            __syncthreads();
            int32_t *out = dst + m.gs + o0;
            // Plain (cached) stores: the next level reads these keys back from L2.
            int start = 0;
            if (aligned16(out)) {
                for (int q = threadIdx.x; q < (tot >> 2); q += NT)
                    reinterpret_cast<int4 *>(out)[q] = *reinterpret_cast<const int4 *>(s + 4 * q);
                start = tot & ~3;
            }
            for (int i = start + threadIdx.x; i < tot; i += NT) out[i] = s[i];
            __syncthreads();
        }
    }
}

template <int NT, int L, int LV>
HS_DEV void sort_segment(const SegDesc &d, uint32_t netset, int32_t *s, int64_t *split) {
    using C = BlockSort3<NT, L, LV>;
    constexpr int T = C::T;
    const int64_t n = d.n;
    if (n <= 1) return;
    if (n <= T) {
        block_sort_tile3<NT, L, LV, true>(d.keys, d.keys, (int)n, netset, aligned16(d.keys), s);
        return;
    }
    int levels = 0;
    for (int64_t w = T; w < n; w *= 2) ++levels;
    // Ping-pong so that the last level lands in d.keys.
    int32_t *cur = (levels % 2 == 0) ? d.keys : d.scratch;
    int32_t *alt = (levels % 2 == 0) ? d.scratch : d.keys;
    const bool vec = aligned16(d.keys) && aligned16(cur);
    for (int64_t base = 0; base < n; base += T) {
        const int cnt = (int)std::min<int64_t>(T, n - base);
        block_sort_tile3<NT, L, LV>(d.keys + base, cur + base, cnt, netset, vec, s);
        __syncthreads();
    }
    for (int64_t w = T; w < n; w *= 2) {
        cta_merge_level<NT, L, LV>(cur, alt, n, w, s, split);
        int32_t *tmp = cur;
        cur = alt;
        alt = tmp;
    }
}

template <int NT, int L, int LV>
__global__ void __launch_bounds__(NT, NT <= 256 ? 3 : 2)
    k_seg_sort(const SegDesc *descs, int64_t ndesc, unsigned long long *head, uint32_t netset) {
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ int64_t s_split[SPLIT_CAP + 1];
    __shared__ unsigned long long s_item[2];
    if (threadIdx.x == 0) s_item[0] = atomicAdd(head, 1ull);
    __syncthreads();
    for (int it = 0;; it ^= 1) {
        const unsigned long long item = s_item[it];
        if (item >= (unsigned long long)ndesc) break;
        // The next item is claimed now; the atomic's round trip overlaps
        // this segment's sort and its result is only consumed at the end.
        unsigned long long next = 0;
        if (threadIdx.x == 0) next = atomicAdd(head, 1ull);
        const SegDesc d = descs[item];
        sort_segment<NT, L, LV>(d, netset, smem, s_split);
        if (threadIdx.x == 0) s_item[it ^ 1] = next;
        __syncthreads();
    }
}

// Descriptors for an offsets array: segment i is keys[off[i], off[i+1]); its
// scratch is the same range of the workspace key area.  Malformed offsets
// raise a status bit and leave the segment empty.
__global__ void k_seg_descs(int32_t *keys, int64_t n_keys, const int64_t *off, int64_t nseg,
                            int32_t *scratch, SegDesc *descs, unsigned *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nseg) return;
    const int64_t b = off[i], e = off[i + 1];
    SegDesc d{};
    if (b < 0 || e < b || e > n_keys) {
        atomicOr(status, kStatusBadOffsets);
    } else {
        d.keys = keys + b;
        d.scratch = scratch + b;
        d.n = e - b;
    }
    descs[i] = d;
}

// ------------------------------------------------------------------ host side

struct SegKernelInfo {
    const void *fn;
    int smem;
    int max_occ;
};

template <int NT, int L, int LV>
static hs_status seg_kernel_info(SegKernelInfo *out) {
    using C = BlockSort3<NT, L, LV>;
    auto kern = k_seg_sort<NT, L, LV>;
    hs_status r = ensure_smem((const void *)kern, C::SMEM_BYTES);
    if (r != HS_OK) return r;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, C::SMEM_BYTES);
    if (e != cudaSuccess) return fail_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    out->fn = (const void *)kern;
    out->smem = C::SMEM_BYTES;
    out->max_occ = occ > 0 ? occ : 1;
    return HS_OK;
}

template <int NT, int LV>
static hs_status seg_kernel_info_nt(int L, SegKernelInfo *out) {
    switch (L) {
        case 1: return seg_kernel_info<NT, 1, LV>(out);
        case 3: return seg_kernel_info<NT, 3, LV>(out);
        case 4: return seg_kernel_info<NT, 4, LV>(out);
        case 5: return seg_kernel_info<NT, 5, LV>(out);
        case 6: return seg_kernel_info<NT, 6, LV>(out);
        case 7: return seg_kernel_info<NT, 7, LV>(out);
        case 8: return seg_kernel_info<NT, 8, LV>(out);
    }
    return fail(HS_ERR_INVALID_ARG, "leaf size outside 1, 3..8");
}

// CTA shapes of the batched kernel: 256 threads hold four leaves each, 512
// threads two leaves each.
static hs_status seg_kernel(int nt, int L, SegKernelInfo *out) {
    if (nt == 256) return seg_kernel_info_nt<256, 4>(L, out);
    if (nt == 512) return seg_kernel_info_nt<512, 2>(L, out);
    return fail(HS_ERR_INVALID_ARG, "plan block_threads must be 256 or 512");
}

static int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return sms > 0 ? sms : 1;
}

hs_plan default_seg_plan(hs_netset s) {
    hs_plan p{};
    p.netset = s;
    p.block_threads = 256;
    p.ctas_per_sm = 0;  // as many as fit
    return p;
}

hs_status check_plan(const hs_plan &p) {
    if (!netset_ok(p.netset)) return fail(HS_ERR_INVALID_ARG, "plan netset is neither a set of sizes 3..8 nor a VarSort configuration");
    if (p.block_threads != 256 && p.block_threads != 512)
        return fail(HS_ERR_INVALID_ARG, "plan block_threads must be 256 or 512");
    if (p.ctas_per_sm < 0 || p.ctas_per_sm > 8)
        return fail(HS_ERR_INVALID_ARG, "plan ctas_per_sm must be 0..8");
    return HS_OK;
}

hs_status seg_launch_descs(const SegDesc *d_descs, int64_t ndesc, unsigned long long *d_head,
                           const hs_plan &plan, cudaStream_t st) {
    hs_status r = check_plan(plan);
    if (r != HS_OK) return r;
    if (ndesc <= 0) return HS_OK;
    SegKernelInfo ki{};
    if ((r = seg_kernel(plan.block_threads, leaf_size(plan.netset), &ki)) != HS_OK) return r;
    const int per_sm = plan.ctas_per_sm > 0 ? std::min(plan.ctas_per_sm, ki.max_occ) : ki.max_occ;
    const int64_t grid = std::min<int64_t>(ndesc, (int64_t)sm_count() * per_sm);
    cudaError_t e = cudaMemsetAsync(d_head, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return fail_cuda(e, "segsort: queue reset");
    uint32_t netset = plan.netset;
    void *args[] = {(void *)&d_descs, (void *)&ndesc, (void *)&d_head, (void *)&netset};
    LaunchToken t = launch_begin(K_SEG_SORT, st);
    e = cudaLaunchKernel(ki.fn, dim3((unsigned)grid), dim3(plan.block_threads), args, ki.smem, st);
    if (e != cudaSuccess) {
        launch_end(t);
        return fail_cuda(e, "segsort launch");
    }
    return launch_end(t);
}

struct SegLayout {
    size_t keys, descs, head, total;
};

static SegLayout seg_layout(size_t n_keys, size_t num_segs) {
    SegLayout l{};
    size_t off = 0;
    l.keys = off;
    off += align_up(n_keys * sizeof(int32_t), 256);
    l.descs = off;
    off += align_up(num_segs * sizeof(SegDesc), 256);
    l.head = off;
    off += 256;
    l.total = off;
    return l;
}

size_t segsort_workspace_bytes(size_t n_keys, size_t num_segs) {
    return seg_layout(n_keys, num_segs).total;
}

hs_status segsort(int32_t *d_keys, size_t n_keys, const int64_t *d_offsets, size_t num_segs,
                  const hs_plan &plan, void *d_ws, size_t ws_bytes, cudaStream_t st) {
    hs_status r = check_plan(plan);
    if (r != HS_OK) return r;
    if (num_segs == 0) return HS_OK;
    if (!d_offsets) return fail(HS_ERR_INVALID_ARG, "hs_segsort_i32: NULL offsets");
    if (n_keys > 0 && (!d_keys || !aligned(d_keys, 4)))
        return fail(HS_ERR_INVALID_ARG, "hs_segsort_i32: NULL or unaligned keys");
    const SegLayout l = seg_layout(n_keys, num_segs);
    if (!d_ws || ws_bytes < l.total)
        return fail(HS_ERR_INVALID_ARG, "hs_segsort_i32: workspace smaller than hs_segsort_workspace_bytes");
    if (!aligned(d_ws, 16)) return fail(HS_ERR_INVALID_ARG, "hs_segsort_i32: workspace not 16-byte aligned");
    char *base = static_cast<char *>(d_ws);
    int32_t *scratch = reinterpret_cast<int32_t *>(base + l.keys);
    SegDesc *descs = reinterpret_cast<SegDesc *>(base + l.descs);
    unsigned long long *head = reinterpret_cast<unsigned long long *>(base + l.head);
    unsigned *status = nullptr;
    if ((r = device_status(&status)) != HS_OK) return r;
    LaunchToken t = launch_begin(K_SEG_CLASSIFY, st);
    k_seg_descs<<<(unsigned)((num_segs + 255) / 256), 256, 0, st>>>(
        d_keys, (int64_t)n_keys, d_offsets, (int64_t)num_segs, scratch, descs, status);
    if ((r = launch_end(t)) != HS_OK) return r;
    return seg_launch_descs(descs, (int64_t)num_segs, head, plan, st);
}

// -------------------------------------------------------------- graphs

struct GraphHandle {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

hs_status segsort_capture(int32_t *d_keys, size_t n_keys, const int64_t *d_offsets,
                          size_t num_segs, const hs_plan &plan, void *d_ws, size_t ws_bytes,
                          void **out) {
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail_cuda(e, "hs_segsort_capture: stream");
    GraphHandle *h = new (std::nothrow) GraphHandle();
    if (!h) {
        cudaStreamDestroy(cs);
        return fail(HS_ERR_NO_MEMORY, "hs_segsort_capture: handle");
    }
    hs_status r = HS_OK;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        r = fail_cuda(e, "hs_segsort_capture: begin capture");
    } else {
        r = segsort(d_keys, n_keys, d_offsets, num_segs, plan, d_ws, ws_bytes, cs);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        if (r == HS_OK && e != cudaSuccess) r = fail_cuda(e, "hs_segsort_capture: end capture");
        h->graph = g;
        if (r == HS_OK) {
            e = cudaGraphInstantiate(&h->exec, g, 0);
            if (e != cudaSuccess) r = fail_cuda(e, "hs_segsort_capture: instantiate");
        }
    }
    cudaStreamDestroy(cs);
    if (r != HS_OK) {
        if (h->exec) cudaGraphExecDestroy(h->exec);
        if (h->graph) cudaGraphDestroy(h->graph);
        delete h;
        return r;
    }
    *out = h;
    return HS_OK;
}

hs_status graph_launch(void *handle, cudaStream_t st) {
    GraphHandle *h = static_cast<GraphHandle *>(handle);
    if (!h || !h->exec) return fail(HS_ERR_INVALID_ARG, "hs_graph_launch: NULL graph");
    cudaError_t e = cudaGraphLaunch(h->exec, st);
    if (e != cudaSuccess) return fail_cuda(e, "hs_graph_launch");
    count_launches(2);  // descriptor build + persistent sort
    return HS_OK;
}

void graph_destroy(void *handle) {
    GraphHandle *h = static_cast<GraphHandle *>(handle);
    if (!h) return;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    delete h;
}

}  // namespace hs
