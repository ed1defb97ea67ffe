// Quick path: the GPU form of Algorithm 2 (Optimized Quick Sort with Sorting
// Networks).
//
// Each level partitions every live segment larger than one block-sort tile
// around its median-of-three pivot (MedianOfThree in Algorithm 2: first,
// middle and last key).  The GPU partition is 3-way (<, =, > pivot) rather
// than Hoare's 2-way scan: keys equal to the pivot are final at once, which
// also ends all-equal segments.  Segments of at most one tile are finished
// by the block sort, whose leaves are the network base cases.
//
// Per level (all segments at once, chunks of QS_C keys):
//   k_qs_partition per chunk: classify against the pivot, compact the < keys
//                  and the > keys per warp in shared memory, reserve one
//                  range for each with an atomic cursor (< from the segment's
//                  front, > from its back), and write both as coalesced runs
//                  to the other buffer: one read and one write per key
//   k_qs_next      per segment: the = range (what the two cursors left in the
//                  middle) is final; short ones are written here, long ones
//                  listed; children go to the next level (> tile, with their
//                  median-of-three pivots) or to the small list (<= tile)
//   k_qs_chunkmap  chunk -> segment map of the next level; publishes the
//                  level's counters to the host
//   k_qs_leaves    (second stream) block sort of each small child into the
//                  caller's array, and the listed = ranges
// The host does not wait for a level before launching the next one.  Each
// level's counters reach it through mapped host memory (written by
// k_qs_chunkmap), and it reads those of the level two back: launch sizes are
// upper bounds derived from the last counters it has seen (segments at most
// double per level, and the chunk count never exceeds the known chunks plus
// one partial chunk per segment); every kernel reads its exact count on the
// device and skips work past it.  The small-segment sorts and the long =
// fills of a level (k_qs_leaves) run on a second stream, overlapped with the
// following levels: their key ranges are final, so no later level touches
// them.  Counters and lists rotate through QS_RING slots so a level's slot is
// reused only after its leaves are done.  The order of the chunks' runs inside
// a < or > range depends on timing; the sorted output does not.
#include <algorithm>
#include <cstring>
#include <vector>

#include "hs_internal.h"
#include "hs_blocksort.cuh"

namespace hs {

constexpr int QS_NT = 256;
constexpr int QS_IPT = 32;
constexpr int QS_C = QS_NT * QS_IPT;  // keys per partition chunk
constexpr int QS_BS_NT = 256;         // small-segment sort: 256 threads x four leaves
constexpr int QS_EQ_INLINE = 64;      // = ranges up to this length are written by k_qs_next
static int64_t qs_tile(int L) { return (int64_t)QS_BS_NT * (4 * L - 1); }

struct QSeg {
    int64_t begin, end, chunk0;
    // Reservation cursors of the < range (from begin) and the > range (back
    // from end); after the partition pass, the segment's < and > counts.
    unsigned long long n_lt, n_gt;
    unsigned long long n_eq;  // 2-way form: ranks handed out to keys equal to the pivot
    int32_t buf, pivot;       // buf 0: caller's array, 1: workspace
};

struct QSmall {
    int64_t begin, end;
    int32_t buf, pad;
};

struct QFill {
    int64_t begin, end;
    int32_t value, pad;
};

// Level k uses counter slot k % QS_RING: nseg and nchunks describe its
// segment list (written by level k - 1); nsmall and nfill count the small
// children and long = ranges that level k itself lists, in its own slot of
// the small and fill lists.
constexpr int QS_RING = 4;
struct QCounters {
    unsigned long long nseg, nchunks, nsmall, nfill;
};

// One level's counters as the host reads them (mapped host memory).
struct QReadback {
    QCounters cur, next;
    unsigned long long status, pad;
};

struct QCaps {
    int64_t seg, chunk, small, fill;
};

static int64_t qs_option_max_levels = -1;  // < 0: automatic

HS_DEV const int32_t *qs_src(int32_t buf, const int32_t *X, const int32_t *Y) { return buf ? Y : X; }

HS_DEV int32_t median_of_three(const int32_t *a, int64_t b, int64_t e) {
    const int32_t x = a[b], y = a[b + (e - b - 1) / 2], z = a[e - 1];
    return hs_max(hs_min(x, y), hs_min(hs_max(x, y), z));
}

HS_DEV int64_t clamp_count(unsigned long long c, int64_t cap) {
    return (int64_t)c < cap ? (int64_t)c : cap;
}

__global__ void k_qs_init(QSeg *segs, int32_t *chunk_seg, int64_t n, int64_t nchunks,
                          const int32_t *X, QCounters *ctr, unsigned long long *status) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        QSeg s{};
        s.begin = 0;
        s.end = n;
        s.chunk0 = 0;
        s.buf = 0;
        s.pivot = median_of_three(X, 0, n);
        segs[0] = s;
        ctr[0] = QCounters{1ull, (unsigned long long)nchunks, 0ull, 0ull};
        for (int i = 1; i < QS_RING; ++i) ctr[i] = QCounters{0ull, 0ull, 0ull, 0ull};
        *status = 0ull;
    }
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
         c += (int64_t)gridDim.x * blockDim.x)
        chunk_seg[c] = 0;
}

// Option "quick_partition" 2: Algorithm 2's 2-way form (every key goes to
// one side: left <= pivot <= right).  Keys equal to the pivot alternate sides
// by their rank among the segment's equal keys (an atomic per chunk hands out
// the ranks), so each side gets half of them: with a median-of-three pivot
// both sides are then non-empty and every level makes progress, as Hoare's
// scan does by stopping on equal keys from both ends.
static int g_qs_two_way = 0;

// One chunk per CTA: each warp classifies its 32*QS_IPT keys (slice j of the
// chunk holds keys j*QS_NT + [0, QS_NT); warp w takes 32 of them) and
// compacts them into its own shared region, < keys from the front and > keys
// from the back, with running offsets that every lane knows from the ballots.
// A scan over the warps' totals gives each warp's place in the chunk's < and
// > runs; one atomic per run reserves the chunk's place in the segment; each
// warp then copies its keys out as coalesced runs.
template <bool TWO_WAY>
__global__ void __launch_bounds__(QS_NT, 4)
    k_qs_partition(QSeg *segs, const int32_t *chunk_seg, const QCounters *ctr, QCaps caps,
                   const int32_t *X, const int32_t *Y, int32_t *Xw, int32_t *Yw) {
    constexpr int NW = QS_NT / 32;
    constexpr int WK = 32 * QS_IPT;  // keys per warp
    __shared__ int32_t stage[QS_C];  // warp w: [w*WK, (w+1)*WK), < from the front, > from the back
    __shared__ int s_wlt[NW], s_wgt[NW], s_weq[NW];
    __shared__ unsigned long long s_base[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    const int64_t c = blockIdx.x;
    if (c >= clamp_count(ctr->nchunks, caps.chunk)) return;
    {
        const int si = chunk_seg[c];
        const QSeg &sg = segs[si];
        const int64_t start = sg.begin + (c - sg.chunk0) * (int64_t)QS_C;
        const int64_t rest = sg.end - start;
        const int len = (int)(rest < QS_C ? rest : QS_C);
        const int32_t p = sg.pivot;
        const int32_t *src = qs_src(sg.buf, X, Y) + start;
        int32_t *dst = sg.buf ? Xw : Yw;

        int32_t k[QS_IPT];
#pragma unroll
        for (int j = 0; j < QS_IPT; ++j) {
            const int i = j * QS_NT + threadIdx.x;
            k[j] = i < len ? ld_stream(src + i) : p;  // padding counts as "=" and is dropped
        }
        // 2-way form: the global rank of each equal key among the segment's
        // equal keys (chunk base from an atomic, then warp and slice order).
        int eq_rank0 = 0;
        if constexpr (TWO_WAY) {
            int neq = 0;
#pragma unroll
            for (int j = 0; j < QS_IPT; ++j)
                neq += __popc(__ballot_sync(0xffffffffu, k[j] == p && j * QS_NT + (int)threadIdx.x < len));
            if (lane == 0) s_weq[warp] = neq;
            __syncthreads();
            int off = 0, tot = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                off += (w < warp) ? s_weq[w] : 0;
                tot += s_weq[w];
            }
            if (threadIdx.x == 0)
                s_base[2] = tot ? atomicAdd(&segs[si].n_eq, (unsigned long long)tot) : 0ull;
            __syncthreads();
            eq_rank0 = (int)(s_base[2] & 1ull) + off;  // only the parity of the rank matters
        }
        int32_t *ws = stage + warp * WK;
        int nlt = 0, ngt = 0, neq_run = 0;  // warp-uniform running counts
#pragma unroll
        for (int j = 0; j < QS_IPT; ++j) {
            bool is_lt = k[j] < p, is_gt = k[j] > p;
            if constexpr (TWO_WAY) {
                const bool is_eq = k[j] == p && j * QS_NT + (int)threadIdx.x < len;
                const unsigned me = __ballot_sync(0xffffffffu, is_eq);
                const int rank = eq_rank0 + neq_run + __popc(me & below);
                is_lt = is_lt || (is_eq && (rank & 1) == 0);
                is_gt = is_gt || (is_eq && (rank & 1) != 0);
                neq_run += __popc(me);
            }
            const unsigned ml = __ballot_sync(0xffffffffu, is_lt);
            const unsigned mg = __ballot_sync(0xffffffffu, is_gt);
            if (is_lt) ws[nlt + __popc(ml & below)] = k[j];
            if (is_gt) ws[WK - 1 - (ngt + __popc(mg & below))] = k[j];
            nlt += __popc(ml);
            ngt += __popc(mg);
        }
        if (lane == 0) {
            s_wlt[warp] = nlt;
            s_wgt[warp] = ngt;
        }
        __syncthreads();
        // Each warp's offsets inside the chunk's runs, and the chunk totals
        // (every thread scans the NW warp counts itself).
        int off_lt = 0, off_gt = 0, tot_lt = 0, tot_gt = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const int a = s_wlt[w], b = s_wgt[w];
            off_lt += (w < warp) ? a : 0;
            off_gt += (w < warp) ? b : 0;
            tot_lt += a;
            tot_gt += b;
        }
        if (threadIdx.x == 0) {
            QSeg &sw = segs[si];
            s_base[0] = tot_lt ? atomicAdd(&sw.n_lt, (unsigned long long)tot_lt) : 0ull;
            s_base[1] = tot_gt ? atomicAdd(&sw.n_gt, (unsigned long long)tot_gt) : 0ull;
        }
        __syncthreads();
        int32_t *lt_dst = dst + sg.begin + (int64_t)s_base[0] + off_lt;
        int32_t *gt_dst = dst + sg.end - (int64_t)s_base[1] - tot_gt + off_gt;
        for (int i = lane; i < nlt; i += 32) st_stream(lt_dst + i, ws[i]);
        for (int i = lane; i < ngt; i += 32) st_stream(gt_dst + i, ws[WK - 1 - i]);
    }
}

HS_DEV void qs_flag(unsigned long long *status) { atomicExch(status, 1ull); }

HS_DEV void qs_emit(int64_t b, int64_t e, int32_t buf, int64_t tile, const int32_t *X,
                    const int32_t *Y, QSeg *next, QCounters *nctr, QSmall *small,
                    QCounters *cctr, const QCaps &caps, unsigned long long *status) {
    const int64_t len = e - b;
    if (len <= 0) return;
    if (len > tile) {
        unsigned long long idx = atomicAdd(&nctr->nseg, 1ull);
        unsigned long long nch = (unsigned long long)((len + QS_C - 1) / QS_C);
        unsigned long long c0 = atomicAdd(&nctr->nchunks, nch);
        if ((int64_t)idx >= caps.seg || (int64_t)(c0 + nch) > caps.chunk) {
            qs_flag(status);
            return;
        }
        QSeg s{};
        s.begin = b;
        s.end = e;
        s.chunk0 = (int64_t)c0;
        s.buf = buf;
        s.pivot = median_of_three(qs_src(buf, X, Y), b, e);
        next[idx] = s;
    } else {
        unsigned long long idx = atomicAdd(&cctr->nsmall, 1ull);
        if ((int64_t)idx >= caps.small) {
            qs_flag(status);
            return;
        }
        small[idx] = QSmall{b, e, buf, 0};
    }
}

__global__ void k_qs_next(const QSeg *segs, QCounters *cctr, QCounters *nctr, QCaps caps,
                          int64_t tile, QSeg *next, QSmall *small, QFill *fill, int32_t *X,
                          const int32_t *Y, unsigned long long *status) {
    const int64_t nseg = clamp_count(cctr->nseg, caps.seg);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nseg;
         i += (int64_t)gridDim.x * blockDim.x) {
        const QSeg s = segs[i];
        const int32_t dbuf = s.buf ^ 1;
        const int64_t lt_end = s.begin + (int64_t)s.n_lt;
        const int64_t gt_begin = s.end - (int64_t)s.n_gt;
        // The = range is final: write the pivot into the caller's array.
        if (gt_begin - lt_end <= QS_EQ_INLINE) {
            for (int64_t x = lt_end; x < gt_begin; ++x) X[x] = s.pivot;
        } else {
            unsigned long long idx = atomicAdd(&cctr->nfill, 1ull);
            if ((int64_t)idx < caps.fill) fill[idx] = QFill{lt_end, gt_begin, s.pivot, 0};
            else qs_flag(status);
        }
        qs_emit(s.begin, lt_end, dbuf, tile, X, Y, next, nctr, small, cctr, caps, status);
        qs_emit(gt_begin, s.end, dbuf, tile, X, Y, next, nctr, small, cctr, caps, status);
    }
}

// Chunk -> segment map of the next level.  Block 0 also publishes the
// level's final counters and status to the host (mapped memory).
__global__ void k_qs_chunkmap(const QSeg *segs, const QCounters *cctr, const QCounters *nctr,
                              QCaps caps, int32_t *chunk_seg, const unsigned long long *status,
                              QReadback *rb) {
    const int64_t nseg = clamp_count(nctr->nseg, caps.seg);
    for (int64_t s = blockIdx.x; s < nseg; s += gridDim.x) {
        const QSeg &g = segs[s];
        const int64_t nch = (g.end - g.begin + QS_C - 1) / QS_C;
        for (int64_t c = threadIdx.x; c < nch; c += blockDim.x)
            if (g.chunk0 + c < caps.chunk) chunk_seg[g.chunk0 + c] = (int32_t)s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        QReadback r{};
        r.cur = *cctr;
        r.next = *nctr;
        r.status = *status;
        *rb = r;
        __threadfence_system();
    }
}

// A level's leaves: item i < nsmall block-sorts small child i into the
// caller's array; the next nfill items write the listed = ranges.
template <int L>
__global__ void __launch_bounds__(QS_BS_NT)
    k_qs_leaves(const QSmall *small, const QFill *fill, const QCounters *cctr, QCaps caps,
                const int32_t *X, const int32_t *Y, int32_t *Xw, uint32_t netset) {
    extern __shared__ __align__(16) int32_t smem[];
    const int64_t nsmall = clamp_count(cctr->nsmall, caps.small);
    const int64_t nfill = clamp_count(cctr->nfill, caps.fill);
    for (int64_t i = blockIdx.x; i < nsmall + nfill; i += gridDim.x) {
        if (i < nsmall) {
            const QSmall s = small[i];
            block_sort_tile3<QS_BS_NT, L, 4, true>(qs_src(s.buf, X, Y) + s.begin, Xw + s.begin,
                                                   (int)(s.end - s.begin), netset, false, smem);
            __syncthreads();
        } else {
            const QFill q = fill[i - nsmall];
            for (int64_t x = q.begin + threadIdx.x; x < q.end; x += blockDim.x) Xw[x] = q.value;
        }
    }
}

// ---------------------------------------------------------------- host side

struct QLayout {
    size_t y, part, seg_a, seg_b, chunk_a, chunk_b, small, fill, ctr, status, total;
    QCaps caps;
};

static QLayout qs_layout(size_t n) {
    QLayout q{};
    // Segments of one level are disjoint and longer than the smallest tile
    // (qs_tile(1) = 768 keys, the set without networks), so a level holds at
    // most n/768 of them; each contributes at most one partial chunk, yields
    // at most two small children and at most one listed = range.
    q.caps.seg = (int64_t)(n / (size_t)qs_tile(1) + 2);
    q.caps.chunk = (int64_t)(n / QS_C) + q.caps.seg + 2;
    q.caps.small = 2 * q.caps.seg + 2;
    q.caps.fill = q.caps.seg;
    // Small and fill lists and counters: one slot per level in flight.
    size_t off = 0;
    q.y = off;
    off += align_up(n * sizeof(int32_t), 256);
    q.part = off;  // merge workspace tail for the depth fallback (contiguous after y)
    off += align_up(merge_workspace_bytes(n, 0) - align_up(n * sizeof(int32_t), 256), 256);
    q.seg_a = off;
    off += align_up((size_t)q.caps.seg * sizeof(QSeg), 256);
    q.seg_b = off;
    off += align_up((size_t)q.caps.seg * sizeof(QSeg), 256);
    q.chunk_a = off;
    off += align_up((size_t)q.caps.chunk * sizeof(int32_t), 256);
    q.chunk_b = off;
    off += align_up((size_t)q.caps.chunk * sizeof(int32_t), 256);
    q.small = off;
    off += align_up(QS_RING * (size_t)q.caps.small * sizeof(QSmall), 256);
    q.fill = off;
    off += align_up(QS_RING * (size_t)q.caps.fill * sizeof(QFill), 256);
    q.ctr = off;
    off += align_up(QS_RING * sizeof(QCounters), 256);
    q.status = off;
    off += 256;
    q.total = off;
    return q;
}

size_t quick_workspace_bytes(size_t n) { return qs_layout(n).total; }

void quick_set_max_levels(int64_t v) { qs_option_max_levels = v; }
void quick_set_two_way(int v) { g_qs_two_way = v; }

template <int L>
static hs_status launch_leaves_t(int64_t grid, const QSmall *small, const QFill *fill,
                                 const QCounters *cctr, const QCaps &caps, const int32_t *X,
                                 const int32_t *Y, int32_t *Xw, hs_netset s, cudaStream_t st) {
    const int smem = BlockSort3<QS_BS_NT, L, 4>::SMEM_BYTES;
    auto kern = k_qs_leaves<L>;
    hs_status r = ensure_smem((const void *)kern, smem);
    if (r != HS_OK) return r;
    LaunchToken t = launch_begin(K_QS_LEAVES, st);
    kern<<<(unsigned)grid, QS_BS_NT, smem, st>>>(small, fill, cctr, caps, X, Y, Xw, s);
    return launch_end(t);
}

static hs_status launch_leaves(int L, int64_t grid, const QSmall *small, const QFill *fill,
                               const QCounters *cctr, const QCaps &caps, const int32_t *X,
                               const int32_t *Y, int32_t *Xw, hs_netset s, cudaStream_t st) {
    switch (L) {
        case 1: return launch_leaves_t<1>(grid, small, fill, cctr, caps, X, Y, Xw, s, st);
        case 3: return launch_leaves_t<3>(grid, small, fill, cctr, caps, X, Y, Xw, s, st);
        case 4: return launch_leaves_t<4>(grid, small, fill, cctr, caps, X, Y, Xw, s, st);
        case 5: return launch_leaves_t<5>(grid, small, fill, cctr, caps, X, Y, Xw, s, st);
        case 6: return launch_leaves_t<6>(grid, small, fill, cctr, caps, X, Y, Xw, s, st);
        case 7: return launch_leaves_t<7>(grid, small, fill, cctr, caps, X, Y, Xw, s, st);
        case 8: return launch_leaves_t<8>(grid, small, fill, cctr, caps, X, Y, Xw, s, st);
    }
    return fail(HS_ERR_INVALID_ARG, "leaf size outside 1, 3..8");
}

// Per host thread and device: the leaves stream, the events of the levels in
// flight and the mapped readback slots.  Created on first use and kept for
// the thread's lifetime.
struct QuickCtx {
    int device = -1;
    cudaStream_t side = nullptr;
    cudaEvent_t level_done[QS_RING] = {}, leaves_done[QS_RING] = {}, side_end = nullptr;
    QReadback *h_rb = nullptr, *d_rb = nullptr;
};

// A level's published counters, once its completion event has been waited
// for (the synchronising call orders the device's writes before this read).
static QReadback read_back(const QuickCtx *qc, int64_t level) {
    QReadback r;
    std::memcpy(&r, &qc->h_rb[level % QS_RING], sizeof(r));
    return r;
}

static hs_status quick_ctx(QuickCtx **out) {
    static thread_local std::vector<QuickCtx *> ctxs;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "quick sort: current device");
    for (QuickCtx *c : ctxs)
        if (c->device == dev) {
            *out = c;
            return HS_OK;
        }
    QuickCtx *c = new (std::nothrow) QuickCtx();
    if (!c) return fail(HS_ERR_NO_MEMORY, "quick sort: context");
    c->device = dev;
    e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    for (int i = 0; i < QS_RING && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&c->level_done[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->leaves_done[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->side_end, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void **>(&c->h_rb), QS_RING * sizeof(QReadback),
                          cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&c->d_rb), c->h_rb, 0);
    if (e != cudaSuccess) {
        // Partly built contexts are released; errors on release are moot.
        if (c->h_rb) cudaFreeHost(c->h_rb);
        for (int i = 0; i < QS_RING; ++i) {
            if (c->level_done[i]) cudaEventDestroy(c->level_done[i]);
            if (c->leaves_done[i]) cudaEventDestroy(c->leaves_done[i]);
        }
        if (c->side_end) cudaEventDestroy(c->side_end);
        if (c->side) cudaStreamDestroy(c->side);
        delete c;
        return fail_cuda(e, "quick sort: context");
    }
    ctxs.push_back(c);
    *out = c;
    return HS_OK;
}

// Depth guard: segments still live after the level cap (adversarial inputs
// for median-of-three) are moved into the caller's array and merge-sorted one
// by one, with the workspace's key area as merge scratch.
static hs_status qs_fallback(int32_t *X, int32_t *Y, const QSeg *d_segs, int64_t nseg,
                             hs_netset s, void *merge_ws, size_t merge_ws_bytes, cudaStream_t st) {
    std::vector<QSeg> h((size_t)nseg);
    cudaError_t e = cudaMemcpyAsync(h.data(), d_segs, (size_t)nseg * sizeof(QSeg),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(e, "quick sort: reading segments");
    for (const QSeg &g : h)
        if (g.buf) {
            e = cudaMemcpyAsync(X + g.begin, Y + g.begin, (size_t)(g.end - g.begin) * sizeof(int32_t),
                                cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return fail_cuda(e, "quick sort: fallback copy");
        }
    for (const QSeg &g : h) {
        hs_status r = merge_sort(X + g.begin, nullptr, (size_t)(g.end - g.begin), s, merge_ws,
                                 merge_ws_bytes, st);
        if (r != HS_OK) return r;
    }
    return HS_OK;
}

hs_status quick_sort(int32_t *d_keys, size_t n_, hs_netset s, void *d_ws, size_t ws_bytes,
                     cudaStream_t st) {
    const int64_t n = (int64_t)n_;
    const int L = leaf_size(s);
    const int64_t tile = qs_tile(L);
    const int vec = aligned(d_keys, 16) ? 1 : 0;
    // Arrays of one tile are the base case: no partition.  Up to the small
    // sort's tile one CTA sorts them in one launch.
    if (n <= small_sort_max(L)) return small_sort(d_keys, n, s, st);
    if (n <= keys_tile(L, n)) return blocksort_launch(L, d_keys, d_keys, n, s, vec, st);

    const QLayout q = qs_layout(n_);
    if (!d_ws || ws_bytes < q.total)
        return fail(HS_ERR_INVALID_ARG, "quick sort: workspace smaller than hs_sort_workspace_bytes");
    if (!aligned(d_ws, 16)) return fail(HS_ERR_INVALID_ARG, "quick sort: workspace not 16-byte aligned");
    char *base = static_cast<char *>(d_ws);
    int32_t *X = d_keys;
    int32_t *Y = reinterpret_cast<int32_t *>(base + q.y);
    QSeg *cur = reinterpret_cast<QSeg *>(base + q.seg_a);
    QSeg *nxt = reinterpret_cast<QSeg *>(base + q.seg_b);
    int32_t *ccur = reinterpret_cast<int32_t *>(base + q.chunk_a);
    int32_t *cnxt = reinterpret_cast<int32_t *>(base + q.chunk_b);
    QSmall *small = reinterpret_cast<QSmall *>(base + q.small);
    QFill *fill = reinterpret_cast<QFill *>(base + q.fill);
    QCounters *ctr = reinterpret_cast<QCounters *>(base + q.ctr);
    unsigned long long *status = reinterpret_cast<unsigned long long *>(base + q.status);

    QuickCtx *qc = nullptr;
    hs_status r = quick_ctx(&qc);
    if (r != HS_OK) return r;

    const int64_t nchunks0 = (n + QS_C - 1) / QS_C;
    LaunchToken t = launch_begin(K_QS_PLAN, st);
    k_qs_init<<<(unsigned)std::min<int64_t>((nchunks0 + 255) / 256, 4096), 256, 0, st>>>(
        cur, ccur, n, nchunks0, X, ctr, status);
    if ((r = launch_end(t)) != HS_OK) return r;

    int lg = 0;
    while ((int64_t(1) << lg) < n) ++lg;
    const int64_t max_levels = qs_option_max_levels >= 0 ? qs_option_max_levels : 4 * lg + 16;
    // Levels launched ahead of the last counters read back.
    constexpr int64_t kAhead = 2;
    // The latest exact counts the host knows: those of level `known`.
    int64_t known = 0;
    int64_t known_nseg = 1, known_nchunks = nchunks0;
    const QCaps &caps = q.caps;
    cudaError_t e = cudaSuccess;
    int64_t level = 0;
    // Waits for everything launched so far (the leaves stream included).
    auto drain = [&]() {
        cudaEventRecord(qc->side_end, qc->side);
        cudaStreamWaitEvent(st, qc->side_end, 0);
        return cudaStreamSynchronize(st);
    };
    for (;; ++level) {
        if (level >= kAhead) {
            const int64_t j = level - kAhead;
            if ((e = cudaEventSynchronize(qc->level_done[j % QS_RING])) != cudaSuccess)
                return fail_cuda(e, "quick sort: waiting for a level");
            const QReadback rb = read_back(qc, j);
            if (rb.status) {
                drain();
                return fail(HS_ERR_CUDA, "quick sort: internal work-list overflow");
            }
            known = j + 1;
            known_nseg = (int64_t)rb.next.nseg;
            known_nchunks = (int64_t)rb.next.nchunks;
            if (known_nseg == 0) break;  // the levels after j were launched empty
        }
        if (level >= max_levels) {
            // Every level up to here has been launched: wait for all of them,
            // then hand the segments still live to the merge path.
            if ((e = drain()) != cudaSuccess) return fail_cuda(e, "quick sort: synchronize");
            int64_t live = 1;  // level 0: the whole array
            if (level > 0) {
                const QReadback rb = read_back(qc, level - 1);
                if (rb.status) return fail(HS_ERR_CUDA, "quick sort: internal work-list overflow");
                live = (int64_t)rb.next.nseg;
            }
            if (live == 0) break;
            return qs_fallback(X, Y, cur, live, s, base + q.y, merge_workspace_bytes(n_, 0), st);
        }
        // Launch sizes: exact for the level whose counts are known, else
        // bounds (segments at most double per level; chunks are at most the
        // known chunks plus one partial chunk per segment).
        const int64_t lag = level - known;
        const int64_t seg_b = lag == 0 ? known_nseg
                                       : std::min<int64_t>(caps.seg, known_nseg << std::min<int64_t>(lag, 32));
        const int64_t chunk_b = lag == 0 ? known_nchunks
                                         : std::min<int64_t>(caps.chunk, known_nchunks + seg_b);
        const int slot = (int)(level % QS_RING), nslot = (int)((level + 1) % QS_RING);
        QCounters *cc = ctr + slot, *nc = ctr + nslot;
        QSmall *small_l = small + (size_t)slot * caps.small;
        QFill *fill_l = fill + (size_t)slot * caps.fill;
        // Slot nslot last served level + 1 - QS_RING: its leaves must be done
        // before its counters are reset.
        if (level + 1 >= QS_RING && (e = cudaStreamWaitEvent(st, qc->leaves_done[nslot], 0)) != cudaSuccess)
            return fail_cuda(e, "quick sort: ordering the leaves");
        if ((e = cudaMemsetAsync(nc, 0, sizeof(QCounters), st)) != cudaSuccess)
            return fail_cuda(e, "quick sort: counter reset");
        if (chunk_b > 0) {
            t = launch_begin(K_QS_PARTITION, st);
            if (g_qs_two_way)
                k_qs_partition<true><<<(unsigned)chunk_b, QS_NT, 0, st>>>(cur, ccur, cc, caps, X, Y, X, Y);
            else
                k_qs_partition<false><<<(unsigned)chunk_b, QS_NT, 0, st>>>(cur, ccur, cc, caps, X, Y, X, Y);
            if ((r = launch_end(t)) != HS_OK) return r;
        }
        t = launch_begin(K_QS_PLAN, st);
        k_qs_next<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((seg_b + 255) / 256, 4096)), 256, 0, st>>>(
            cur, cc, nc, caps, tile, nxt, small_l, fill_l, X, Y, status);
        if ((r = launch_end(t)) != HS_OK) return r;
        t = launch_begin(K_QS_PLAN, st);
        k_qs_chunkmap<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(2 * seg_b, 4096)), 256, 0, st>>>(
            nxt, cc, nc, caps, cnxt, status, qc->d_rb + slot);
        if ((r = launch_end(t)) != HS_OK) return r;
        if ((e = cudaEventRecord(qc->level_done[slot], st)) != cudaSuccess)
            return fail_cuda(e, "quick sort: level event");
        // This level's small children and long = ranges, on the leaves stream.
        if ((e = cudaStreamWaitEvent(qc->side, qc->level_done[slot], 0)) != cudaSuccess)
            return fail_cuda(e, "quick sort: ordering the leaves");
        const int64_t leaves_b = std::min<int64_t>(caps.small + caps.fill, 3 * seg_b);
        if (leaves_b > 0 &&
            (r = launch_leaves(L, std::min<int64_t>(leaves_b, 8192), small_l, fill_l, cc, caps, X, Y,
                               X, s, qc->side)) != HS_OK)
            return r;
        if ((e = cudaEventRecord(qc->leaves_done[slot], qc->side)) != cudaSuccess)
            return fail_cuda(e, "quick sort: leaves event");
        std::swap(cur, nxt);
        std::swap(ccur, cnxt);
    }
    // The sort ends on `st`: it waits for the leaves stream's last work.
    if ((e = cudaEventRecord(qc->side_end, qc->side)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(st, qc->side_end, 0)) != cudaSuccess)
        return fail_cuda(e, "quick sort: joining the leaves stream");
    return HS_OK;
}

}  // namespace hs
