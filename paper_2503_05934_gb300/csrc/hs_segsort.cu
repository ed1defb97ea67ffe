// Batched form: many independent arrays sorted by one persistent launch.
//
// Every array ("segment") is sorted by a single CTA, as Algorithm 1 would sort
// it: network leaves and shared-memory merge levels (the block sort's) for a
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

#include "hs_bulk.cuh"
#include "hs_internal.h"
#include "hs_blocksort.cuh"
#include "hs_segsort.h"

namespace hs {

constexpr int SPLIT_CAP = 256;  // merge-level chunk boundaries searched per batch

// Bulk-copy staging of the batched form.  Segments start anywhere, so a run
// g[0, cnt) of keys is placed at s[0, cnt) with s congruent to g modulo 16
// bytes (s = a 16-byte aligned base + (g mod 16) / 4 words): its 16-byte
// aligned interior then moves as one bulk copy, and at most three keys at
// each end move by plain loads and stores.  The copies never touch a word
// outside the run.
struct StageCut {
    int head, body;  // keys before the first 16-byte boundary, then whole 16-byte words (keys)
};
HS_DEV StageCut stage_cut(const int32_t *g, int cnt) {
    const int h = (int)(((16u - (uint32_t)(reinterpret_cast<uintptr_t>(g) & 15u)) & 15u) >> 2);
    StageCut c;
    c.head = h < cnt ? h : cnt;
    c.body = ((cnt - c.head) >> 2) << 2;
    return c;
}
HS_DEV int32_t *congruent(int32_t *sbase, const int32_t *g) {
    return sbase + ((reinterpret_cast<uintptr_t>(g) & 15u) >> 2);
}
// Thread 0: the interior copy (its bytes are counted by the caller's expect_tx).
HS_DEV void stage_issue(int32_t *s, const int32_t *g, const StageCut &c, uint64_t *bar,
                        uint64_t pol) {
    if (c.body > 0) bulk_load(s + c.head, g + c.head, (unsigned)c.body * 4u, bar, pol);
}
template <int NT>
HS_DEV void stage_edges(int32_t *s, const int32_t *g, int cnt, const StageCut &c) {
    for (int i = threadIdx.x; i < c.head; i += NT) s[i] = g[i];
    for (int i = c.head + c.body + threadIdx.x; i < cnt; i += NT) s[i] = g[i];
}
// Writes s[0, cnt) back to g (congruent as above).  The caller has made every
// thread's writes to s visible to the copy engine (fence_proxy_async_smem and
// a barrier); thread 0 waits until the bulk store has read s, so s may be
// reused after the caller's next barrier.
template <int NT>
HS_DEV void unstage(const int32_t *s, int32_t *g, int cnt, uint64_t pol) {
    const StageCut c = stage_cut(g, cnt);
    if (threadIdx.x == 0 && c.body > 0) {
        bulk_store(g + c.head, s + c.head, (unsigned)c.body * 4u, pol);
        bulk_wait_read();
    }
    for (int i = threadIdx.x; i < c.head; i += NT) g[i] = s[i];
    for (int i = c.head + c.body + threadIdx.x; i < cnt; i += NT) g[i] = s[i];
}

// Makes everything the CTA stored so far (thread 0's bulk stores, every
// thread's plain stores) visible to the CTA's later reads by either proxy.
HS_DEV void stores_done() {
    if (threadIdx.x == 0) bulk_wait_writes();
    fence_proxy_async_global();
    __syncthreads();
}

// Per-CTA state of the bulk-copy staging: one mbarrier, its phase parity,
// the L2 policy and the status word for a wait that gives up.
struct Stager {
    uint64_t *bar;
    unsigned phase;
    uint64_t pol;
    unsigned *status;
    // Every thread calls it after the interior copies were issued; false if
    // the wait gave up (the status word is raised, and the copies in flight
    // get one more bounded wait).  Callers separate consecutive waits by a
    // barrier, so no thread lags a phase behind; after a false the CTA stops
    // using the barrier.
    HS_DEV bool wait() {
        const bool ok = mbar_wait(bar, phase);
        if (!ok) {
            atomicOr(status, kStatusTimeout);
            mbar_wait(bar, phase);
        }
        phase ^= 1u;
        return ok;
    }
};


// One merge level over a single segment by one CTA: runs of w in src are
// merged into runs of 2w in dst.  Output chunks of T keys: their merge-path
// splits are found by one warp per chunk boundary; each chunk's A and B
// ranges are then placed congruent to their global addresses in two regions
// of the buffer (A first, B from the next 16-byte boundary after it), each
// thread merges exactly its own EO outputs (exact window, end split from the
// next lane), and the merged chunk leaves from a copy congruent to its
// destination (src and dst need not be congruent to each other).  False if a
// copy wait gave up or the chunk's split sizes do not fit the buffer.
template <int NT, int L, int LV>
HS_DEV bool cta_merge_level_staged(const int32_t *src, int32_t *dst, int64_t n, int64_t w,
                                   int32_t *sbase, int64_t *split, Stager &sg) {
    using C = BlockSort3<NT, L, LV>;
    constexpr int T = C::T, EO = C::EO, P = C::P;
    const int64_t span = 2 * w;
    const int64_t ngroups = (n + span - 1) / span;
    const int64_t tpg = (span + T - 1) / T;
    const int64_t last = n - (ngroups - 1) * span;
    const int64_t nchunks = (ngroups - 1) * tpg + (last + T - 1) / T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // Past the A and B regions (at most T + 9 + P words with the window slack).
    int *wsplit = sbase + C::T + C::P + 32;
    for (int64_t c0 = 0; c0 < nchunks; c0 += SPLIT_CAP) {
        const int64_t c1 = std::min<int64_t>(nchunks, c0 + SPLIT_CAP);
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
            // Consistent splits give 0 <= na, nb <= tot <= T; anything else would
            // stage outside the buffer, so it is reported and the segment dropped
            // (the values are the same in every thread: uniform).
            if (na < 0 || nb < 0 || tot > T) {
                if (threadIdx.x == 0) atomicOr(sg.status, kStatusInconsistent);
                return false;
            }
            const int32_t *gA = src + m.gs + a0, *gB = src + m.gs + w + (o0 - a0);
            int32_t *sA = congruent(sbase, gA);
            int32_t *sB = congruent(sbase + ((int)(sA - sbase) + na + 3) / 4 * 4, gB);
            fence_proxy_async_smem();  // earlier generic writes to the buffer before the copies
            __syncthreads();
            const StageCut ca = stage_cut(gA, na), cb = stage_cut(gB, nb);
            if (threadIdx.x == 0) {
                mbar_arrive_expect_tx(sg.bar, (unsigned)(ca.body + cb.body) * 4u);
                stage_issue(sA, gA, ca, sg.bar, sg.pol);
                stage_issue(sB, gB, cb, sg.bar, sg.pol);
            }
            stage_edges<NT>(sA, gA, na, ca);
            stage_edges<NT>(sB, gB, nb, cb);
            const bool ok = sg.wait();
            if (__syncthreads_or(!ok)) return false;
            const int32_t *A = sA, *B = sB;
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
            int32_t *out = dst + m.gs + o0;
            int32_t *so = congruent(sbase, out);
            if (cnt > 0) {
#pragma unroll
                for (int k = 0; k < EO; ++k)
                    if (k < cnt) so[diag + k] = x[k];
            }
            fence_proxy_async_smem();
            __syncthreads();
            unstage<NT>(so, out, tot, sg.pol);
            __syncthreads();
        }
    }
    // The next level reads this one's output back: its bulk stores must be
    // done, and both the bulk stores and the threads' plain stores of the
    // chunk ends must be ordered before the next reads of either proxy.
    stores_done();
    return true;
}

// One block-sort tile of a segment through bulk-copy staging: keys src[0,
// cnt) sorted into dst[0, cnt).  The tile is placed congruent to src; when
// dst is congruent to src too (in place, or the same offset of a congruent
// scratch area) it leaves by a bulk store, else by plain stores.  Slots past
// cnt hold +infinity sentinels.  False if a copy wait gave up.
template <int NT, int L, int LV, bool SKIP>
HS_DEV bool sort_tile_staged(int32_t *sbase, const int32_t *src, int32_t *dst, int cnt,
                             uint32_t netset, Stager &sg) {
    using C = BlockSort3<NT, L, LV>;
    constexpr int T = C::T, EO = C::EO, P = C::P;
    int32_t *s = congruent(sbase, src);
    int *wsplit = s + T + P + 32;
    fence_proxy_async_smem();  // earlier generic writes to the buffer before the copy
    __syncthreads();
    const StageCut c = stage_cut(src, cnt);
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(sg.bar, (unsigned)c.body * 4u);
        stage_issue(s, src, c, sg.bar, sg.pol);
    }
    stage_edges<NT>(s, src, cnt, c);
    for (int i = cnt + threadIdx.x; i < T; i += NT) s[i] = kKeyMax;
    const bool ok = sg.wait();
    if (__syncthreads_or(!ok)) return false;
    const int my0 = threadIdx.x * EO;
    int32_t k[EO];
#pragma unroll
    for (int j = 0; j < EO; ++j) k[j] = s[my0 + j];
    if (!SKIP || my0 < cnt) sort_thread_leaves<L, LV, P>(k, cnt - my0, netset);
    block_merge_levels<NT, EO, P, SKIP>(s, wsplit, k, cnt);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < EO; ++j) s[my0 + j] = k[j];
    fence_proxy_async_smem();
    __syncthreads();
    if (((reinterpret_cast<uintptr_t>(src) ^ reinterpret_cast<uintptr_t>(dst)) & 15u) == 0) {
        unstage<NT>(s, dst, cnt, sg.pol);
    } else {
        for (int i = threadIdx.x; i < cnt; i += NT) dst[i] = s[i];
    }
    __syncthreads();
    return true;
}

// Every tile and merge chunk moves by bulk copies of its 16-byte aligned
// interior (sg).  False (uniform across the CTA) if a copy wait gave up.
template <int NT, int L, int LV>
HS_DEV bool sort_segment(const SegDesc &d, uint32_t netset, int32_t *s, int64_t *split,
                         Stager &sg) {
    using C = BlockSort3<NT, L, LV>;
    constexpr int T = C::T;
    const int64_t n = d.n;
    if (n <= 1) return true;
    if (n <= T) return sort_tile_staged<NT, L, LV, true>(s, d.keys, d.keys, (int)n, netset, sg);
    int levels = 0;
    for (int64_t w = T; w < n; w *= 2) ++levels;
    // Ping-pong so that the last level lands in d.keys.
    int32_t *cur = (levels % 2 == 0) ? d.keys : d.scratch;
    int32_t *alt = (levels % 2 == 0) ? d.scratch : d.keys;
    for (int64_t base = 0; base < n; base += T) {
        const int cnt = (int)std::min<int64_t>(T, n - base);
        if (!sort_tile_staged<NT, L, LV, false>(s, d.keys + base, cur + base, cnt, netset, sg))
            return false;
    }
    // The merge levels read the tiles back.
    stores_done();
    for (int64_t w = T; w < n; w *= 2) {
        if (!cta_merge_level_staged<NT, L, LV>(cur, alt, n, w, s, split, sg)) return false;
        int32_t *tmp = cur;
        cur = alt;
        alt = tmp;
    }
    return true;
}

// A segment of at most one warp tile (32 * EO keys) sorted by one warp alone:
// the block sort's leaves and merge levels with warp barriers only, in the
// warp's own part of shared memory, so a CTA keeps one small segment in
// flight per warp instead of one per CTA.
template <int L, int LV>
HS_DEV void warp_sort_segment(int32_t *keys, int n, uint32_t netset, int32_t *s) {
    using W = BlockSort3<32, L, LV>;
    constexpr int EO = W::EO, P = W::P, T = W::T;
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < T; i += 32) {
        if (i < n) cp_async4(s + i, keys + i);
        else s[i] = kKeyMax;
    }
    cp_async_wait_all();
    __syncwarp();
    const int my0 = lane * EO;
    int32_t k[EO];
#pragma unroll
    for (int j = 0; j < EO; ++j) k[j] = s[my0 + j];
    if (my0 < n) sort_thread_leaves<L, LV, P>(k, n - my0, netset);
    block_merge_levels<32, EO, P, true, int32_t, true>(s, nullptr, k, n);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < EO; ++j) s[my0 + j] = k[j];
    __syncwarp();
    for (int i = lane; i < n; i += 32) keys[i] = s[i];
    __syncwarp();
}

// Queue counters of one launch (zeroed before the classify step):
// [0] large-list head, [1] small-list head, [2] large count, [3] small count.
constexpr int kCtrlWords = 4;

// Dynamic shared memory of the batched kernel: the block tile, or one warp
// tile per warp, whichever is larger.
template <int NT, int L, int LV>
constexpr int seg_smem_bytes() {
    constexpr int blk = BlockSort3<NT, L, LV>::SMEM_BYTES + 16;  // + a congruent shift of up to 3 words
    constexpr int wrp = (NT / 32) * BlockSort3<32, L, LV>::SMEM_BYTES;
    return blk > wrp ? blk : wrp;
}

// Persistent sort over the classified descriptors: CTAs first take the large
// list (cdesc[0, nlarge), one segment per CTA), then each warp takes small
// segments from the back of the array (cdesc[ndesc - 1 - j]) until both
// lists are drained.  Large segments first also balances the load: the
// short items fill the gaps at the end.
// Resident CTAs of 256 threads the register budget allows (measured: 3 with
// 80 registers against 4 with 64 registers and spills, 14.8 against 15.9 ms
// for the 200,000-array batch).
constexpr int kSegMinCtas = 3;
template <int NT, int L, int LV>
__global__ void __launch_bounds__(NT, NT <= 256 ? kSegMinCtas : 2)
    k_seg_sort(const SegDesc *cdesc, int64_t ndesc, unsigned long long *ctrl, uint32_t netset,
               unsigned *status) {
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ int64_t s_split[SPLIT_CAP + 1];
    __shared__ unsigned long long s_item[2];
    __shared__ __align__(8) uint64_t s_bar;
    Stager sg{&s_bar, 0u, l2_evict_normal_policy(), status};
    // The congruent staging relies on a 16-byte aligned dynamic buffer.
    if ((smem_addr(smem) & 15u) != 0) {
        if (threadIdx.x == 0) atomicOr(status, kStatusMisaligned);
        return;
    }
    if (threadIdx.x == 0) mbar_init(&s_bar, 1);
    const unsigned long long nlarge = ctrl[2], nsmall = ctrl[3];
    if (threadIdx.x == 0) s_item[0] = atomicAdd(&ctrl[0], 1ull);
    __syncthreads();
    for (int it = 0;; it ^= 1) {
        const unsigned long long item = s_item[it];
        if (item >= nlarge) break;
        // The next item is claimed now; the atomic's round trip overlaps
        // this segment's sort and its result is only consumed at the end.
        unsigned long long next = 0;
        if (threadIdx.x == 0) next = atomicAdd(&ctrl[0], 1ull);
        const SegDesc d = cdesc[item];
        // A copy wait that gave up (status raised) ends this CTA's work.
        if (!sort_segment<NT, L, LV>(d, netset, smem, s_split, sg)) return;
        if (threadIdx.x == 0) s_item[it ^ 1] = next;
        __syncthreads();
    }
    // Every thread left the loop after the same barrier: the block's shared
    // memory is free for the warps' own tiles.
    constexpr int WSZ = BlockSort3<32, L, LV>::SZ;
    int32_t *ws = smem + (threadIdx.x >> 5) * WSZ;
    for (;;) {
        unsigned long long j = 0;
        if ((threadIdx.x & 31) == 0) j = atomicAdd(&ctrl[1], 1ull);
        j = __shfl_sync(0xffffffffu, j, 0);
        if (j >= nsmall) break;
        const SegDesc d = cdesc[ndesc - 1 - (int64_t)j];
        warp_sort_segment<L, LV>(d.keys, (int)d.n, netset, ws);
    }
}

// Files descriptor d (when valid) into the classified array: large segments
// (more than small_max keys) from the front, small ones (2..small_max keys)
// from the back; empty and one-key segments are already sorted and dropped.
// One atomic per warp and class.  Every lane of the warp must call it.
HS_DEV void classify_desc(const SegDesc &d, bool valid, int64_t ndesc, int64_t small_max,
                          SegDesc *cdesc, unsigned long long *ctrl) {
    const bool big = valid && d.n > small_max;
    const bool sml = valid && d.n > 1 && d.n <= small_max;
    const unsigned mb = __ballot_sync(0xffffffffu, big), ms = __ballot_sync(0xffffffffu, sml);
    const int lane = threadIdx.x & 31;
    unsigned long long bb = 0, sb = 0;
    if (lane == 0) {
        if (mb) bb = atomicAdd(&ctrl[2], (unsigned long long)__popc(mb));
        if (ms) sb = atomicAdd(&ctrl[3], (unsigned long long)__popc(ms));
    }
    bb = __shfl_sync(0xffffffffu, bb, 0);
    sb = __shfl_sync(0xffffffffu, sb, 0);
    const unsigned below = (1u << lane) - 1u;
    if (big) cdesc[bb + __popc(mb & below)] = d;
    if (sml) cdesc[ndesc - 1 - (int64_t)(sb + __popc(ms & below))] = d;
}

// Classifies caller-built descriptors (the serving loop's batches).
__global__ void k_seg_classify(const SegDesc *descs, int64_t ndesc, int64_t small_max,
                               SegDesc *cdesc, unsigned long long *ctrl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    SegDesc d{};
    const bool valid = i < ndesc;
    if (valid) d = descs[i];
    classify_desc(d, valid, ndesc, small_max, cdesc, ctrl);
}

// Descriptors for an offsets array, classified as they are built: segment i
// is keys[off[i], off[i+1]); its scratch is the same range of the workspace
// key area.  Malformed offsets raise a status bit and drop the segment.
__global__ void k_seg_descs(int32_t *keys, int64_t n_keys, const int64_t *off, int64_t nseg,
                            int32_t *scratch, int64_t small_max, SegDesc *cdesc,
                            unsigned long long *ctrl, unsigned *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    SegDesc d{};
    bool valid = false;
    if (i < nseg) {
        const int64_t b = off[i], e = off[i + 1];
        if (b < 0 || e < b || e > n_keys) {
            atomicOr(status, kStatusBadOffsets);
        } else {
            d.keys = keys + b;
            d.scratch = scratch + b;
            d.n = e - b;
            valid = true;
        }
    }
    classify_desc(d, valid, nseg, small_max, cdesc, ctrl);
}

// ------------------------------------------------------------------ host side

struct SegKernelInfo {
    const void *fn;
    int smem;
    int max_occ;
    int64_t small_max;  // segments of up to this many keys are sorted by one warp
};

template <int NT, int L, int LV>
static hs_status seg_kernel_info(SegKernelInfo *out) {
    constexpr int SMEM = seg_smem_bytes<NT, L, LV>();
    auto kern = k_seg_sort<NT, L, LV>;
    hs_status r = ensure_smem((const void *)kern, SMEM);
    if (r != HS_OK) return r;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, SMEM);
    if (e != cudaSuccess) return fail_cuda(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    out->fn = (const void *)kern;
    out->smem = SMEM;
    out->max_occ = occ > 0 ? occ : 1;
    out->small_max = BlockSort3<32, L, LV>::T;
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

// The persistent sort over classified descriptors (ctrl already holds the
// class counts and zeroed heads).
static hs_status seg_launch_sort(const SegKernelInfo &ki, const SegDesc *d_cdesc, int64_t ndesc,
                                 unsigned long long *d_ctrl, const hs_plan &plan, cudaStream_t st) {
    const int per_sm = plan.ctas_per_sm > 0 ? std::min(plan.ctas_per_sm, ki.max_occ) : ki.max_occ;
    const int64_t grid = std::min<int64_t>(ndesc, (int64_t)sm_count() * per_sm);
    uint32_t netset = plan.netset;
    unsigned *status = nullptr;
    hs_status r = device_status(&status);
    if (r != HS_OK) return r;
    void *args[] = {(void *)&d_cdesc, (void *)&ndesc, (void *)&d_ctrl, (void *)&netset,
                    (void *)&status};
    LaunchToken t = launch_begin(K_SEG_SORT, st);
    cudaError_t e = cudaLaunchKernel(ki.fn, dim3((unsigned)grid), dim3(plan.block_threads), args,
                                     ki.smem, st);
    if (e != cudaSuccess) {
        launch_end(t);
        return fail_cuda(e, "segsort launch");
    }
    return launch_end(t);
}

hs_status seg_launch_descs(const SegDesc *d_descs, int64_t ndesc, SegDesc *d_cdesc,
                           unsigned long long *d_ctrl, const hs_plan &plan, cudaStream_t st) {
    hs_status r = check_plan(plan);
    if (r != HS_OK) return r;
    if (ndesc <= 0) return HS_OK;
    SegKernelInfo ki{};
    if ((r = seg_kernel(plan.block_threads, leaf_size(plan.netset), &ki)) != HS_OK) return r;
    cudaError_t e = cudaMemsetAsync(d_ctrl, 0, kCtrlWords * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return fail_cuda(e, "segsort: queue reset");
    LaunchToken t = launch_begin(K_SEG_CLASSIFY, st);
    k_seg_classify<<<(unsigned)((ndesc + 255) / 256), 256, 0, st>>>(d_descs, ndesc, ki.small_max,
                                                                    d_cdesc, d_ctrl);
    if ((r = launch_end(t)) != HS_OK) return r;
    return seg_launch_sort(ki, d_cdesc, ndesc, d_ctrl, plan, st);
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
    SegKernelInfo ki{};
    if ((r = seg_kernel(plan.block_threads, leaf_size(plan.netset), &ki)) != HS_OK) return r;
    char *base = static_cast<char *>(d_ws);
    int32_t *scratch = reinterpret_cast<int32_t *>(base + l.keys);
    SegDesc *cdesc = reinterpret_cast<SegDesc *>(base + l.descs);
    unsigned long long *ctrl = reinterpret_cast<unsigned long long *>(base + l.head);
    unsigned *status = nullptr;
    if ((r = device_status(&status)) != HS_OK) return r;
    cudaError_t e = cudaMemsetAsync(ctrl, 0, kCtrlWords * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return fail_cuda(e, "segsort: queue reset");
    LaunchToken t = launch_begin(K_SEG_CLASSIFY, st);
    k_seg_descs<<<(unsigned)((num_segs + 255) / 256), 256, 0, st>>>(
        d_keys, (int64_t)n_keys, d_offsets, (int64_t)num_segs, scratch, ki.small_max, cdesc, ctrl,
        status);
    if ((r = launch_end(t)) != HS_OK) return r;
    return seg_launch_sort(ki, cdesc, (int64_t)num_segs, ctrl, plan, st);
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
