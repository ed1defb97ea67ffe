// Shared device/host helpers of the hsort CUDA library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define HS_HD __host__ __device__ __forceinline__
#define HS_DEV __device__ __forceinline__

namespace hs {

// +infinity sentinel for padded leaves.  It is never stored: only the first
// n outputs of a padded tile are written back, and sentinels sort last.
constexpr int32_t kKeyMax = INT32_MAX;

// Shared-memory index with one pad word per 32: thread t reading element
// t*E + j (E = 8 or 16) then hits 32 distinct banks.
HS_HD int pad32(int i) { return i + (i >> 5); }

template <class T>
HS_HD T hs_min(T a, T b) { return b < a ? b : a; }
template <class T>
HS_HD T hs_max(T a, T b) { return a < b ? b : a; }

// Streaming global loads/stores: every key is read once and written once per
// pass, and a pass moves far more than L2 holds, so mark them evict-first.
HS_DEV int4 ld_stream(const int4 *p) {
    int4 v;
    asm volatile("ld.global.cs.v4.s32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}
HS_DEV int32_t ld_stream(const int32_t *p) {
    int32_t v;
    asm volatile("ld.global.cs.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
HS_DEV void st_stream(int4 *p, int4 v) {
    asm volatile("st.global.cs.v4.s32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}
HS_DEV void st_stream(int32_t *p, int32_t v) {
    asm volatile("st.global.cs.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

}  // namespace hs

// ---------------------------------------------------------------------------
// Bulk-copy (TMA) and mbarrier helpers for one CTA (no cluster, no multicast).
namespace hs {

HS_DEV uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

HS_DEV void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Makes initialised barriers visible to the async proxy (bulk copies).
HS_DEV void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders earlier generic-proxy shared-memory accesses before later bulk copies.
HS_DEV void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One arrival that also announces `bytes` of incoming bulk-copy data.
HS_DEV void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared; src and dst 16-byte aligned, bytes % 16 == 0.
HS_DEV void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

HS_DEV bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

HS_DEV uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase with the given parity: gives up after about one
// second (or 2^28 polls) and returns false instead of spinning forever.
HS_DEV bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int i = 0; i < 32; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < (1u << 28); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) break;
    }
    return false;
}

// Device status bits raised by kernels instead of trapping.
constexpr unsigned kStatusTimeout = 1u;
constexpr unsigned kStatusBadOffsets = 2u;

}  // namespace hs
