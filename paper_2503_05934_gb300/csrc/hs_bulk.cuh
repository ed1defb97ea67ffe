// Bulk asynchronous copies (the TMA engine's untiled form, cp.async.bulk)
// between global and shared memory, completed through an mbarrier (loads) or
// a bulk group (stores).  One thread issues a whole tile's copy, so the
// load/store units carry none of the tile's global traffic: they are left to
// the merge's own shared-memory reads and writes.
//
// Rules of the untiled form: both addresses 16-byte aligned and the size a
// multiple of 16 bytes.  Every wait here is bounded.
#pragma once

#include "hs_common.cuh"

namespace hs {

// Polls of a bounded mbarrier wait (each try_wait may also suspend the
// thread for a while): far beyond any healthy copy, far below a hang.
constexpr long kBulkSpinLimit = 1L << 22;

HS_DEV void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
    // Make the initialised barrier visible to the async proxy (the copy engine).
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

HS_DEV void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// True once the barrier's phase `parity` has completed; false after `limit`
// polls.
HS_DEV bool mbar_wait(uint64_t *bar, unsigned parity, long limit = kBulkSpinLimit) {
    const uint32_t a = smem_addr(bar);
    for (long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// L2 policy for streamed data: evict first, so that small reused arrays (the
// partition samples) stay resident while whole passes stream through.
HS_DEV uint64_t l2_evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// L2 policy for data read again soon (a segment's merge levels in the
// batched form): the normal eviction priority.
HS_DEV uint64_t l2_evict_normal_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Global -> shared, `bytes` (multiple of 16, both ends 16-byte aligned),
// completing `bytes` of transaction count on `bar`.
HS_DEV void bulk_load(void *sdst, const void *gsrc, unsigned bytes, uint64_t *bar,
                      uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(sdst)),
        "l"(gsrc), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// Shared -> global in the calling thread's bulk group.
HS_DEV void bulk_store(void *gdst, const void *ssrc, unsigned bytes, uint64_t policy) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;"
                 ::"l"(gdst), "r"(smem_addr(ssrc)), "r"(bytes), "l"(policy)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Waits until the calling thread's bulk stores have read their shared source
// (the CTA's shared memory must outlive those reads).
HS_DEV void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Waits until the calling thread's bulk stores have completed their writes
// (for kernels that read back what they stored).
HS_DEV void bulk_wait_writes() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Orders this thread's global-memory accesses by the generic proxy (plain
// loads and stores) with those of the async proxy (bulk copies) on either
// side of it; a barrier after it extends the order to the rest of the CTA.
HS_DEV void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Orders this thread's generic shared-memory writes before later bulk copies
// (async proxy) that read them.
HS_DEV void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// x[k] for a run-time k in [0, N) without local memory: a select tree on k's bits.
template <int N, class K>
HS_HD K select_dyn(const K (&x)[N], int k) {
    constexpr int P = N <= 1 ? 1 : N <= 2 ? 2 : N <= 4 ? 4 : N <= 8 ? 8 : N <= 16 ? 16 : N <= 32 ? 32 : 64;
    static_assert(N <= P, "select_dyn covers arrays of up to 64 entries");
    K v[P];
#pragma unroll
    for (int i = 0; i < P; ++i) v[i] = x[i < N ? i : 0];
#pragma unroll
    for (int h = P / 2; h >= 1; h /= 2) {
        const bool up = (k & h) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) v[i] = up ? v[i + h] : v[i];
    }
    return v[0];
}

}  // namespace hs
