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
HS_DEV int64_t ld_stream(const int64_t *p) {
    int64_t v;
    asm volatile("ld.global.cs.s64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
HS_DEV void st_stream(int64_t *p, int64_t v) {
    asm volatile("st.global.cs.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

}  // namespace hs

// ---------------------------------------------------------------------------
namespace hs {

// Shared-window address of a shared-memory pointer (for PTX operands).
HS_DEV uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Device status bits raised by kernels instead of trapping.
constexpr unsigned kStatusTimeout = 1u;  // a bounded device-side wait gave up
constexpr unsigned kStatusBadOffsets = 2u;
constexpr unsigned kStatusMisaligned = 4u;  // a bulk copy's addresses were not 16-byte aligned
constexpr unsigned kStatusInconsistent = 8u;  // merge splits that would stage outside a buffer

}  // namespace hs
