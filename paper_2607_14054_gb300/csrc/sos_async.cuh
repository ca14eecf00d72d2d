// Asynchronous-copy and mbarrier helpers shared by the forward kernels
// (inline PTX, sm_90+ forms available on sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sosf {

__device__ __forceinline__ unsigned smem_u32(const void* a) {
    return (unsigned)__cvta_generic_to_shared(a);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
    // src-size 0 fills the destination with zeros and reads nothing
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                     smem_u32(b))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Store of the hand-off value and arrive, both predicated on `pred` inside
// the asm block (no branch, so the warp stays converged).
__device__ __forceinline__ void mbar_publish(float2* v, float a, float b, unsigned long long* bar,
                                             bool pred) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b64 st;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "@p st.shared.v2.f32 [%0], {%1, %2};\n\t"
        "@p mbarrier.arrive.shared::cta.b64 st, [%3];\n\t}" ::"r"(smem_u32(v)),
        "f"(a), "f"(b), "r"(smem_u32(bar)), "r"((unsigned)pred)
        : "memory");
}

// bound on try_wait calls in one hand-off (each call may suspend the warp
// for a while before returning false)
constexpr uint32_t kHandOffLimit = 1u << 20;

}  // namespace sosf
