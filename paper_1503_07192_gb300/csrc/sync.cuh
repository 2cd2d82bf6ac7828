// Device-side flag synchronisation between CTAs of one launch (the back-substitution's
// tile flags, the elimination rounds' task flags): release stores, acquire loads and the
// global timer that bounds every wait.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spq {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bound of one device-side dependency wait in ns, and whether launches withhold their
// releases (both from the test hook spq_test_backsub_wait; elim.cu).
unsigned long long wait_bound_ns();
int wait_withhold();

}  // namespace spq
