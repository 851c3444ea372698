// Dependency waits between CTAs of one launch (tree-scheduled sweeps).  A flag
// is published with a release store after the producer's data, read with an
// acquire load, and every wait is bounded: after DC_SPIN_LIMIT polls it sets the
// launch's sticky fault word and gives up, so that no kernel can hang the GPU.
#pragma once

constexpr int DC_SPIN_LIMIT = 1 << 20;

static __device__ __forceinline__ int dc_ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
static __device__ __forceinline__ void dc_st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
static __device__ __forceinline__ bool dc_fault_set(const unsigned long long* fault) {
    return *reinterpret_cast<const volatile unsigned long long*>(fault) != 0ull;
}
// Waits until *flag is nonzero; false when the fault word is (or gets) set.
static __device__ bool dc_wait_flag(const int* flag, unsigned long long* fault) {
    for (int i = 0; i < DC_SPIN_LIMIT; ++i) {
        if (dc_ld_acquire(flag)) {
            __threadfence();
            return true;
        }
        if ((i & 31) == 31 && dc_fault_set(fault)) return false;
        __nanosleep(i < 64 ? 32 : 256);
    }
    atomicExch(fault, 1ull);
    return false;
}
