// Fifth-generation tensor-core helpers (sm_103a): tcgen05 MMA with operands in
// shared memory and the accumulator in tensor memory (TMEM), used for the dense
// rank-32 trailing updates of the preconditioner's multifrontal factorisation.
//
// Operands are K-major without swizzle: a matrix of R rows and 32 FP32/TF32
// columns is stored as "core matrices" of 8 rows x 16 bytes (4 elements), each
// core 128 contiguous bytes (row i of the core at byte 16 i).  The 8 cores along
// K of one 8-row group are consecutive (leading-dimension byte offset 128) and
// the 8-row groups follow each other every 1024 bytes (stride byte offset).
// Element (r, k) is thus at byte (r / 8) 1024 + (k / 4) 128 + (r % 8) 16 + (k % 4) 4.
//
// FP32 accuracy from TF32 inputs: x = hi + lo with hi = tf32(x), lo = tf32(x - hi);
// A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi, accumulated in FP32 (the dropped
// A_lo B_lo term is 2^-22 relative), i.e. three MMA passes.
#pragma once
#include <cstdint>

constexpr uint32_t TC_CORE_K_BYTES = 128;    // next core along K
constexpr uint32_t TC_GROUP_BYTES = 1024;    // next 8-row group (K = 32)
constexpr int TC_K = 32;                     // K of one trailing update (the panel width)

static __device__ __forceinline__ uint32_t tc_smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (r, k) of a K = 32 operand in the layout above.
static __device__ __forceinline__ uint32_t tc_off(int r, int k) {
    return (uint32_t)(r >> 3) * TC_GROUP_BYTES + (uint32_t)(k >> 2) * TC_CORE_K_BYTES + (uint32_t)(r & 7) * 16u +
           (uint32_t)(k & 3) * 4u;
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (row
// group) byte offsets, all >> 4; bits 46-47 = 1 (the tcgen05 descriptor
// version); base offset 0; no swizzle (bits 61-63 = 0).
static __device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((TC_CORE_K_BYTES >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((TC_GROUP_BYTES >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::tf32: D in F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
static __host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A B^T for one K = 8 slice (one thread issues).
static __device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                                   uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrives once on the mbarrier when every MMA issued so far by this thread is done.
static __device__ __forceinline__ void tc_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     tc_smem_u32(mbar))
                 : "memory");
}

static __device__ __forceinline__ void tc_mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem_u32(mbar)), "r"(count) : "memory");
}
static __device__ __forceinline__ void tc_mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Polls the phase `parity` of the mbarrier at most `limit` times; true once it completed.
static __device__ __forceinline__ bool tc_mbar_wait(uint64_t* mbar, uint32_t parity, int limit) {
    const uint32_t a = tc_smem_u32(mbar);
    for (int i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred q;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (i > 64) __nanosleep(64);
    }
    return false;
}

// Generic-proxy writes to shared memory -> visible to the tensor core (async proxy).
static __device__ __forceinline__ void tc_fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
static __device__ __forceinline__ void tc_fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
static __device__ __forceinline__ void tc_fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// TMEM columns: allocated by one whole warp; the base address goes to *slot.
static __device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
static __device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive accumulator columns of this thread's TMEM lane (warp w of a
// warpgroup reads lanes 32 (w % 4) .. + 31; taddr carries the lane in bits 16-31).
static __device__ __forceinline__ void tc_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// TF32 rounding (round to nearest, ties away) and the hi/lo split.
static __device__ __forceinline__ float tc_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
static __device__ __forceinline__ void tc_split(float x, float& hi, float& lo) {
    hi = tc_tf32(x);
    lo = tc_tf32(x - hi);
}
