// Thin inline-PTX wrappers for the sm_100-family tensor-core path: tcgen05
// (TMEM allocation, MMA, commit, TMEM loads), mbarriers and bulk async
// copies.  Every wait is bounded by a %globaltimer deadline.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace opta {
namespace tc5 {

__device__ inline uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ inline uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- mbarrier ---------------------------------------------------------------
__device__ inline void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ inline void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ inline void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// One arrival (release: this thread's earlier writes are visible to a
// thread that observes the completed phase).
__device__ inline void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of `bar`; gives up after `budget_ns` and returns false.
__device__ inline bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t budget_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > budget_ns) return false;
    }
    return true;
}

// ---- bulk async copy global -> shared (completes on an mbarrier) -------------
__device__ inline void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Generic-proxy shared-memory writes become visible to the async proxy
// (tensor-core operand reads).
__device__ inline void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- TMEM -------------------------------------------------------------------
__device__ inline void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ inline void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ inline void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ inline void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// ---- descriptors ----------------------------------------------------------------
// Shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// core matrices of 8 rows x 16 bytes (rows 16 B apart); `lbo` = byte distance
// between core matrices along K, `sbo` = along M/N.  Version field 1.
__device__ inline uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: F16 x F16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// D(tmem) (+)= A(smem) * B(smem)^T, issued by one thread (kind::f16: the
// operands' type, bf16 or fp16 for both, is in the instruction descriptor).
__device__ inline void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                bool accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// Arrive on `bar` once every MMA issued so far by this thread has completed.
__device__ inline void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// 32 lanes x 8 columns of zeros into TMEM: thread i of the warp clears
// columns [col, col+8) of TMEM lane (warp's lane base + i).  Completion is
// awaited by tmem_wait_st.
__device__ inline void tmem_st8_zero(uint32_t taddr) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
        "r"(0u)
        : "memory");
}
__device__ inline void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// ---- tensor-map (TMA) copies --------------------------------------------------
// 2-D tile of the tensor map `tmap` (a __grid_constant__ kernel parameter)
// at element coordinates (x, y) into shared memory, completing on `bar`.
// x times the element size must be a multiple of 16 bytes.
__device__ inline void tma_load_2d(void *dst_smem, const void *tmap, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst_smem)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// ---- operand conversion ----------------------------------------------------------
// bf16 pair (low half first) of bytes k and k + 1 of w, each minus 128:
// a byte b placed under the exponent of 2^23 (bit pattern 0x4B0000bb) is the
// float 2^23 + b, so subtracting 2^23 + 128 gives b - 128 exactly, and a
// float integer of at most 8 significant bits is exact in its top 16 bits.
template <int K>
__device__ __forceinline__ uint32_t bytes_bf16x2(uint32_t w) {
    const float f0 = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7650 + K)) - 8388736.f;
    const float f1 = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7650 + K + 1)) - 8388736.f;
    return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

// Bytes K and K + 1 of w as the fp16 pair (b - 128) (low half = byte K):
// 0x64bb is the fp16 value 1024 + b (exponent of 2^10, b in the mantissa),
// and 1024 + b - 1152 = b - 128 is exact.
template <int K>
__device__ __forceinline__ uint32_t bytes_f16x2(uint32_t w) {
    const uint32_t h = __byte_perm(w, 0x6464u, 0x5040u + (uint32_t)K + ((uint32_t)(K + 1) << 8));
    const __half2 v = __hsub2(*reinterpret_cast<const __half2 *>(&h), __half2half2(__ushort_as_half(0x6480u)));
    return *reinterpret_cast<const uint32_t *>(&v);
}

// 32 lanes x 8 columns of 32-bit TMEM data: thread i of the warp gets
// columns [col, col+8) of TMEM lane (warp's lane base + i).
__device__ inline void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    // load and wait in one statement so no use of r[] can be scheduled before the wait
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

}  // namespace tc5
}  // namespace opta
