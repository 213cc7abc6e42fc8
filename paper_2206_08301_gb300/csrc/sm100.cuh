// Inline-PTX helpers for sm_103a: mbarriers with bounded waits, bulk (TMA)
// copies, tensor memory (TMEM) allocation and loads, and tcgen05.mma with
// shared-memory matrix descriptors.  Written from the public PTX ISA
// description of these instructions.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

namespace deinsum {
namespace sm100 {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bit of the device status word that a bounded wait sets when it gives up.
constexpr int kStatusTimeout = 1;
// Default limit of a pipeline wait, and the limit of a drain (below), in nanoseconds.
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kDrainLimitNs = 2000000000ull;

// try_wait with an explicit suspend-time hint (ns): the thread is suspended at most about
// that long before the test returns false.
__device__ __forceinline__ bool mbar_try_wait_hint(uint32_t bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}


// Non-blocking test of a phase (never suspends the thread).
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Limits below this are a test regime (deinsum_set_wait_limit_ns): polls that never
// suspend, with the clock read after each one.  A suspending try_wait may sleep until the
// phase completes whatever its hint says, which would outlast a limit of a few ns.
constexpr uint64_t kShortWaitNs = 1000000ull;

// The polling part of mbar_wait, out of line: the waits sit in every pipeline loop, and
// inlined polling loops at each of them measurably slowed the kernels (instruction fetch).
static __device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity, volatile int *abort, int *status,
                                            uint64_t limit_ns) {
    const uint64_t t0 = globaltimer_ns();
    if (limit_ns < kShortWaitNs) {
        while (true) {
            if (mbar_test_wait(bar, parity)) return true;
            if (*abort) return false;
            if (globaltimer_ns() - t0 > limit_ns) break;
        }
    } else {
        while (true) {
            #pragma unroll 1
            for (int i = 0; i < 32; ++i)
                if (mbar_try_wait_hint(bar, parity, 10000000u)) return true;
            if (*abort) return false;
            if (globaltimer_ns() - t0 > limit_ns) break;
        }
    }
    atomicOr(status, kStatusTimeout);
    *abort = 1;
    return false;
}

// Wait for the phase of parity `parity` to complete, for at most `limit_ns`.
// On time-out (or when another role already gave up, *abort != 0) it records
// a failure in the device status word, raises *abort and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort, int *status,
                                          uint64_t limit_ns) {
    if (limit_ns >= kShortWaitNs && mbar_try_wait_hint(bar, parity, 10000000u)) return true;
    return mbar_wait_slow(bar, parity, abort, status, limit_ns);
}

// Wait for the phase of parity `parity` to complete whether or not another role gave up:
// used before a role exits, for the completion of bulk copies or MMAs that this thread
// issued itself (they finish on their own, so this returns promptly even after an abort;
// the limit only guards against a broken pipeline).  On time-out it sets the status word.
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity, int *status) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        #pragma unroll 1
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > kDrainLimitNs) {
            atomicOr(status, kStatusTimeout);
            return false;
        }
    }
}

// --------------------------------------------------------- bulk async copy
// 1-D bulk copy global -> shared (both 16-byte aligned, bytes % 16 == 0),
// completing `bytes` transactions on mbarrier `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Tiled TMA loads global -> shared through a tensor map (kernel-parameter
// address `tmap`); the innermost coordinate must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(tmap), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void *tmap, int c0, int c1, int c2, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const void *tmap, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(dst), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Order earlier generic-proxy writes of a tensor map in global memory before
// its use by the TMA (the descriptor may have been rewritten since a previous launch).
__device__ __forceinline__ void fence_tensormap_acquire(const void *tmap) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
}

// Asynchronous prefetch of `bytes` (multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ------------------------------------------------------------------ TMEM
__device__ __forceinline__ void tmem_alloc(uint32_t holder_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(holder_smem), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 lanes x 32 bit, 16 consecutive columns per thread (lane = TMEM lane of the warp's quadrant).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ------------------------------------------------------------ tcgen05.mma
// Shared-memory matrix descriptor, K-major operand in the 128-byte swizzle
// layout: 8-row x 128-byte atoms (rows 128 B apart, 16-byte chunk c of row r
// stored at chunk c ^ (r % 8)), atoms of 8 rows stacked 1024 B apart (SBO).
// The leading-byte offset is unused for this layout (encoded as 1).
__device__ __forceinline__ uint64_t desc_kmajor_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFF) >> 4);       // start address >> 4, bits 0-13
    d |= uint64_t(1) << 16;                      // leading byte offset (unused), bits 16-29
    d |= uint64_t(1024 >> 4) << 32;              // stride byte offset, bits 32-45
    d |= uint64_t(1) << 46;                      // descriptor version, bits 46-47
    d |= uint64_t(2) << 61;                      // layout: 128-byte swizzle, bits 61-63
    return d;
}

// Shared-memory matrix descriptor, MN-major operand in the 128-byte swizzle
// layout: atoms of 64 MN elements (128 B) x 8 k (k-rows 128 B apart, 16-byte
// chunk c of k-row r stored at chunk c ^ (r % 8)); the leading-byte offset is
// the stride between atoms along MN, the stride-byte offset the stride between
// groups of 8 k.
__device__ __forceinline__ uint64_t desc_mnmajor_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFF) >> 4);       // start address >> 4, bits 0-13
    d |= uint64_t((lbo >> 4) & 0x3FFF) << 16;    // leading byte offset, bits 16-29
    d |= uint64_t((sbo >> 4) & 0x3FFF) << 32;    // stride byte offset, bits 32-45
    d |= uint64_t(1) << 46;                      // descriptor version, bits 46-47
    d |= uint64_t(2) << 61;                      // layout: 128-byte swizzle, bits 61-63
    return d;
}

// Instruction-descriptor bit selecting an MN-major A operand (bit 15, "transpose A").
constexpr uint32_t kIdescAMnMajor = 1u << 15;

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 accumulator,
// both operands K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4)                       // D format: F32
         | (1u << 7)                       // A format: BF16
         | (1u << 10)                      // B format: BF16
         | (uint32_t(N >> 3) << 17)        // N / 8
         | (uint32_t(M >> 4) << 24);       // M / 16
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on `bar` when every tcgen05 operation this thread issued so far has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(bar) : "memory");
}

// ----------------------------------------------------------- conversions
// Split two floats into packed BF16 (x0 in the low half) hi parts and lo parts
// with hi = bf16_rn(x), lo = bf16_rn(x - hi).
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &hi, uint32_t &lo) {
    __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    hi = *reinterpret_cast<uint32_t *>(&h);
    const float h0 = __uint_as_float(hi << 16);
    const float h1 = __uint_as_float(hi & 0xFFFF0000u);
    __nv_bfloat162 l = __floats2bfloat162_rn(x0 - h0, x1 - h1);
    lo = *reinterpret_cast<uint32_t *>(&l);
}

__device__ __forceinline__ float4 ldg_stream4(const float *p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ float ldg_stream1(const float *p) {
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void sts64(uint32_t addr, uint32_t a, uint32_t b) {
    asm volatile("st.shared.v2.b32 [%0], {%1,%2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// Byte offset of element (m, k) of an MN-major 128B-swizzled bf16 operand tile of
// 128 rows x 64 k: atom (k / 8, m / 64) at byte (2 (k / 8) + m / 64) * 1024, so the
// MN atom stride is 1024 B and the stride between groups of 8 k is 2048 B.
__host__ __device__ __forceinline__ uint32_t sw128_mn_offset(uint32_t m, uint32_t k) {
    return ((k >> 3) * 2u + (m >> 6)) * 1024u + (k & 7u) * 128u + (((((m & 63u) >> 3) ^ (k & 7u)) & 7u) << 4) +
           (m & 7u) * 2u;
}
constexpr uint32_t kMnAtomStride = 1024;   // between the two 64-row halves
constexpr uint32_t kMnKGroupStride = 2048; // between groups of 8 k

// The same for an MN-major tile of 64 rows (one atom along MN) x any k: atom k / 8
// at byte (k / 8) * 1024 (stride 1024 B between groups of 8 k).
__host__ __device__ __forceinline__ uint32_t sw128_mn64_offset(uint32_t n, uint32_t k) {
    return (k >> 3) * 1024u + (k & 7u) * 128u + ((((n >> 3) ^ (k & 7u)) & 7u) << 4) + (n & 7u) * 2u;
}
// Instruction-descriptor bit selecting an MN-major B operand (bit 16, "transpose B").
constexpr uint32_t kIdescBMnMajor = 1u << 16;

// Byte offset of element (row, k) of a K-major 128B-swizzled bf16 operand tile
// (64 k per row): atoms of 8 rows x 128 B.
__host__ __device__ __forceinline__ uint32_t sw128_offset(uint32_t row, uint32_t k) {
    return (row >> 3) * 1024u + (row & 7u) * 128u + ((((k >> 3) ^ (row & 7u)) & 7u) << 4) + (k & 7u) * 2u;
}

}  // namespace sm100
}  // namespace deinsum
