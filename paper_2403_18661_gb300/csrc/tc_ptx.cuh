// Inline-PTX wrappers for the Blackwell (sm_103a) tensor-core path:
// mbarriers, async-proxy fences, TMEM allocation, tcgen05.mma (kind::f16,
// BF16 operands from shared memory, FP32 accumulators in TMEM), commit and
// TMEM loads, plus the shared-memory matrix descriptor and the instruction
// descriptor encodings.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity to complete.  Bounded: returns
// false if it has not completed after timeout_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > timeout_ns) return false;
    }
}

// non-blocking test of the phase (never suspends the thread)
__device__ __forceinline__ uint32_t mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok;
}

// try_wait that may suspend the thread for up to hint_ns while the phase is incomplete (it
// resumes when the phase completes), so that a waiting warp does not compete for issue slots
__device__ __forceinline__ uint32_t mbar_try_wait_suspend(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok;
}

// A warp waits for the phase: lane 0 polls, suspending for at most hint_ns between polls (0: a
// spin on the non-blocking test, for latency-critical waits), the other lanes wait at the warp
// barrier; the result (false: gave up after timeout_ns) is the same in every lane and the warp is
// converged afterwards.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity, uint64_t timeout_ns,
                                               uint32_t hint_ns = 200u) {
    uint32_t ok = 1;
    if ((threadIdx.x & 31) == 0) {
        auto poll = [&]() { return hint_ns ? mbar_try_wait_suspend(bar, parity, hint_ns) : mbar_test_wait(bar, parity); };
        if (!poll()) {
            const uint64_t t0 = globaltimer_ns();
            while (!(ok = poll()))
                if (globaltimer_ns() - t0 > timeout_ns) break;
        }
    }
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// mbar_wait_warp for waits that have usually completed already: lane 0 first tests the phase without
// blocking (a blocking try_wait costs its latency even on a completed phase), then polls with
// try_wait, suspending up to 200 ns per poll, and reads the clock for timeout_ns every 16 polls.
__device__ __forceinline__ bool mbar_wait_warp_tested(uint64_t *bar, uint32_t parity, uint64_t timeout_ns) {
    uint32_t ok = 1;
    if ((threadIdx.x & 31) == 0 && !mbar_test_wait(bar, parity) && !mbar_try_wait_suspend(bar, parity, 200u)) {
        const uint64_t t0 = globaltimer_ns();
        for (uint32_t i = 1;; ++i) {
            if ((ok = mbar_try_wait_suspend(bar, parity, 200u))) break;
            if ((i & 15) == 0 && globaltimer_ns() - t0 > timeout_ns) break;
        }
    }
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// A warp polls the non-blocking test until the phase completes (latency-critical waits): lane 0
// polls, sleeping about sleep_ns between polls (0: a pure spin) so that the waiting warp takes few
// issue slots, and reads the clock for the timeout only every 64 polls; same result in every lane.
__device__ __forceinline__ bool mbar_spin_warp(uint64_t *bar, uint32_t parity, uint64_t timeout_ns,
                                               uint32_t sleep_ns = 0) {
    uint32_t ok = 1;
    if ((threadIdx.x & 31) == 0 && !mbar_test_wait(bar, parity)) {
        const uint64_t t0 = globaltimer_ns();
        for (uint32_t i = 1;; ++i) {
            if (sleep_ns) __nanosleep(sleep_ns);
            if ((ok = mbar_test_wait(bar, parity))) break;
            if ((i & 63) == 0 && globaltimer_ns() - t0 > timeout_ns) break;
        }
    }
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// ---------------------------------------------------------------- bulk copies
// contiguous global -> shared copy of `bytes` (multiple of 16, both 16-byte aligned)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// ---------------------------------------------------------------- fences
// generic-proxy shared-memory writes -> visible to the async proxy (tensor core, TMA)
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---------------------------------------------------------------- TMEM (warp-wide)
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---------------------------------------------------------------- MMA (one thread)
// D[tmem] (+)= A[smem desc] x B[smem desc]^T, BF16 x BF16 -> FP32, cta_group::1
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The same MMA issued by a whole warp executing uniformly: one elected lane issues it, so
// the operands stay warp-uniform (no per-lane divergence around the issue).
__device__ __forceinline__ void mma_bf16_elect(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred P, Q;\n\t"
        "elect.sync _|P, 0xffffffff;\n\t"
        "setp.ne.b32 Q, %4, 0;\n\t"
        "@P tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, Q;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// mma_bf16_elect issued only if `live` (a warp-uniform value): the skip is a predicate, not a
// branch, so the surrounding loop stays uniform
__device__ __forceinline__ void mma_bf16_elect_if(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                                  uint32_t accumulate, uint32_t live) {
    asm volatile(
        "{\n\t.reg .pred P, Q, R;\n\t"
        "elect.sync _|P, 0xffffffff;\n\t"
        "setp.ne.b32 Q, %4, 0;\n\t"
        "setp.ne.and.b32 R, %5, 0, P;\n\t"
        "@R tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, Q;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate), "r"(live)
        : "memory");
}

__device__ __forceinline__ void mma_commit_elect_if(uint64_t *bar, uint32_t live) {
    asm volatile(
        "{\n\t.reg .pred P, R;\n\telect.sync _|P, 0xffffffff;\n\t"
        "setp.ne.and.b32 R, %1, 0, P;\n\t"
        "@R tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(
            smem_addr(bar)), "r"(live)
        : "memory");
}

// commit from the elected lane of a uniform warp (the lane that issued with mma_bf16_elect)
__device__ __forceinline__ void mma_commit_elect(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .pred P;\n\telect.sync _|P, 0xffffffff;\n\t"
        "@P tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(
            smem_addr(bar))
        : "memory");
}

// arrive once on `bar` when every MMA this thread issued before has completed
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// ---------------------------------------------------------------- TMEM -> registers
// 32 lanes x 32 bit, 16 consecutive columns per thread (thread i of the warp
// reads lane (taddr.lane + i)); warp w may address lanes 32*(w%4) .. +31.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// the same load without the wait (issue several, then tmem_wait_ld once)
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Mark 16 registers filled by earlier *_nowait loads as (re)defined here, so that the compiler
// cannot move their uses above the wait that precedes this call.
__device__ __forceinline__ void tmem_regs_ready(uint32_t (&r)[16]) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
}

// 16 lanes x 8 columns per repetition (the MMA accumulator fragment): thread t receives
// (lane t/4, columns 2(t%4) and 2(t%4)+1) and (lane 8 + t/4, the same columns) of each
// 8-column group, group g in r[4g .. 4g + 3]
__device__ __forceinline__ void tmem_ld16x256b_x2_nowait(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.16x256b.x2.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16x256b_x4_nowait(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x4.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// 8 x 8 b16 matrix transposes through shared memory (threads 0..15 give the row addresses
// of matrices 0 and 1: matrix t / 8, row t % 8)
__device__ __forceinline__ void stmatrix_x2_trans(uint32_t saddr, uint32_t r0, uint32_t r1) {
    asm volatile("stmatrix.sync.aligned.m8n8.x2.trans.shared.b16 [%0], {%1, %2};" ::"r"(saddr), "r"(r0), "r"(r1)
                 : "memory");
}
__device__ __forceinline__ void ldmatrix_x2_trans(uint32_t saddr, uint32_t &r0, uint32_t &r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(saddr)
                 : "memory");
}

// two FP32 values to BF16x2 (lo in the low half), round to nearest even, optional ReLU
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ uint32_t pack_bf16x2_relu(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// relu(a * b + c) on BF16 pairs, rounded once to BF16
__device__ __forceinline__ uint32_t fma_relu_bf16x2(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("fma.rn.relu.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// named barrier `id` (1..15) over `count` threads (a multiple of 32)
__device__ __forceinline__ void named_bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// 32 consecutive columns per thread, waited
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- descriptors
// Shared-memory matrix descriptor, no swizzle ("interleaved" canonical
// layout of 8-row x 16-byte core matrices), K-major:
//   element (row i, k) at start + (i % 8) * 16 + (i / 8) * SBO + (k / 8) * LBO + (k % 8) * 2
// bits [0,14) start >> 4, [16,30) LBO >> 4, [32,46) SBO >> 4, [46,48) version 1,
// [49,52) base offset 0, bit 52 LBO mode 0, [61,64) layout 0 (no swizzle).
__device__ __forceinline__ uint64_t desc_kmajor_noswizzle(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5 = 1),
// A and B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

}  // namespace tc
