// Bulk-copy ring for streaming kernels (sm_90 and later, used on sm_103a).
//
// One producer lane streams contiguous tiles of global memory into a ring of
// shared-memory slots with cp.async.bulk; each copy completes on the slot's
// "full" mbarrier (transaction count = the tile's bytes). Consumer warps wait
// on the full barrier, read the slot, and release it with one arrive per warp
// on the slot's "empty" barrier, which the producer waits on before it reuses
// the slot. The copy engine keeps many tiles in flight while the consumers
// compute, without a register per byte in flight.
//
// Every wait is bounded in time (globaltimer, through WaitClock). A wait that runs out sets the
// block's abort word; from then on no wait of the block blocks again, the
// kernel walks the rest of its control flow (every named barrier included)
// without data and reports NaN, and the producer waits, again bounded, for
// the copies it already issued before the block exits. A consumer that gives
// up still releases its slot, so the producer re-reads the abort word after
// every wait on a released slot and issues no copy into a slot whose last
// copy may still be landing (the abort store is ordered before the release).
#pragma once
#include <cstdint>

namespace helm {
namespace pipe {

constexpr unsigned long long kWaitNs = 500ull * 1000 * 1000;   // 0.5 s per wait

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

// make initialised barriers visible to the other threads and to the copy engine
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// non-blocking test of the same phase (try_wait may suspend the thread for a
// while before it reports an unfinished phase; test_wait returns at once)
__device__ __forceinline__ bool mbar_test_wait(uint64_t *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Time spent in one wait, from %globaltimer read at each check. Only forward
// steps below kStepCapNs count, so a reading behind the previous one (which a
// plain unsigned now - start would turn into an instant timeout) or a leap
// longer than a check interval can take adds nothing; the iteration caps of
// the waits bound them whatever the timer does.
constexpr unsigned long long kStepCapNs = 50ull * 1000 * 1000;   // 50 ms between two checks

struct WaitClock {
    unsigned long long prev, spent;
    __device__ __forceinline__ WaitClock() : prev(global_ns()), spent(0) {}
    // true once the counted time exceeds limit_ns
    __device__ __forceinline__ bool over(unsigned long long limit_ns) {
        const unsigned long long now = global_ns();
        const long long d = (long long)(now - prev);
        prev = now;
        if (d > 0 && (unsigned long long)d < kStepCapNs) spent += (unsigned long long)d;
        return spent > limit_ns;
    }
};

// Wait until the phase of parity `parity` of barrier b has completed. Returns
// false at once when *abort is set, and false (setting *abort) after limit_ns.
// A limit below 1 us gives up at the first check that finds the phase
// unfinished (a non-blocking test): the form tests use to make waits run out.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, unsigned parity, volatile int *abort,
                                          unsigned long long limit_ns = kWaitNs) {
    if (*abort) return false;
    if (limit_ns < 1000ull) {
        if (mbar_test_wait(b, parity)) return true;
        *abort = 1;
        return false;
    }
    if (mbar_try_wait(b, parity)) return true;
    WaitClock clk;
    for (unsigned n = 1;; ++n) {
        if (mbar_try_wait(b, parity)) return true;
        if ((n & 31) == 0) {
            if (*abort) return false;
            if (clk.over(limit_ns) || n > (1u << 30)) {
                *abort = 1;
                return false;
            }
        }
    }
}

// The same wait without the abort short-cut (teardown of copies in flight).
__device__ __forceinline__ bool mbar_wait_drain(uint64_t *b, unsigned parity) {
    WaitClock clk;
    for (unsigned n = 0;; ++n) {
        if (mbar_try_wait(b, parity)) return true;
        if ((n & 31) == 31 && (clk.over(kWaitNs) || n > (1u << 30))) return false;
    }
}

// global -> shared copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned), completing as transactions on barrier `bar`
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// named barrier over the first `n` threads of the block (n a multiple of 32)
__device__ __forceinline__ void named_sync(unsigned id, unsigned n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

}  // namespace pipe
}  // namespace helm
