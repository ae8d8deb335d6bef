// hd_device.cuh -- device helpers shared by the decoder kernels: code
// parameters, inline-PTX wrappers for mbarriers and 1-D bulk (TMA) copies, and
// the bounded wait that every spin on an mbarrier goes through.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hd {

// ---------------------------------------------------------------------------
// Code parameters of the full-length code n = 2^m - 1.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int log2_exact(int v) { return v <= 1 ? 0 : 1 + log2_exact(v >> 1); }

template <int N_>
struct Code {
    static constexpr int n = N_;
    static constexpr int m = log2_exact(N_ + 1);
    static constexpr int k = N_ - m;
    // Words of the "position domain" y: bit p of y is position p (bit 0 unused),
    // so a codeword of n = 2^m - 1 bits fills exactly 2^m bits.
    static constexpr int Wy = (N_ + 1) <= 32 ? 1 : (N_ + 1) / 32;
    static_assert((1 << m) - 1 == N_, "n must be 2^m - 1");
};

// Positions p in [1, n] with bit i of p set, as a bit mask over the position
// domain (bit p).  Index set I_i of Sec. III-A, restricted to one 32-bit word.
__host__ __device__ constexpr uint32_t qmask(int n, int i)
{
    uint32_t mk = 0;
    for (int p = 1; p <= n && p < 32; ++p)
        if ((p >> i) & 1) mk |= 1u << p;
    return mk;
}

// Data run j (j >= 1) covers positions 2^j + 1 .. 2^(j+1) - 1; in the compacted
// data word it starts at bit 2^j - j - 1.  This is the mask of its bits there.
__host__ __device__ constexpr uint32_t run_mask(int j)
{
    return (uint32_t)(((1ull << ((1 << j) - 1)) - 1ull) << ((1 << j) - j - 1));
}

// shl.b32 clamps shift amounts above 32 to 32, which yields 0: used for the
// branch-free flip of a bit that may live in another word.
__device__ __forceinline__ uint32_t shl_clamp(uint32_t v, uint32_t sh)
{
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(sh));
    return r;
}

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy wrappers (sm_90+ PTX, used on sm_103a).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Every wait on an mbarrier is bounded: after this many nanoseconds the wait
// gives up and the caller reports HD_ERR_TIMEOUT instead of spinning forever.
constexpr uint64_t kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0 && global_ns() - t0 > kWaitLimitNs) return false;
    }
}

// Global -> shared bulk copy completing on an mbarrier (both addresses and the
// size are multiples of 16 bytes; the callers guarantee it).
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Shared -> global bulk copy tracked by bulk groups.
__device__ __forceinline__ void bulk_s2g(void *dst_gmem, const void *src_smem, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(smem_addr(src_smem)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

template <int N>
__device__ __forceinline__ void bulk_wait_all()
{
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// Programmatic dependent launch (sm_90+).  A kernel launched with the
// programmatic-serialisation attribute may start before the kernel ahead of
// it in the stream has finished, once every CTA of that kernel has executed
// launch_dependents; wait blocks the executing thread until the kernels ahead
// have completed and their memory operations are visible.  Without such a
// dependency wait returns at once.
__device__ __forceinline__ void grid_dep_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace hd
