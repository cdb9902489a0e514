// sl_async.cuh -- asynchronous copies into shared memory (inline PTX): per-element copies
// (cp.async), mbarriers with bounded waits, and bulk-tensor box copies (cp.async.bulk.tensor,
// no multicast); the host side encodes the tensor maps.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace {

// asynchronous global -> shared copies (LDGSTS); a CTA issues its whole window, then waits once
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem_dst, const void *gmem_src)
{
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(dst), "l"(gmem_src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// this thread's earlier cp.async copies arrive on the barrier when they complete (the pending count
// is raised first, so the phase still needs the barrier's own arrival)
__device__ __forceinline__ void mbar_track_cp_async(unsigned long long *bar)
{
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// as mbar_track_cp_async, without raising the pending count: the barrier's expected arrivals
// count this thread (one such arrival per thread and phase)
__device__ __forceinline__ void mbar_track_cp_async_noinc(unsigned long long *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// as mbar_test, but a thread whose phase is not complete is suspended (issuing nothing) until it
// completes or about `ns` nanoseconds pass
__device__ __forceinline__ bool mbar_test_suspend(unsigned long long *bar, unsigned parity, unsigned ns)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of the barrier, suspended between tests, giving up after 0.2 s (a copy
// that never lands).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_test_suspend(bar, parity, 20000u)) return true;
        if (global_ns() - t0 > 200000000ull) return false;
    }
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_addr(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}
// order this thread's generic-proxy accesses of shared memory before later async-proxy writes
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace

// Tensor map of a dense FP32 array of `rank` (2 or 3) dimensions, dims[0] innermost, strides[k]
// the byte distance between consecutive indices of dimension k + 1, copied in boxes of box[]
// elements (no interleave, no swizzle, out-of-range elements read as zero).  False when the
// driver's encoder is unavailable or rejects the layout (base not 16-byte aligned, a stride not a
// multiple of 16 bytes, a box's row not a multiple of 16 bytes).
bool encode_tensor_f32(CUtensorMap *m, const void *base, int rank, const unsigned long long *dims,
                       const unsigned long long *strides, const unsigned *box);
