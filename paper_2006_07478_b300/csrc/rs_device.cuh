// rs_device.cuh -- device helpers shared by the kernels of rs_kernel.cu (signal
// strategy, planner) and rs_tag.cu (tag strategy): hashing, PTX wrappers for
// mbarriers, bulk copies and streaming loads, warp scans, and the per-processor view
// of dynamic shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rs_internal.h"

#define FULLMASK 0xFFFFFFFFu

// ---------------------------------------------------------------------------
// small device helpers

__device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    // MurmurHash3 32-bit finalizer
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity)
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

// 1-D bulk copy global -> shared, completion counted on an mbarrier (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// streaming loads (read once: no L1 allocation) of 4 / 2 consecutive words
__device__ __forceinline__ uint4 ld_stream_v4(const uint32_t *p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// read-only 8-byte load that allocates in L1 (the words are read again soon)
__device__ __forceinline__ uint2 ld_nc_v2(const uint32_t *p)
{
    uint2 v;
    asm volatile("ld.global.nc.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

// 4-byte asynchronous copy global -> shared (no register staging)
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// arrive on an mbarrier once all of this thread's earlier cp.async copies have landed
__device__ __forceinline__ void cp_async_arrive(unsigned long long *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test_wait(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// relaxed gpu-scope 64-bit store and load: single-copy atomic and coherent across SMs,
// with no ordering of the thread's other memory operations (no fence), for words that
// carry their whole message themselves
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Reductions into global memory that return nothing (red.global: the L2 applies them and
// sends no value back, where an atomic that returns the old value would)
__device__ __forceinline__ void red_add_u32(uint32_t *p, uint32_t v)
{
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_min_u32(uint32_t *p, uint32_t v)
{
    asm volatile("red.relaxed.gpu.global.min.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULLMASK, v, d);
    return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v, uint32_t lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(FULLMASK, v, d);
        if (lane >= (uint32_t)d) v += y;
    }
    return v;
}

// sum of 32-bit values over the warp as a 64-bit total (inactive lanes pass 0)
__device__ __forceinline__ unsigned long long warp_sum_u32_wide(uint32_t v)
{
    uint32_t lo = __reduce_add_sync(FULLMASK, v & 0xFFFFu);
    uint32_t hi = __reduce_add_sync(FULLMASK, v >> 16);
    return ((unsigned long long)hi << 16) + lo;
}

// ---------------------------------------------------------------------------
// Compile-time pipeline signature: the enumerate op and the element-stage ops
// (0 = no such stage; the aggregate follows the last one).  OE == 0 marks the generic
// kernel, which reads every op from the parameters at run time.  A specialised
// kernel carries only the code its own nodes execute, which keeps its hot loop small
// enough for the instruction cache.
template <int OE_, int O1_, int O2_, int O3_, int O4_, int SK_ = D_AGG>
struct Sig {
    static constexpr bool generic = OE_ == 0;
    // the sink: an aggregate, or an emit sink (Section 4's results stripped of context)
    static constexpr bool emit = !generic && SK_ == D_EMIT;
    static constexpr int n = generic ? 0 : 2 + (O1_ != 0) + (O2_ != 0) + (O3_ != 0) + (O4_ != 0);
    template <int I>
    __host__ __device__ static constexpr int op()
    {
        return I == 0 ? OE_ : (I == n - 1 ? SK_ : (I == 1 ? O1_ : I == 2 ? O2_ : I == 3 ? O3_ : O4_));
    }
    template <int I>
    __host__ __device__ static constexpr bool present() { return generic ? (I < RS_MAX_STAGES) : (I < n); }
    template <int I>
    __host__ __device__ static constexpr bool maybe_last() { return generic ? true : (I == n - 1); }
    template <int I>
    __host__ __device__ static constexpr bool maybe_elem() { return generic ? (I + 1 < RS_MAX_STAGES) : (I < n - 1); }
};
using GenericSig = Sig<0, 0, 0, 0, 0>;

// ---------------------------------------------------------------------------
// Shared memory: one dynamic array; every per-processor array is addressed by a
// 32-bit element index into it, so all accesses are shared-memory loads and stores
// with 32-bit address arithmetic.

extern __shared__ __align__(128) unsigned char smem_raw[];

template <typename T>
struct SArr {
    uint32_t base;   // index of element 0, in units of T, from the start of smem_raw
    __device__ __forceinline__ T &operator[](uint32_t i) const { return reinterpret_cast<T *>(smem_raw)[base + i]; }
    __device__ __forceinline__ T *ptr() const { return reinterpret_cast<T *>(smem_raw) + base; }
};

template <typename T>
__device__ __forceinline__ SArr<T> sarr(uint32_t byte_off)
{
    SArr<T> a;
    a.base = byte_off / (uint32_t)sizeof(T);
    return a;
}
