// async.cuh -- thin inline-PTX wrappers for the asynchronous data movement of
// sm_90+ (mbarrier objects, bulk global->shared copies, remote stores into a
// cluster peer's shared memory).  Every wait is bounded (0.2 s of global time)
// and reports a timeout instead of spinning forever.
#pragma once
#include <stdint.h>

namespace miugks {

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// mbarrier with `count` expected arrivals per phase
__device__ __forceinline__ void mbar_init(uint64_t* mb, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(mb)), "r"(count) : "memory");
}

// make initialised mbarriers visible to the other CTAs of the cluster
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// arrive once and add `bytes` to the transaction count of the current phase
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* mb, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(mb)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* mb, unsigned parity)
{
    unsigned done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(smem_addr(mb)), "r"(parity)
                 : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
    return t;
}

constexpr uint64_t kWaitNs = 200000000ull;   // a wait gives up after 0.2 s ...
constexpr int kWaitRounds = 1 << 26;         // ... or this many try_wait rounds

// wait for the phase with the given parity to complete; false when the bound
// (limit_ns of global time, or kWaitRounds rounds) is reached.  limit 0 gives
// up without testing the phase at all: it drives the caller's timeout path on
// purpose (the inputs of a sweep step are normally complete at the first test,
// so a short bound alone would not reach that path).
__device__ __forceinline__ bool mbar_wait(uint64_t* mb, unsigned parity, uint64_t limit_ns = kWaitNs)
{
    if (limit_ns == 0) return false;
    if (mbar_try_wait(mb, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int it = 0; it < kWaitRounds; ++it) {
        if (mbar_try_wait(mb, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// order this thread's generic-proxy global writes before later async-proxy (bulk copy) reads
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;\n" ::: "memory"); }

// bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from global
// memory into this CTA's shared memory, completing on the local mbarrier mb
__device__ __forceinline__ void bulk_g2s(void* sdst, const void* gsrc, unsigned bytes, uint64_t* mb)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_addr(sdst)),
                 "l"(gsrc), "r"(bytes), "r"(smem_addr(mb))
                 : "memory");
}

// address of the same shared-memory location in cluster CTA `rank`
__device__ __forceinline__ unsigned peer_addr(const void* p, unsigned rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(smem_addr(p)), "r"(rank));
    return r;
}

// store into a peer CTA's shared memory; completes `sizeof(v)` bytes on the peer's mbarrier
__device__ __forceinline__ void st_async(unsigned raddr, float v, unsigned rmb)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];\n" ::"r"(raddr),
                 "r"(__float_as_uint(v)), "r"(rmb)
                 : "memory");
}
__device__ __forceinline__ void st_async(unsigned raddr, double v, unsigned rmb)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];\n" ::"r"(raddr),
                 "l"(__double_as_longlong(v)), "r"(rmb)
                 : "memory");
}

// asynchronous 16-byte global -> shared copy (LDGSTS, cached in L2 only; both
// addresses 16-byte aligned), completed per commit group of the issuing thread
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's most recent commit groups are pending
template <int N>
__device__ __forceinline__ void cp_async_wait_n()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace miugks
