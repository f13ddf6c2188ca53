// Device-side building blocks shared by the library's kernels:
// - value traits for the four storages of the folded matrices;
// - cache-control loads and stores;
// - the bounded grid barrier.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/splitsart.h"

namespace splitsart {

// ---------------------------------------------------------------------------
// Value traits. The two split systems always travel together: matrix values
// and vectors are stored as interleaved pairs (x1, x2). One pass over the
// shared index pattern then serves A1 and A2 at once.
//
// Norm2 is the stored type of the normalisers 1/R and 1/C. KNorm2 is the
// type the iteration applies. For BF16/FP16 the FP64 normalisers are kept
// for export, and the kernels read FP32 copies: 1/R times the row scale,
// and 1/C, each an FP64 value rounded once to FP32. Then u and f cost no
// FP64 arithmetic (FP64 runs at a small fraction of the FP32 rate on this
// GPU).
// ---------------------------------------------------------------------------
struct TF64 {
    using Pair = double2;  // (a1, a2)
    using Acc = double;
    using Vec2 = double2;  // (x1, x2) vectors: f, p, u
    using Norm2 = double2; // 1/R, 1/C
    using KNorm2 = double2;
    static constexpr bool kQuant = false;
    static constexpr int kDtype = SPLITSART_F64;
    __device__ static inline void decode(Pair v, Acc& a1, Acc& a2) { a1 = v.x; a2 = v.y; }
};
struct TF32 {
    using Pair = float2;
    using Acc = float;
    using Vec2 = float2;
    using Norm2 = float2;
    using KNorm2 = float2;
    static constexpr bool kQuant = false;
    static constexpr int kDtype = SPLITSART_F32;
    __device__ static inline void decode(Pair v, Acc& a1, Acc& a2) { a1 = v.x; a2 = v.y; }
};
struct TBF16 {
    using Pair = __nv_bfloat162;
    using Acc = float;
    using Vec2 = float2;
    using Norm2 = double2;
    using KNorm2 = float2;
    static constexpr bool kQuant = true;
    static constexpr int kDtype = SPLITSART_BF16;
    __device__ static inline void decode(Pair v, Acc& a1, Acc& a2) {
        float2 f = __bfloat1622float2(v);
        a1 = f.x;
        a2 = f.y;
    }
    __device__ static inline Pair encode(float q1, float q2) {
        return __halves2bfloat162(__float2bfloat16_rn(q1), __float2bfloat16_rn(q2));
    }
};
struct TF16 {
    using Pair = __half2;
    using Acc = float;
    using Vec2 = float2;
    using Norm2 = double2;
    using KNorm2 = float2;
    static constexpr bool kQuant = true;
    static constexpr int kDtype = SPLITSART_F16;
    __device__ static inline void decode(Pair v, Acc& a1, Acc& a2) {
        float2 f = __half22float2(v);
        a1 = f.x;
        a2 = f.y;
    }
    __device__ static inline Pair encode(float q1, float q2) {
        return __halves2half2(__float2half_rn(q1), __float2half_rn(q2));
    }
};

// Read-only (non-coherent path) loads, for data that no kernel writes
// during the launch.
template <class T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }
template <>
__device__ __forceinline__ __nv_bfloat162 ldg(const __nv_bfloat162* p) {
    unsigned v = __ldg(reinterpret_cast<const unsigned*>(p));
    return *reinterpret_cast<__nv_bfloat162*>(&v);
}
template <>
__device__ __forceinline__ __half2 ldg(const __half2* p) {
    unsigned v = __ldg(reinterpret_cast<const unsigned*>(p));
    return *reinterpret_cast<__half2*>(&v);
}

// Loads and stores of the vectors that CTAs of one persistent launch rewrite
// between grid barriers.
// - Stores go to L2 (st.global.cg).
// - Gathers may use L1 (ld.global.ca). Every such load follows the grid
//   barrier's acquire and a CTA barrier, so under the PTX memory model it
//   observes every write made before the barrier's release; no stale line
//   can be read.
// - ldcg reads L2 directly, for data read once.
__device__ __forceinline__ float2 ldca(const float2* p) { return __ldca(p); }
__device__ __forceinline__ double2 ldca(const double2* p) { return __ldca(p); }
__device__ __forceinline__ float2 ldcg(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldcg(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ void stcg(float2* p, float2 v) { __stcg(p, v); }
__device__ __forceinline__ void stcg(double2* p, double2 v) { __stcg(p, v); }

// One thread's share of ||r||^2. Squares are formed in the working precision
// and summed in groups of 16 before they join an FP64 total, so FP32 systems
// take one FP64 add per 16 rows. For FP64 systems every step is FP64.
template <class Acc>
struct SqAcc {
    double tot = 0.0;
    Acc part = 0;
    int n = 0;
    __device__ __forceinline__ void add(Acc x, Acc y) {
        part += x * x + y * y;
        if (++n == 16) {
            tot += (double)part;
            part = 0;
            n = 0;
        }
    }
    __device__ __forceinline__ double sum() const { return tot + (double)part; }
};

template <class T>
__device__ __forceinline__ T warp_sum(T v, unsigned width = 32) {
    for (unsigned o = width >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, width);
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Control block of one persistent launch. The host zeroes it before each launch.
struct LaunchCtl {
    unsigned long long bar_count;  // barrier arrivals; bit 63 set once an error is recorded
    int err;                       // 0, or a SPLITSART_ERR_* code
    int err_where;                 // barrier index at which a wait ran out
    unsigned work[2];              // work counters of dynamically scheduled passes (forward, back)
};
constexpr unsigned long long kBarError = 1ull << 63;

// Record a launch error (the first one recorded wins) and raise the error bit
// of the barrier count, so that every CTA leaves at its next grid barrier.
__device__ __forceinline__ void record_error(LaunchCtl* ctl, int code, int where) {
    if (atomicCAS(&ctl->err, 0, code) == 0) ctl->err_where = where;
    atomicOr(&ctl->bar_count, kBarError);
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).
// ctl->bar_count only ever grows during a launch:
// - thread 0 of each CTA adds 1 with a release reduction (a posted write that
//   needs no round trip; no separate fence);
// - it then waits until the count reaches `target`, which is
//   expected x (barrier index + 1).
// An error recorded by any CTA sets bit 63 of the same word, so one acquire
// load per poll sees both the arrivals and the error. The wait has a
// wall-clock limit (checked every 64 polls) and a spin cap. If either runs
// out, the wait records SPLITSART_ERR_TIMEOUT and stops waiting. `expected`
// is normally gridDim.x; a test passes gridDim.x + 1 to make the wait run out
// on purpose.
// Returns false, for every thread of the CTA, if this CTA saw an error
// recorded by any CTA while it waited. The caller must then return. (A CTA
// that passes a barrier just as another records an error learns of it at the
// next barrier, which the failed CTA never reaches.)
__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ bool grid_sync(LaunchCtl* ctl, unsigned long long target, unsigned long long timeout_ns,
                                          int where) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        // The release orders this CTA's earlier writes: the CTA barrier above puts
        // them before this thread's release, and release is cumulative.
        red_release_add(&ctl->bar_count, 1ull);
        const unsigned long long max_spins = timeout_ns / 32ull + (1ull << 20);
        unsigned long long t0 = 0, spins = 0;
        for (;;) {
            const unsigned long long count = ld_acquire_gpu(&ctl->bar_count);
            if (count & kBarError) {
                ok = 0;
                break;
            }
            if (count >= target) break;
            if (spins == 0) t0 = global_ns();
            if (++spins > max_spins || ((spins & 63) == 0 && global_ns() - t0 > timeout_ns)) {
                record_error(ctl, SPLITSART_ERR_TIMEOUT, where);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        // The acquire load, and the CTA barrier below, put the other CTAs' writes
        // before every later load of this CTA.
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (global -> shared) completed on an mbarrier.
// Both addresses must be 16-byte aligned and the size a multiple of 16.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
// One arrival (no transaction bytes), with release semantics at CTA scope.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
                 : "memory");
}
// Wait for the completion of the given phase parity, with a wall-clock limit
// and a spin cap. Returns false if either runs out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned long long timeout_ns) {
    const uint32_t addr = smem_addr(bar);
    const unsigned long long t0 = global_ns();
    const unsigned long long max_spins = timeout_ns / 16ull + (1ull << 20);
    for (unsigned long long spins = 0;; ++spins) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (spins > max_spins || global_ns() - t0 > timeout_ns) return false;
    }
}
// Order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// An L2 policy that marks the lines it touches for eviction first: for data
// that a pass reads once, so that it does not push out what the gathers reuse.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// bulk_g2s with an L2 cache policy.
__device__ __forceinline__ void bulk_g2s_l2(void* dst, const void* src, unsigned bytes, uint64_t* bar,
                                            uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// One warp: the sum of partials[2b + which] over b < nparts, in a fixed
// order. Every CTA obtains bitwise the same total.
__device__ __forceinline__ double grid_total(const double* partials, int nparts, int lane, int which) {
    double t = 0.0;
#pragma unroll 4
    for (int b = lane; b < nparts; b += 32) t += __ldcg(partials + 2 * b + which);
    return warp_sum(t);
}

// Warp 0: sum the per-CTA pairs partials[2b], partials[2b+1] (b < nparts) in
// a fixed order. Every CTA obtains bitwise the same totals.
__device__ __forceinline__ void grid_totals(const double* partials, int nparts, int lane, double& t0, double& t1) {
    t0 = 0.0;
    t1 = 0.0;
#pragma unroll 4
    for (int b = lane; b < nparts; b += 32) {
        t0 += __ldcg(partials + 2 * b);
        t1 += __ldcg(partials + 2 * b + 1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        t0 += __shfl_xor_sync(0xffffffffu, t0, o);
        t1 += __shfl_xor_sync(0xffffffffu, t1, o);
    }
}

}  // namespace splitsart
