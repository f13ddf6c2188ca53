// Types and launch phases shared by the compacted streaming kernels (stream.cu:
// kernels 5 and 6; ring.cu: kernels 7 and 8). Internal to the library.
//
// The compacted format renumbers the rows and columns that have entries in
// increasing order; p, u, f and the normalisers are held in that order for a
// launch. These kernels share the launch prologue (p and f gathered into
// compacted order, the norms of p), the stop test after each forward pass
// and the write-back of f.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "device_common.cuh"
#include "system.h"

namespace splitsart {

constexpr uint32_t kSignBit = 0x80000000u;
constexpr uint32_t kIndexMask = 0x7fffffffu;


// Storage traits of the streamed matrix: how one entry gives its compacted
// index and the pair (a1, a2).
template <class T, bool kImplicit>
struct Stor;
template <class T>
struct Stor<T, false> {  // explicit fold: index, (a1, a2)
    using Val = typename T::Pair;
    __device__ static __forceinline__ int col(int32_t idx) { return idx; }
    __device__ static __forceinline__ void get(int32_t idx, Val v, int& j, typename T::Acc& a1,
                                               typename T::Acc& a2) {
        j = idx;
        T::decode(v, a1, a2);
    }
};
template <class T>
struct Stor<T, true> {  // implicit fold: index with A1's sign in bit 31, w
    using Val = decltype(typename T::Vec2{}.x);
    __device__ static __forceinline__ int col(int32_t idx) { return (int)((uint32_t)idx & kIndexMask); }
    __device__ static __forceinline__ void get(int32_t idx, Val v, int& j, typename T::Acc& a1,
                                               typename T::Acc& a2) {
        j = (int)((uint32_t)idx & kIndexMask);
        a2 = v;
        a1 = idx < 0 ? -v : v;
    }
};

template <class T, bool kImplicit>
struct StArgs {
    using Val = typename Stor<T, kImplicit>::Val;
    using V2 = typename T::Vec2;
    using N2 = typename T::KNorm2;
    const int32_t* __restrict__ rp;
    const int32_t* __restrict__ ci;
    const Val* __restrict__ cv;
    const int32_t* __restrict__ cp;
    const int32_t* __restrict__ ri;
    const Val* __restrict__ rv;
    const N2* __restrict__ ir;
    const N2* __restrict__ ic;
    const float2* __restrict__ sc;  // BF16/FP16: compacted row scales
    V2* pc;
    V2* uc;
    V2* fc;
    double* rr;
    const int32_t* __restrict__ qs;
    const int32_t* __restrict__ cs;
    double* pz;
    const V2* __restrict__ p12;
    V2* f12;
    const int32_t* __restrict__ nzr;
    const int32_t* __restrict__ nzc;
    const int32_t* __restrict__ zr;
    const FoldStats* stats;
    double* partials;
    LaunchCtl* ctl;
    SolveResultDev* result;
    int Mh;
    int ns;
    const long long* sl_rows;
    SliceSolve* sl_solve;
    int* ndone;
    int max_iters, check_every;
    double lambda, tol, tol2_hi;
    unsigned long long timeout_ns;
    unsigned expected;
};

// Index and value loads with the streaming hint (each is read once per pass).
__device__ __forceinline__ int32_t st_ld(const int32_t* p) { return __ldcs(p); }
__device__ __forceinline__ float st_ld(const float* p) { return __ldcs(p); }
__device__ __forceinline__ double st_ld(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float2 st_ld(const float2* p) { return __ldcs(p); }
__device__ __forceinline__ double2 st_ld(const double2* p) { return __ldcs(p); }
__device__ __forceinline__ __nv_bfloat162 st_ld(const __nv_bfloat162* p) {
    const unsigned v = __ldcs(reinterpret_cast<const unsigned*>(p));
    return *reinterpret_cast<const __nv_bfloat162*>(&v);
}
__device__ __forceinline__ __half2 st_ld(const __half2* p) {
    const unsigned v = __ldcs(reinterpret_cast<const unsigned*>(p));
    return *reinterpret_cast<const __half2*>(&v);
}

// The entries one lane holds for a step: U of each of R rows (or columns).
template <class Val, int R, int U>
struct StepBuf {
    int32_t ia[R][U];
    Val va[R][U];
};


// ---------------------------------------------------------------------------
// Launch phases. Every thread of the CTA calls each of them.
// ---------------------------------------------------------------------------

// Prologue: p and f into compacted order and the norms of p. Batch: each
// slice's ||p||^2 into sl_solve[s].pp and its empty rows' share into pz[s]
// (one warp per slice). Single system: this CTA's share of ||p||^2 into
// partials[2b + 1]; the return value (thread 0) is its share of the empty
// rows' ||p||^2, which the forward pass adds to its residual.
template <class T, bool kImplicit, bool kBatch>
__device__ __forceinline__ double st_prologue(const StArgs<T, kImplicit>& a, double* s_red) {
    using V2 = typename T::Vec2;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5, nwarps = blockDim.x >> 5, BD = blockDim.x;
    const int gw = blockIdx.x * nwarps + wib, nw_grid = gridDim.x * nwarps;
    const int n_nzr = a.stats->n_nzr, n_nzc = a.stats->n_nzc, n_zr = a.stats->n_zr;
    for (int q = blockIdx.x * BD + tid; q < n_nzr; q += gridDim.x * BD) stcg(a.pc + q, ldg(a.p12 + __ldg(a.nzr + q)));
    for (int q = blockIdx.x * BD + tid; q < n_nzc; q += gridDim.x * BD) stcg(a.fc + q, ldcg(a.f12 + __ldg(a.nzc + q)));
    double ppz = 0.0;
    if constexpr (kBatch) {
        for (int sl = gw; sl < a.ns; sl += nw_grid) {
            const long long r0 = __ldg(a.sl_rows + sl), r1 = __ldg(a.sl_rows + sl + 1);
            double t = 0.0;
            for (long long i = r0 + lane; i < r1; i += 32) {
                const V2 p = ldg(a.p12 + i);
                t += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
            }
            // The slice's empty rows: a range of the increasing list zr.
            int lo = 0, hi = n_zr;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((long long)__ldg(a.zr + mid) < r0) lo = mid + 1;
                else hi = mid;
            }
            double z = 0.0;
            for (int k = lo + lane; k < n_zr && (long long)__ldg(a.zr + k) < r1; k += 32) {
                const V2 p = ldg(a.p12 + __ldg(a.zr + k));
                z += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
            }
            t = warp_sum(t);
            z = warp_sum(z);
            if (lane == 0) {
                a.sl_solve[sl] = SliceSolve{-1, 0, 0.0, 0.0, t};
                a.pz[sl] = z;
            }
        }
    } else {
        const long long G = gridDim.x, b = blockIdx.x;
        const int z0 = (int)(n_zr * b / G), z1 = (int)(n_zr * (b + 1) / G);
        const long long m0 = (long long)a.Mh * b / G, m1 = (long long)a.Mh * (b + 1) / G;
        double tz = 0.0, ta = 0.0;
        for (int z = z0 + tid; z < z1; z += BD) {
            const V2 p = ldg(a.p12 + __ldg(a.zr + z));
            tz += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
        }
        for (long long i = m0 + tid; i < m1; i += BD) {
            const V2 p = ldg(a.p12 + i);
            ta += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
        }
        tz = warp_sum(tz);
        ta = warp_sum(ta);
        if (lane == 0) s_red[wib] = tz;
        __syncthreads();
        if (tid == 0)
            for (int w = 0; w < nwarps; ++w) ppz += s_red[w];
        __syncthreads();
        if (lane == 0) s_red[wib] = ta;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < nwarps; ++w) t += s_red[w];
            __stcg(a.partials + 2 * blockIdx.x + 1, t);
        }
    }
    return ppz;
}

// Single system, after a forward pass: this CTA's ||r||^2 (its warps' sums
// `warp_rr` plus the empty rows' ppz) into partials[2b].
__device__ __forceinline__ void st_rr_partial(double warp_rr, double ppz, double* partials, double* s_red) {
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5, nwarps = blockDim.x >> 5;
    const double t = warp_sum(warp_rr);
    if (lane == 0) s_red[wib] = t;
    __syncthreads();
    if (tid == 0) {
        double tot = ppz;  // an empty row's residual is its p
        for (int w = 0; w < nwarps; ++w) tot += s_red[w];
        __stcg(partials + 2 * blockIdx.x, tot);
    }
}

// f back from compacted order (every CTA its share).
template <class T, bool kImplicit>
__device__ __forceinline__ void st_write_back(const StArgs<T, kImplicit>& a) {
    const int n_nzc = a.stats->n_nzc;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_nzc; q += gridDim.x * blockDim.x)
        stcg(a.f12 + __ldg(a.nzc + q), ldcg(a.fc + q));
}

// The stop test after forward pass k (which a grid barrier has closed). Batch:
// one CTA per unfinished slice sums its rows' residuals in a fixed order and
// marks the slice done at rho <= tol, then a grid barrier; the launch stops
// when every slice is done. Single system: every CTA sums the partials in the
// same order and takes the same decision. Returns 1 when the launch is to stop
// (f written back), -1 when a barrier wait failed (return at once), 0 to go on
// with the back pass. s_tpp (single system) holds ||p||^2.
template <class T, bool kImplicit, bool kBatch>
__device__ __forceinline__ int st_stop_test(const StArgs<T, kImplicit>& a, int k, double* s_red, double s_tpp,
                                            int* s_stop, unsigned& nbar) {
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5, nwarps = blockDim.x >> 5, BD = blockDim.x;
    const bool last = k >= a.max_iters;
    if constexpr (kBatch) {
        if (last || (k % a.check_every == 0)) {
            for (int sl = blockIdx.x; sl < a.ns; sl += gridDim.x) {
                if (__ldcg(&a.sl_solve[sl].done)) continue;  // uniform over the CTA
                double t = 0.0;
                for (int q = __ldg(a.qs + sl) + tid; q < __ldg(a.qs + sl + 1); q += BD) t += __ldcg(a.rr + q);
                t = warp_sum(t);
                if (lane == 0) s_red[wib] = t;
                __syncthreads();
                if (tid == 0) {
                    double trr = __ldcg(a.pz + sl);
                    for (int w = 0; w < nwarps; ++w) trr += s_red[w];
                    const double tpp = __ldcg(&a.sl_solve[sl].pp);
                    const bool above = !last && tpp > 0.0 && trr > tpp * a.tol2_hi;
                    const double rho = (above || !(tpp > 0.0)) ? 0.0 : sqrt(trr / tpp);
                    if (!above && (last || rho <= a.tol)) {
                        a.sl_solve[sl] = SliceSolve{k, 1, rho, trr, tpp};
                        atomicAdd(a.ndone, 1);
                    }
                }
                __syncthreads();
            }
        }
        if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return -1;
        if (ld_volatile(a.ndone) >= a.ns) {
            if (blockIdx.x == 0 && tid == 0) {
                a.result->iters = k;
                a.result->status = SPLITSART_OK;
                a.result->rho = 0.0;
                a.result->rr = 0.0;
                a.result->pp = 0.0;
            }
            st_write_back(a);
            return 1;
        }
    } else if (last || (k % a.check_every == 0)) {
        if (wib == 0) {
            const double trr = grid_total(a.partials, gridDim.x, lane, 0);
            if (lane == 0) {
                const double tpp = s_tpp;
                int stop = 0;
                if (last || !(tpp > 0.0) || trr <= tpp * a.tol2_hi) {
                    const double rho = tpp > 0.0 ? sqrt(trr / tpp) : 0.0;
                    stop = (last || rho <= a.tol) ? 1 : 0;
                    if (stop && blockIdx.x == 0) {
                        a.result->iters = k;
                        a.result->status = SPLITSART_OK;
                        a.result->rho = rho;
                        a.result->rr = trr;
                        a.result->pp = tpp;
                    }
                }
                *s_stop = stop;
            }
        }
        __syncthreads();
        if (*s_stop) {
            st_write_back(a);
            return 1;
        }
    }
    return 0;
}

// Kernel arguments of a compacted launch on format F of system s (host).
template <class T, bool kImplicit>
inline StArgs<T, kImplicit> st_args(splitsart_system* s, const StreamFmt& F, const void* p12, void* f12,
                                    const splitsart_solve_opts& o, int grid) {
    using V2 = typename T::Vec2;
    using N2 = typename T::KNorm2;
    using Val = typename Stor<T, kImplicit>::Val;
    StArgs<T, kImplicit> a{};
    a.rp = F.rp;
    a.ci = F.ci;
    a.cv = (const Val*)F.cv;
    a.cp = F.cp;
    a.ri = F.ri;
    a.rv = (const Val*)F.rv;
    a.ir = (const N2*)F.ir;
    a.ic = (const N2*)F.ic;
    a.sc = F.sc;
    a.pc = (V2*)F.pc;
    a.uc = (V2*)F.uc;
    a.fc = (V2*)F.fc;
    a.rr = F.rr;
    a.qs = F.qs;
    a.cs = F.cs;
    a.pz = F.pz;
    a.p12 = (const V2*)p12;
    a.f12 = (V2*)f12;
    a.nzr = s->nzr;
    a.nzc = s->nzc;
    a.zr = s->zr;
    a.stats = s->stats;
    a.partials = s->partials;
    a.ctl = s->ctl;
    a.result = s->result;
    a.Mh = (int)s->Mh;
    a.ns = s->ns;
    a.sl_rows = s->sl_rows;
    a.sl_solve = s->sl_solve;
    a.ndone = s->ndone;
    a.max_iters = o.max_iters;
    a.check_every = effective_check_every(o);
    a.lambda = o.lambda;
    a.tol = o.tol;
    a.tol2_hi = o.tol * o.tol * (1.0 + 1e-12);
    const double tms = o.timeout_ms > 0 ? o.timeout_ms : 2000.0;
    a.timeout_ns = (unsigned long long)(tms * 1e6);
    a.expected = (unsigned)grid + (o.inject_barrier_fault ? 1u : 0u);
    return a;
}

// Reset the launch's control block, result and (batch) finished-slice count.
inline int st_reset(splitsart_system* s, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(s->ctl, 0, sizeof(LaunchCtl), st)) != cudaSuccess) return cuda_fail(e, "solve: memset");
    if ((e = cudaMemsetAsync(s->result, 0xff, sizeof(SolveResultDev), st)) != cudaSuccess)
        return cuda_fail(e, "solve: memset");
    if (s->ns > 1 && (e = cudaMemsetAsync(s->ndone, 0, sizeof(int), st)) != cudaSuccess)
        return cuda_fail(e, "solve: memset");
    return SPLITSART_OK;
}

}  // namespace splitsart
