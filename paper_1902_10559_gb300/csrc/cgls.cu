// CGLS on both split systems in one persistent cooperative launch.
//
// The normal matrix of each split system is the fold of the full one (text
// after Eq. 18): B_s = A_s^T A_s. CGLS solves A_s^T A_s f = A_s^T p_s by
// conjugate gradients without forming B_s, two sparse passes per iteration.
// For each system s, from x^0:
//     r^0 = p - A x^0,  s^0 = A^T r^0,  d^{-1} = 0,  beta^{-1} = 0,  gamma_0 = ||s^0||^2
//     d^k = s^k + beta^{k-1} d^{k-1},  q^k = A d^k,  alpha_k = gamma_k / ||q^k||^2
//     x^{k+1} = x^k + alpha_k d^k,  r^{k+1} = r^k - alpha_k q^k
//     s^{k+1} = A^T r^{k+1},  gamma_{k+1} = ||s^{k+1}||^2,  beta_k = gamma_{k+1} / gamma_k
// with 0/0 := 0. The two systems share every pass over the index pattern and
// have their own scalars; the stop test is the joint one of the SART solver,
// rho_k = sqrt(||r1^k||^2 + ||r2^k||^2) / ||p||, tested before step k.
//
// Passes of iteration k, with two grid barriers:
//   rows:    r_i -= alpha_{k-1} q_i (k >= 1); ||r^k||^2; q_i = (A d^k)_i where
//            d^k_j = s_j + beta_{k-1} d_j is formed at the gather; ||q^k||^2.
//   barrier: stop test on ||r^k||; alpha_k.
//   columns: d_j = s_j + beta_{k-1} d_j (stored); x_j += alpha_k d_j;
//            s_j = sum_i a_ij (r_i - alpha_k q_i) = (A^T r^{k+1})_j; ||s||^2.
//   barrier: beta_k, gamma_{k+1}.
// The expressions formed at a gather and by the owner of the row or column
// are the same fused multiply-adds, so both sides see the same values. Every
// reduction is FP64 across threads, warps and CTAs, in a fixed order, so all
// CTAs hold bitwise the same scalars and the launch is reproducible.
#include <cmath>
#include <cstdio>
#include <algorithm>

#include "device_common.cuh"
#include "system.h"

namespace splitsart {

namespace {

constexpr int kCgSlots = 6;  // per-CTA partials: rr, qq1, qq2, ss1, ss2, pp

template <class T>
struct CgArgs {
    const int32_t* __restrict__ nzr;
    const int32_t* __restrict__ nzrp;
    const int32_t* __restrict__ zr;
    const int32_t* __restrict__ nzc;
    const int32_t* __restrict__ nzcp;
    const int32_t* __restrict__ col;
    const typename T::Pair* __restrict__ val;
    const int32_t* __restrict__ row;
    const typename T::Pair* __restrict__ valT;
    const typename T::Vec2* __restrict__ p12;
    typename T::Vec2* x12;  // f: in x^0, out the returned iterate
    typename T::Vec2* r12;  // [Mh] residuals
    typename T::Vec2* q12;  // [Mh] A d
    typename T::Vec2* s12;  // [Nh] A^T r
    typename T::Vec2* d12;  // [Nh] search directions
    double* part;           // [kCgSlots][gridDim.x]
    LaunchCtl* ctl;
    SolveResultDev* result;
    const FoldStats* stats;
    int Mh, Nh;
    int max_iters, check_every;
    double tol, tol2_hi;
    unsigned long long timeout_ns;
    unsigned expected;
};

template <class S>
__device__ __forceinline__ S fma_(S a, S b, S c);
template <>
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

// Sum over the CTA of each thread's values v[0..N) that lane 0 of each warp
// holds; thread 0 writes them to part[slot[n]][blockIdx.x]. Fixed order.
template <int N>
__device__ __forceinline__ void cta_publish(const double (&v)[N], const int (&slot)[N], double* part,
                                            double (*red)[32]) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (lane == 0)
        for (int n = 0; n < N; ++n) red[n][wib] = v[n];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int n = 0; n < N; ++n) {
            double t = 0.0;
            for (int w = 0; w < nwarps; ++w) t += red[n][w];
            __stcg(part + (size_t)slot[n] * gridDim.x + blockIdx.x, t);
        }
    __syncthreads();
}

// Warp 0: the grid total of one slot, in a fixed order (the same in every CTA).
__device__ __forceinline__ double slot_total(const double* part, int slot, int lane) {
    double t = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(part + (size_t)slot * gridDim.x + b);
    return warp_sum(t);
}

template <class T, int LPC>
__global__ void __launch_bounds__(512, 1) cgls_kernel(CgArgs<T> a) {
    using Acc = typename T::Acc;
    using V2 = typename T::Vec2;
    constexpr int kGroups = 32 / LPC;
    __shared__ double s_red[3][32];
    __shared__ double s_sc[8];  // pp, alpha1, alpha2, beta1, beta2, gamma1, gamma2, stop
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5, nwarps = blockDim.x >> 5, BD = blockDim.x;
    const int sub = lane % LPC;
    const int gw = blockIdx.x * nwarps + wib, nw_grid = gridDim.x * nwarps;
    const int n_nzr = a.stats->n_nzr, n_nzc = a.stats->n_nzc, n_zr = a.stats->n_zr;
    unsigned nbar = 0;

    // Row q's sum of a_ij v_j, where v_j = op(j) is formed at the gather. Lane 0 holds it.
    auto row_dot = [&](int q, auto&& op, Acc& s1, Acc& s2) {
        const int lo = __ldg(a.nzrp + q), hi = __ldg(a.nzrp + q + 1);
        s1 = 0;
        s2 = 0;
        for (int e = lo + lane; e < hi; e += 32) {
            Acc v1, v2;
            T::decode(ldg(a.val + e), v1, v2);
            const V2 g = op(__ldg(a.col + e));
            s1 += v1 * g.x;
            s2 += v2 * g.y;
        }
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
    };
    // Column q's sum of a_ij w_i over its LPC lanes, w_i = op(i).
    auto col_dot = [&](int q, auto&& op, Acc& b1, Acc& b2) {
        const int lo = q < n_nzc ? __ldg(a.nzcp + q) : 0, hi = q < n_nzc ? __ldg(a.nzcp + q + 1) : 0;
        b1 = 0;
        b2 = 0;
        for (int e = lo + sub; e < hi; e += LPC) {
            Acc v1, v2;
            T::decode(ldg(a.valT + e), v1, v2);
            const V2 w = op(__ldg(a.row + e));
            b1 += v1 * w.x;
            b2 += v2 * w.y;
        }
        b1 = warp_sum(b1, LPC);
        b2 = warp_sum(b2, LPC);
    };

    // ---- prologue 1: r^0 = p - A x^0 (empty rows: r = p), ||r^0||^2 and ||p||^2 ----
    {
        double rr = 0.0, pp = 0.0;
        for (int q = gw; q < n_nzr; q += nw_grid) {
            Acc s1, s2;
            row_dot(q, [&](int j) { return ldcg(a.x12 + j); }, s1, s2);
            if (lane == 0) {
                const int i = __ldg(a.nzr + q);
                const V2 p = ldg(a.p12 + i);
                const V2 r = V2{p.x - s1, p.y - s2};
                stcg(a.r12 + i, r);
                stcg(a.q12 + i, V2{0, 0});
                rr += (double)r.x * (double)r.x + (double)r.y * (double)r.y;
                pp += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
            }
        }
        double rz = 0.0;
        for (int z = blockIdx.x * BD + tid; z < n_zr; z += gridDim.x * BD) {
            const int i = __ldg(a.zr + z);
            const V2 p = ldg(a.p12 + i);
            stcg(a.r12 + i, p);
            stcg(a.q12 + i, V2{0, 0});
            rz += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
        }
        rz = warp_sum(rz);  // every lane's share; lane 0 publishes the warp's total
        const double v[2] = {rr + rz, pp + rz};
        const int sl[2] = {0, 5};
        cta_publish(v, sl, a.part, s_red);
    }
    if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
    // ---- prologue 2: s^0 = A^T r^0, d^{-1} = 0, gamma_0 ----
    {
        double g1 = 0.0, g2 = 0.0;
        for (int g0 = gw * kGroups; g0 < n_nzc; g0 += nw_grid * kGroups) {
            const int q = g0 + lane / LPC;
            Acc b1, b2;
            col_dot(q, [&](int i) { return ldcg(a.r12 + i); }, b1, b2);
            if (sub == 0 && q < n_nzc) {
                const int j = __ldg(a.nzc + q);
                stcg(a.s12 + j, V2{b1, b2});
                stcg(a.d12 + j, V2{0, 0});
                g1 += (double)b1 * (double)b1;
                g2 += (double)b2 * (double)b2;
            }
        }
        g1 = warp_sum(g1);
        g2 = warp_sum(g2);
        const double v[2] = {g1, g2};
        const int sl[2] = {3, 4};
        cta_publish(v, sl, a.part, s_red);
    }
    if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
    if (wib == 0) {
        const double pp = slot_total(a.part, 5, lane);
        const double g1 = slot_total(a.part, 3, lane);
        const double g2 = slot_total(a.part, 4, lane);
        if (lane == 0) {
            s_sc[0] = pp;
            s_sc[1] = s_sc[2] = 0.0;  // alpha_{-1}
            s_sc[3] = s_sc[4] = 0.0;  // beta_{-1}
            s_sc[5] = g1;
            s_sc[6] = g2;
        }
    }
    __syncthreads();

    for (int k = 0;; ++k) {
        // ---- rows: r^k, ||r^k||^2, q^k = A d^k, ||q^k||^2 ----
        const Acc am1 = (Acc)s_sc[1], am2 = (Acc)s_sc[2];  // alpha_{k-1}
        const Acc bm1 = (Acc)s_sc[3], bm2 = (Acc)s_sc[4];  // beta_{k-1}
        {
            double rr = 0.0, q1 = 0.0, q2 = 0.0;
            for (int q = gw; q < n_nzr; q += nw_grid) {
                Acc s1, s2;
                row_dot(q, [&](int j) {
                    const V2 s = ldcg(a.s12 + j), d = ldcg(a.d12 + j);
                    return V2{fma_(bm1, d.x, s.x), fma_(bm2, d.y, s.y)};
                }, s1, s2);
                if (lane == 0) {
                    const int i = __ldg(a.nzr + q);
                    V2 r = ldcg(a.r12 + i);
                    if (k > 0) {
                        const V2 qo = ldcg(a.q12 + i);
                        r = V2{fma_(-am1, qo.x, r.x), fma_(-am2, qo.y, r.y)};
                        stcg(a.r12 + i, r);
                    }
                    stcg(a.q12 + i, V2{s1, s2});
                    rr += (double)r.x * (double)r.x + (double)r.y * (double)r.y;
                    q1 += (double)s1 * (double)s1;
                    q2 += (double)s2 * (double)s2;
                }
            }
            double rz = 0.0;  // empty rows: r = p and q = 0 throughout
            for (int z = blockIdx.x * BD + tid; z < n_zr; z += gridDim.x * BD) {
                const V2 p = ldg(a.p12 + __ldg(a.zr + z));
                rz += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
            }
            rz = warp_sum(rz);
            const double v[3] = {rr + rz, q1, q2};
            const int sl[3] = {0, 1, 2};
            cta_publish(v, sl, a.part, s_red);
        }
        if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
        // ---- stop test on ||r^k||, then alpha_k (one thread; every CTA alike) ----
        const bool last = k >= a.max_iters;
        if (wib == 0) {
            const double trr = slot_total(a.part, 0, lane);
            const double tq1 = slot_total(a.part, 1, lane);
            const double tq2 = slot_total(a.part, 2, lane);
            if (lane == 0) {
                int stop = 0;
                if (last || k % a.check_every == 0) {
                    const double tpp = s_sc[0];
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
                }
                s_sc[7] = stop;
                s_sc[1] = tq1 > 0.0 ? s_sc[5] / tq1 : 0.0;
                s_sc[2] = tq2 > 0.0 ? s_sc[6] / tq2 : 0.0;
            }
        }
        __syncthreads();
        if (s_sc[7] != 0.0) return;

        // ---- columns: d^k, x^{k+1}, s^{k+1} = A^T (r^k - alpha_k q^k), gamma_{k+1} ----
        const Acc al1 = (Acc)s_sc[1], al2 = (Acc)s_sc[2];
        {
            double g1 = 0.0, g2 = 0.0;
            for (int g0 = gw * kGroups; g0 < n_nzc; g0 += nw_grid * kGroups) {
                const int q = g0 + lane / LPC;
                Acc b1, b2;
                col_dot(q, [&](int i) {
                    const V2 r = ldcg(a.r12 + i), qv = ldcg(a.q12 + i);
                    return V2{fma_(-al1, qv.x, r.x), fma_(-al2, qv.y, r.y)};
                }, b1, b2);
                if (sub == 0 && q < n_nzc) {
                    const int j = __ldg(a.nzc + q);
                    const V2 s = ldcg(a.s12 + j), d0 = ldcg(a.d12 + j);
                    const V2 d = V2{fma_(bm1, d0.x, s.x), fma_(bm2, d0.y, s.y)};
                    V2 x = ldcg(a.x12 + j);
                    x = V2{fma_(al1, d.x, x.x), fma_(al2, d.y, x.y)};
                    stcg(a.d12 + j, d);
                    stcg(a.x12 + j, x);
                    stcg(a.s12 + j, V2{b1, b2});
                    g1 += (double)b1 * (double)b1;
                    g2 += (double)b2 * (double)b2;
                }
            }
            g1 = warp_sum(g1);
            g2 = warp_sum(g2);
            const double v[2] = {g1, g2};
            const int sl[2] = {3, 4};
            cta_publish(v, sl, a.part, s_red);
        }
        if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
        // ---- beta_k and gamma_{k+1} ----
        if (wib == 0) {
            const double g1 = slot_total(a.part, 3, lane);
            const double g2 = slot_total(a.part, 4, lane);
            if (lane == 0) {
                s_sc[3] = s_sc[5] > 0.0 ? g1 / s_sc[5] : 0.0;
                s_sc[4] = s_sc[6] > 0.0 ? g2 / s_sc[6] : 0.0;
                s_sc[5] = g1;
                s_sc[6] = g2;
            }
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace splitsart

namespace splitsart {
namespace {

size_t cg_align(size_t x) { return (x + 255) & ~size_t(255); }

template <class T, int LPC>
int launch_cgls(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st) {
    using V2 = typename T::Vec2;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "solve_cgls: cudaGetDevice");
    int nsm = 0, coop = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return fail(SPLITSART_ERR_CUDA, "solve_cgls: device lacks cooperative launch");
    int threads = o.block_threads > 0 ? o.block_threads : 512;
    if (threads % 32 != 0 || threads > 1024 || threads < 64)
        return fail(SPLITSART_ERR_ARG, "solve_cgls: block_threads must be a multiple of 32 in [64, 1024]");
    if (threads > 512) threads = 512;
    if (!s->cg_alloc) {
        const size_t bm = cg_align(sizeof(V2) * (size_t)s->Mh), bn = cg_align(sizeof(V2) * (size_t)s->Nh);
        const size_t bp = cg_align(sizeof(double) * kCgSlots * (size_t)kMaxCtas);
        if ((e = cudaMalloc(&s->cg_alloc, 2 * bm + 2 * bn + bp)) != cudaSuccess) {
            s->cg_alloc = nullptr;
            return fail(SPLITSART_ERR_NOMEM, "solve_cgls: %zu bytes of work vectors", 2 * bm + 2 * bn + bp);
        }
    }
    const size_t bm = cg_align(sizeof(V2) * (size_t)s->Mh), bn = cg_align(sizeof(V2) * (size_t)s->Nh);
    char* w = (char*)s->cg_alloc;

    auto kern = cgls_kernel<T, LPC>;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
    if (e != cudaSuccess) return cuda_fail(e, "solve_cgls: occupancy");
    if (per_sm < 1) return fail(SPLITSART_ERR_CUDA, "solve_cgls: kernel does not fit on an SM");
    if (o.ctas_per_sm > 0 && o.ctas_per_sm < per_sm) per_sm = o.ctas_per_sm;
    int grid = nsm * per_sm;
    if (grid > kMaxCtas) grid = kMaxCtas;

    CgArgs<T> a{};
    a.nzr = s->nzr;
    a.nzrp = s->nzrp;
    a.zr = s->zr;
    a.nzc = s->nzc;
    a.nzcp = s->nzcp;
    a.col = s->col;
    a.val = (const typename T::Pair*)s->val;
    a.row = s->row;
    a.valT = (const typename T::Pair*)s->valT;
    a.p12 = (const V2*)p12;
    a.x12 = (V2*)f12;
    a.r12 = (V2*)w;
    a.q12 = (V2*)(w + bm);
    a.s12 = (V2*)(w + 2 * bm);
    a.d12 = (V2*)(w + 2 * bm + bn);
    a.part = (double*)(w + 2 * bm + 2 * bn);
    a.ctl = s->ctl;
    a.result = s->result;
    a.stats = s->stats;
    a.Mh = (int)s->Mh;
    a.Nh = (int)s->Nh;
    a.max_iters = o.max_iters;
    a.check_every = effective_check_every(o);
    a.tol = o.tol;
    a.tol2_hi = o.tol * o.tol * (1.0 + 1e-12);
    const double tms = o.timeout_ms > 0 ? o.timeout_ms : 2000.0;
    a.timeout_ns = (unsigned long long)(tms * 1e6);
    a.expected = (unsigned)grid + (o.inject_barrier_fault ? 1u : 0u);

    if ((e = cudaMemsetAsync(s->ctl, 0, sizeof(LaunchCtl), st)) != cudaSuccess) return cuda_fail(e, "solve_cgls: memset");
    if ((e = cudaMemsetAsync(s->result, 0xff, sizeof(SolveResultDev), st)) != cudaSuccess)
        return cuda_fail(e, "solve_cgls: memset");
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(threads), args, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "solve_cgls: cooperative launch");
    return SPLITSART_OK;
}

template <class T>
int launch_cgls_typed(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o,
                      cudaStream_t st) {
    switch (o.lanes_per_col > 0 ? o.lanes_per_col : 4) {
        case 1: return launch_cgls<T, 1>(s, p12, f12, o, st);
        case 2: return launch_cgls<T, 2>(s, p12, f12, o, st);
        case 4: return launch_cgls<T, 4>(s, p12, f12, o, st);
        case 8: return launch_cgls<T, 8>(s, p12, f12, o, st);
        case 16: return launch_cgls<T, 16>(s, p12, f12, o, st);
        case 32: return launch_cgls<T, 32>(s, p12, f12, o, st);
    }
    return fail(SPLITSART_ERR_ARG, "solve_cgls: lanes_per_col must be 1, 2, 4, 8, 16 or 32");
}

}  // namespace

int run_solve_cgls(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st) {
    if (s->ns != 1) return fail(SPLITSART_ERR_ARG, "solve_cgls: batch systems are not supported; solve each slice");
    if (s->Mh <= 0) return fail(SPLITSART_ERR_ARG, "solve_cgls: empty system");
    switch (s->dtype) {
        case SPLITSART_F64: return launch_cgls_typed<TF64>(s, p12, f12, o, st);
        case SPLITSART_F32: return launch_cgls_typed<TF32>(s, p12, f12, o, st);
    }
    return fail(SPLITSART_ERR_ARG, "solve_cgls: FP64 and FP32 systems only");
}

}  // namespace splitsart
