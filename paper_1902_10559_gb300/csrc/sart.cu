// Persistent split-SART: both folded systems, every iteration, in one cooperative launch.
//
// SART is the accepted iterative method (Section 1, reference [001]). The
// simultaneous form is applied to each split system s in {1, 2} (Eqs. 3, 4):
//     r^k = p^s - A_s f^k,   u^k = r^k / R,   f^{k+1} = f^k + lambda (A_s^T u^k) / C,
// where R and C are absolute row and column sums with 1/0 := 0. The two
// systems are independent (Theorem 1). They are run together because they
// share the index pattern: one pass over col/row indices feeds both.
//
// One iteration is two grid-wide phases:
//   forward:  one warp per folded row. It gathers the pair (f1, f2) at each
//             column, reduces (A1 f1, A2 f2) with a fixed shuffle tree, and
//             writes the pair u = r / R. ||r||^2 and ||p||^2 are summed in
//             FP64 into per-CTA partials.
//   barrier, then the stop test: every CTA sums the partials in the same
//             order, so all CTAs take the same decision.
//   back:     LPC lanes per column walk the CSC (rows ascending), gather u,
//             reduce with a fixed tree, and update the pair f in place.
//   barrier.
// No atomics touch values, so results are bitwise reproducible for a given
// launch shape.
//
// Vectors rewritten during the launch (f12 and u12) are read through L2
// (ld.global.cg), so a CTA never sees a stale L1 copy. The matrix, p, and
// the normalisers use the read-only path.
#include <cstdio>

#include "device_common.cuh"
#include "system.h"

namespace splitsart {

namespace {

template <class T>
struct SartArgs {
    const int32_t* __restrict__ rp;
    const int32_t* __restrict__ col;
    const typename T::Pair* __restrict__ val;
    const int32_t* __restrict__ cp;
    const int32_t* __restrict__ row;
    const typename T::Pair* __restrict__ valT;
    const typename T::Norm2* __restrict__ invR;
    const typename T::Norm2* __restrict__ invC;
    const float2* __restrict__ scale;
    const typename T::Vec2* __restrict__ p12;
    typename T::Vec2* f12;
    typename T::Vec2* u12;
    double* partials;  // [2 * gridDim.x]: (rr, pp) per CTA
    LaunchCtl* ctl;
    SolveResultDev* result;
    int Mh, Nh;
    int max_iters, check_every;
    double lambda, tol;
    unsigned long long timeout_ns;
    unsigned expected;  // CTAs the barrier waits for
};

constexpr int kUnroll = 4;

// Forward projection of one row for both systems, by one warp.
template <class T>
__device__ __forceinline__ void row_dot(const SartArgs<T>& a, int i, int lane, typename T::Acc& s1,
                                        typename T::Acc& s2) {
    using Acc = typename T::Acc;
    using V2 = typename T::Vec2;
    const int e0 = __ldg(a.rp + i), e1 = __ldg(a.rp + i + 1);
    s1 = 0;
    s2 = 0;
    for (int base = e0; base < e1; base += 32 * kUnroll) {
        int c[kUnroll];
        typename T::Pair v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int e = base + u * 32 + lane;
            if (e < e1) {
                c[u] = ldg(a.col + e);
                v[u] = ldg(a.val + e);
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int e = base + u * 32 + lane;
            if (e < e1) {
                const V2 fv = ldcg(a.f12 + c[u]);
                Acc a1, a2;
                T::decode(v[u], a1, a2);
                s1 += a1 * fv.x;
                s2 += a2 * fv.y;
            }
        }
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
}

template <class T, int LPC>
__global__ void __launch_bounds__(256, 4) sart_persistent_kernel(SartArgs<T> a) {
    using Acc = typename T::Acc;
    using V2 = typename T::Vec2;
    __shared__ double s_red[2][32];
    __shared__ double s_rho[3];

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int nwarps_blk = blockDim.x >> 5;
    const int gwarp = blockIdx.x * nwarps_blk + wib;
    const int nwarps = gridDim.x * nwarps_blk;
    constexpr int kGroupsPerWarp = 32 / LPC;
    const int sub = lane % LPC;
    const Acc lam = (Acc)a.lambda;

    int barrier_no = 0;
    for (int k = 0;; ++k) {
        // ---- forward: r = p - A f, u = r / R, and the norm partials ----
        double rr = 0.0, pp = 0.0;
        for (int i = gwarp; i < a.Mh; i += nwarps) {
            Acc s1, s2;
            row_dot<T>(a, i, lane, s1, s2);
            if (lane == 0) {
                const V2 p = ldg(a.p12 + i);
                if constexpr (T::kQuant) {
                    const float2 sc = ldg(a.scale + i);
                    s1 *= sc.x;
                    s2 *= sc.y;
                }
                const Acc r1 = p.x - s1, r2 = p.y - s2;
                const typename T::Norm2 ir = ldg(a.invR + i);
                V2 u;
                if constexpr (T::kQuant) {
                    // Back-projection reuses the codes, so fold the row scale into u.
                    const float2 sc = ldg(a.scale + i);
                    u.x = (Acc)((double)r1 * ir.x * (double)sc.x);
                    u.y = (Acc)((double)r2 * ir.y * (double)sc.y);
                } else {
                    u.x = r1 * ir.x;
                    u.y = r2 * ir.y;
                }
                stcg(a.u12 + i, u);
                rr += (double)r1 * (double)r1 + (double)r2 * (double)r2;
                pp += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
            }
        }
        if (lane == 0) {
            s_red[0][wib] = rr;
            s_red[1][wib] = pp;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t0 = 0.0, t1 = 0.0;
            for (int w = 0; w < nwarps_blk; ++w) {
                t0 += s_red[0][w];
                t1 += s_red[1][w];
            }
            __stcg(a.partials + 2 * blockIdx.x, t0);
            __stcg(a.partials + 2 * blockIdx.x + 1, t1);
        }
        if (!grid_barrier(a.ctl, a.expected, a.timeout_ns, barrier_no++)) return;

        // ---- stop test ----
        const bool last = (k >= a.max_iters);
        const bool check = last || (k % a.check_every == 0);
        if (check) {
            if (wib == 0) {
                double t0 = 0.0, t1 = 0.0;
                for (int b = lane; b < (int)gridDim.x; b += 32) {
                    t0 += __ldcg(a.partials + 2 * b);
                    t1 += __ldcg(a.partials + 2 * b + 1);
                }
                t0 = warp_sum(t0);
                t1 = warp_sum(t1);
                if (lane == 0) {
                    s_rho[0] = t0;
                    s_rho[1] = t1;
                    s_rho[2] = t1 > 0.0 ? sqrt(t0 / t1) : 0.0;
                }
            }
            __syncthreads();
            const double rho = s_rho[2];
            if (last || rho <= a.tol) {
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    a.result->iters = k;
                    a.result->status = SPLITSART_OK;
                    a.result->rho = rho;
                    a.result->rr = s_rho[0];
                    a.result->pp = s_rho[1];
                }
                return;
            }
        }

        // ---- back-projection and update: f += lambda (A^T u) / C ----
        // The outer loop is warp-uniform, so every lane reaches the shuffles.
        for (int jb = gwarp * kGroupsPerWarp; jb < a.Nh; jb += nwarps * kGroupsPerWarp) {
            const int j = jb + lane / LPC;
            Acc b1 = 0, b2 = 0;
            if (j < a.Nh) {
                const int e0 = __ldg(a.cp + j), e1 = __ldg(a.cp + j + 1);
                for (int e = e0 + sub; e < e1; e += LPC) {
                    const int r = ldg(a.row + e);
                    const typename T::Pair v = ldg(a.valT + e);
                    const V2 u = ldcg(a.u12 + r);
                    Acc a1, a2;
                    T::decode(v, a1, a2);
                    b1 += a1 * u.x;
                    b2 += a2 * u.y;
                }
            }
            b1 = warp_sum(b1, LPC);
            b2 = warp_sum(b2, LPC);
            if (sub == 0 && j < a.Nh) {
                const typename T::Norm2 ic = ldg(a.invC + j);
                V2 f = ldcg(a.f12 + j);
                if constexpr (T::kQuant) {
                    f.x += (Acc)((double)(lam * b1) * ic.x);
                    f.y += (Acc)((double)(lam * b2) * ic.y);
                } else {
                    f.x += lam * b1 * ic.x;
                    f.y += lam * b2 * ic.y;
                }
                stcg(a.f12 + j, f);
            }
        }
        if (!grid_barrier(a.ctl, a.expected, a.timeout_ns, barrier_no++)) return;
    }
}

template <class T, int LPC>
int launch_lpc(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st) {
    auto kern = sart_persistent_kernel<T, LPC>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "solve: cudaGetDevice");
    int nsm = 0, coop = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return fail(SPLITSART_ERR_CUDA, "solve: device lacks cooperative launch");
    const int threads = o.block_threads > 0 ? o.block_threads : 256;
    if (threads % 32 != 0 || threads > 256 || threads < LPC)
        return fail(SPLITSART_ERR_ARG, "solve: block_threads must be a multiple of 32 in [32, 256]");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
    if (e != cudaSuccess) return cuda_fail(e, "solve: occupancy");
    if (o.ctas_per_sm > 0 && o.ctas_per_sm < per_sm) per_sm = o.ctas_per_sm;
    int grid = nsm * per_sm;
    if (grid > kMaxCtas) grid = kMaxCtas;
    if (grid < 1) return fail(SPLITSART_ERR_CUDA, "solve: kernel does not fit on an SM");

    SartArgs<T> a;
    a.rp = s->rp;
    a.col = s->col;
    a.val = (const typename T::Pair*)s->val;
    a.cp = s->cp;
    a.row = s->row;
    a.valT = (const typename T::Pair*)s->valT;
    a.invR = (const typename T::Norm2*)s->invR;
    a.invC = (const typename T::Norm2*)s->invC;
    a.scale = s->scale;
    a.p12 = (const typename T::Vec2*)p12;
    a.f12 = (typename T::Vec2*)f12;
    a.u12 = (typename T::Vec2*)s->u12;
    a.partials = s->partials;
    a.ctl = s->ctl;
    a.result = s->result;
    a.Mh = (int)s->Mh;
    a.Nh = (int)s->Nh;
    a.max_iters = o.max_iters;
    a.check_every = o.check_every > 0 ? o.check_every : 1;
    a.lambda = o.lambda;
    a.tol = o.tol;
    const double tms = o.timeout_ms > 0 ? o.timeout_ms : 2000.0;
    a.timeout_ns = (unsigned long long)(tms * 1e6);
    a.expected = (unsigned)grid + (o.inject_barrier_fault ? 1u : 0u);

    if ((e = cudaMemsetAsync(s->ctl, 0, sizeof(LaunchCtl), st)) != cudaSuccess) return cuda_fail(e, "solve: memset");
    // A result the launch never writes (a timeout) reads back as iters = -1.
    if ((e = cudaMemsetAsync(s->result, 0xff, sizeof(SolveResultDev), st)) != cudaSuccess)
        return cuda_fail(e, "solve: memset");
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(threads), args, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "solve: cooperative launch");
    return SPLITSART_OK;
}

template <class T>
int launch_typed(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st) {
    switch (o.lanes_per_col > 0 ? o.lanes_per_col : 8) {
        case 1: return launch_lpc<T, 1>(s, p12, f12, o, st);
        case 2: return launch_lpc<T, 2>(s, p12, f12, o, st);
        case 4: return launch_lpc<T, 4>(s, p12, f12, o, st);
        case 8: return launch_lpc<T, 8>(s, p12, f12, o, st);
        case 16: return launch_lpc<T, 16>(s, p12, f12, o, st);
        case 32: return launch_lpc<T, 32>(s, p12, f12, o, st);
    }
    return fail(SPLITSART_ERR_ARG, "solve: lanes_per_col must be 1, 2, 4, 8, 16 or 32");
}

}  // namespace

int run_solve(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st) {
    switch (s->dtype) {
        case SPLITSART_F64: return launch_typed<TF64>(s, p12, f12, o, st);
        case SPLITSART_F32: return launch_typed<TF32>(s, p12, f12, o, st);
        case SPLITSART_BF16: return launch_typed<TBF16>(s, p12, f12, o, st);
        case SPLITSART_F16: return launch_typed<TF16>(s, p12, f12, o, st);
    }
    return fail(SPLITSART_ERR_ARG, "solve: unknown dtype %d", s->dtype);
}

}  // namespace splitsart
