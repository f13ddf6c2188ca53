// Ordered-subsets SART (OS-SART) on both split systems, with the optional
// non-negativity cone, in one persistent cooperative launch.
//
// SART as Andersen and Kak state it (Section 1, reference [001]) updates the
// image once per projection view. The folded rows are taken in T subsets of
// consecutive rows (by default one folded view pair each: rows t nb .. t nb +
// nb - 1 hold the rays of sources t and K-1-t). Within one iteration, for
// t = 0 .. T-1 and each system s in {1, 2}:
//     u_i = (p^s_i - (A_s f)_i) / R_i                       rows i of subset t
//     f_j += lambda (sum_{i in subset t} a_ij u_i) / C_t,j   C_t,j = sum_{i in t} |a_ij|
// With one subset this is the simultaneous SART of sart.cu.
//
// The cone: the image is non-negative iff f2_j >= |f1_j| for every voxel pair
// (Eq. 5). Its Euclidean projection is: recombine the pair (a = (f2+f1)/2,
// b = (f2-f1)/2), clip a and b at zero, fold again (f1 = a - b, f2 = a + b).
// It is applied to the start and after every subset update, per voxel pair.
//
// Work layout, per subset: a forward pass over the subset's rows (a warp per
// row, lanes strided over the row's entries, a fixed shuffle tree), a grid
// barrier, a back pass over every non-empty column (LPC lanes per column)
// that reads only the column's entries from rows of the subset, and a grid
// barrier. The CSC keeps each column's rows in increasing order, so a
// subset's entries are a contiguous range of the column; a table built once
// per subset size holds where each range starts, and 1/C_t per column.
//
// Stopping: before sweep k, when k is a multiple of check_every or k =
// max_iters, a forward pass over all rows forms ||r||^2 (FP64 across threads,
// warps and CTAs, in a fixed order) and every CTA takes the same decision.
// With one subset that pass is the subset's own forward pass.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <vector>

#include "device_common.cuh"
#include "system.h"

namespace splitsart {

namespace {

// ---------------------------------------------------------------------------
// Tables of a subset size rs: T = ceil(Mh / rs) subsets.
// ---------------------------------------------------------------------------

// qr[t] = first compacted row q with nzr[q] >= t rs (qr[T] = n_nzr).
__global__ void os_row_ranges_kernel(const int32_t* __restrict__ nzr, const FoldStats* __restrict__ stats, int rs,
                                     int T, int32_t* __restrict__ qr) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > T) return;
    const int n = stats->n_nzr;
    const long long key = (long long)t * rs;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((long long)nzr[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    qr[t] = lo;
}

// One warp per compacted column q: off[t][q] = first entry of the column
// whose row is >= t rs (t = 0 .. T; off[T][q] is the column's end), and
// invC[t][q] = 1 / sum of |a| over the entries of subset t (0 if the sum is 0),
// summed in FP64 in increasing row order.
template <class T>
__global__ void os_col_tables_kernel(const int32_t* __restrict__ nzcp, const int32_t* __restrict__ row,
                                     const typename T::Pair* __restrict__ valT, const FoldStats* __restrict__ stats,
                                     int rs, int Tn, int32_t* __restrict__ off, typename T::Vec2* __restrict__ invC) {
    using V2 = typename T::Vec2;
    using S = decltype(V2{}.x);
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int n = stats->n_nzc;
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < n; q += nw) {
        const int e0 = nzcp[q], e1 = nzcp[q + 1];
        for (int t = lane; t <= Tn; t += 32) {
            const long long key = (long long)t * rs;
            int lo = e0, hi = e1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((long long)row[mid] < key) lo = mid + 1;
                else hi = mid;
            }
            off[(size_t)t * n + q] = lo;
        }
        __syncwarp();
        for (int t = lane; t < Tn; t += 32) {
            const int a0 = off[(size_t)t * n + q], a1 = off[(size_t)(t + 1) * n + q];
            double c1 = 0.0, c2 = 0.0;
            for (int e = a0; e < a1; ++e) {
                typename T::Acc v1, v2;
                T::decode(valT[e], v1, v2);
                c1 += fabs((double)v1);
                c2 += fabs((double)v2);
            }
            invC[(size_t)t * n + q] = V2{(S)(c1 > 0.0 ? 1.0 / c1 : 0.0), (S)(c2 > 0.0 ? 1.0 / c2 : 0.0)};
        }
    }
}

// ---------------------------------------------------------------------------
// The solve kernel.
// ---------------------------------------------------------------------------
template <class T>
struct OsArgs {
    const int32_t* __restrict__ nzr;
    const int32_t* __restrict__ nzrp;
    const int32_t* __restrict__ zr;
    const int32_t* __restrict__ nzc;
    const int32_t* __restrict__ col;
    const typename T::Pair* __restrict__ val;
    const int32_t* __restrict__ row;
    const typename T::Pair* __restrict__ valT;
    const typename T::KNorm2* __restrict__ invR;
    const typename T::Vec2* __restrict__ p12;
    typename T::Vec2* f12;
    typename T::Vec2* u12;
    const int32_t* __restrict__ qr;               // [T + 1]
    const int32_t* __restrict__ off;              // [(T + 1) x n_nzc]
    const typename T::Vec2* __restrict__ invCt;   // [T x n_nzc]
    double* partials;  // [2 * gridDim.x]: (rr, pp) per CTA
    LaunchCtl* ctl;
    SolveResultDev* result;
    const FoldStats* stats;
    int Tn;            // subsets
    int Nh;            // folded columns (the cone projects every one at the start)
    int cone;
    int max_iters, check_every;
    double lambda, tol, tol2_hi;
    unsigned long long timeout_ns;
    unsigned expected;
};

// Project one voxel pair onto f2 >= |f1|: recombine (Eq. 5), clip, fold.
template <class V2>
__device__ __forceinline__ V2 cone_project(V2 f) {
    using S = decltype(f.x);
    const S half = (S)0.5;
    S a = half * (f.y + f.x), b = half * (f.y - f.x);
    a = a > (S)0 ? a : (S)0;
    b = b > (S)0 ? b : (S)0;
    return V2{a - b, a + b};
}

// The joint stop test (one thread), as in the simultaneous solve: rho =
// sqrt(rr / pp), 0 when pp = 0; rr > pp tol^2 (1 + 1e-12) proves rho > tol
// without the division and the square root. CTA 0 records the stopping pass.
template <class A>
__device__ __forceinline__ int os_stop_test(const A& a, int k, bool last, double trr, double tpp) {
    if (!last && tpp > 0.0 && trr > tpp * a.tol2_hi) return 0;
    const double rho = tpp > 0.0 ? sqrt(trr / tpp) : 0.0;
    const bool stop = last || rho <= a.tol;
    if (stop && blockIdx.x == 0) {
        a.result->iters = k;
        a.result->status = SPLITSART_OK;
        a.result->rho = rho;
        a.result->rr = trr;
        a.result->pp = tpp;
    }
    return stop ? 1 : 0;
}

template <class T, int LPC>
__global__ void __launch_bounds__(512, 1) os_sart_kernel(OsArgs<T> a) {
    using Acc = typename T::Acc;
    using V2 = typename T::Vec2;
    using N2 = typename T::KNorm2;
    constexpr int kGroups = 32 / LPC;
    __shared__ double s_red[32];
    __shared__ double s_tpp;
    __shared__ int s_stop;

    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5, nwarps = blockDim.x >> 5, BD = blockDim.x;
    const int sub = lane % LPC;
    const int gw = blockIdx.x * nwarps + wib, nw_grid = gridDim.x * nwarps;
    const Acc lam = (Acc)a.lambda;
    const int n_nzr = a.stats->n_nzr, n_nzc = a.stats->n_nzc, n_zr = a.stats->n_zr;

    // ---- prologue: ||p||^2 of every row, ||p||^2 of the empty rows, the cone on the start ----
    double ppz = 0.0;  // thread 0: this CTA's share of the empty rows' ||p||^2 (their residual is p)
    {
        const long long G = gridDim.x, b = blockIdx.x;
        const int z0 = (int)(n_zr * b / G), z1 = (int)(n_zr * (b + 1) / G);
        const long long Mall = (long long)n_nzr + n_zr;
        const long long m0 = Mall * b / G, m1 = Mall * (b + 1) / G;
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
        if (a.cone)
            for (int j = blockIdx.x * BD + tid; j < a.Nh; j += gridDim.x * BD) stcg(a.f12 + j, cone_project(ldcg(a.f12 + j)));
    }
    unsigned nbar = 0;
    if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
    if (wib == 0) {
        const double t = grid_total(a.partials, gridDim.x, lane, 1);
        if (lane == 0) s_tpp = t;
    }

    // Row q's residual pair (lane 0 holds the result): r = p - A f.
    auto residual = [&](int q, Acc& r1, Acc& r2, int& i) {
        const int lo = __ldg(a.nzrp + q), hi = __ldg(a.nzrp + q + 1);
        Acc s1 = 0, s2 = 0;
        for (int e = lo + lane; e < hi; e += 32) {
            Acc v1, v2;
            T::decode(ldg(a.val + e), v1, v2);
            const V2 f = ldca(a.f12 + __ldg(a.col + e));
            s1 += v1 * f.x;
            s2 += v2 * f.y;
        }
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        i = __ldg(a.nzr + q);
        const V2 p = ldg(a.p12 + i);
        r1 = p.x - s1;
        r2 = p.y - s2;
    };
    // The CTA's sum of its warps' ||r||^2 (lane 0 values), plus the empty rows', to partials[2b].
    auto publish_rr = [&](double mine) {
        if (lane == 0) s_red[wib] = mine;
        __syncthreads();
        if (tid == 0) {
            double t = ppz;
            for (int w = 0; w < nwarps; ++w) t += s_red[w];
            __stcg(a.partials + 2 * blockIdx.x, t);
        }
    };
    // Every CTA sums the partials in the same order; thread 0 decides.
    auto decide = [&](int k, bool last) {
        if (wib == 0) {
            const double trr = grid_total(a.partials, gridDim.x, lane, 0);
            if (lane == 0) s_stop = os_stop_test(a, k, last, trr, s_tpp);
        }
        __syncthreads();
        return s_stop != 0;
    };

    for (int k = 0;; ++k) {
        const bool last = k >= a.max_iters;
        const bool check = last || (k % a.check_every == 0);
        if (check && a.Tn > 1) {
            // ---- test pass: ||A f^k - p||^2 over all rows ----
            double mine = 0.0;
            for (int q = gw; q < n_nzr; q += nw_grid) {
                Acc r1, r2;
                int i;
                residual(q, r1, r2, i);
                mine += (double)(r1 * r1 + r2 * r2);
            }
            publish_rr(mine);
            if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
            if (decide(k, last)) return;
        }
        for (int t = 0; t < a.Tn; ++t) {
            // ---- forward over the subset's rows: u = (p - A f) / R ----
            const int q0 = __ldg(a.qr + t), q1 = __ldg(a.qr + t + 1);
            double mine = 0.0;
            for (int q = q0 + gw; q < q1; q += nw_grid) {
                Acc r1, r2;
                int i;
                residual(q, r1, r2, i);
                if (lane == 0) {
                    const N2 ir = ldg(a.invR + i);
                    stcg(a.u12 + i, V2{r1 * ir.x, r2 * ir.y});
                    mine += (double)(r1 * r1 + r2 * r2);
                }
            }
            if (a.Tn == 1 && check) publish_rr(mine);
            if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
            if (a.Tn == 1 && check && decide(k, last)) return;

            // ---- back over every non-empty column: f += lambda (A_t^T u) / C_t, then the cone ----
            const int32_t* off0 = a.off + (size_t)t * n_nzc;
            const int32_t* off1 = off0 + n_nzc;
            const V2* ic_t = a.invCt + (size_t)t * n_nzc;
            for (int g0 = gw * kGroups; g0 < n_nzc; g0 += nw_grid * kGroups) {
                const int q = g0 + lane / LPC;
                const int lo = q < n_nzc ? __ldg(off0 + q) : 0, hi = q < n_nzc ? __ldg(off1 + q) : 0;
                Acc b1 = 0, b2 = 0;
                for (int e = lo + sub; e < hi; e += LPC) {
                    Acc v1, v2;
                    T::decode(ldg(a.valT + e), v1, v2);
                    const V2 u = ldca(a.u12 + __ldg(a.row + e));
                    b1 += v1 * u.x;
                    b2 += v2 * u.y;
                }
                b1 = warp_sum(b1, LPC);
                b2 = warp_sum(b2, LPC);
                if (sub == 0 && q < n_nzc && (hi > lo || a.cone)) {
                    const int j = __ldg(a.nzc + q);
                    V2 f = ldcg(a.f12 + j);
                    if (hi > lo) {
                        const V2 ic = ldg(ic_t + q);
                        f.x += lam * b1 * ic.x;
                        f.y += lam * b2 * ic.y;
                    }
                    if (a.cone) f = cone_project(f);
                    stcg(a.f12 + j, f);
                }
            }
            if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
        }
    }
}

}  // namespace
}  // namespace splitsart

namespace splitsart {
namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Build (once per subset size) the subset tables of a system.
template <class T>
int os_tables(splitsart_system* s, const FoldStats& fs, int rs, cudaStream_t st) {
    if (s->os_rows == rs && s->os_alloc) return SPLITSART_OK;
    using V2 = typename T::Vec2;
    const long long Tn = (s->Mh + rs - 1) / rs;
    if (Tn < 1 || Tn > 65536) return fail(SPLITSART_ERR_ARG, "solve_os: %lld subsets (1 to 65536 allowed)", Tn);
    const size_t nc = (size_t)(fs.n_nzc > 0 ? fs.n_nzc : 1);
    const size_t b_qr = align256(sizeof(int32_t) * (size_t)(Tn + 1));
    const size_t b_off = align256(sizeof(int32_t) * (size_t)(Tn + 1) * nc);
    const size_t b_ic = align256(sizeof(V2) * (size_t)Tn * nc);
    if (s->os_alloc) {
        cudaStreamSynchronize(st);
        cudaFree(s->os_alloc);
        s->os_alloc = nullptr;
        s->os_rows = 0;
    }
    void* base = nullptr;
    cudaError_t e = cudaMalloc(&base, b_qr + b_off + b_ic);
    if (e != cudaSuccess) return fail(SPLITSART_ERR_NOMEM, "solve_os: %zu bytes of subset tables", b_qr + b_off + b_ic);
    char* p = (char*)base;
    s->os_qr = (int32_t*)p;
    s->os_off = (int32_t*)(p + b_qr);
    s->os_invC = p + b_qr + b_off;
    s->os_alloc = base;
    s->os_T = (int)Tn;
    os_row_ranges_kernel<<<(unsigned)((Tn + 1 + 127) / 128), 128, 0, st>>>(s->nzr, s->stats, rs, (int)Tn, s->os_qr);
    const int blocks = (int)std::min<long long>(((long long)nc * 32 + 255) / 256, 152LL * 16);
    os_col_tables_kernel<T><<<blocks, 256, 0, st>>>(s->nzcp, s->row, (const typename T::Pair*)s->valT, s->stats, rs,
                                                   (int)Tn, s->os_off, (V2*)s->os_invC);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "solve_os: table kernels");
    s->os_rows = rs;
    return SPLITSART_OK;
}

template <class T, int LPC>
int launch_os(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o,
              const splitsart_os_opts& os, cudaStream_t st) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "solve_os: cudaGetDevice");
    int nsm = 0, coop = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return fail(SPLITSART_ERR_CUDA, "solve_os: device lacks cooperative launch");
    int threads = o.block_threads > 0 ? o.block_threads : 512;
    if (threads % 32 != 0 || threads > 1024 || threads < 64)
        return fail(SPLITSART_ERR_ARG, "solve_os: block_threads must be a multiple of 32 in [64, 1024]");
    if (threads > 512) threads = 512;
    FoldStats fs;
    int rc = system_host_stats(s, &fs);
    if (rc) return rc;
    const int rs = os.subset_rows > 0 ? os.subset_rows : s->nb;
    rc = os_tables<T>(s, fs, rs, st);
    if (rc) return rc;

    auto kern = os_sart_kernel<T, LPC>;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
    if (e != cudaSuccess) return cuda_fail(e, "solve_os: occupancy");
    if (per_sm < 1) return fail(SPLITSART_ERR_CUDA, "solve_os: kernel does not fit on an SM");
    if (o.ctas_per_sm > 0 && o.ctas_per_sm < per_sm) per_sm = o.ctas_per_sm;
    int grid = nsm * per_sm;
    if (grid > kMaxCtas) grid = kMaxCtas;

    OsArgs<T> a{};
    a.nzr = s->nzr;
    a.nzrp = s->nzrp;
    a.zr = s->zr;
    a.nzc = s->nzc;
    a.col = s->col;
    a.val = (const typename T::Pair*)s->val;
    a.row = s->row;
    a.valT = (const typename T::Pair*)s->valT;
    a.invR = (const typename T::KNorm2*)s->invR;
    a.p12 = (const typename T::Vec2*)p12;
    a.f12 = (typename T::Vec2*)f12;
    a.u12 = (typename T::Vec2*)s->u12;
    a.qr = s->os_qr;
    a.off = s->os_off;
    a.invCt = (const typename T::Vec2*)s->os_invC;
    a.partials = s->partials;
    a.ctl = s->ctl;
    a.result = s->result;
    a.stats = s->stats;
    a.Tn = s->os_T;
    a.Nh = (int)s->Nh;
    a.cone = os.cone ? 1 : 0;
    a.max_iters = o.max_iters;
    a.check_every = effective_check_every(o);
    a.lambda = o.lambda;
    a.tol = o.tol;
    a.tol2_hi = o.tol * o.tol * (1.0 + 1e-12);
    const double tms = o.timeout_ms > 0 ? o.timeout_ms : 2000.0;
    a.timeout_ns = (unsigned long long)(tms * 1e6);
    a.expected = (unsigned)grid + (o.inject_barrier_fault ? 1u : 0u);

    if ((e = cudaMemsetAsync(s->ctl, 0, sizeof(LaunchCtl), st)) != cudaSuccess) return cuda_fail(e, "solve_os: memset");
    if ((e = cudaMemsetAsync(s->result, 0xff, sizeof(SolveResultDev), st)) != cudaSuccess)
        return cuda_fail(e, "solve_os: memset");
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(threads), args, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "solve_os: cooperative launch");
    return SPLITSART_OK;
}

template <class T>
int launch_os_typed(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o,
                    const splitsart_os_opts& os, cudaStream_t st) {
    switch (o.lanes_per_col > 0 ? o.lanes_per_col : 4) {
        case 1: return launch_os<T, 1>(s, p12, f12, o, os, st);
        case 2: return launch_os<T, 2>(s, p12, f12, o, os, st);
        case 4: return launch_os<T, 4>(s, p12, f12, o, os, st);
        case 8: return launch_os<T, 8>(s, p12, f12, o, os, st);
        case 16: return launch_os<T, 16>(s, p12, f12, o, os, st);
        case 32: return launch_os<T, 32>(s, p12, f12, o, os, st);
    }
    return fail(SPLITSART_ERR_ARG, "solve_os: lanes_per_col must be 1, 2, 4, 8, 16 or 32");
}

}  // namespace

int run_solve_os(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o,
                 const splitsart_os_opts& os, cudaStream_t st) {
    if (s->ns != 1) return fail(SPLITSART_ERR_ARG, "solve_os: batch systems are not supported; solve each slice");
    if (os.subset_rows < 0) return fail(SPLITSART_ERR_ARG, "solve_os: subset_rows must be >= 0");
    if (os.subset_rows == 0 && s->nb <= 0)
        return fail(SPLITSART_ERR_ARG, "solve_os: subset_rows = 0 needs a system folded from acquisition parameters");
    if (os.reserved[0] || os.reserved[1]) return fail(SPLITSART_ERR_ARG, "solve_os: reserved fields must be zero");
    if (s->Mh <= 0) return fail(SPLITSART_ERR_ARG, "solve_os: empty system");
    switch (s->dtype) {
        case SPLITSART_F64: return launch_os_typed<TF64>(s, p12, f12, o, os, st);
        case SPLITSART_F32: return launch_os_typed<TF32>(s, p12, f12, o, os, st);
    }
    return fail(SPLITSART_ERR_ARG, "solve_os: FP64 and FP32 systems only");
}

}  // namespace splitsart
