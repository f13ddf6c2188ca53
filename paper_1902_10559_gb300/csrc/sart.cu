// Persistent split-SART: both folded systems, every iteration, in one cooperative launch.
//
// SART is the accepted iterative method (Section 1, reference [001]). The
// simultaneous form is applied to each split system s in {1, 2} (Eqs. 3, 4):
//     r^k = p^s - A_s f^k,   u^k = r^k / R,   f^{k+1} = f^k + lambda (A_s^T u^k) / C,
// where R and C are absolute row and column sums with 1/0 := 0. The two
// systems are independent (Theorem 1). They are run together because they
// share the index pattern: one pass over the col/row indices feeds both.
//
// Work layout. One CTA per SM (1024 threads), launched cooperatively.
// - Each CTA owns a contiguous range of the non-empty rows with about S/G
//   entries, and likewise a range of the non-empty columns. Empty rows and
//   columns were compacted away by the fold.
// - A range is cut into tiles of at most TE entries that end on row
//   (column) boundaries. The tile boundaries are computed once per launch.
//
// Per iteration:
//   forward: for each tile, all threads stream the tile's col/value pairs
//            with coalesced loads, gather the pair (f1, f2) at each column,
//            and stage the products in shared memory. One warp per row then
//            reduces its products (lane-strided, fixed shuffle tree) and
//            writes u = r / R. ||r||^2 and ||p||^2 accumulate in FP64.
//   barrier: the last CTA to arrive sums the per-CTA norm partials in a
//            fixed order and publishes rho. All CTAs take the same stop
//            decision.
//   back:    the same tiling over the CSC (rows ascending within a column).
//            It gathers u. LPC lanes reduce each column and update f in place.
//   barrier.
// Each row's and each column's sum is formed in an order that depends on
// neither the tiling nor the grid, so f is bitwise reproducible across
// launch shapes with the same LPC. No atomics touch values.
//
// Vectors rewritten during the launch (f12, u12) are read through L2
// (ld.global.cg), so a CTA never sees a stale L1 copy. The matrix, p and the
// normalisers use the read-only path.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <initializer_list>
#include <vector>
#include <type_traits>

#include "device_common.cuh"
#include "system.h"

namespace splitsart {

namespace {

constexpr int kMaxTiles = 1024;  // tiles per CTA and phase
constexpr int kUnroll = 4;

template <class T>
struct SartArgs {
    const int32_t* __restrict__ nzr;
    const int32_t* __restrict__ nzrp;
    const int32_t* __restrict__ zr;
    const int32_t* __restrict__ nzc;
    const int32_t* __restrict__ nzcp;
    const int32_t* __restrict__ col;
    const typename T::Pair* __restrict__ val;
    const int32_t* __restrict__ row;
    const typename T::Pair* __restrict__ valT;
    const typename T::KNorm2* __restrict__ invR;  // as applied (BF16/FP16: scale / R in FP32)
    const typename T::KNorm2* __restrict__ invC;
    const float2* __restrict__ scale;
    const typename T::Vec2* __restrict__ p12;
    typename T::Vec2* f12;
    typename T::Vec2* u12;
    double* partials;  // [2 * gridDim.x]: (rr, pp) per CTA; pp is written once per launch
    LaunchCtl* ctl;
    SolveResultDev* result;
    const FoldStats* stats;
    int max_iters, check_every;
    double lambda, tol;
    double tol2_hi;  // tol^2 (1 + 1e-12): rr > pp tol2_hi proves rho > tol without a division or square root
    unsigned long long timeout_ns;
    unsigned expected;  // CTAs the barrier waits for
    int tile_entries;   // TE
    int direct_rows;    // kDirect only: Mh (nzrp = rp, row q is row q, no empty-row list)
    int direct_cols;    // kDirect only: Nh (nzcp = cp, column q is column q)
    // kBatch only: slices with their own stopping tests.
    int ns;
    const long long* sl_rows;  // [ns+1] folded-row prefix
    const long long* sl_cols;  // [ns+1] folded-column prefix
    SliceSolve* sl_solve;      // [ns]
    double* rr_row;            // [Mh] per-row residual^2
    int* ndone;                // slices finished
    // Resident kernel only: the row plan (null: contiguous row ranges).
    const int32_t* res_rows;
    const int32_t* res_off;
    const int32_t* res_loc;
};

// Per-slice stop tests of a batch: one CTA per slice sums the slice's per-row
// residual^2 (thread-strided, then a fixed tree), and one thread decides.
// red: 32 doubles of shared scratch. Called by every thread of the CTA.
template <class A>
__device__ void slice_stop_tests(const A& a, int k, bool last, double* red) {
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5, nwarps = blockDim.x >> 5;
    for (int sl = blockIdx.x; sl < a.ns; sl += gridDim.x) {
        if (__ldcg(&a.sl_solve[sl].done)) continue;  // uniform over the CTA
        double t = 0.0;
        for (long long i = __ldg(a.sl_rows + sl) + tid; i < __ldg(a.sl_rows + sl + 1); i += blockDim.x)
            t += __ldcg(a.rr_row + i);
        t = warp_sum(t);
        if (lane == 0) red[wib] = t;
        __syncthreads();
        if (wib == 0) {
            const double trr = warp_sum(lane < nwarps ? red[lane] : 0.0);
            if (lane == 0) {
                const double tpp = __ldcg(&a.sl_solve[sl].pp);
                const bool above = !last && tpp > 0.0 && trr > tpp * a.tol2_hi;  // rho > tol for certain
                const double rho = (above || !(tpp > 0.0)) ? 0.0 : sqrt(trr / tpp);
                if (!above && (last || rho <= a.tol)) {
                    a.sl_solve[sl] = SliceSolve{k, 1, rho, trr, tpp};
                    atomicAdd(a.ndone, 1);
                }
            }
        }
        __syncthreads();
    }
}

// The joint stop test (one thread): rho = sqrt(rr / pp), 0 when pp = 0. CTA 0
// records the result of the stopping pass. Returns 1 to stop.
// rr > pp tol^2 (1 + 1e-12) proves rho > tol whatever the rounding of the
// division and the square root (a few ulps), so the common case skips both:
// FP64 division and square root are long dependent chains on this GPU.
template <class A>
__device__ __forceinline__ int stop_test(const A& a, int k, bool last, double trr, double tpp) {
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

// The slice holding global index i (largest s with off[s] <= i).
__device__ __forceinline__ int slice_index(const long long* off, int ns, long long i) {
    int lo = 0, hi = ns;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Warp-cooperative search: the first q in [lo, hi] with ptr[q] >= t, where
// ptr is non-decreasing and q = hi if no probed index qualifies. Only indices
// below hi are read. Each round probes 32 evenly spaced indices; the probes
// below t form a prefix, so their count narrows the range 32-fold.
__device__ __forceinline__ int warp_lower_bound(const int32_t* ptr, int lo, int hi, long long t, int lane) {
    while (hi - lo > 32) {
        const int step = (hi - lo + 31) / 32;
        const int idx = lo + lane * step;
        const bool below = idx < hi && (long long)__ldg(ptr + idx) < t;
        const int c = __popc(__ballot_sync(0xffffffffu, below));
        if (c == 0) return lo;
        const int nlo = lo + (c - 1) * step + 1;
        hi = min(lo + c * step, hi);
        lo = nlo;
    }
    const int idx = lo + lane;
    const bool below = idx < hi && (long long)__ldg(ptr + idx) < t;
    return lo + __popc(__ballot_sync(0xffffffffu, below));
}

// One warp: cut this CTA's share of [0, n) (balanced by the entry counts of
// ptr[0..n]) into tiles of at most TE entries that end on boundaries. Lane 0
// writes the boundaries to tiles[]. Returns the tile count, or -1 if more
// than kMaxTiles would be needed.
__device__ int plan_tiles(const int32_t* ptr, int n, int TE, int* tiles, int lane) {
    const long long S = __ldg(ptr + n);
    const long long G = gridDim.x, b = blockIdx.x;
    const int q0 = warp_lower_bound(ptr, 0, n, S * b / G, lane);
    const int q1 = (b == G - 1) ? n : warp_lower_bound(ptr, 0, n, S * (b + 1) / G, lane);
    int nt = 0;
    int q = q0;
    while (q < q1) {
        if (nt >= kMaxTiles) return -1;
        if (lane == 0) tiles[nt] = q;
        ++nt;
        // Largest q' in (q, q1] with ptr[q'] <= ptr[q] + TE, and at least q + 1.
        const long long lim = (long long)__ldg(ptr + q) + TE;
        const int x = warp_lower_bound(ptr, q + 1, q1 + 1, lim + 1, lane);
        q = max(q + 1, x - 1);
    }
    if (lane == 0) tiles[nt] = q1;
    return nt;
}

// kDirect: the caller's plain folded CSR/CSC is used as is (no compacted
// lists). Empty rows then pass through the row loop with no entries.
// kBatch: the system is a block-diagonal batch of independent slices, each
// with its own stopping test (per-slice rho, iteration count and done flag).
template <class T, int LPC, bool kDirect = false, bool kBatch = false>
__global__ void __launch_bounds__(1024, 1) sart_stream_kernel(SartArgs<T> a) {
    using Acc = typename T::Acc;
    using V2 = typename T::Vec2;
    using Pair = typename T::Pair;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V2* prod = reinterpret_cast<V2*>(smem_raw);
    __shared__ int s_rt[kMaxTiles + 1];
    __shared__ int s_ct[kMaxTiles + 1];
    __shared__ int s_nrt, s_nct;
    __shared__ double s_red[2][32];
    __shared__ double s_tpp;
    __shared__ int s_stop;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int wib = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int BD = blockDim.x;
    const int TE = a.tile_entries;
    constexpr int kGroupsPerWarp = 32 / LPC;
    const int sub = lane % LPC;
    const Acc lam = (Acc)a.lambda;

    // ---- launch prologue: tiles, and the empty rows' share of ||p||^2 ----
    const int n_nzr = kDirect ? a.direct_rows : a.stats->n_nzr;
    const int n_nzc = kDirect ? a.direct_cols : a.stats->n_nzc;
    const int n_zr = kDirect ? 0 : a.stats->n_zr;
    if (wib == 0) {
        const int nt = plan_tiles(a.nzrp, n_nzr, TE, s_rt, lane);
        if (lane == 0) {
            s_nrt = nt;
            if (nt < 0) record_error(a.ctl, SPLITSART_ERR_ARG, 0);
        }
    } else if (wib == 1) {
        const int nt = plan_tiles(a.nzcp, n_nzc, TE, s_ct, lane);
        if (lane == 0) {
            s_nct = nt;
            if (nt < 0) record_error(a.ctl, SPLITSART_ERR_ARG, 0);
        }
    }
    // ||p||^2 is fixed for the launch: this CTA's share of it over all rows
    // (to partials[2b + 1]), and over the empty rows, whose residual is p.
    double ppz = 0.0;  // meaningful in thread 0 only
    if constexpr (!kBatch) {
        const long long G = gridDim.x, b = blockIdx.x;
        const int z0 = (int)(n_zr * b / G), z1 = (int)(n_zr * (b + 1) / G);
        const long long Mall = kDirect ? a.direct_rows : (long long)n_nzr + n_zr;
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
        if (lane == 0) {
            s_red[0][wib] = tz;
            s_red[1][wib] = ta;
        }
        __syncthreads();
        if (wib == 0) {
            tz = warp_sum(lane < nwarps ? s_red[0][lane] : 0.0);
            ta = warp_sum(lane < nwarps ? s_red[1][lane] : 0.0);
            if (lane == 0) {
                ppz = tz;
                __stcg(a.partials + 2 * blockIdx.x + 1, ta);
            }
        }
    }
    unsigned nbar = 0;
    const int gw = blockIdx.x * nwarps + wib, nw_grid = gridDim.x * nwarps;
    if constexpr (kBatch) {
        // Empty rows keep residual p; each slice's ||p||^2 is summed once.
        const long long Mh = a.sl_rows[a.ns];
        for (int z = blockIdx.x * BD + tid; z < n_zr; z += gridDim.x * BD) {
            const int i = __ldg(a.zr + z);
            const V2 p = ldg(a.p12 + i);
            a.rr_row[i] = (double)p.x * (double)p.x + (double)p.y * (double)p.y;
        }
        for (int sl = gw; sl < a.ns; sl += nw_grid) {
            double t = 0.0;
            for (long long i = __ldg(a.sl_rows + sl) + lane; i < __ldg(a.sl_rows + sl + 1); i += 32) {
                const V2 p = ldg(a.p12 + i);
                t += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
            }
            t = warp_sum(t);
            if (lane == 0) a.sl_solve[sl] = SliceSolve{-1, 0, 0.0, 0.0, t};
        }
        (void)Mh;
    }
    if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
    const int nrt = s_nrt, nct = s_nct;
    if (!kBatch && wib == 0) {
        const double t = grid_total(a.partials, gridDim.x, lane, 1);
        if (lane == 0) s_tpp = t;  // read after later CTA barriers
    }

    for (int k = 0;; ++k) {
        // ---- forward: r = p - A f, u = r / R, and the norm partials ----
        SqAcc<Acc> rr;  // lane 0 of each warp: its rows' ||r||^2
        for (int t = 0; t < nrt; ++t) {
            const int qa = s_rt[t], qb = s_rt[t + 1];
            const int ea = __ldg(a.nzrp + qa), eb = __ldg(a.nzrp + qb);
            const int n = eb - ea;
            const bool staged = n <= TE;
            if (staged) {
                for (int base = 0; base < n; base += BD * kUnroll) {
                    int c[kUnroll];
                    Pair v[kUnroll];
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        const int e = base + u * BD + tid;
                        if (e < n) {
                            c[u] = ldg(a.col + ea + e);
                            v[u] = ldg(a.val + ea + e);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        const int e = base + u * BD + tid;
                        if (e < n) {
                            const V2 fv = ldca(a.f12 + c[u]);
                            Acc a1, a2;
                            T::decode(v[u], a1, a2);
                            prod[e] = V2{a1 * fv.x, a2 * fv.y};
                        }
                    }
                }
                __syncthreads();
            }
            for (int q = qa + wib; q < qb; q += nwarps) {
                const int i = kDirect ? q : __ldg(a.nzr + q);
                const int lo = __ldg(a.nzrp + q) - ea, hi = __ldg(a.nzrp + q + 1) - ea;
                V2 p{};
                typename T::KNorm2 ir{};
                float2 sc{};
                if (lane == 0) {
                    p = ldg(a.p12 + i);
                    ir = ldg(a.invR + i);
                    if constexpr (T::kQuant) sc = ldg(a.scale + i);
                }
                Acc s1 = 0, s2 = 0;
                if (staged) {
                    for (int e = lo + lane; e < hi; e += 32) {
                        const V2 pr = prod[e];
                        s1 += pr.x;
                        s2 += pr.y;
                    }
                } else {
                    // A row longer than a tile: stream it straight from memory.
                    for (int e = lo + lane; e < hi; e += 32) {
                        const V2 fv = ldcg(a.f12 + ldg(a.col + ea + e));
                        Acc a1, a2;
                        T::decode(ldg(a.val + ea + e), a1, a2);
                        s1 += a1 * fv.x;
                        s2 += a2 * fv.y;
                    }
                }
                s1 = warp_sum(s1);
                s2 = warp_sum(s2);
                if (lane == 0) {
                    if constexpr (T::kQuant) {
                        s1 *= sc.x;
                        s2 *= sc.y;
                    }
                    const Acc r1 = p.x - s1, r2 = p.y - s2;
                    // For BF16/FP16, ir already holds the row scale: the back-projection
                    // reuses the codes, so the scale moves into u.
                    const V2 u{r1 * ir.x, r2 * ir.y};
                    stcg(a.u12 + i, u);
                    if constexpr (kBatch) {
                        __stcg(a.rr_row + i, (double)(r1 * r1 + r2 * r2));
                    } else {
                        rr.add(r1, r2);
                    }
                }
            }
            __syncthreads();  // prod is reused by the next tile
        }
        if constexpr (!kBatch) {
            if (lane == 0) s_red[0][wib] = rr.sum();
            __syncthreads();
            if (wib == 0) {
                const double t = warp_sum(lane < nwarps ? s_red[0][lane] : 0.0);
                if (lane == 0) __stcg(a.partials + 2 * blockIdx.x, t + ppz);  // an empty row's residual is its p
            }
        }
        if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;

        const bool last = (k >= a.max_iters);
        if constexpr (kBatch) {
            // ---- per-slice stop tests: one CTA per slice, fixed order ----
            if (last || (k % a.check_every == 0)) slice_stop_tests(a, k, last, s_red[0]);
            if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
            if (ld_volatile(a.ndone) >= a.ns) {
                if (blockIdx.x == 0 && tid == 0) {
                    a.result->iters = k;
                    a.result->status = SPLITSART_OK;
                    a.result->rho = 0.0;
                    a.result->rr = 0.0;
                    a.result->pp = 0.0;
                }
                return;
            }
        } else if (last || (k % a.check_every == 0)) {
            // ---- stop test: every CTA sums the partials in the same order ----
            // One thread decides, so the FP64 division and square root run once per CTA.
            if (wib == 0) {
                const double trr = grid_total(a.partials, gridDim.x, lane, 0);
                if (lane == 0) s_stop = stop_test(a, k, last, trr, s_tpp);
            }
            __syncthreads();
            if (s_stop) return;
        }

        // ---- back-projection and update: f += lambda (A^T u) / C ----
        for (int t = 0; t < nct; ++t) {
            const int qa = s_ct[t], qb = s_ct[t + 1];
            const int ea = __ldg(a.nzcp + qa), eb = __ldg(a.nzcp + qb);
            const int n = eb - ea;
            const bool staged = n <= TE;
            if (staged) {
                for (int base = 0; base < n; base += BD * kUnroll) {
                    int r[kUnroll];
                    Pair v[kUnroll];
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        const int e = base + u * BD + tid;
                        if (e < n) {
                            r[u] = ldg(a.row + ea + e);
                            v[u] = ldg(a.valT + ea + e);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        const int e = base + u * BD + tid;
                        if (e < n) {
                            const V2 uv = ldca(a.u12 + r[u]);
                            Acc a1, a2;
                            T::decode(v[u], a1, a2);
                            prod[e] = V2{a1 * uv.x, a2 * uv.y};
                        }
                    }
                }
                __syncthreads();
            }
            // Warp-uniform loop over groups of columns, so every lane reaches the shuffles.
            for (int qb0 = qa + wib * kGroupsPerWarp; qb0 < qb; qb0 += nwarps * kGroupsPerWarp) {
                const int q = qb0 + lane / LPC;
                Acc b1 = 0, b2 = 0;
                int j = -1;
                if (q < qb) {
                    j = kDirect ? q : __ldg(a.nzc + q);
                    const int lo = __ldg(a.nzcp + q) - ea, hi = __ldg(a.nzcp + q + 1) - ea;
                    if (staged) {
                        for (int e = lo + sub; e < hi; e += LPC) {
                            const V2 pr = prod[e];
                            b1 += pr.x;
                            b2 += pr.y;
                        }
                    } else {
                        for (int e = lo + sub; e < hi; e += LPC) {
                            const V2 uv = ldcg(a.u12 + ldg(a.row + ea + e));
                            Acc a1, a2;
                            T::decode(ldg(a.valT + ea + e), a1, a2);
                            b1 += a1 * uv.x;
                            b2 += a2 * uv.y;
                        }
                    }
                }
                b1 = warp_sum(b1, LPC);
                b2 = warp_sum(b2, LPC);
                bool frozen = false;  // the slice of column j has stopped: keep its returned iterate
                if constexpr (kBatch) {
                    if (sub == 0 && j >= 0) frozen = __ldcg(&a.sl_solve[slice_index(a.sl_cols, a.ns, j)].done) != 0;
                }
                if (sub == 0 && j >= 0 && !frozen) {
                    const typename T::KNorm2 ic = ldg(a.invC + j);
                    V2 f = ldcg(a.f12 + j);
                    f.x += lam * b1 * ic.x;
                    f.y += lam * b2 * ic.y;
                    stcg(a.f12 + j, f);
                }
            }
            __syncthreads();
        }
        if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
    }
}

// ---------------------------------------------------------------------------
// Shared-memory-resident variant, for systems whose per-CTA share fits on chip.
//
// Each CTA copies its part of the folded matrix into shared memory once per
// launch:
// - its rows: a contiguous range of non-empty rows from the host's row plan
//   (balanced by entries plus a fixed weight per row, since a row's fixed
//   cost is of the order of its gathers), or, without a plan, a range
//   balanced by shared-memory bytes;
// - a contiguous range of non-empty columns, balanced by bytes;
// - values, 16-bit indices, and the per-row/column metadata (p, 1/R, 1/C,
//   its own f).
// After that, an iteration's global traffic is only the gathers of f (forward)
// and of u (back), the stores of u and f, and the norm partials.
//
// Inside a CTA:
// - forward: one warp per row, NR rows per warp in flight. Lane l takes the
//   entries l, l + 32, ... of a row; each lane issues up to U gathers per row
//   before it consumes any, then a shuffle tree sums the row. Every lane ends
//   with the sums, and lane k finishes row k of the step (r, u and its store),
//   so the NR rows finish in parallel rather than one after another on lane 0.
// - back: LPC lanes per column, two groups of columns per warp in flight,
//   up to UB gathers per lane and column, then a shuffle tree over the group;
//   the group's lanes 0 and 1 finish its two columns.
// - The stop test of iteration k is decided by one thread per CTA while the
//   first back-projection gathers are in flight.
// The sums have a fixed order, so results are deterministic for a given
// launch shape. The block is at most 512 threads (128 registers each).
// ---------------------------------------------------------------------------

// Shared-memory bytes per entry and per row/column of the resident layout.
template <class T>
struct ResidentBytes {
    static constexpr int kEntry = (int)sizeof(typename T::Pair) + 2;
    static constexpr int kRow = 4 + 4 + (int)sizeof(typename T::Vec2) + (int)sizeof(typename T::KNorm2) +
                                (T::kQuant ? (int)sizeof(float2) : 0);
    static constexpr int kCol = 4 + 4 + (int)sizeof(typename T::KNorm2) + (int)sizeof(typename T::Vec2);
    static constexpr int kThread = 0;
    static constexpr int kSlack = 12 * 16 + 16;  // alignment of 12 segments, plus the end pointers
    static constexpr int kChunk = sizeof(typename T::Vec2) == 16 ? 2 : 4;  // gathers in flight per lane and item
};

// First q in [lo, hi] with WE*ptr[q] + WR*q >= t (a non-decreasing key).
__device__ __forceinline__ int warp_lower_bound_w(const int32_t* ptr, int lo, int hi, long long t, int WE, int WR,
                                                  int lane) {
    while (hi - lo > 32) {
        const int step = (hi - lo + 31) / 32;
        const int idx = lo + lane * step;
        const bool below = idx < hi && (long long)WE * __ldg(ptr + idx) + (long long)WR * idx < t;
        const int c = __popc(__ballot_sync(0xffffffffu, below));
        if (c == 0) return lo;
        const int nlo = lo + (c - 1) * step + 1;
        hi = min(lo + c * step, hi);
        lo = nlo;
    }
    const int idx = lo + lane;
    const bool below = idx < hi && (long long)WE * __ldg(ptr + idx) + (long long)WR * idx < t;
    return lo + __popc(__ballot_sync(0xffffffffu, below));
}

// One warp: this CTA's range [q0, q1) of [0, n), balanced by WE*entries + WR*items.
// One warp: part `part` of `nparts` of [0, n), balanced by WE*entries + WR*items.
__device__ __forceinline__ int2 part_range(const int32_t* ptr, int n, int WE, int WR, long long part, long long nparts,
                                           int lane) {
    const long long total = (long long)WE * __ldg(ptr + n) + (long long)WR * n;
    const int q0 = warp_lower_bound_w(ptr, 0, n, total * part / nparts, WE, WR, lane);
    const int q1 =
        (part == nparts - 1) ? n : warp_lower_bound_w(ptr, 0, n, total * (part + 1) / nparts, WE, WR, lane);
    return make_int2(q0, q1);
}

__device__ __forceinline__ int2 resident_range(const int32_t* ptr, int n, int WE, int WR, int lane) {
    return part_range(ptr, n, WE, WR, blockIdx.x, gridDim.x, lane);
}

__device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Gathers of NI items at once, lane-strided by W: one round issues up to UU
// gathers per item from shared-memory indices, the next consumes them.
template <class T, int NI, int UU>
__device__ __forceinline__ void issue_round(const uint16_t* idx, const typename T::Vec2* src, const int (&lo)[NI],
                                            const int (&hi)[NI], int base, int W, typename T::Vec2 (&g)[NI][UU]) {
#pragma unroll
    for (int k = 0; k < NI; ++k)
#pragma unroll
        for (int u = 0; u < UU; ++u) {
            const int e = lo[k] + base + u * W;
            if (e < hi[k]) g[k][u] = ldca(src + idx[e]);
        }
}
template <class T, int NI, int UU>
__device__ __forceinline__ void consume_round(const typename T::Pair* vals, const int (&lo)[NI], const int (&hi)[NI],
                                              int base, int W, const typename T::Vec2 (&g)[NI][UU],
                                              typename T::Acc (&s1)[NI], typename T::Acc (&s2)[NI]) {
#pragma unroll
    for (int k = 0; k < NI; ++k)
#pragma unroll
        for (int u = 0; u < UU; ++u) {
            const int e = lo[k] + base + u * W;
            if (e < hi[k]) {
                typename T::Acc v1, v2;
                T::decode(vals[e], v1, v2);
                s1[k] += v1 * g[k][u].x;
                s2[k] += v2 * g[k][u].y;
            }
        }
}
// All rounds from `base` on, for the items' remaining entries.
template <class T, int NI, int UU>
__device__ __forceinline__ void gather_rounds(const uint16_t* idx, const typename T::Pair* vals,
                                              const typename T::Vec2* src, const int (&lo)[NI], const int (&hi)[NI],
                                              int first, int base, int W, typename T::Acc (&s1)[NI],
                                              typename T::Acc (&s2)[NI]) {
    int n = 0;
#pragma unroll
    for (int k = 0; k < NI; ++k) n = max(n, hi[k] - lo[k]);
    for (; base - first < n; base += UU * W) {
        typename T::Vec2 g[NI][UU];
        issue_round<T, NI, UU>(idx, src, lo, hi, base, W, g);
        consume_round<T, NI, UU>(vals, lo, hi, base, W, g, s1, s2);
    }
}

template <class T, int LPC>
__global__ void __launch_bounds__(512, 1) sart_resident_kernel(SartArgs<T> a, int smem_bytes) {
    using Acc = typename T::Acc;
    using V2 = typename T::Vec2;
    using N2 = typename T::KNorm2;
    using Pair = typename T::Pair;
    using B = ResidentBytes<T>;
    constexpr int U = B::kChunk;                   // forward: gathers in flight per lane and row
    constexpr int NR = sizeof(V2) == 16 ? 2 : 3;   // forward: rows per warp in flight
    constexpr int UB = sizeof(V2) == 16 ? 4 : 8;   // back: gathers in flight per lane and column
    constexpr int kGroupsPerWarp = 32 / LPC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int2 s_rows, s_cols;
    __shared__ double s_rrw[32];  // per warp: ||r||^2 of its rows
    __shared__ double2 s_pw[32];  // per warp, once: ||p||^2 over the empty rows, and over all rows
    __shared__ double s_tot[2];   // totals over the grid: ||r||^2 (per check), ||p||^2 (once)
    __shared__ int s_stop;
    __shared__ double s_ppz;      // this CTA's ||p||^2 over its share of the empty rows

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int wib = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int BD = blockDim.x;
    const int sub = lane % LPC;
    const Acc lam = (Acc)a.lambda;

    // ---- launch prologue: ranges, shared-memory layout, and the copy-in ----
    const int n_nzr = a.stats->n_nzr, n_nzc = a.stats->n_nzc, n_zr = a.stats->n_zr;
    if (wib == 0) {
        const int2 r = resident_range(a.nzrp, n_nzr, B::kEntry, B::kRow, lane);
        if (lane == 0) s_rows = r;
    } else if (wib == 1) {
        const int2 r = resident_range(a.nzcp, n_nzc, B::kEntry, B::kCol, lane);
        if (lane == 0) s_cols = r;
    }
    __syncthreads();
    // Rows: the host's plan (contiguous ranges balanced by time), or a range
    // balanced by bytes.
    const bool planned = a.res_rows != nullptr;
    const int rg0 = planned ? __ldg(a.res_off + blockIdx.x) : 0;
    const int q0 = planned ? 0 : s_rows.x;
    const int nr = planned ? __ldg(a.res_off + blockIdx.x + 1) - rg0 : s_rows.y - s_rows.x;
    const int32_t* loc = planned ? a.res_loc + rg0 + blockIdx.x : nullptr;
    auto row_pos = [&](int q) { return planned ? __ldg(a.res_rows + rg0 + q) : q0 + q; };  // compacted position
    const int c0 = s_cols.x, nc = s_cols.y - s_cols.x;
    const int fea = planned ? 0 : __ldg(a.nzrp + q0);
    const int nfe = planned ? __ldg(loc + nr) : __ldg(a.nzrp + q0 + nr) - fea;
    const int bea = __ldg(a.nzcp + c0), nbe = __ldg(a.nzcp + c0 + nc) - bea;

    size_t off = 0;
    Pair* f_val = reinterpret_cast<Pair*>(smem_raw + off);
    off = align16(off + sizeof(Pair) * nfe);
    uint16_t* f_idx = reinterpret_cast<uint16_t*>(smem_raw + off);
    off = align16(off + 2 * (size_t)nfe);
    int* r_ptr = reinterpret_cast<int*>(smem_raw + off);
    off = align16(off + 4 * (size_t)(nr + 1));
    int* r_id = reinterpret_cast<int*>(smem_raw + off);
    off = align16(off + 4 * (size_t)nr);
    V2* r_p = reinterpret_cast<V2*>(smem_raw + off);
    off = align16(off + sizeof(V2) * nr);
    N2* r_ir = reinterpret_cast<N2*>(smem_raw + off);
    off = align16(off + sizeof(N2) * nr);
    float2* r_sc = reinterpret_cast<float2*>(smem_raw + off);
    off = align16(off + (T::kQuant ? sizeof(float2) * nr : 0));
    Pair* b_val = reinterpret_cast<Pair*>(smem_raw + off);
    off = align16(off + sizeof(Pair) * nbe);
    uint16_t* b_idx = reinterpret_cast<uint16_t*>(smem_raw + off);
    off = align16(off + 2 * (size_t)nbe);
    int* c_ptr = reinterpret_cast<int*>(smem_raw + off);
    off = align16(off + 4 * (size_t)(nc + 1));
    int* c_id = reinterpret_cast<int*>(smem_raw + off);
    off = align16(off + 4 * (size_t)nc);
    N2* c_ic = reinterpret_cast<N2*>(smem_raw + off);
    off = align16(off + sizeof(N2) * nc);
    V2* c_f = reinterpret_cast<V2*>(smem_raw + off);
    off = align16(off + sizeof(V2) * nc);

    if (off > (size_t)smem_bytes) {
        // Cannot happen when the host's bound holds; fail cleanly rather than overrun.
        if (tid == 0) record_error(a.ctl, SPLITSART_ERR_ARG, 0);
        grid_sync(a.ctl, a.expected, a.timeout_ns, 1);
        return;
    }
    if (planned) {
        for (int q = wib; q < nr; q += nwarps) {  // one warp per row
            const int src = __ldg(a.nzrp + row_pos(q)), len = __ldg(a.nzrp + row_pos(q) + 1) - src;
            const int dst = __ldg(loc + q);
            for (int t = lane; t < len; t += 32) {
                f_val[dst + t] = ldg(a.val + src + t);
                f_idx[dst + t] = (uint16_t)__ldg(a.col + src + t);
            }
        }
    } else {
        for (int e = tid; e < nfe; e += BD) {
            f_val[e] = ldg(a.val + fea + e);
            f_idx[e] = (uint16_t)__ldg(a.col + fea + e);
        }
    }
    for (int q = tid; q < nr; q += BD) {
        const int i = __ldg(a.nzr + row_pos(q));
        r_ptr[q] = planned ? __ldg(loc + q) : __ldg(a.nzrp + q0 + q) - fea;
        r_id[q] = i;
        r_p[q] = ldg(a.p12 + i);
        r_ir[q] = ldg(a.invR + i);
        if constexpr (T::kQuant) r_sc[q] = ldg(a.scale + i);
    }
    if (tid == 0) r_ptr[nr] = nfe;
    for (int e = tid; e < nbe; e += BD) {
        b_val[e] = ldg(a.valT + bea + e);
        b_idx[e] = (uint16_t)__ldg(a.row + bea + e);
    }
    for (int q = tid; q < nc; q += BD) {
        const int j = __ldg(a.nzc + c0 + q);
        c_ptr[q] = __ldg(a.nzcp + c0 + q) - bea;
        c_id[q] = j;
        c_ic[q] = ldg(a.invC + j);
        c_f[q] = ldcg(a.f12 + j);
    }
    if (tid == 0) c_ptr[nc] = nbe;
    // ||p||^2 is fixed for the launch. This CTA's share over its empty rows
    // (whose residual is p) and over all of its rows, summed once.
    {
        const long long G = gridDim.x, b = blockIdx.x;
        const int z0 = (int)(n_zr * b / G), z1 = (int)(n_zr * (b + 1) / G);
        double tz = 0.0, ta = 0.0;
        for (int z = z0 + tid; z < z1; z += BD) {
            const V2 p = ldg(a.p12 + __ldg(a.zr + z));
            tz += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
        }
        for (int q = tid; q < nr; q += BD) {
            const V2 p = ldg(a.p12 + __ldg(a.nzr + row_pos(q)));
            ta += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
        }
        ta += tz;
        tz = warp_sum(tz);
        ta = warp_sum(ta);
        if (lane == 0) s_pw[wib] = make_double2(tz, ta);
        __syncthreads();
        if (wib == 0) {
            const double2 v = lane < nwarps ? s_pw[lane] : make_double2(0.0, 0.0);
            const double t0 = warp_sum(v.x), t1 = warp_sum(v.y);
            if (lane == 0) {
                s_ppz = t0;
                __stcg(a.partials + 2 * blockIdx.x + 1, t1);
            }
        }
    }
    unsigned nbar = 0;
    if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
    if (wib == 0) {
        const double t = grid_total(a.partials, gridDim.x, lane, 1);
        if (lane == 0) s_tot[1] = t;  // read after later CTA barriers
    }
    const double ppz = s_ppz;

    for (int k = 0;; ++k) {
        // ---- forward: r = p - A f, u = r / R, and the norm partials ----
        SqAcc<Acc> rr;  // per lane: the ||r||^2 of the rows it finished
        auto fin_row = [&](int q, Acc s1, Acc s2) {
            const V2 p = r_p[q];
            const N2 ir = r_ir[q];
            if constexpr (T::kQuant) {
                const float2 sc = r_sc[q];
                s1 *= sc.x;
                s2 *= sc.y;
            }
            const Acc r1 = p.x - s1, r2 = p.y - s2;
            // For BF16/FP16, ir already holds the row scale: the back-projection
            // reuses the codes, so the scale moves into u.
            stcg(a.u12 + r_id[q], V2{r1 * ir.x, r2 * ir.y});
            rr.add(r1, r2);
        };
        // NR rows per warp in flight: q, q + nwarps, q + 2 nwarps, ...
        for (int q = wib; q < nr; q += NR * nwarps) {
            int lo[NR], hi[NR];
            Acc s1[NR], s2[NR];
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const int qk = q + k * nwarps;
                lo[k] = qk < nr ? r_ptr[qk] : 0;
                hi[k] = qk < nr ? r_ptr[qk + 1] : 0;
                s1[k] = 0;
                s2[k] = 0;
            }
            gather_rounds<T, NR, U>(f_idx, f_val, a.f12, lo, hi, lane, lane, 32, s1, s2);
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                s1[k] = warp_sum(s1[k]);
                s2[k] = warp_sum(s2[k]);
            }
            // Every lane holds the sums: lane k finishes row q + k nwarps.
            if (lane < NR) {
                Acc t1 = s1[0], t2 = s2[0];
#pragma unroll
                for (int k = 1; k < NR; ++k)
                    if (lane == k) {
                        t1 = s1[k];
                        t2 = s2[k];
                    }
                if (q + lane * nwarps < nr) fin_row(q + lane * nwarps, t1, t2);
            }
        }
        const bool last = (k >= a.max_iters);
        const bool check = last || (k % a.check_every == 0);
        if (check) {  // the CTA's ||r||^2, only where the stop test reads it (uniform over the grid)
            const double tw = warp_sum(rr.sum());
            if (lane == 0) s_rrw[wib] = tw;
            __syncthreads();
            if (wib == 0) {
                const double t = warp_sum(lane < nwarps ? s_rrw[lane] : 0.0);
                if (lane == 0) __stcg(a.partials + 2 * blockIdx.x, t + ppz);  // an empty row's residual is its p
            }
        }
        if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;

        // ---- back-projection; the stop test reads its totals while the first gathers fly ----
        auto fin_col = [&](int q, Acc b1, Acc b2) {
            const N2 ic = c_ic[q];
            V2 f = c_f[q];
            f.x += lam * b1 * ic.x;
            f.y += lam * b2 * ic.y;
            c_f[q] = f;
            stcg(a.f12 + c_id[q], f);
        };
        const int stride = 2 * nwarps * kGroupsPerWarp;
        bool first_pass = true;
        for (int g0 = wib * kGroupsPerWarp; g0 < nc || first_pass; g0 += stride) {
            const int qA = g0 + lane / LPC, qB = qA + nwarps * kGroupsPerWarp;
            const int lo[2] = {qA < nc ? c_ptr[qA] : 0, qB < nc ? c_ptr[qB] : 0};
            const int hi[2] = {qA < nc ? c_ptr[qA + 1] : 0, qB < nc ? c_ptr[qB + 1] : 0};
            V2 g[2][UB];
            issue_round<T, 2, UB>(b_idx, a.u12, lo, hi, sub, LPC, g);
            if (first_pass) {
                first_pass = false;
                if (check) {  // uniform over the CTA
                    // One thread decides, so the FP64 division and square root run once per CTA.
                    if (wib == 0) {
                        const double trr = grid_total(a.partials, gridDim.x, lane, 0);
                        if (lane == 0) s_stop = stop_test(a, k, last, trr, s_tot[1]);
                    }
                    __syncthreads();
                    if (s_stop) return;
                }
                if (g0 >= nc) break;  // uniform within the warp
            }
            Acc b1[2] = {0, 0}, b2[2] = {0, 0};
            consume_round<T, 2, UB>(b_val, lo, hi, sub, LPC, g, b1, b2);
            gather_rounds<T, 2, UB>(b_idx, b_val, a.u12, lo, hi, sub, sub + UB * LPC, LPC, b1, b2);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                b1[k] = warp_sum(b1[k], LPC);
                b2[k] = warp_sum(b2[k], LPC);
            }
            if constexpr (LPC == 1) {
                if (qA < nc) fin_col(qA, b1[0], b2[0]);
                if (qB < nc) fin_col(qB, b1[1], b2[1]);
            } else {  // every lane of the group holds the sums: two lanes finish the two columns
                if (sub == 0 && qA < nc) fin_col(qA, b1[0], b2[0]);
                if (sub == 1 && qB < nc) fin_col(qB, b1[1], b2[1]);
            }
        }
        if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
    }
}

// ---------------------------------------------------------------------------
// Row-streaming variant, for systems far larger than on-chip memory (the
// batch of slices).
//
// The matrix is streamed from HBM once per pass, so the kernel must keep
// enough loads in flight to cover DRAM latency. It has no CTA barriers
// inside a pass:
// - Work is scheduled dynamically. A warp takes the next chunk of 16
//   non-empty rows (or 8 x 32/LPC non-empty columns) from a global counter,
//   fetched one chunk ahead, so no warp waits at the pass's end for a slow
//   static share. Chunks go out in order, so the warps of the grid work on
//   neighbouring rows and the gathered vector stays hot in L2.
// - Within a chunk a warp takes two adjacent rows at a time. Each lane first
//   issues the index and value loads of up to U entries of both rows, then
//   the U gathers, then the products; a row longer than 32 U entries
//   continues in further rounds.
// - The back-projection is the same over the CSC with LPC lanes per column
//   and two groups of columns per warp.
// Matrix loads use the streaming cache hint (read once per pass). Per-row
// sums use the same lane-strided order and shuffle tree as the other
// kernels, so f does not depend on the grid or the schedule. The FP32 group
// sums of ||r||^2 do, so rho may differ in its last bits between runs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ldcs(const int32_t* p) { return __ldcs(p); }
__device__ __forceinline__ float2 ldcs(const float2* p) { return __ldcs(p); }
__device__ __forceinline__ double2 ldcs(const double2* p) { return __ldcs(p); }
__device__ __forceinline__ __nv_bfloat162 ldcs(const __nv_bfloat162* p) {
    unsigned v = __ldcs(reinterpret_cast<const unsigned*>(p));
    return *reinterpret_cast<__nv_bfloat162*>(&v);
}
__device__ __forceinline__ __half2 ldcs(const __half2* p) {
    unsigned v = __ldcs(reinterpret_cast<const unsigned*>(p));
    return *reinterpret_cast<__half2*>(&v);
}

// UF: entries in flight per lane and row (two rows per warp step). UB: per
// lane and column; with UB > 6 each lane group takes one column per step,
// otherwise two.
template <class T, int LPC, bool kBatch, int UF, int UB>
__global__ void __launch_bounds__(512, 1) sart_rows_kernel(SartArgs<T> a) {
    using Acc = typename T::Acc;
    using V2 = typename T::Vec2;
    using N2 = typename T::KNorm2;
    using Pair = typename T::Pair;
    constexpr bool kOneCol = UB > 6;
    constexpr int kGroupsPerWarp = 32 / LPC;
    constexpr int kRowChunk = 16;  // rows per scheduled chunk
    __shared__ double s_red[2][32];
    __shared__ double s_tpp;
    __shared__ int s_stop;

    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5, nwarps = blockDim.x >> 5, BD = blockDim.x;
    const int sub = lane % LPC;
    const Acc lam = (Acc)a.lambda;
    const int n_nzr = a.stats->n_nzr, n_nzc = a.stats->n_nzc, n_zr = a.stats->n_zr;

    // ---- launch prologue: the fixed ||p||^2 terms ----
    double ppz = 0.0;  // meaningful in thread 0 only
    const int gw = blockIdx.x * nwarps + wib, nw_grid = gridDim.x * nwarps;
    if constexpr (kBatch) {
        // Empty rows keep residual p; each slice's ||p||^2 is summed once.
        for (int z = blockIdx.x * BD + tid; z < n_zr; z += gridDim.x * BD) {
            const int i = __ldg(a.zr + z);
            const V2 p = ldg(a.p12 + i);
            a.rr_row[i] = (double)p.x * (double)p.x + (double)p.y * (double)p.y;
        }
        for (int sl = gw; sl < a.ns; sl += nw_grid) {
            double t = 0.0;
            for (long long i = __ldg(a.sl_rows + sl) + lane; i < __ldg(a.sl_rows + sl + 1); i += 32) {
                const V2 p = ldg(a.p12 + i);
                t += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
            }
            t = warp_sum(t);
            if (lane == 0) a.sl_solve[sl] = SliceSolve{-1, 0, 0.0, 0.0, t};
        }
    } else {
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
        if (lane == 0) {
            s_red[0][wib] = tz;
            s_red[1][wib] = ta;
        }
        __syncthreads();
        if (wib == 0) {
            tz = warp_sum(lane < nwarps ? s_red[0][lane] : 0.0);
            ta = warp_sum(lane < nwarps ? s_red[1][lane] : 0.0);
            if (lane == 0) {
                ppz = tz;
                __stcg(a.partials + 2 * blockIdx.x + 1, ta);
            }
        }
    }
    unsigned nbar = 0;
    if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
    if (!kBatch && wib == 0) {
        const double t = grid_total(a.partials, gridDim.x, lane, 1);
        if (lane == 0) s_tpp = t;  // read after later CTA barriers
    }
    // Rounds over one or two items: each lane issues the index and value loads
    // of up to UU entries per item (lane-strided by W), then their gathers,
    // then the products. UC is std::integral_constant<int, UU>.
    auto two_items = [&](auto UC, const int32_t* idx, const Pair* vals, const V2* src, int loA, int hiA, int loB,
                         int hiB, int first, int W, Acc& sA1, Acc& sA2, Acc& sB1, Acc& sB2) {
        constexpr int UU = decltype(UC)::value;
        const int nA = hiA - loA, nB = hiB - loB, n = nA > nB ? nA : nB;
        for (int base = first; base - first < n; base += UU * W) {
            int ixA[UU], ixB[UU];
            Pair vA[UU], vB[UU];
            V2 gA[UU], gB[UU];
#pragma unroll
            for (int u = 0; u < UU; ++u) {
                const int eA = loA + base + u * W, eB = loB + base + u * W;
                if (eA < hiA) {
                    ixA[u] = ldcs(idx + eA);
                    vA[u] = ldcs(vals + eA);
                }
                if (eB < hiB) {
                    ixB[u] = ldcs(idx + eB);
                    vB[u] = ldcs(vals + eB);
                }
            }
#pragma unroll
            for (int u = 0; u < UU; ++u) {
                if (loA + base + u * W < hiA) gA[u] = ldca(src + ixA[u]);
                if (loB + base + u * W < hiB) gB[u] = ldca(src + ixB[u]);
            }
#pragma unroll
            for (int u = 0; u < UU; ++u) {
                Acc v1, v2;
                if (loA + base + u * W < hiA) {
                    T::decode(vA[u], v1, v2);
                    sA1 += v1 * gA[u].x;
                    sA2 += v2 * gA[u].y;
                }
                if (loB + base + u * W < hiB) {
                    T::decode(vB[u], v1, v2);
                    sB1 += v1 * gB[u].x;
                    sB2 += v2 * gB[u].y;
                }
            }
        }
    };
    auto one_item = [&](auto UC, const int32_t* idx, const Pair* vals, const V2* src, int lo, int hi, int first, int W,
                        Acc& s1, Acc& s2) {
        constexpr int UU = decltype(UC)::value;
        for (int base = first; base - first < hi - lo; base += UU * W) {
            int ix[UU];
            Pair v[UU];
            V2 g[UU];
#pragma unroll
            for (int u = 0; u < UU; ++u) {
                const int e = lo + base + u * W;
                if (e < hi) {
                    ix[u] = ldcs(idx + e);
                    v[u] = ldcs(vals + e);
                }
            }
#pragma unroll
            for (int u = 0; u < UU; ++u)
                if (lo + base + u * W < hi) g[u] = ldca(src + ix[u]);
#pragma unroll
            for (int u = 0; u < UU; ++u) {
                if (lo + base + u * W < hi) {
                    Acc v1, v2;
                    T::decode(v[u], v1, v2);
                    s1 += v1 * g[u].x;
                    s2 += v2 * g[u].y;
                }
            }
        }
    };
    constexpr std::integral_constant<int, UF> kUF{};
    constexpr std::integral_constant<int, UB> kUB{};

    for (int k = 0;; ++k) {
        // ---- forward: r = p - A f, u = r / R, and the norm partials ----
        SqAcc<Acc> rr;  // lane 0 of each warp: its rows' ||r||^2
        auto fin_row = [&](int q, Acc s1, Acc s2) {
            const int i = __ldg(a.nzr + q);
            const V2 p = ldg(a.p12 + i);
            const N2 ir = ldg(a.invR + i);
            if constexpr (T::kQuant) {
                const float2 sc = ldg(a.scale + i);
                s1 *= sc.x;
                s2 *= sc.y;
            }
            const Acc r1 = p.x - s1, r2 = p.y - s2;
            // For BF16/FP16, ir already holds the row scale: the back-projection
            // reuses the codes, so the scale moves into u.
            stcg(a.u12 + i, V2{r1 * ir.x, r2 * ir.y});
            if constexpr (kBatch) __stcg(a.rr_row + i, (double)(r1 * r1 + r2 * r2));
            else rr.add(r1, r2);
        };
        if (blockIdx.x == 0 && tid == 0) a.ctl->work[1] = 0;  // the back pass's counter, idle until the barrier
        int grab = 0;  // lane 0: the next chunk, fetched one chunk ahead
        if (lane == 0) grab = atomicAdd(&a.ctl->work[0], 1u);
        for (int chunk = __shfl_sync(0xffffffffu, grab, 0); chunk < (n_nzr + kRowChunk - 1) / kRowChunk;
             chunk = __shfl_sync(0xffffffffu, grab, 0)) {
            if (lane == 0) grab = atomicAdd(&a.ctl->work[0], 1u);
            const int q1 = min((chunk + 1) * kRowChunk, n_nzr);
            for (int q = chunk * kRowChunk; q < q1; q += 2) {
                const bool hasB = q + 1 < q1;
                const int loA = __ldg(a.nzrp + q), hiA = __ldg(a.nzrp + q + 1);
                const int hiB = hasB ? __ldg(a.nzrp + q + 2) : hiA;
                Acc sA1 = 0, sA2 = 0, sB1 = 0, sB2 = 0;
                two_items(kUF, a.col, a.val, a.f12, loA, hiA, hiA, hiB, lane, 32, sA1, sA2, sB1, sB2);
                sA1 = warp_sum(sA1);
                sA2 = warp_sum(sA2);
                sB1 = warp_sum(sB1);
                sB2 = warp_sum(sB2);
                if (lane == 0) {
                    fin_row(q, sA1, sA2);
                    if (hasB) fin_row(q + 1, sB1, sB2);
                }
            }
        }
        if constexpr (!kBatch) {
            if (lane == 0) s_red[0][wib] = rr.sum();
            __syncthreads();
            if (wib == 0) {
                const double t = warp_sum(lane < nwarps ? s_red[0][lane] : 0.0);
                if (lane == 0) __stcg(a.partials + 2 * blockIdx.x, t + ppz);  // an empty row's residual is its p
            }
        }
        if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;

        const bool last = (k >= a.max_iters);
        if constexpr (kBatch) {
            // ---- per-slice stop tests: one CTA per slice, fixed order ----
            if (last || (k % a.check_every == 0)) slice_stop_tests(a, k, last, s_red[0]);
            if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
            if (ld_volatile(a.ndone) >= a.ns) {
                if (blockIdx.x == 0 && tid == 0) {
                    a.result->iters = k;
                    a.result->status = SPLITSART_OK;
                    a.result->rho = 0.0;
                    a.result->rr = 0.0;
                    a.result->pp = 0.0;
                }
                return;
            }
        } else if (last || (k % a.check_every == 0)) {
            // ---- stop test: every CTA sums the partials in the same order ----
            // One thread decides, so the FP64 division and square root run once per CTA.
            if (wib == 0) {
                const double trr = grid_total(a.partials, gridDim.x, lane, 0);
                if (lane == 0) s_stop = stop_test(a, k, last, trr, s_tpp);
            }
            __syncthreads();
            if (s_stop) return;
        }

        // ---- back-projection and update: f += lambda (A^T u) / C ----
        // A lane's columns increase (chunks are handed out in order), so its
        // slice is found by walking forward.
        int sl = 0;
        auto fin_col = [&](int q, Acc b1, Acc b2) {
            const int j = __ldg(a.nzc + q);
            if constexpr (kBatch) {
                while (j >= __ldg(a.sl_cols + sl + 1)) ++sl;
                if (__ldcg(&a.sl_solve[sl].done)) return;  // the slice has stopped: keep its returned iterate
            }
            const N2 ic = ldg(a.invC + j);
            V2 f = ldcg(a.f12 + j);
            f.x += lam * b1 * ic.x;
            f.y += lam * b2 * ic.y;
            stcg(a.f12 + j, f);
        };
        if (blockIdx.x == 0 && tid == 0) a.ctl->work[0] = 0;  // the forward pass's counter, idle until the barrier
        constexpr int kColsPerStep = (kOneCol ? 1 : 2) * kGroupsPerWarp;
        constexpr int kColChunk = 8 * kGroupsPerWarp;
        if (lane == 0) grab = atomicAdd(&a.ctl->work[1], 1u);
        for (int chunk = __shfl_sync(0xffffffffu, grab, 0); chunk < (n_nzc + kColChunk - 1) / kColChunk;
             chunk = __shfl_sync(0xffffffffu, grab, 0)) {
            if (lane == 0) grab = atomicAdd(&a.ctl->work[1], 1u);
            const int c1 = min((chunk + 1) * kColChunk, n_nzc);
            // Warp-uniform loop over steps of column groups, so every lane reaches the shuffles.
            for (int g0 = chunk * kColChunk; g0 < c1; g0 += kColsPerStep) {
                if constexpr (kOneCol) {
                    const int q = g0 + lane / LPC;
                    const int lo = q < c1 ? __ldg(a.nzcp + q) : 0, hi = q < c1 ? __ldg(a.nzcp + q + 1) : 0;
                    Acc b1 = 0, b2 = 0;
                    one_item(kUB, a.row, a.valT, a.u12, lo, hi, sub, LPC, b1, b2);
                    b1 = warp_sum(b1, LPC);
                    b2 = warp_sum(b2, LPC);
                    if (sub == 0 && q < c1) fin_col(q, b1, b2);
                    continue;
                }
                const int qA = g0 + lane / LPC, qB = qA + kGroupsPerWarp;
                const int loA = qA < c1 ? __ldg(a.nzcp + qA) : 0, hiA = qA < c1 ? __ldg(a.nzcp + qA + 1) : 0;
                const int loB = qB < c1 ? __ldg(a.nzcp + qB) : 0, hiB = qB < c1 ? __ldg(a.nzcp + qB + 1) : 0;
                Acc bA1 = 0, bA2 = 0, bB1 = 0, bB2 = 0;
                two_items(kUB, a.row, a.valT, a.u12, loA, hiA, loB, hiB, sub, LPC, bA1, bA2, bB1, bB2);
                bA1 = warp_sum(bA1, LPC);
                bA2 = warp_sum(bA2, LPC);
                bB1 = warp_sum(bB1, LPC);
                bB2 = warp_sum(bB2, LPC);
                if (sub == 0) {
                    if (qA < c1) fin_col(qA, bA1, bA2);
                    if (qB < c1) fin_col(qB, bB1, bB2);
                }
            }
        }
        if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
    }
}

// ---------------------------------------------------------------------------
// Bulk-staged streaming, for systems far larger than on-chip memory.
//
// Every warp of the grid owns a contiguous range of non-empty rows and one
// of non-empty columns, balanced by bytes. It walks each range in jobs of
// two rows (forward) or 2 x 32/LPC columns (back).
// - A job's indices and values are staged into one of the warp's two
//   shared-memory slots by bulk asynchronous copies (cp.async.bulk),
//   completed on the slot's mbarrier.
// - The copy of job j + 1 is issued before job j is processed, and the
//   pointers and metadata (p, 1/R and the row scale; or f and 1/C) of later
//   jobs load meanwhile. The matrix stream therefore never waits for the
//   warp's gathers, and registers hold only the gathers in flight.
// - A job larger than a slot is read straight from global memory.
// Warps never wait for one another inside a pass: the only CTA-wide
// synchronisation is the grid barrier between passes. Each row and column
// sum has the same lane-strided order and shuffle tree as in the other
// kernels.
// ---------------------------------------------------------------------------
template <class T, int LPC, bool kBatch>
__global__ void __launch_bounds__(384, 1) sart_bulk_kernel(SartArgs<T> a, int te) {
    using Acc = typename T::Acc;
    using V2 = typename T::Vec2;
    using N2 = typename T::KNorm2;
    using Pair = typename T::Pair;
    // Gathers in flight per lane and item: for staged jobs, and for jobs read from global memory.
    constexpr std::integral_constant<int, sizeof(V2) == 16 ? 2 : 8> kUS{};
    constexpr std::integral_constant<int, 2> kUD{};
    constexpr int kEB = 4 + (int)sizeof(Pair);  // staged bytes per entry
    constexpr int GPW = 32 / LPC;                // column groups per warp
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar[16][2];
    __shared__ double s_red[2][32];
    __shared__ double s_tpp;
    __shared__ int s_stop;

    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5, nwarps = blockDim.x >> 5, BD = blockDim.x;
    const int sub = lane % LPC;
    const Acc lam = (Acc)a.lambda;
    const int n_nzr = a.stats->n_nzr, n_nzc = a.stats->n_nzc, n_zr = a.stats->n_zr;
    const int cap = te + 8;  // entries per slot: a tile plus the 16-byte alignment of both ends
    unsigned char* wslots = smem_raw + (size_t)wib * 2 * cap * kEB;
    uint64_t* bar = s_bar[wib];
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    unsigned phase = 0;     // bit s: parity of slot s's next completion
    unsigned inflight = 0;  // bit s: a copy into slot s was issued and not yet waited for

    // ---- launch prologue: ranges, and the fixed ||p||^2 terms ----
    const int gw = blockIdx.x * nwarps + wib, nw_grid = gridDim.x * nwarps;
    const int2 rrange = part_range(a.nzrp, n_nzr, 12, 32, gw, nw_grid, lane);
    const int2 crange = part_range(a.nzcp, n_nzc, 12, 32, gw, nw_grid, lane);
    double ppz = 0.0;  // meaningful in thread 0 only
    if constexpr (kBatch) {
        for (int z = blockIdx.x * BD + tid; z < n_zr; z += gridDim.x * BD) {
            const int i = __ldg(a.zr + z);
            const V2 p = ldg(a.p12 + i);
            a.rr_row[i] = (double)p.x * (double)p.x + (double)p.y * (double)p.y;
        }
        for (int sl = gw; sl < a.ns; sl += nw_grid) {
            double t = 0.0;
            for (long long i = __ldg(a.sl_rows + sl) + lane; i < __ldg(a.sl_rows + sl + 1); i += 32) {
                const V2 p = ldg(a.p12 + i);
                t += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
            }
            t = warp_sum(t);
            if (lane == 0) a.sl_solve[sl] = SliceSolve{-1, 0, 0.0, 0.0, t};
        }
    } else {
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
        if (lane == 0) {
            s_red[0][wib] = tz;
            s_red[1][wib] = ta;
        }
        __syncthreads();
        if (wib == 0) {
            tz = warp_sum(lane < nwarps ? s_red[0][lane] : 0.0);
            ta = warp_sum(lane < nwarps ? s_red[1][lane] : 0.0);
            if (lane == 0) {
                ppz = tz;
                __stcg(a.partials + 2 * blockIdx.x + 1, ta);
            }
        }
    }
    unsigned nbar = 0;
    if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
    if (!kBatch && wib == 0) {
        const double t = grid_total(a.partials, gridDim.x, lane, 1);
        if (lane == 0) s_tpp = t;  // read after later CTA barriers
    }
    int sl_first = 0;  // the slice of this warp's first column
    if constexpr (kBatch) {
        if (crange.x < crange.y) sl_first = slice_index(a.sl_cols, a.ns, __ldg(a.nzc + crange.x));
    }

    // ---- jobs and their staging (warp-uniform) ----
    // A job is J consecutive items of this warp's range: two rows (forward) or
    // two column groups of GPW columns each (back). Lane k < J + 1 holds the
    // job's pointer ptr[q + k] (clamped at the job's end), so every bound is
    // one shuffle away. Jobs are pipelined three deep:
    //   job j + 2: pointers and the first level of metadata (row or column index) load;
    //   job j + 1: its bulk copy is issued and its remaining metadata loads;
    //   job j:     waits for its copy and is processed.
    auto load_ptrs = [&](const int32_t* ptr, int q, int qe) { return __ldg(ptr + min(q + lane, qe)); };
    auto issue = [&](const int32_t* idx, const Pair* vals, int s, int lo, int hi) {
        if (lane == 0) {
            unsigned char* slot = wslots + (size_t)s * cap * kEB;
            const unsigned nbi = 4u * (unsigned)(hi - lo), nbv = (unsigned)sizeof(Pair) * (unsigned)(hi - lo);
            fence_proxy_async_smem();
            mbar_expect_tx(&bar[s], nbi + nbv);
            bulk_g2s(slot, idx + lo, nbi, &bar[s]);
            bulk_g2s(slot + (size_t)cap * 4, vals + lo, nbv, &bar[s]);
        }
        inflight |= 1u << s;
    };
    // Wait (bounded) for every copy still in flight; used before leaving on an error.
    auto drain = [&]() {
        for (int s = 0; s < 2; ++s)
            if (inflight & (1u << s)) mbar_wait_bounded(&bar[s], (phase >> s) & 1u, a.timeout_ns);
        inflight = 0;
    };
    // Sums of two items' entries [loA, hiA) and [loB, hiB) (already offset), lane-strided by W.
    // UC is std::integral_constant<int, gathers in flight per lane and item>.
    auto two_items = [&](auto UC, const int32_t* idx, const Pair* vals, const V2* src, int loA, int hiA, int loB,
                         int hiB, int first, int W, Acc& sA1, Acc& sA2, Acc& sB1, Acc& sB2) {
        constexpr int U = decltype(UC)::value;
        const int nA = hiA - loA, nB = hiB - loB, n = nA > nB ? nA : nB;
        for (int base = first; base - first < n; base += U * W) {
            V2 gA[U], gB[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int eA = loA + base + u * W, eB = loB + base + u * W;
                if (eA < hiA) gA[u] = ldca(src + idx[eA]);
                if (eB < hiB) gB[u] = ldca(src + idx[eB]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int eA = loA + base + u * W, eB = loB + base + u * W;
                Acc v1, v2;
                if (eA < hiA) {
                    T::decode(vals[eA], v1, v2);
                    sA1 += v1 * gA[u].x;
                    sA2 += v2 * gA[u].y;
                }
                if (eB < hiB) {
                    T::decode(vals[eB], v1, v2);
                    sB1 += v1 * gB[u].x;
                    sB2 += v2 * gB[u].y;
                }
            }
        }
    };
    // One pass over the items [r0, r1). Meta is the per-item metadata one lane holds.
    //   first(q, qe)        -> the first-level metadata load for job [q, qe) (returns an int);
    //   second(q, qe, lvl1) -> the remaining metadata of the job (returns Meta);
    //   body(q, qe, pv, soff, off, meta) processes the job. With soff >= 0 the job is
    //   staged at byte soff of shared memory (entry e at position e - off); with
    //   soff < 0 it is read from global memory.
    // Returns false if a copy timed out.
    auto run_pass = [&](const int32_t* ptr, const int32_t* idx, const Pair* vals, int r0, int r1, int J,
                        auto&& first, auto&& second, auto&& body) {
        if (r0 >= r1) return true;
        int slot = 0;
        // Job 0: pointers, copy and metadata, synchronously.
        int q = r0, qe = min(q + J, r1);
        int pv = load_ptrs(ptr, q, qe);
        int lo = __shfl_sync(0xffffffffu, pv, 0) & ~3, hi = (__shfl_sync(0xffffffffu, pv, qe - q) + 3) & ~3;
        bool st = hi - lo <= cap;
        if (st) issue(idx, vals, slot, lo, hi);
        auto meta = second(q, qe, first(q, qe));
        // Job 1: pointers and first-level metadata.
        int nq = qe, nqe = min(nq + J, r1);
        int npv = nq < r1 ? load_ptrs(ptr, nq, nqe) : 0;
        int nl1 = nq < r1 ? first(nq, nqe) : 0;
        while (q < r1) {
            // Job j + 1: copy and remaining metadata.
            bool nst = false;
            int nlo = 0;
            decltype(meta) nmeta{};
            if (nq < r1) {
                nlo = __shfl_sync(0xffffffffu, npv, 0) & ~3;
                const int nhi = (__shfl_sync(0xffffffffu, npv, nqe - nq) + 3) & ~3;
                nst = nhi - nlo <= cap;
                if (nst) issue(idx, vals, slot ^ 1, nlo, nhi);
                nmeta = second(nq, nqe, nl1);
            }
            // Job j + 2: pointers and first-level metadata.
            const int nnq = nqe, nnqe = min(nnq + J, r1);
            const int nnpv = nnq < r1 ? load_ptrs(ptr, nnq, nnqe) : 0;
            const int nnl1 = nnq < r1 ? first(nnq, nnqe) : 0;
            // Job j.
            if (st) {
                if (!mbar_wait_bounded(&bar[slot], (phase >> slot) & 1u, a.timeout_ns)) {
                    if (lane == 0) record_error(a.ctl, SPLITSART_ERR_TIMEOUT, -1);
                    inflight &= ~(1u << slot);
                    drain();
                    return false;
                }
                phase ^= 1u << slot;
                inflight &= ~(1u << slot);
                body(q, qe, pv, (int)(wslots - smem_raw) + slot * cap * kEB, lo, meta);
            } else {
                body(q, qe, pv, -1, 0, meta);
            }
            __syncwarp();
            q = nq;
            qe = nqe;
            pv = npv;
            st = nst;
            lo = nlo;
            meta = nmeta;
            nq = nnq;
            nqe = nnqe;
            npv = nnpv;
            nl1 = nnl1;
            slot ^= 1;
        }
        return true;
    };

    struct RowMeta {
        int i;
        V2 p;
        N2 ir;
        float2 sc;
    };
    struct ColMeta {
        int j;  // -1: no column, or its slice has stopped
        N2 ic;
        V2 f;
    };
    constexpr int JB = 2 * GPW <= 31 ? 2 * GPW : 31;  // columns per back job (J + 1 pointers fit in a warp)

    for (int k = 0;; ++k) {
        // ---- forward: r = p - A f, u = r / R, and the norm partials ----
        SqAcc<Acc> rr;  // lanes 0 and 1: their rows' ||r||^2
        // Lane 0 holds row q's metadata, lane 1 row q + 1's.
        auto f_first = [&](int q, int qe) { return (lane < 2 && q + lane < qe) ? __ldg(a.nzr + q + lane) : -1; };
        auto f_second = [&](int, int, int i) {
            RowMeta m{i, V2{}, N2{}, float2{}};
            if (i >= 0) {
                m.p = ldg(a.p12 + i);
                m.ir = ldg(a.invR + i);
                if constexpr (T::kQuant) m.sc = ldg(a.scale + i);
            }
            return m;
        };
        auto f_body = [&](int q, int qe, int pv, int soff, int off, const RowMeta& m) {
            const int loA = __shfl_sync(0xffffffffu, pv, 0) - off, hiA = __shfl_sync(0xffffffffu, pv, 1) - off;
            const int hiB = __shfl_sync(0xffffffffu, pv, qe - q) - off;  // = hiA when the job has one row
            Acc sA1 = 0, sA2 = 0, sB1 = 0, sB2 = 0;
            if (soff >= 0)
                two_items(kUS, reinterpret_cast<const int32_t*>(smem_raw + soff),
                          reinterpret_cast<const Pair*>(smem_raw + soff + cap * 4), a.f12, loA, hiA, hiA, hiB, lane, 32,
                          sA1, sA2, sB1, sB2);
            else
                two_items(kUD, a.col, a.val, a.f12, loA, hiA, hiA, hiB, lane, 32, sA1, sA2, sB1, sB2);
            sA1 = warp_sum(sA1);
            sA2 = warp_sum(sA2);
            sB1 = warp_sum(sB1);
            sB2 = warp_sum(sB2);
            if (m.i >= 0) {
                Acc s1 = lane == 0 ? sA1 : sB1, s2 = lane == 0 ? sA2 : sB2;
                if constexpr (T::kQuant) {
                    s1 *= m.sc.x;
                    s2 *= m.sc.y;
                }
                const Acc r1 = m.p.x - s1, r2 = m.p.y - s2;
                // For BF16/FP16, ir already holds the row scale (the codes are reused by the back-projection).
                stcg(a.u12 + m.i, V2{r1 * m.ir.x, r2 * m.ir.y});
                if constexpr (kBatch) __stcg(a.rr_row + m.i, (double)(r1 * r1 + r2 * r2));
                else rr.add(r1, r2);
            }
        };
        const bool ok_f = run_pass(a.nzrp, a.col, a.val, rrange.x, rrange.y, 2, f_first, f_second, f_body);
        if constexpr (!kBatch) {
            const double t = warp_sum(rr.sum());
            if (lane == 0) s_red[0][wib] = t;
            __syncthreads();
            if (wib == 0) {
                const double tc = warp_sum(lane < nwarps ? s_red[0][lane] : 0.0);
                if (lane == 0) __stcg(a.partials + 2 * blockIdx.x, tc + ppz);  // an empty row's residual is its p
            }
        }
        (void)ok_f;  // a failed copy has recorded an error; the barrier below then returns false
        if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;

        const bool last = (k >= a.max_iters);
        if constexpr (kBatch) {
            if (last || (k % a.check_every == 0)) slice_stop_tests(a, k, last, s_red[0]);
            if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
            if (ld_volatile(a.ndone) >= a.ns) {
                if (blockIdx.x == 0 && tid == 0) {
                    a.result->iters = k;
                    a.result->status = SPLITSART_OK;
                    a.result->rho = 0.0;
                    a.result->rr = 0.0;
                    a.result->pp = 0.0;
                }
                return;
            }
        } else if (last || (k % a.check_every == 0)) {
            // One thread decides, so the FP64 division and square root run once per CTA.
            if (wib == 0) {
                const double trr = grid_total(a.partials, gridDim.x, lane, 0);
                if (lane == 0) s_stop = stop_test(a, k, last, trr, s_tpp);
            }
            __syncthreads();
            if (s_stop) return;
        }

        // ---- back-projection and update: f += lambda (A^T u) / C ----
        // Group g of LPC lanes takes columns q + g (A) and q + g + GPW (B). Its lane 0
        // holds A's metadata, its lane 1 (lane 0 if LPC = 1) B's.
        int sl = sl_first;  // this lane's slice, advanced as its columns increase
        auto b_col = [&](int q, int qe) {
            // With LPC = 1 every lane is a group's lane 0, and B is never in the job (J = 31).
            const int g = lane / LPC;
            int c = -1;
            if (sub == 0) c = q + g;
            else if (LPC > 1 && sub == 1) c = q + g + GPW;
            return c < qe ? c : -1;
        };
        auto b_first = [&](int q, int qe) {
            const int c = b_col(q, qe);
            return c >= 0 ? __ldg(a.nzc + c) : -1;
        };
        auto b_second = [&](int, int, int j) {
            ColMeta m{j, N2{}, V2{}};
            if (j >= 0) {
                if constexpr (kBatch) {
                    while (j >= __ldg(a.sl_cols + sl + 1)) ++sl;
                    if (__ldcg(&a.sl_solve[sl].done)) {  // the slice has stopped: keep its returned iterate
                        m.j = -1;
                        return m;
                    }
                }
                m.ic = ldg(a.invC + j);
                m.f = ldcg(a.f12 + j);
            }
            return m;
        };
        auto b_body = [&](int q, int qe, int pv, int soff, int off, const ColMeta& m) {
            const int g = lane / LPC;
            const int qA = q + g, qB = qA + GPW;
            const int kA = min(g, 31), kB = min(g + GPW, 31);
            const int pA0 = __shfl_sync(0xffffffffu, pv, kA), pA1 = __shfl_sync(0xffffffffu, pv, min(kA + 1, 31));
            const int pB0 = __shfl_sync(0xffffffffu, pv, kB), pB1 = __shfl_sync(0xffffffffu, pv, min(kB + 1, 31));
            const int loA = qA < qe ? pA0 - off : 0, hiA = qA < qe ? pA1 - off : 0;
            const int loB = qB < qe ? pB0 - off : 0, hiB = qB < qe ? pB1 - off : 0;
            Acc bA1 = 0, bA2 = 0, bB1 = 0, bB2 = 0;
            if (soff >= 0)
                two_items(kUS, reinterpret_cast<const int32_t*>(smem_raw + soff),
                          reinterpret_cast<const Pair*>(smem_raw + soff + cap * 4), a.u12, loA, hiA, loB, hiB, sub, LPC,
                          bA1, bA2, bB1, bB2);
            else
                two_items(kUD, a.row, a.valT, a.u12, loA, hiA, loB, hiB, sub, LPC, bA1, bA2, bB1, bB2);
            bA1 = warp_sum(bA1, LPC);
            bA2 = warp_sum(bA2, LPC);
            bB1 = warp_sum(bB1, LPC);
            bB2 = warp_sum(bB2, LPC);
            if (m.j >= 0) {
                const bool isA = LPC == 1 || sub == 0;
                const Acc b1 = isA ? bA1 : bB1, b2 = isA ? bA2 : bB2;
                V2 f = m.f;
                f.x += lam * b1 * m.ic.x;
                f.y += lam * b2 * m.ic.y;
                stcg(a.f12 + m.j, f);
            }
        };
        const bool ok_b = run_pass(a.nzcp, a.row, a.valT, crange.x, crange.y, JB, b_first, b_second, b_body);
        (void)ok_b;
        if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
    }
}

template <class T>
constexpr int default_tile_entries() {
    return sizeof(typename T::Vec2) == 16 ? 8192 : 12288;
}

// Row-streaming kernel: entries in flight per lane and item. Five per row
// cover most rows of the batch (about 136 entries) in one round; FP64 pairs
// are twice as wide, so they keep fewer in flight.
template <class T, int LPC>
void* rows_kernel(bool batch) {
    constexpr bool kWide = sizeof(typename T::Vec2) == 16;
    constexpr int kUF = kWide ? 2 : 5, kUB = kWide ? 2 : 4;
    return batch ? (void*)sart_rows_kernel<T, LPC, true, kUF, kUB> : (void*)sart_rows_kernel<T, LPC, false, kUF, kUB>;
}

template <class T>
void fill_args(SartArgs<T>& a, splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o,
               unsigned grid) {
    a.nzr = s->nzr;
    a.nzrp = s->nzrp;
    a.zr = s->zr;
    a.nzc = s->nzc;
    a.nzcp = s->nzcp;
    a.col = s->col;
    a.val = (const typename T::Pair*)s->val;
    a.row = s->row;
    a.valT = (const typename T::Pair*)s->valT;
    using KN2 = typename T::KNorm2;
    a.invR = (const KN2*)(T::kQuant ? (const void*)s->wR : s->invR);
    a.invC = (const KN2*)(T::kQuant ? (const void*)s->wC : s->invC);
    a.scale = s->scale;
    a.p12 = (const typename T::Vec2*)p12;
    a.f12 = (typename T::Vec2*)f12;
    a.u12 = (typename T::Vec2*)s->u12;
    a.partials = s->partials;
    a.ctl = s->ctl;
    a.result = s->result;
    a.stats = s->stats;
    a.max_iters = o.max_iters;
    a.check_every = effective_check_every(o);
    a.lambda = o.lambda;
    a.tol = o.tol;
    a.tol2_hi = o.tol * o.tol * (1.0 + 1e-12);
    const double tms = o.timeout_ms > 0 ? o.timeout_ms : 2000.0;
    a.timeout_ns = (unsigned long long)(tms * 1e6);
    a.expected = grid + (o.inject_barrier_fault ? 1u : 0u);
    a.tile_entries = o.tile_entries > 0 ? o.tile_entries : default_tile_entries<T>();
    a.direct_rows = 0;
    a.direct_cols = 0;
    a.ns = s->ns;
    a.sl_rows = s->sl_rows;
    a.sl_cols = s->sl_cols;
    a.sl_solve = s->sl_solve;
    a.rr_row = s->rr_row;
    a.ndone = s->ndone;
    a.res_rows = nullptr;
    a.res_off = nullptr;
    a.res_loc = nullptr;
}

// Row plan of the resident kernel for a grid of G CTAs: contiguous ranges of
// the non-empty rows, balanced by time rather than by bytes. A warp step costs
// about one gather round trip whatever its rows' lengths, so a CTA's forward
// pass takes time in proportion to its rows as well as to its entries; on the
// realistic slice a byte-balanced split gave CTAs from 29 to 134 rows and
// forward passes from 2.8 to 6.6 us, with every CTA then waiting for the
// slowest at the grid barrier. Here each row weighs row_weight entries more
// than its length (default 240: on the realistic slice 200 iterations took
// 2.62 ms with weight 0, 2.37 ms with 160, 2.33 ms with 240, 2.67 ms with 480). Ranges keep the rows' order, so neighbouring rays (which
// gather neighbouring voxels) stay together. Built on the first resident solve
// and kept: the rows do not change across refolds.
template <class T>
int resident_plan(splitsart_system* s, const FoldStats& fs, int G, int row_weight, cudaStream_t st) {
    if (s->res_G == G && s->res_weight == row_weight) return SPLITSART_OK;
    using B = ResidentBytes<T>;
    const int n = fs.n_nzr;
    if (s->res_ptr.size() != (size_t)n + 1) {
        std::vector<int32_t> ptr((size_t)n + 1);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e == cudaSuccess)
            e = cudaMemcpy(ptr.data(), s->nzrp, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "solve: read the row pointers for the resident plan");
        s->res_ptr.swap(ptr);
    }
    const std::vector<int32_t>& ptr = s->res_ptr;
    // Prefix of the time weights; CTA b takes the rows whose prefix falls in [b W/G, (b+1) W/G).
    std::vector<long long> cum((size_t)n + 1, 0);
    for (int q = 0; q < n; ++q) cum[q + 1] = cum[q] + (ptr[q + 1] - ptr[q]) + row_weight;
    const long long total = cum[n];
    std::vector<int32_t> rows((size_t)n), off((size_t)G + 1), loc;
    loc.reserve((size_t)n + G);
    for (int q = 0; q < n; ++q) rows[q] = q;
    long long worst = 0;
    int q = 0;
    for (int b = 0; b < G; ++b) {
        const long long lim = total * (b + 1) / G;
        off[b] = q;
        int32_t run = 0;
        long long bytes = 0;
        const int q_end = (b == G - 1) ? n : (int)(std::lower_bound(cum.begin() + q, cum.end(), lim) - cum.begin());
        for (; q < q_end && q < n; ++q) {
            loc.push_back(run);
            const int len = ptr[q + 1] - ptr[q];
            run += len;
            bytes += (long long)B::kEntry * len + B::kRow;
        }
        loc.push_back(run);
        worst = std::max(worst, bytes);
    }
    off[G] = n;
    cudaError_t e;
    if (s->res_alloc) {
        cudaFree(s->res_alloc);
        s->res_alloc = nullptr;
        s->res_G = 0;
    }
    const size_t bytes = sizeof(int32_t) * (rows.size() + off.size() + loc.size());
    if ((e = cudaMalloc(&s->res_alloc, bytes > 0 ? bytes : 4)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SPLITSART_ERR_NOMEM, "solve: cudaMalloc of the resident plan (%zu bytes) failed", bytes);
    }
    s->res_rows = (int32_t*)s->res_alloc;
    s->res_off = s->res_rows + rows.size();
    s->res_loc = s->res_off + off.size();
    e = cudaMemcpy(s->res_rows, rows.data(), sizeof(int32_t) * rows.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->res_off, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->res_loc, loc.data(), sizeof(int32_t) * loc.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "solve: upload the resident plan");
    s->res_G = G;
    s->res_weight = row_weight;
    s->res_row_bytes = worst;
    return SPLITSART_OK;
}

// Upper bound of one CTA's resident shared-memory bytes for a grid of G CTAs.
template <class T>
long long resident_bound(const FoldStats& fs, long long G) {
    using B = ResidentBytes<T>;
    const long long Wr = (long long)B::kEntry * fs.S + (long long)B::kRow * fs.n_nzr;
    const long long Wc = (long long)B::kEntry * fs.S + (long long)B::kCol * fs.n_nzc;
    return (Wr + G - 1) / G + (long long)B::kEntry * fs.max_row + B::kRow + (Wc + G - 1) / G +
           (long long)B::kEntry * fs.max_col + B::kCol + B::kSlack;
}

template <class T, int LPC>
int launch_lpc(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "solve: cudaGetDevice");
    int nsm = 0, coop = 0, smem_optin = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop) return fail(SPLITSART_ERR_CUDA, "solve: device lacks cooperative launch");
    const int threads = o.block_threads > 0 ? o.block_threads : 1024;
    if (threads % 32 != 0 || threads > 1024 || threads < 64)
        return fail(SPLITSART_ERR_ARG, "solve: block_threads must be a multiple of 32 in [64, 1024]");
    if (o.row_weight < 0 || o.row_weight > 100000)
        return fail(SPLITSART_ERR_ARG, "solve: row_weight must be in [0, 100000]");
    FoldStats fs;
    int rc = system_host_stats(s, &fs);
    if (rc) return rc;

    // Shared-memory residency: one CTA per SM, 16-bit indices.
    void* rkern = (void*)sart_resident_kernel<T, LPC>;
    const int res_threads = (o.block_threads > 0 && o.block_threads <= 512) ? o.block_threads : 512;
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, (const void*)rkern);
    if (e != cudaSuccess) return cuda_fail(e, "solve: kernel attributes");
    const long long res_avail = (long long)smem_optin - (long long)fa.sharedSizeBytes -
                                (long long)ResidentBytes<T>::kThread * res_threads - 32;
    const bool batch = s->ns > 1;
    const bool res_shape = !batch && s->Mh <= 65536 && s->Nh <= 65536;
    long long need = resident_bound<T>(fs, nsm);
    bool use_plan = false;
    if (res_shape && (o.kernel == 0 || o.kernel == 2)) {
        // The asked row weight, else the heaviest default whose plan fits in
        // shared memory (weight 0 balances entries alone).
        using B = ResidentBytes<T>;
        const long long Wc = (long long)B::kEntry * fs.S + (long long)B::kCol * fs.n_nzc;
        const long long col_part = (Wc + nsm - 1) / nsm + (long long)B::kEntry * fs.max_col + B::kCol + B::kSlack;
        const int asked = o.row_weight > 0 ? o.row_weight : 240;
        for (int w : {asked, 240, 160, 80, 40, 0}) {
            if (w > asked) continue;
            rc = resident_plan<T>(s, fs, nsm, w, st);
            if (rc) return rc;
            if (s->res_row_bytes + col_part <= res_avail) {
                use_plan = true;
                need = s->res_row_bytes + col_part;
                break;
            }
        }
    }
    const bool res_ok = res_shape && need <= res_avail;
    if (o.kernel == 2 && !res_ok)
        return fail(SPLITSART_ERR_ARG, "solve: the system does not fit in shared memory (need %lld of %lld bytes per SM)",
                    need, res_avail);
    const bool use_res = o.kernel == 2 || (o.kernel == 0 && res_ok);
    const bool use_rows = o.kernel == 3 || (o.kernel == 0 && !res_ok);
    const bool use_bulk = o.kernel == 4;
    if (o.kernel < 0 || o.kernel > 4) return fail(SPLITSART_ERR_ARG, "solve: kernel must be 0, 1, 2, 3 or 4");

    SartArgs<T> a;
    void* kern;
    size_t dyn;
    int grid;
    int smem_bytes = 0;
    int block = threads;
    int te_bulk = 0;
    if (use_res) {
        kern = rkern;
        dyn = (size_t)res_avail;
        smem_bytes = (int)dyn;
        grid = nsm;
        block = res_threads;
    } else if (use_rows) {
        kern = rows_kernel<T, LPC>(batch);
        dyn = 0;
        block = threads > 512 ? 512 : threads;
    } else if (use_bulk) {
        // Built for 4 and 8 lanes per column only (the shapes the autotuner tries).
        if constexpr (LPC != 4 && LPC != 8) {
            return fail(SPLITSART_ERR_ARG, "solve: kernel 4 supports lanes_per_col 4 or 8");
        } else {
            kern = batch ? (void*)sart_bulk_kernel<T, LPC, true> : (void*)sart_bulk_kernel<T, LPC, false>;
        }
        block = threads > 384 ? 384 : threads;
        cudaFuncAttributes ba{};
        if ((e = cudaFuncGetAttributes(&ba, (const void*)kern)) != cudaSuccess) return cuda_fail(e, "solve: attributes");
        // Two slots per warp, each a tile of te entries plus 8 of alignment slack.
        const long long eb = 4 + (long long)sizeof(typename T::Pair);
        const long long per_slot = ((long long)smem_optin - (long long)ba.sharedSizeBytes - 256) / (2LL * (block / 32) * eb);
        te_bulk = (int)((per_slot - 8) & ~3LL);
        if (te_bulk < 64) return fail(SPLITSART_ERR_ARG, "solve: too little shared memory for the bulk-staged kernel");
        dyn = (size_t)(block / 32) * 2 * (size_t)(te_bulk + 8) * (size_t)eb;
    } else {
        kern = batch ? (void*)sart_stream_kernel<T, LPC, false, true> : (void*)sart_stream_kernel<T, LPC>;
        dyn = sizeof(typename T::Vec2) * (size_t)(o.tile_entries > 0 ? o.tile_entries : default_tile_entries<T>());
    }
    if (!use_res && !use_bulk) {
        cudaFuncAttributes sa{};
        if ((e = cudaFuncGetAttributes(&sa, (const void*)kern)) != cudaSuccess) return cuda_fail(e, "solve: attributes");
        if (dyn + sa.sharedSizeBytes > (size_t)smem_optin)
            return fail(SPLITSART_ERR_ARG, "solve: tile_entries too large for shared memory (%zu bytes)", dyn);
    }
    e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return cuda_fail(e, "solve: shared memory attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)kern, block, dyn);
    if (e != cudaSuccess) return cuda_fail(e, "solve: occupancy");
    if (per_sm < 1) return fail(SPLITSART_ERR_CUDA, "solve: kernel does not fit on an SM");
    if (!use_res) {
        if (o.ctas_per_sm > 0 && o.ctas_per_sm < per_sm) per_sm = o.ctas_per_sm;
        grid = nsm * per_sm;
        if (grid > kMaxCtas) grid = kMaxCtas;
    }
    fill_args<T>(a, s, p12, f12, o, (unsigned)grid);
    if (use_res && use_plan) {
        a.res_rows = s->res_rows;
        a.res_off = s->res_off;
        a.res_loc = s->res_loc;
    }

    if ((e = cudaMemsetAsync(s->ctl, 0, sizeof(LaunchCtl), st)) != cudaSuccess) return cuda_fail(e, "solve: memset");
    // A result the launch never writes (a timeout) reads back as iters = -1.
    if ((e = cudaMemsetAsync(s->result, 0xff, sizeof(SolveResultDev), st)) != cudaSuccess)
        return cuda_fail(e, "solve: memset");
    if (batch && (e = cudaMemsetAsync(s->ndone, 0, sizeof(int), st)) != cudaSuccess)
        return cuda_fail(e, "solve: memset");
    void* args_stream[] = {&a};
    void* args_res[] = {&a, &smem_bytes};
    void* args_bulk[] = {&a, &te_bulk};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(block),
                                    use_res ? args_res : (use_bulk ? args_bulk : args_stream), dyn, st);
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

// ---------------------------------------------------------------------------
// Allocation-free solve.
//
// Some callers cannot call cudaMalloc. Examples: a process that reserves all
// of its device memory up front and forbids allocation afterwards, and a
// plugin that runs inside a host application which owns the GPU's memory
// budget. Such a caller cannot create a system with splitsart_fold_system,
// because that allocates. It can still hand in a folded system that it
// placed in its own buffers.
//
// This variant runs the same persistent kernel on a plain folded CSR/CSC
// (no compacted lists). Its working memory lives in one file-scope
// static __device__ array of fixed size:
//   the launch control block, the result, the per-CTA norm partials, and
//   u12 for at most kStaticMaxRows rows.
// Every GPU that loads the library holds this array until the process exits.
// ---------------------------------------------------------------------------
namespace splitsart {
namespace {

constexpr int kStaticMaxRows = 65536;

struct StaticScratch {
    LaunchCtl ctl;  // cleared at every call
    SolveResultDev result;
    double partials[2 * kMaxCtas];
    float2 u12[kStaticMaxRows];
};

static __device__ __align__(256) unsigned char g_static_scratch[sizeof(StaticScratch)];

// Device address of g_static_scratch in the current device's context. In host
// code the array's name is only a host-side stand-in, so the address is looked
// up on every call: a context that was torn down and created again (after
// cudaDeviceReset, say) reloads the library's device code, and the array may
// then sit at another address. The lookup is a host-side table read once the
// device code is loaded; the first call in a context also loads it.
int static_scratch_address(StaticScratch** out) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "solve_static: cudaGetSymbolAddress");
    *out = reinterpret_cast<StaticScratch*>(ptr);
    return SPLITSART_OK;
}

__global__ void static_result_kernel(const StaticScratch* sc, splitsart_solve_info* info) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (sc->ctl.err != 0) {
        info->iters = -1;
        info->status = sc->ctl.err;
        info->rho = NAN;
        info->rr = NAN;
        info->pp = NAN;
    } else {
        info->iters = sc->result.iters;
        info->status = sc->result.status;
        info->rho = sc->result.rho;
        info->rr = sc->result.rr;
        info->pp = sc->result.pp;
    }
}

template <int LPC>
int launch_static(StaticScratch* sc, int Mh, int Nh, const int32_t* rp, const int32_t* col, const float2* val,
                  const int32_t* cp, const int32_t* row, const float2* valT, const float2* invR, const float2* invC,
                  const float2* p12, float2* f12, const splitsart_solve_opts& o, cudaStream_t st) {
    auto kern = sart_stream_kernel<TF32, LPC, true>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "solve_static: cudaGetDevice");
    int nsm = 0, coop = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return fail(SPLITSART_ERR_CUDA, "solve_static: device lacks cooperative launch");
    const int threads = o.block_threads > 0 ? o.block_threads : 1024;
    if (threads % 32 != 0 || threads > 1024 || threads < 64)
        return fail(SPLITSART_ERR_ARG, "solve_static: block_threads must be a multiple of 32 in [64, 1024]");
    const int TE = default_tile_entries<TF32>();
    const size_t dyn = sizeof(float2) * (size_t)TE;
    e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return cuda_fail(e, "solve_static: shared memory attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, dyn);
    if (e != cudaSuccess) return cuda_fail(e, "solve_static: occupancy");
    if (o.ctas_per_sm > 0 && o.ctas_per_sm < per_sm) per_sm = o.ctas_per_sm;
    int grid = nsm * per_sm;
    if (grid > kMaxCtas) grid = kMaxCtas;
    if (grid < 1) return fail(SPLITSART_ERR_CUDA, "solve_static: kernel does not fit on an SM");

    SartArgs<TF32> a{};
    a.nzrp = rp;
    a.nzcp = cp;
    a.col = col;
    a.val = val;
    a.row = row;
    a.valT = valT;
    a.invR = invR;
    a.invC = invC;
    a.p12 = p12;
    a.f12 = f12;
    a.u12 = sc->u12;
    a.partials = sc->partials;
    a.ctl = &sc->ctl;
    a.result = &sc->result;
    a.max_iters = o.max_iters;
    a.check_every = effective_check_every(o);
    a.lambda = o.lambda;
    a.tol = o.tol;
    a.tol2_hi = o.tol * o.tol * (1.0 + 1e-12);
    const double tms = o.timeout_ms > 0 ? o.timeout_ms : 2000.0;
    a.timeout_ns = (unsigned long long)(tms * 1e6);
    a.expected = (unsigned)grid + (o.inject_barrier_fault ? 1u : 0u);
    a.tile_entries = TE;
    a.direct_rows = Mh;
    a.direct_cols = Nh;
    // The array keeps the previous call's contents: the control block must start at zero.
    if ((e = cudaMemsetAsync(&sc->ctl, 0, sizeof(LaunchCtl), st)) != cudaSuccess)
        return cuda_fail(e, "solve_static: clear control block");
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(threads), args, dyn, st);
    if (e != cudaSuccess) return cuda_fail(e, "solve_static: cooperative launch");
    return SPLITSART_OK;
}

}  // namespace

}  // namespace splitsart

extern "C" int splitsart_solve_static(int64_t Mh, int64_t Nh, const int32_t* rp_dev, const int32_t* col_dev,
                                      const void* val_dev, const int32_t* cp_dev, const int32_t* row_dev,
                                      const void* valT_dev, const void* invR_dev, const void* invC_dev,
                                      const void* p12_dev, void* f12_dev, const splitsart_solve_opts* opts,
                                      splitsart_solve_info* info_dev, void* stream) {
    splitsart::NvtxRange nvtx_range("splitsart_solve_static");
    using namespace splitsart;
    if (!opts || !info_dev || !rp_dev || !col_dev || !val_dev || !cp_dev || !row_dev || !valT_dev || !p12_dev ||
        !f12_dev || !invR_dev || !invC_dev)
        return fail(SPLITSART_ERR_ARG, "solve_static: NULL argument");
    if (Mh <= 0 || Nh <= 0) return fail(SPLITSART_ERR_ARG, "solve_static: Mh and Nh must be positive");
    if (Mh > kStaticMaxRows)
        return fail(SPLITSART_ERR_ARG,
                    "solve_static: Mh = %lld rows exceeds the static scratch capacity of %d rows; use splitsart_solve",
                    (long long)Mh, kStaticMaxRows);
    if (Nh > INT32_MAX) return fail(SPLITSART_ERR_ARG, "solve_static: Nh exceeds int32");
    if (opts->max_iters < 0) return fail(SPLITSART_ERR_ARG, "solve_static: max_iters must be >= 0");
    if (!(opts->lambda > 0.0) || !std::isfinite(opts->lambda))
        return fail(SPLITSART_ERR_ARG, "solve_static: lambda must be > 0");
    if (!(opts->tol >= 0.0)) return fail(SPLITSART_ERR_ARG, "solve_static: tol must be >= 0");
    if (opts->check_every < 0 || !(opts->timeout_ms >= 0.0))
        return fail(SPLITSART_ERR_ARG, "solve_static: bad check_every or timeout_ms");
    StaticScratch* sc = nullptr;
    int rc = static_scratch_address(&sc);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const auto* val = (const float2*)val_dev;
    const auto* valT = (const float2*)valT_dev;
    const auto* iR = (const float2*)invR_dev;
    const auto* iC = (const float2*)invC_dev;
    const auto* p12 = (const float2*)p12_dev;
    auto* f12 = (float2*)f12_dev;
    switch (opts->lanes_per_col > 0 ? opts->lanes_per_col : 8) {
        case 1: rc = launch_static<1>(sc, (int)Mh, (int)Nh, rp_dev, col_dev, val, cp_dev, row_dev, valT, iR, iC, p12, f12, *opts, st); break;
        case 2: rc = launch_static<2>(sc, (int)Mh, (int)Nh, rp_dev, col_dev, val, cp_dev, row_dev, valT, iR, iC, p12, f12, *opts, st); break;
        case 4: rc = launch_static<4>(sc, (int)Mh, (int)Nh, rp_dev, col_dev, val, cp_dev, row_dev, valT, iR, iC, p12, f12, *opts, st); break;
        case 8: rc = launch_static<8>(sc, (int)Mh, (int)Nh, rp_dev, col_dev, val, cp_dev, row_dev, valT, iR, iC, p12, f12, *opts, st); break;
        case 16: rc = launch_static<16>(sc, (int)Mh, (int)Nh, rp_dev, col_dev, val, cp_dev, row_dev, valT, iR, iC, p12, f12, *opts, st); break;
        case 32: rc = launch_static<32>(sc, (int)Mh, (int)Nh, rp_dev, col_dev, val, cp_dev, row_dev, valT, iR, iC, p12, f12, *opts, st); break;
        default: return fail(SPLITSART_ERR_ARG, "solve_static: lanes_per_col must be 1, 2, 4, 8, 16 or 32");
    }
    if (rc) return rc;
    static_result_kernel<<<1, 32, 0, st>>>(sc, info_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "solve_static: result launch");
}
