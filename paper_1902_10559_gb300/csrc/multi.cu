// Many right-hand sides on one folded system: the split-SART iteration as a
// sparse matrix times a block of vectors (SpMM).
//
// The method is SART on each split system (Section 1, reference [001];
// Eqs. 3, 4). Every right-hand side is an independent solve with its own
// stopping test; only the matrix is shared.
//
// Layout. The whole folded system (CSR, CSC, normalisers) is copied into each
// CTA's shared memory once per launch. Each CTA has RC slots, each holding one
// right-hand side's p, u and two buffers of f (f^k read, f^{k+1} written),
// also in shared memory. An iteration therefore touches no global memory, and
// its two phases are separated by two CTA barriers. The stop test of pass k
// runs on one warp per slot while the other warps back-project; a slot that
// stops returns f^k from the buffer the pass did not write. The launch needs
// no grid-wide synchronisation.
//
// Scheduling. The launch is persistent: as many CTAs as are resident at once.
// When a slot's right-hand side stops, its f and stop record are written out
// and the slot takes the next right-hand side from a global queue. The launch
// time then follows the total iterations of all right-hand sides, not the
// slowest one per CTA. Each right-hand side is computed within one slot in a
// fixed order, so results do not depend on the schedule.
//
// SpMM. A warp takes RPW rows (forward) or columns (back) at a time. Its 32
// lanes are split into RPW x RC groups, one per (row, slot). Every matrix
// entry read from shared memory (a broadcast) is applied to all RC slots.
#include <cmath>
#include <cstdio>

#include "device_common.cuh"
#include "system.h"

namespace splitsart {

namespace {

template <class T>
struct MultiArgs {
    const int32_t* rp;
    const int32_t* col;
    const typename T::Pair* val;
    const int32_t* cp;
    const int32_t* row;
    const typename T::Pair* valT;
    const typename T::KNorm2* invR;  // as applied (BF16/FP16: scale / R in FP32)
    const typename T::KNorm2* invC;
    const float2* scale;
    const typename T::Vec2* p12;  // [nrhs][Mh]
    typename T::Vec2* f12;        // [nrhs][Nh]
    splitsart_solve_info* info;   // [nrhs]
    unsigned* queue;              // next right-hand side after the first wave (zeroed before the launch)
    const int32_t* order;         // [nrhs] queue position -> right-hand side (null: in index order)
    int Mh, Nh, S, nrhs;
    int max_iters, check_every;
    double lambda, tol;
    double tol2_hi;  // tol^2 (1 + 1e-12): rr > pp tol2_hi proves rho > tol without a division or square root
};

__device__ __forceinline__ size_t align16m(size_t x) { return (x + 15) & ~size_t(15); }

// RC right-hand sides per CTA; RPW rows (or columns) per warp at a time; the
// 32 lanes split into RPW x RC groups of LPR = 32 / (RPW RC) lanes.
template <class T, int RC, int RPW>
__global__ void __launch_bounds__(1024, 1) sart_multi_kernel(MultiArgs<T> a) {
    using Acc = typename T::Acc;
    using V2 = typename T::Vec2;
    using N2 = typename T::KNorm2;
    using Pair = typename T::Pair;
    constexpr int LPR = 32 / (RC * RPW);  // lanes per (row, right-hand side)
    static_assert(LPR >= 1, "too many groups per warp");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_rr[32][RC];  // per warp (at most 32) and slot: ||r||^2 of the warp's rows
    __shared__ double s_pp[RC];
    __shared__ int s_rhs[RC];    // right-hand side held by each slot, or -1
    __shared__ int s_k[RC];      // iterations done by the slot's right-hand side
    __shared__ unsigned s_fin;   // slots whose right-hand side stopped in this pass
    __shared__ int s_active;

    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5, nwarps = blockDim.x >> 5;
    const int grp = lane / LPR, sub = lane % LPR;
    const int g = grp % RC, rw = grp / RC;        // slot and row of this lane group
    const int Mh = a.Mh, Nh = a.Nh, S = a.S;
    const Acc lam = (Acc)a.lambda;

    size_t off = 0;
    int* s_rp = reinterpret_cast<int*>(smem + off);
    off = align16m(off + 4 * (size_t)(Mh + 1));
    int* s_col = reinterpret_cast<int*>(smem + off);
    off = align16m(off + 4 * (size_t)S);
    Pair* s_val = reinterpret_cast<Pair*>(smem + off);
    off = align16m(off + sizeof(Pair) * (size_t)S);
    int* s_cp = reinterpret_cast<int*>(smem + off);
    off = align16m(off + 4 * (size_t)(Nh + 1));
    int* s_row = reinterpret_cast<int*>(smem + off);
    off = align16m(off + 4 * (size_t)S);
    Pair* s_valT = reinterpret_cast<Pair*>(smem + off);
    off = align16m(off + sizeof(Pair) * (size_t)S);
    N2* s_ir = reinterpret_cast<N2*>(smem + off);
    off = align16m(off + sizeof(N2) * (size_t)Mh);
    N2* s_ic = reinterpret_cast<N2*>(smem + off);
    off = align16m(off + sizeof(N2) * (size_t)Nh);
    float2* s_sc = reinterpret_cast<float2*>(smem + off);
    off = align16m(off + (T::kQuant ? sizeof(float2) * (size_t)Mh : 0));
    V2* s_p = reinterpret_cast<V2*>(smem + off);  // [Mh][RC]
    off = align16m(off + sizeof(V2) * (size_t)Mh * RC);
    V2* s_u = reinterpret_cast<V2*>(smem + off);  // [Mh][RC]
    off = align16m(off + sizeof(V2) * (size_t)Mh * RC);
    V2* s_f = reinterpret_cast<V2*>(smem + off);  // [Nh][RC]: f^k, read by this pass
    off = align16m(off + sizeof(V2) * (size_t)Nh * RC);
    V2* s_fn = reinterpret_cast<V2*>(smem + off);  // [Nh][RC]: f^{k+1}, written by this pass

    for (int i = tid; i <= Mh; i += blockDim.x) s_rp[i] = a.rp[i];
    for (int j = tid; j <= Nh; j += blockDim.x) s_cp[j] = a.cp[j];
    for (int e = tid; e < S; e += blockDim.x) {
        s_col[e] = a.col[e];
        s_val[e] = a.val[e];
        s_row[e] = a.row[e];
        s_valT[e] = a.valT[e];
    }
    for (int i = tid; i < Mh; i += blockDim.x) {
        s_ir[i] = a.invR[i];
        if constexpr (T::kQuant) s_sc[i] = a.scale[i];
    }
    for (int j = tid; j < Nh; j += blockDim.x) s_ic[j] = a.invC[j];
    // ---- slots: load, store, and ||p||^2 of newly loaded right-hand sides ----
    auto load_slots = [&](unsigned mask, V2* fdst) {
        for (int t = tid; t < Mh * RC; t += blockDim.x) {
            const int i = t / RC, r = t % RC;
            if (mask >> r & 1u) s_p[t] = s_rhs[r] >= 0 ? a.p12[(size_t)s_rhs[r] * Mh + i] : V2{};
        }
        for (int t = tid; t < Nh * RC; t += blockDim.x) {
            const int j = t / RC, r = t % RC;
            if (mask >> r & 1u) fdst[t] = s_rhs[r] >= 0 ? a.f12[(size_t)s_rhs[r] * Nh + j] : V2{};
        }
        __syncthreads();
        // ||p||^2 once per right-hand side: one warp per slot, lane-strided, fixed tree.
        for (int r = wib; r < RC; r += nwarps) {
            if (!(mask >> r & 1u)) continue;
            double t1 = 0.0;
            for (int i = lane; i < Mh; i += 32) {
                const V2 p = s_p[i * RC + r];
                t1 += (double)p.x * (double)p.x + (double)p.y * (double)p.y;
            }
            t1 = warp_sum(t1);
            if (lane == 0) s_pp[r] = t1;
        }
    };
    auto store_slots = [&](unsigned mask) {
        for (int t = tid; t < Nh * RC; t += blockDim.x) {
            const int j = t / RC, r = t % RC;
            if ((mask >> r & 1u) && s_rhs[r] >= 0) a.f12[(size_t)s_rhs[r] * Nh + j] = s_f[t];
        }
    };

    // The first wave takes queue positions blockIdx.x * RC + r; later ones come from the queue.
    // Position q holds right-hand side order[q] (q itself without an order).
    if (tid < RC) {
        const int r = blockIdx.x * RC + tid;
        s_rhs[tid] = r < a.nrhs ? (a.order ? a.order[r] : r) : -1;
        s_k[tid] = 0;
    }
    __syncthreads();
    load_slots((1u << RC) - 1u, s_f);
    __syncthreads();

    // Every thread's copy of s_k, kept in step at points where s_rhs is not being written.
    int kl[RC];
#pragma unroll
    for (int r = 0; r < RC; ++r) kl[r] = 0;
    for (;;) {
        // Whether any slot tests rho after this pass (uniform over the CTA): the
        // residual norms are formed only then.
        bool tested = false;
#pragma unroll
        for (int r = 0; r < RC; ++r) tested |= s_rhs[r] >= 0 && (kl[r] >= a.max_iters || kl[r] % a.check_every == 0);
        // ---- forward: RPW rows per warp, one lane group per (row, slot) ----
        SqAcc<Acc> rr;  // this lane group's ||r||^2 over its rows
        for (int i0 = wib * RPW; i0 < Mh; i0 += nwarps * RPW) {
            const int i = i0 + rw;
            Acc s1 = 0, s2 = 0;
            if (i < Mh) {
                const int lo = s_rp[i], hi = s_rp[i + 1];
                for (int e = lo + sub; e < hi; e += LPR) {
                    Acc a1, a2;
                    T::decode(s_val[e], a1, a2);
                    const V2 fv = s_f[s_col[e] * RC + g];
                    s1 += a1 * fv.x;
                    s2 += a2 * fv.y;
                }
            }
            s1 = warp_sum(s1, LPR);
            s2 = warp_sum(s2, LPR);
            if (sub == 0 && i < Mh) {
                const V2 p = s_p[i * RC + g];
                const N2 ir = s_ir[i];
                if constexpr (T::kQuant) {
                    const float2 sc = s_sc[i];
                    s1 *= sc.x;
                    s2 *= sc.y;
                }
                const Acc r1 = p.x - s1, r2 = p.y - s2;
                // For BF16/FP16, ir already holds the row scale (the codes are reused by the back-projection).
                s_u[i * RC + g] = V2{r1 * ir.x, r2 * ir.y};
                if (tested) rr.add(r1, r2);
            }
        }
        if (tested) {
            // The warp's sum per slot: a fixed xor tree over its RPW lane groups of the slot
            // (lanes with sub != 0 hold 0 and pair only with each other).
            double t = rr.sum();
#pragma unroll
            for (int o = RC * LPR; o < 32; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane < RC * LPR && sub == 0) s_rr[wib][g] = t;
        }
        if (tid == 0) s_fin = 0u;
        __syncthreads();
        // ---- stop tests, overlapped with the back-projection ----
        // One warp per slot sums the warps' partials (lane-strided, fixed tree; FP64
        // is slow on this GPU, so no serial chain) and its lane 0 decides. The last
        // warps take the tests: when the columns do not fill every warp, they have
        // no back-projection work. The other warps back-project meanwhile: that
        // writes f^{k+1} into the second buffer, so a slot that stops still holds
        // f^k in the first.
        for (int r = nwarps - 1 - wib; r < RC; r += nwarps) {
            if (s_rhs[r] < 0) continue;  // uniform over the warp
            const int k = s_k[r];
            const bool last = k >= a.max_iters;
            if (!(last || (k % a.check_every == 0))) continue;
            double t0 = 0.0;
            for (int x = lane; x < nwarps; x += 32) t0 += s_rr[x][r];
            t0 = warp_sum(t0);
            if (lane == 0) {
                const double t1 = s_pp[r];
                // The common case (rho > tol for certain) needs no FP64 division or square root.
                const bool above = !last && t1 > 0.0 && t0 > t1 * a.tol2_hi;
                const double rho = (above || !(t1 > 0.0)) ? 0.0 : sqrt(t0 / t1);
                if (!above && (last || rho <= a.tol)) {
                    a.info[s_rhs[r]] = splitsart_solve_info{k, SPLITSART_OK, rho, t0, t1};
                    atomicOr(&s_fin, 1u << r);
                }
            }
        }
        for (int j0 = wib * RPW; j0 < Nh; j0 += nwarps * RPW) {
            const int j = j0 + rw;
            Acc b1 = 0, b2 = 0;
            if (j < Nh) {
                const int lo = s_cp[j], hi = s_cp[j + 1];
                for (int e = lo + sub; e < hi; e += LPR) {
                    Acc a1, a2;
                    T::decode(s_valT[e], a1, a2);
                    const V2 uv = s_u[s_row[e] * RC + g];
                    b1 += a1 * uv.x;
                    b2 += a2 * uv.y;
                }
            }
            b1 = warp_sum(b1, LPR);
            b2 = warp_sum(b2, LPR);
            if (sub == 0 && j < Nh) {
                const N2 ic = s_ic[j];
                V2 f = s_f[j * RC + g];
                f.x += lam * b1 * ic.x;
                f.y += lam * b2 * ic.y;
                s_fn[j * RC + g] = f;
            }
        }
        __syncthreads();
        const unsigned fin = s_fin;  // read by every thread before any later write of s_fin
        if (tid < RC && s_rhs[tid] >= 0) ++s_k[tid];
#pragma unroll
        for (int r = 0; r < RC; ++r) kl[r] += s_rhs[r] >= 0 ? 1 : 0;
        if (fin) {
            // Return the stopped right-hand sides' f^k and refill their slots from
            // the queue; a new right-hand side's f0 goes into the buffer that the
            // next pass reads.
            store_slots(fin);
            __syncthreads();
            if (tid == 0) {
                int active = 0;
                for (int r = 0; r < RC; ++r) {
                    if (fin >> r & 1u) {
                        const int nxt = (int)atomicAdd(a.queue, 1u) + (int)gridDim.x * RC;
                        s_rhs[r] = nxt < a.nrhs ? (a.order ? a.order[nxt] : nxt) : -1;
                        s_k[r] = 0;
                    }
                    active += s_rhs[r] >= 0;
                }
                s_active = active;
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < RC; ++r)
                if (fin >> r & 1u) kl[r] = 0;
            if (s_active == 0) break;
            load_slots(fin, s_fn);
            __syncthreads();
        }
        V2* const t = s_f;
        s_f = s_fn;
        s_fn = t;
    }
}

template <class T>
size_t multi_smem_bytes(const splitsart_system* s, int S, int RC) {
    auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
    const size_t pb = sizeof(typename T::Pair), nb = sizeof(typename T::KNorm2), vb = sizeof(typename T::Vec2);
    return al(4 * (s->Mh + 1)) + al(4 * (size_t)S) + al(pb * S) + al(4 * (s->Nh + 1)) + al(4 * (size_t)S) +
           al(pb * S) + al(nb * s->Mh) + al(nb * s->Nh) + (T::kQuant ? al(8 * s->Mh) : 0) + 2 * al(vb * s->Mh * RC) +
           2 * al(vb * s->Nh * RC);
}

template <class T, int RC, int RPW>
int launch_multi(splitsart_system* s, int S, int nrhs, const void* p12, void* f12, const splitsart_solve_opts& o,
                 const int32_t* order, splitsart_solve_info* info, cudaStream_t st) {
    auto kern = sart_multi_kernel<T, RC, RPW>;
    const size_t dyn = multi_smem_bytes<T>(s, S, RC);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)kern);
    if (e != cudaSuccess) return cuda_fail(e, "solve_multi: kernel attributes");
    if (dyn + fa.sharedSizeBytes > (size_t)optin)
        return fail(SPLITSART_ERR_ARG, "solve_multi: the system and %d right-hand sides need %zu bytes of shared memory "
                                       "per CTA (limit %d); use fewer per CTA or splitsart_solve",
                    RC, dyn + fa.sharedSizeBytes, optin);
    e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return cuda_fail(e, "solve_multi: shared memory attribute");
    MultiArgs<T> a;
    a.rp = s->rp;
    a.col = s->col;
    a.val = (const typename T::Pair*)s->val;
    a.cp = s->cp;
    a.row = s->row;
    a.valT = (const typename T::Pair*)s->valT;
    using KN2 = typename T::KNorm2;
    a.invR = (const KN2*)(T::kQuant ? (const void*)s->wR : s->invR);
    a.invC = (const KN2*)(T::kQuant ? (const void*)s->wC : s->invC);
    a.scale = s->scale;
    a.p12 = (const typename T::Vec2*)p12;
    a.f12 = (typename T::Vec2*)f12;
    a.info = info;
    a.Mh = (int)s->Mh;
    a.Nh = (int)s->Nh;
    a.S = S;
    a.nrhs = nrhs;
    a.max_iters = o.max_iters;
    a.check_every = effective_check_every(o);
    a.lambda = o.lambda;
    a.tol = o.tol;
    a.tol2_hi = o.tol * o.tol * (1.0 + 1e-12);
    const int threads = o.block_threads > 0 ? o.block_threads : 512;
    if (threads % 32 || threads > 1024 || threads < 32)
        return fail(SPLITSART_ERR_ARG, "solve_multi: block_threads must be a multiple of 32 in [32, 1024]");
    // Persistent: as many CTAs as are resident at once; a CTA refills a slot from
    // the queue as soon as its right-hand side stops.
    int nsm = 0, per_sm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)kern, threads, dyn);
    if (e != cudaSuccess) return cuda_fail(e, "solve_multi: occupancy");
    if (per_sm < 1) return fail(SPLITSART_ERR_ARG, "solve_multi: the kernel does not fit on an SM");
    const int groups = (nrhs + RC - 1) / RC;
    const int grid = groups < nsm * per_sm ? groups : nsm * per_sm;
    a.queue = &s->ctl->work[0];
    a.order = order;
    if ((e = cudaMemsetAsync(s->ctl, 0, sizeof(LaunchCtl), st)) != cudaSuccess)
        return cuda_fail(e, "solve_multi: memset");
    kern<<<grid, threads, dyn, st>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "solve_multi: launch");
}

// Lanes per (row, right-hand side): LPR = 32 / (RC RPW). With 2 lanes (the
// default) a warp of one right-hand side per CTA sums 16 rows at once, and the
// tiny slice's 320 rows and 256 columns take one sweep each of a 512-thread
// CTA. On 64 right-hand sides of the tiny slice (one per CTA, 200 iterations)
// 2 lanes ran 0.765 ms at 512 threads, against 0.964 ms for 8 lanes at 1024
// threads (the earlier fixed shape), 0.815 ms for 4 lanes and 0.790 ms for 1.
template <class T, int RC>
int multi_lpr(splitsart_system* s, int S, int nrhs, const void* p12, void* f12, const splitsart_solve_opts& o,
              const int32_t* order, splitsart_solve_info* info, cudaStream_t st) {
    const int lpr = o.lanes_per_row > 0 ? o.lanes_per_row : 2;
    if (lpr == 2 && RC <= 16) return launch_multi<T, RC, (RC <= 16 ? 16 / RC : 1)>(s, S, nrhs, p12, f12, o, order, info, st);
    if (lpr == 4 && RC <= 8) return launch_multi<T, RC, (RC <= 8 ? 8 / RC : 1)>(s, S, nrhs, p12, f12, o, order, info, st);
    if (lpr == 8 && RC <= 4) return launch_multi<T, RC, (RC <= 4 ? 4 / RC : 1)>(s, S, nrhs, p12, f12, o, order, info, st);
    return fail(SPLITSART_ERR_ARG, "solve_multi: lanes_per_row must be 2, 4 or 8, with rhs_per_cta x lanes_per_row <= 32");
}

template <class T>
int multi_typed(splitsart_system* s, int S, int nrhs, int rc, const void* p12, void* f12,
                const splitsart_solve_opts& o, const int32_t* order, splitsart_solve_info* info, cudaStream_t st) {
    switch (rc) {
        case 1: return multi_lpr<T, 1>(s, S, nrhs, p12, f12, o, order, info, st);
        case 2: return multi_lpr<T, 2>(s, S, nrhs, p12, f12, o, order, info, st);
        case 4: return multi_lpr<T, 4>(s, S, nrhs, p12, f12, o, order, info, st);
        case 8: return multi_lpr<T, 8>(s, S, nrhs, p12, f12, o, order, info, st);
        case 16: return multi_lpr<T, 16>(s, S, nrhs, p12, f12, o, order, info, st);
    }
    return fail(SPLITSART_ERR_ARG, "solve_multi: rhs_per_cta must be 1, 2, 4, 8 or 16");
}

// Per right-hand side: keep the warm start only if its residual is lower.
template <class V2>
__global__ void pick_start_kernel(int nrhs, long long Nh, const V2* __restrict__ warm,
                                  const splitsart_solve_info* __restrict__ iw, const splitsart_solve_info* __restrict__ ib,
                                  V2* __restrict__ f12, int* __restrict__ picked) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nrhs * Nh) return;
    const int r = (int)(t / Nh);
    const bool use = iw[r].rho < ib[r].rho;
    if (use) f12[t] = warm[t];
    if (picked && t % Nh == 0) picked[r] = use ? 1 : 0;
}

}  // namespace

}  // namespace splitsart

using namespace splitsart;

extern "C" int splitsart_pick_start(const splitsart_system* s, int nrhs, const void* f12_warm_dev,
                                    const splitsart_solve_info* info_warm_dev,
                                    const splitsart_solve_info* info_base_dev, void* f12_dev, int* picked_dev,
                                    void* stream) {
    if (!s || nrhs < 1 || !f12_warm_dev || !info_warm_dev || !info_base_dev || !f12_dev)
        return fail(SPLITSART_ERR_ARG, "pick_start: bad argument");
    const long long n = (long long)nrhs * s->Nh;
    const unsigned g = (unsigned)((n + 255) / 256);
    cudaStream_t st = (cudaStream_t)stream;
    if (s->dtype == SPLITSART_F64)
        pick_start_kernel<double2><<<g, 256, 0, st>>>(nrhs, s->Nh, (const double2*)f12_warm_dev, info_warm_dev,
                                                       info_base_dev, (double2*)f12_dev, picked_dev);
    else
        pick_start_kernel<float2><<<g, 256, 0, st>>>(nrhs, s->Nh, (const float2*)f12_warm_dev, info_warm_dev,
                                                     info_base_dev, (float2*)f12_dev, picked_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "pick_start: launch");
}

extern "C" int splitsart_solve_multi_ordered(splitsart_system* s, int nrhs, const void* p12_dev, void* f12_dev,
                                             const splitsart_solve_opts* o, int rhs_per_cta, const int32_t* order_dev,
                                             splitsart_solve_info* info_dev, void* stream) {
    splitsart::NvtxRange nvtx_range("splitsart_solve_multi");
    if (!s || !o || !p12_dev || !f12_dev || !info_dev) return fail(SPLITSART_ERR_ARG, "solve_multi: NULL argument");
    if (nrhs < 1) return fail(SPLITSART_ERR_ARG, "solve_multi: nrhs must be >= 1");
    if (s->ns != 1) return fail(SPLITSART_ERR_ARG, "solve_multi: needs a single-slice system");
    if (o->max_iters < 0 || o->max_iters > 500000) return fail(SPLITSART_ERR_ARG, "solve_multi: bad max_iters");
    if (!(o->lambda > 0.0) || !std::isfinite(o->lambda)) return fail(SPLITSART_ERR_ARG, "solve_multi: lambda must be > 0");
    if (!(o->tol >= 0.0) || o->check_every < 0) return fail(SPLITSART_ERR_ARG, "solve_multi: bad tol or check_every");
    FoldStats fs;
    int rc = system_host_stats(s, &fs);
    if (rc) return rc;
    const int per = rhs_per_cta > 0 ? rhs_per_cta : 4;
    cudaStream_t st = (cudaStream_t)stream;
    s->last = st;
    const int S = (int)fs.S;
    switch (s->dtype) {
        case SPLITSART_F64: return multi_typed<TF64>(s, S, nrhs, per, p12_dev, f12_dev, *o, order_dev, info_dev, st);
        case SPLITSART_F32: return multi_typed<TF32>(s, S, nrhs, per, p12_dev, f12_dev, *o, order_dev, info_dev, st);
        case SPLITSART_BF16: return multi_typed<TBF16>(s, S, nrhs, per, p12_dev, f12_dev, *o, order_dev, info_dev, st);
        case SPLITSART_F16: return multi_typed<TF16>(s, S, nrhs, per, p12_dev, f12_dev, *o, order_dev, info_dev, st);
    }
    return fail(SPLITSART_ERR_ARG, "solve_multi: unknown dtype");
}

extern "C" int splitsart_solve_multi(splitsart_system* s, int nrhs, const void* p12_dev, void* f12_dev,
                                     const splitsart_solve_opts* o, int rhs_per_cta, splitsart_solve_info* info_dev,
                                     void* stream) {
    return splitsart_solve_multi_ordered(s, nrhs, p12_dev, f12_dev, o, rhs_per_cta, nullptr, info_dev, stream);
}
