// Row-streaming split-SART fed through a shared-memory ring by a producer warp
// (solve kernels 7 and 8).
//
// The iteration and the compacted index order are those of kernels 5 and 6
// (stream.cu): the simultaneous SART on both split systems (Eqs. 3, 4), rows
// and columns with entries renumbered in order. What differs is who waits for
// HBM. In kernels 5 and 6 every warp loads its own next entries into
// registers and then waits for them before its gathers can start, so each
// warp alternates between an HBM round trip and an L2 round trip. Here the two
// are split between warps:
// - Chunks. The rows (columns) of a pass are cut into chunks by entry count:
//   chunk c holds the rows whose first entry lies in [c E, (c + 1) E). CTAs
//   take batches of consecutive chunks from the pass's work counter.
// - Producer. One warp per CTA copies its chunks, in order, into a circular
//   byte ring in shared memory with bulk asynchronous copies (each chunk is
//   its row pointers, its indices and its values, three copies completed on
//   the chunk slot's mbarrier). A chunk takes exactly its own bytes of the
//   ring, so no space is set aside for the longest row; the producer waits
//   for the oldest chunks to be released before it writes over their bytes.
//   A sentinel chunk without bytes ends each pass.
// - Consumers. The other warps (23, or 15 for FP64 vectors) take the rows of
//   each chunk in groups, dealt round robin across chunks, read the entries
//   from shared memory and spend their waits on the gathers of f (of u in the
//   back pass) alone. Each warp releases a chunk on its slot's second mbarrier
//   when it is done with its groups.
// With the whole warp on a row (lanes_per_row 32, the default) the per-row and
// per-column sums keep the lane-strided order and shuffle tree of kernels 5
// and 6, so at equal lanes_per_col kernel 7 returns kernel 5's f and kernel 8
// kernel 6's, bit for bit.
#include <algorithm>
#include <cstdio>

#include "stream_common.cuh"

namespace splitsart {
namespace {

constexpr int kRingSlots = 32;  // chunks outstanding per CTA at most

// Header of a chunk in the ring, written by the producer before its arrival on
// the slot's full barrier.
struct RingHdr {
    int q0, q1;  // rows (columns) [q0, q1)
    int q0a;     // first pointer staged (q0 rounded down to a multiple of 4)
    int e0a;     // first entry staged (the chunk's first entry rounded down to a multiple of 4)
    int off;     // byte offset of the chunk in the ring
    int nqa;     // pointers staged (a multiple of 4)
    int nea;     // entries staged (a multiple of 4)
    int pad;
};

// Longest row (column) of a compacted pointer array ptr[0..n].
__global__ void ring_maxlen_kernel(const int32_t* __restrict__ ptr, const int* __restrict__ n_ptr,
                                   int* __restrict__ out) {
    const int n = *n_ptr;
    int m = 0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
        m = max(m, ptr[q + 1] - ptr[q]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Chunk plan: desc[c] = (first row q with ptr[q] >= c E, ptr[q]) for c < nch,
// desc[nch] = (n, ptr[n]). Chunk c is the rows [desc[c].x, desc[c + 1].x):
// those that start in its window of E entries. Every row has an entry, so a
// chunk has at most E rows and at most E + L - 1 entries (L the longest row).
// A chunk can be empty: the last one, or one whose window a row longer than E
// spans.
__global__ void ring_plan_kernel(const int32_t* __restrict__ ptr, const int* __restrict__ n_ptr, int E, int nch,
                                 int2* __restrict__ desc) {
    const int n = *n_ptr;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= nch; c += gridDim.x * blockDim.x) {
        int q = n;
        if (c < nch) {
            const long long target = (long long)c * E;
            int lo = 0, hi = n;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((long long)ptr[mid] < target) lo = mid + 1;
                else hi = mid;
            }
            q = lo;
        }
        desc[c] = make_int2(q, ptr[q]);
    }
}

template <class T, bool kImplicit>
struct RingArgs {
    StArgs<T, kImplicit> st;
    const int2* __restrict__ desc[2];  // chunk plans: [0] rows (forward pass), [1] columns (back pass)
    int nch[2];                        // chunks per pass
    int batch;                         // chunks per grab from a pass's work counter (at most 31)
    int ring_bytes;                    // bytes of the ring, a multiple of 16
};

constexpr int kRingPrefix = 2 * kRingSlots * 8 + kRingSlots * (int)sizeof(RingHdr);  // barriers and headers
static_assert(kRingPrefix % 128 == 0, "the ring starts 128-byte aligned");

__device__ __forceinline__ bool ring_try(uint32_t addr, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for an mbarrier phase with a time and spin limit; gives up as soon as
// another warp of the CTA has recorded an abort. The clock is read only once
// a first try has failed, and then every 256 tries: most waits here find the
// phase already complete, and a clock read costs far more than a try.
__device__ __forceinline__ bool ring_wait(uint64_t* bar, unsigned parity, unsigned long long timeout_ns,
                                          const volatile int* abort) {
    const uint32_t addr = smem_addr(bar);
    if (ring_try(addr, parity)) return true;
    const unsigned long long t0 = global_ns();
    const unsigned long long max_spins = timeout_ns / 16ull + (1ull << 20);
    for (unsigned long long spins = 1;; ++spins) {
        if (ring_try(addr, parity)) return true;
        if (*abort) return false;
        if (spins > max_spins || ((spins & 255) == 0 && global_ns() - t0 > timeout_ns)) return false;
    }
}

// Record a ring wait that ran out (where: -2 a consumer's wait for a chunk,
// -3 the producer's wait for a release) and tell the CTA to stop.
__device__ __forceinline__ void ring_abort(LaunchCtl* ctl, int where, volatile int* abort) {
    record_error(ctl, SPLITSART_ERR_TIMEOUT, where);
    *abort = 1;
}

// LPC, LPR: lanes per column (back pass) and per row (forward pass); UF, UB:
// entries in flight per lane and item (forward, back); R: items per lane group
// and step; W: consumer warps (the CTA has W + 1).
template <class T, bool kImplicit, bool kBatch, int LPC, int LPR, int UF, int UB, int R, int W>
__global__ void __launch_bounds__(32 * (W + 1), 1) sart_ring_kernel(RingArgs<T, kImplicit> ra) {
    using Acc = typename T::Acc;
    using V2 = typename T::Vec2;
    using N2 = typename T::KNorm2;
    using St = Stor<T, kImplicit>;
    using Val = typename St::Val;
    constexpr int kGroups = 32 / LPC;
    constexpr int kColStep = R * kGroups;  // columns per consumer step
    constexpr int kW = W;
    constexpr unsigned kFull = 0xffffffffu;
    static_assert(kColStep <= 32 && R * (32 / LPR) <= 32, "a lane holds the data of one item of a step");
    const StArgs<T, kImplicit>& a = ra.st;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kRingSlots;
    RingHdr* hdr = reinterpret_cast<RingHdr*>(empty + kRingSlots);
    unsigned char* ring = smem + kRingPrefix;
    __shared__ double s_red[32];
    __shared__ double s_tpp;
    __shared__ int s_stop;
    __shared__ int s_abort;

    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const bool producer = wib == kW;
    const int sub = lane % LPC, grp = lane / LPC;
    const Acc lam = (Acc)a.lambda;
    volatile int* abort = &s_abort;

    if (tid == 0) {
        for (int i = 0; i < kRingSlots; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kW);
        }
        mbar_init_fence();
        s_abort = 0;
    }
    const double ppz = st_prologue<T, kImplicit, kBatch>(a, s_red);  // thread 0: empty rows' ||p||^2
    unsigned nbar = 0;
    // The barrier also publishes the mbarrier initialisation to the CTA.
    if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
    if (!kBatch && wib == 0) {
        const double t = grid_total(a.partials, gridDim.x, lane, 1);
        if (lane == 0) s_tpp = t;
    }

    // ---- producer state (warp-uniform): chunks issued (kp) and seen released (kt); the ring
    // bytes in use (used: from the oldest outstanding chunk up to pos, where the next one goes) ----
    unsigned kp = 0, kt = 0;
    unsigned used = 0, pos = 0;
    unsigned foot = 0;  // lane i: bytes that the chunk last issued on slot i holds (with any skipped ring tail)
    // ---- consumer state: chunks taken, and the warp that takes a chunk's first group ----
    unsigned kc = 0;
    int rot = 0;

    // Room for a chunk of `bytes` bytes (the host checked bytes <= the ring): a free slot and
    // contiguous bytes; a chunk that does not fit before the end of the ring starts at its
    // beginning. Waits for the oldest chunks' release. Returns the offset, or -1 after an abort.
    auto room = [&](unsigned bytes, unsigned RB) __attribute__((always_inline)) -> int {
        unsigned skip;
        for (;;) {
            if (kp == kt) used = pos = 0;  // nothing outstanding
            skip = pos + bytes > RB ? RB - pos : 0u;
            if (kp - kt < (unsigned)kRingSlots && used + skip + bytes <= RB) break;
            const unsigned ts = kt % kRingSlots;
            if (!ring_wait(&empty[ts], (kt / kRingSlots) & 1u, a.timeout_ns, abort)) {
                if (!*abort) ring_abort(a.ctl, -3, abort);
                return -1;
            }
            used -= __shfl_sync(kFull, foot, ts);
            ++kt;
        }
        const unsigned off = skip ? 0u : pos;
        if (lane == (int)(kp % kRingSlots)) foot = skip + bytes;
        used += skip + bytes;
        pos = off + bytes == RB ? 0u : off + bytes;
        return (int)off;
    };

    // Producer: copy the chunks of pass `pass` into the ring, in order, taking batches of
    // ra.batch consecutive chunks from the pass's work counter; then a sentinel chunk (q0 = -1)
    // that ends the pass for the consumers. Lane j prepares chunk j of a batch and issues its copies.
    auto produce = [&](int pass) __attribute__((always_inline)) -> bool {
        const int32_t* ptr = pass ? a.cp : a.rp;
        const int32_t* idx = pass ? a.ri : a.ci;
        const Val* val = pass ? a.rv : a.cv;
        const int2* __restrict__ desc = ra.desc[pass];
        const uint64_t l2_stream = l2_evict_first();
        const int nch = ra.nch[pass], B = ra.batch;
        const int nbt = (nch + B - 1) / B;  // batches of the pass
        const unsigned RB = (unsigned)ra.ring_bytes;
        unsigned* ctr = &a.ctl->work[pass];
        // Lane j <= B: the bounds desc[t B + j] of batch t (clamped to the pass's end).
        auto bounds = [&](int t) __attribute__((always_inline)) -> int2 {
            int2 d = make_int2(0, 0);
            if (t < nbt && lane <= B) d = __ldg(desc + min(t * B + lane, nch));
            return d;
        };
        // Two grabs run ahead of the batch being issued; lane 0 holds their raw results.
        unsigned g1 = 0, g2 = 0;
        if (lane == 0) {
            g1 = atomicAdd(ctr, 1u);
            g2 = atomicAdd(ctr, 1u);
        }
        int t = __shfl_sync(kFull, (int)g1, 0);
        int2 d = bounds(t);
        while (t < nbt) {
            const int tn = __shfl_sync(kFull, (int)g2, 0);
            if (lane == 0) g2 = atomicAdd(ctr, 1u);
            const int2 dn = bounds(tn);  // the next batch's bounds load while this one issues
            const int m = min(B, nch - t * B);
            // This lane's chunk: pointers q0 .. q1 and entries [e0, e1) staged, each range widened
            // to multiples of 4 elements so that every copy starts and ends on a 16-byte boundary.
            const int q1 = __shfl_down_sync(kFull, d.x, 1), e1 = __shfl_down_sync(kFull, d.y, 1);
            RingHdr h;
            h.q0 = d.x;
            h.q1 = q1;
            h.q0a = h.q0 & ~3;
            h.e0a = d.y & ~3;
            h.nqa = h.q1 > h.q0 ? ((h.q1 + 4) & ~3) - h.q0a : 0;
            h.nea = h.q1 > h.q0 ? ((e1 + 3) & ~3) - h.e0a : 0;
            h.off = 0;
            h.pad = 0;
            const unsigned my_bytes = 4u * h.nqa + (4u + (unsigned)sizeof(Val)) * h.nea;
            for (int j = 0; j < m; ++j) {
                if (*abort) return false;
                const unsigned bytes = __shfl_sync(kFull, my_bytes, j);
                const unsigned slot = kp % kRingSlots;
                const int off = room(bytes, RB);
                if (off < 0) return false;
                if (lane == j) {
                    h.off = off;
                    hdr[slot] = h;
                    mbar_expect_tx(&full[slot], bytes);  // the producer's arrival, with the bytes to come
                    unsigned char* dst = ring + off;
                    if (h.nqa) bulk_g2s(dst, ptr + h.q0a, 4u * h.nqa, &full[slot]);
                    if (h.nea) {  // indices and values are read once per pass: evict them first
                        bulk_g2s_l2(dst + 4 * h.nqa, idx + h.e0a, 4u * h.nea, &full[slot], l2_stream);
                        bulk_g2s_l2(dst + 4 * h.nqa + 4 * h.nea, val + h.e0a, (unsigned)sizeof(Val) * h.nea,
                                    &full[slot], l2_stream);
                    }
                }
                __syncwarp();
                ++kp;
            }
            t = tn;
            d = dn;
        }
        // The sentinel: a slot without bytes.
        const unsigned slot = kp % kRingSlots;
        if (room(0u, RB) < 0) return false;
        if (lane == 0) {
            RingHdr h{};
            h.q0 = -1;
            hdr[slot] = h;
            mbar_arrive(&full[slot]);
        }
        __syncwarp();
        ++kp;
        return true;
    };
    // Producer, after an abort: wait (bounded) for the copies still in flight.
    auto drain = [&]() __attribute__((always_inline)) {
        for (unsigned j = kt; j != kp; ++j)
            mbar_wait_bounded(&full[j % kRingSlots], (j / kRingSlots) & 1u, a.timeout_ns);
        kt = kp;
    };
    // Consumer: wait for the next chunk; false after an abort.
    auto take = [&](unsigned& slot, RingHdr& h) __attribute__((always_inline)) -> bool {
        slot = kc % kRingSlots;
        if (!ring_wait(&full[slot], (kc / kRingSlots) & 1u, a.timeout_ns, abort)) {
            if (!*abort) ring_abort(a.ctl, -2, abort);
            return false;
        }
        h = hdr[slot];
        return true;
    };
    auto release = [&](unsigned slot) __attribute__((always_inline)) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        ++kc;
    };

    // Consumer, forward: r = p - A f and u = r / R for the rows of its chunks. A step takes
    // kRowStep rows: item g of lane group grpr (LPR lanes) is row cb + g kRG + grpr. With
    // LPR = 32 a step is R rows, each summed by the whole warp as in kernels 5 and 6.
    auto consume_rows = [&](SqAcc<Acc>& rr) __attribute__((always_inline)) -> bool {
        constexpr int kRG = 32 / LPR;
        constexpr int kRowStep = R * kRG;
        const int subr = lane % LPR, grpr = lane / LPR;
        for (;;) {
            unsigned slot;
            RingHdr h;
            if (!take(slot, h)) return false;
            if (h.q0 < 0) {  // the pass's end
                release(slot);
                return true;
            }
            const int32_t* sp = reinterpret_cast<const int32_t*>(ring + h.off);
            const int32_t* sidx = sp + h.nqa;
            const Val* sval = reinterpret_cast<const Val*>(sidx + h.nea);
            const int nq = h.q1 - h.q0, nst = (nq + kRowStep - 1) / kRowStep;
            for (int si = (wib - rot + kW) % kW; si < nst; si += kW) {
                const int cb = si * kRowStep;
                int lo[R], hi[R], len = 0;
#pragma unroll
                for (int g = 0; g < R; ++g) {
                    const int krow = cb + g * kRG + grpr;
                    const bool has = krow < nq;
                    const int r = h.q0 - h.q0a + krow;
                    lo[g] = has ? sp[r] - h.e0a : 0;
                    hi[g] = has ? sp[r + 1] - h.e0a : 0;
                    len = max(len, hi[g] - lo[g]);
                }
                if constexpr (LPR < 32) len = (int)__reduce_max_sync(kFull, (unsigned)len);
                // Lane t < kRowStep finishes row cb + t; its p, 1/R (and scale) load during the sums.
                const int qr = h.q0 + cb + lane;
                const bool mine = lane < kRowStep && cb + lane < nq;
                V2 pm{};
                N2 irm{};
                float2 scm{1.f, 1.f};
                if (mine) {
                    pm = ldcg(a.pc + qr);
                    irm = ldg(a.ir + qr);
                    if constexpr (T::kQuant) scm = ldg(a.sc + qr);
                }
                Acc s1[R], s2[R];
#pragma unroll
                for (int g = 0; g < R; ++g) s1[g] = s2[g] = 0;
                // A round: the gathers of up to UF entries per lane and row in flight together; the
                // values are read from shared memory again once the gathers are back.
                for (int off = 0; off < len; off += LPR * UF) {
                    int32_t ia[R][UF];
                    V2 gv[R][UF];
#pragma unroll
                    for (int g = 0; g < R; ++g)
#pragma unroll
                        for (int u = 0; u < UF; ++u) {
                            const int e = lo[g] + off + subr + LPR * u;
                            if (e < hi[g]) {
                                ia[g][u] = sidx[e];
                                gv[g][u] = ldca(a.fc + St::col(ia[g][u]));
                            }
                        }
#pragma unroll
                    for (int g = 0; g < R; ++g)
#pragma unroll
                        for (int u = 0; u < UF; ++u) {
                            const int e = lo[g] + off + subr + LPR * u;
                            if (e < hi[g]) {
                                int jj;
                                Acc v1, v2;
                                St::get(ia[g][u], sval[e], jj, v1, v2);
                                s1[g] += v1 * gv[g][u].x;
                                s2[g] += v2 * gv[g][u].y;
                            }
                        }
                }
#pragma unroll
                for (int g = 0; g < R; ++g) {
                    s1[g] = warp_sum(s1[g], LPR);
                    s2[g] = warp_sum(s2[g], LPR);
                }
                // Row cb + t was item t / kRG of lane group t mod kRG.
                const int src = (mine ? lane % kRG : 0) * LPR, item = mine ? lane / kRG : 0;
                Acc t1 = 0, t2 = 0;
#pragma unroll
                for (int g = 0; g < R; ++g) {
                    const Acc z1 = __shfl_sync(kFull, s1[g], src), z2 = __shfl_sync(kFull, s2[g], src);
                    if (item == g) {
                        t1 = z1;
                        t2 = z2;
                    }
                }
                if (mine) {
                    if constexpr (T::kQuant) {  // codes times the row's scale; 1/R already holds it for u
                        t1 *= scm.x;
                        t2 *= scm.y;
                    }
                    const Acc r1 = pm.x - t1, r2 = pm.y - t2;
                    stcg(a.uc + qr, V2{r1 * irm.x, r2 * irm.y});
                    if constexpr (kBatch) __stcg(a.rr + qr, (double)(r1 * r1 + r2 * r2));
                    else rr.add(r1, r2);
                }
            }
            rot = (rot + nst) % kW;
            release(slot);
        }
    };

    // Consumer, back: f += lambda (A^T u) / C for the columns of its chunks.
    auto consume_cols = [&]() __attribute__((always_inline)) -> bool {
        for (;;) {
            unsigned slot;
            RingHdr h;
            if (!take(slot, h)) return false;
            if (h.q0 < 0) {  // the pass's end
                release(slot);
                return true;
            }
            const int32_t* sp = reinterpret_cast<const int32_t*>(ring + h.off);
            const int32_t* sidx = sp + h.nqa;
            const Val* sval = reinterpret_cast<const Val*>(sidx + h.nea);
            const int nc = h.q1 - h.q0, nst = (nc + kColStep - 1) / kColStep;
            for (int si = (wib - rot + kW) % kW; si < nst; si += kW) {
                const int cb = si * kColStep;
                // Item g of lane group grp: column cb + g kGroups + grp of the chunk.
                int lo[R], hi[R], len = 0;
#pragma unroll
                for (int g = 0; g < R; ++g) {
                    const int kcol = cb + g * kGroups + grp;
                    const bool has = kcol < nc;
                    const int r = h.q0 - h.q0a + kcol;
                    lo[g] = has ? sp[r] - h.e0a : 0;
                    hi[g] = has ? sp[r + 1] - h.e0a : 0;
                    len = max(len, hi[g] - lo[g]);
                }
                len = (int)__reduce_max_sync(kFull, (unsigned)len);
                // Lane t < kColStep finishes column cb + t; its 1/C, f and slice state load during the sums.
                const int c = h.q0 + cb + lane;
                const bool mine = lane < kColStep && cb + lane < nc;
                N2 icm{};
                V2 fm{};
                int skip = 1;
                if (mine) {
                    icm = ldg(a.ic + c);
                    fm = ldcg(a.fc + c);
                    skip = 0;
                    if constexpr (kBatch) skip = __ldcg(&a.sl_solve[__ldg(a.cs + c)].done);
                }
                Acc b1[R], b2[R];
#pragma unroll
                for (int g = 0; g < R; ++g) b1[g] = b2[g] = 0;
                for (int off = 0; off < len; off += LPC * UB) {
                    int32_t ia[R][UB];
                    V2 gv[R][UB];
#pragma unroll
                    for (int g = 0; g < R; ++g)
#pragma unroll
                        for (int u = 0; u < UB; ++u) {
                            const int e = lo[g] + off + sub + LPC * u;
                            if (e < hi[g]) {
                                ia[g][u] = sidx[e];
                                gv[g][u] = ldca(a.uc + St::col(ia[g][u]));
                            }
                        }
#pragma unroll
                    for (int g = 0; g < R; ++g)
#pragma unroll
                        for (int u = 0; u < UB; ++u) {
                            const int e = lo[g] + off + sub + LPC * u;
                            if (e < hi[g]) {
                                int ii;
                                Acc v1, v2;
                                St::get(ia[g][u], sval[e], ii, v1, v2);
                                b1[g] += v1 * gv[g][u].x;
                                b2[g] += v2 * gv[g][u].y;
                            }
                        }
                }
#pragma unroll
                for (int g = 0; g < R; ++g) {
                    b1[g] = warp_sum(b1[g], LPC);
                    b2[g] = warp_sum(b2[g], LPC);
                }
                // Column cb + t was item t / kGroups of lane group t mod kGroups.
                const int src = (mine ? lane % kGroups : 0) * LPC, item = mine ? lane / kGroups : 0;
                Acc y1 = 0, y2 = 0;
#pragma unroll
                for (int g = 0; g < R; ++g) {
                    const Acc z1 = __shfl_sync(kFull, b1[g], src), z2 = __shfl_sync(kFull, b2[g], src);
                    if (item == g) {
                        y1 = z1;
                        y2 = z2;
                    }
                }
                if (mine && !skip) {
                    fm.x += lam * y1 * icm.x;
                    fm.y += lam * y2 * icm.y;
                    stcg(a.fc + c, fm);
                }
            }
            rot = (rot + nst) % kW;
            release(slot);
        }
    };

    for (int k = 0;; ++k) {
        // pass 0: forward, then the stop test; pass 1: back-projection and update
        for (int pass = 0; pass < 2; ++pass) {
            // The other pass's work counter is idle until the barrier that ends this pass.
            if (blockIdx.x == 0 && tid == 0) a.ctl->work[1 - pass] = 0;
            SqAcc<Acc> rr;
            if (producer) {
                if (!produce(pass)) drain();
            } else if (pass == 0) {
                consume_rows(rr);
            } else {
                consume_cols();
            }
            if (pass == 0) {
                if constexpr (!kBatch) st_rr_partial(rr.sum(), ppz, a.partials, s_red);
                if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
                const int stop = st_stop_test<T, kImplicit, kBatch>(a, k, s_red, s_tpp, &s_stop, nbar);
                if (stop != 0) return;  // stopped (f written back), or a barrier wait failed
            } else if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) {
                return;
            }
        }
    }
}

// Consumer step shape for LPR lanes per row: W consumer warps (the CTA has
// W + 1), R items per lane group and step, UF (UB) entries in flight per lane
// and item in the forward (back) pass. kWide: FP64 vectors. On the 256-slice
// batch (FP32, 200 iterations, 4096 entries per chunk, LPR = 32) 23 warps with
// one row per step ran 532 ms explicit and 477 ms implicit (6144 entries per
// chunk), against 558/493 ms for 15 warps with two rows, 546/645 ms for 23
// warps with two rows and 532/491 ms for 31 warps with one row.
constexpr int kRingDefaultLPR = 32;  // forward-pass lanes per row when lanes_per_row is 0

template <bool kWide, int LPR>
struct RingShape {
    static constexpr int W = kWide ? 15 : 23;
    static constexpr int R = kWide ? 2 : 1;
    static constexpr int UF = (kWide ? 2 : 4) * (LPR == 32 ? 1 : 2);
    static constexpr int UB = kWide ? 2 : 4;
};

// Chunk entry target when tile_entries is 0, and the ring's size. On the
// 256-slice batch (200 iterations, lanes_per_col 4; ms for chunks of
// 2048/4096 entries explicit FP32, 3072/6144 for the 8-byte forms):
//   ring          explicit FP32   implicit FP32   BF16 codes
//   228 KB        539 / 510       497 / 458       501 / 462
//   164 KB        532 / 566       441 / 454       439 / 452
//   132 KB        564 / 711       453 / 560       451 / 557
// so the explicit FP32 fold keeps the full ring with 4096-entry chunks (about
// 48 KB), and 8-byte entries take a 164 KB ring with 3072-entry chunks: the
// shared memory given back becomes L1, where their gathers, 1.5 times as many
// per byte streamed, hit more often. Other widths take about 48 KB chunks.
template <class Val>
constexpr int ring_default_E() {
    constexpr int entry = 4 + (int)sizeof(Val);
    if (entry == 8) return 3072;
    const int e = 49152 / entry / 1024 * 1024;
    return e < 1024 ? 1024 : e;
}
// The whole shared memory of a CTA (ring, barriers and headers, static
// variables and the 1 KB the SM reserves per CTA) stays within this, so that
// the rest of the SM's 256 KB array serves as L1.
template <class Val>
constexpr long long ring_smem_cap() {
    return 4 + sizeof(Val) == 8 ? 164LL * 1024 : (1LL << 40);
}

// The chunk plans of format F (kind 0 explicit, 1 implicit) for entry target
// E, made once per target: the longest row and column, then both plans.
int ring_plans(splitsart_system* s, StreamFmt& F, int kind, int E, cudaStream_t st) {
    if (F.ring_E == E) return SPLITSART_OK;
    cudaError_t e;
    if (F.ring_alloc) {
        cudaStreamSynchronize(st);
        cudaFree(F.ring_alloc);
        F.ring_alloc = nullptr;
        F.ring_E = 0;
    }
    FoldStats fs;
    int rc = system_host_stats(s, &fs);
    if (rc) return rc;
    const long long nnz = kind ? (long long)s->nnz_half : fs.S;
    if (nnz + 2LL * E + 64 > 0x7fffffffLL)
        return fail(SPLITSART_ERR_ARG, "solve: kernels 7 and 8 index entries in 32 bits (%lld entries)", nnz);
    const int nch = (int)((nnz + E - 1) / E);
    const size_t dbytes = ((sizeof(int2) * (size_t)(nch + 1)) + 255) & ~size_t(255);
    void* base = nullptr;
    if ((e = cudaMalloc(&base, 256 + 2 * dbytes)) != cudaSuccess)
        return fail(SPLITSART_ERR_NOMEM, "solve: %zu bytes of chunk plans", 256 + 2 * dbytes);
    int* lens = (int*)base;
    int2* d0 = (int2*)((char*)base + 256);
    int2* d1 = (int2*)((char*)base + 256 + dbytes);
    const int G = 152 * 4, B = 256;
    cudaMemsetAsync(lens, 0, 2 * sizeof(int), st);
    ring_maxlen_kernel<<<G, B, 0, st>>>(F.rp, &s->stats->n_nzr, lens);
    ring_maxlen_kernel<<<G, B, 0, st>>>(F.cp, &s->stats->n_nzc, lens + 1);
    ring_plan_kernel<<<G, B, 0, st>>>(F.rp, &s->stats->n_nzr, E, nch, d0);
    ring_plan_kernel<<<G, B, 0, st>>>(F.cp, &s->stats->n_nzc, E, nch, d1);
    int hl[2] = {0, 0};
    e = cudaMemcpyAsync(hl, lens, sizeof(hl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(base);
        return cuda_fail(e, "solve: chunk plans");
    }
    F.ring_alloc = base;
    F.ring_desc[0] = d0;
    F.ring_desc[1] = d1;
    F.ring_nch[0] = F.ring_nch[1] = nch;
    F.ring_len[0] = hl[0];
    F.ring_len[1] = hl[1];
    F.ring_E = E;
    return SPLITSART_OK;
}

template <class T, bool kImplicit, int LPC, int LPR>
int launch_ring(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st) {
    using V2 = typename T::Vec2;
    using Val = typename Stor<T, kImplicit>::Val;
    using Shape = RingShape<sizeof(V2) == 16, LPR>;
    constexpr int R = Shape::R, UF = Shape::UF, UB = Shape::UB, W = Shape::W;
    constexpr int threads = 32 * (W + 1);
    const int kind = kImplicit ? 1 : 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "solve: cudaGetDevice");
    int nsm = 0, coop = 0, optin = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop) return fail(SPLITSART_ERR_CUDA, "solve: device lacks cooperative launch");
    int rc = stream_format(s, kind, st);
    if (rc) return rc;
    StreamFmt& F = s->st[kind];
    const int E = o.tile_entries > 0 ? o.tile_entries : ring_default_E<Val>();
    if ((rc = ring_plans(s, F, kind, E, st)) != SPLITSART_OK) return rc;
    const bool batch = s->ns > 1;
    const void* kern = batch ? (const void*)sart_ring_kernel<T, kImplicit, true, LPC, LPR, UF, UB, R, W>
                             : (const void*)sart_ring_kernel<T, kImplicit, false, LPC, LPR, UF, UB, R, W>;
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return cuda_fail(e, "solve: kernel attributes");
    const long long fixed = (long long)fa.sharedSizeBytes + kRingPrefix;
    const long long ring = std::min((long long)optin - fixed, ring_smem_cap<Val>() - 1024 - fixed) / 128 * 128;
    // The largest chunk: at most E + 8 pointers and E + L + 8 entries staged (L the longest row or column).
    long long chunk = 0;
    for (int k = 0; k < 2; ++k)
        chunk = std::max(chunk, 4LL * (E + 8) + (4LL + (long long)sizeof(Val)) * ((long long)E + F.ring_len[k] + 8));
    if (chunk > ring)
        return fail(SPLITSART_ERR_ARG,
                    "solve: kernels 7 and 8: a chunk of up to %lld bytes (tile_entries %d, longest row %d, "
                    "longest column %d) exceeds the %lld-byte ring; lower tile_entries",
                    chunk, E, F.ring_len[0], F.ring_len[1], ring);
    const int dyn = kRingPrefix + (int)ring;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess)
        return cuda_fail(e, "solve: ring shared memory");
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, dyn)) != cudaSuccess)
        return cuda_fail(e, "solve: occupancy");
    if (per_sm < 1) return fail(SPLITSART_ERR_CUDA, "solve: kernel does not fit on an SM");
    const int grid = std::min(nsm, kMaxCtas);

    RingArgs<T, kImplicit> ra{};
    ra.st = st_args<T, kImplicit>(s, F, p12, f12, o, grid);
    ra.desc[0] = F.ring_desc[0];
    ra.desc[1] = F.ring_desc[1];
    ra.nch[0] = F.ring_nch[0];
    ra.nch[1] = F.ring_nch[1];
    ra.batch = std::min(16, std::max(1, 16384 / E));  // about 16K entries per grab
    ra.ring_bytes = (int)ring;
    if ((rc = st_reset(s, st)) != SPLITSART_OK) return rc;
    void* args[] = {&ra};
    e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(threads), args, (size_t)dyn, st);
    if (e != cudaSuccess) return cuda_fail(e, "solve: cooperative launch");
    return SPLITSART_OK;
}

template <class T, bool kImplicit, int LPC>
int launch_ring_lpr(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st) {
    switch (o.lanes_per_row > 0 ? o.lanes_per_row : kRingDefaultLPR) {
        case 8: return launch_ring<T, kImplicit, LPC, 8>(s, p12, f12, o, st);
        case 16: return launch_ring<T, kImplicit, LPC, 16>(s, p12, f12, o, st);
        case 32: return launch_ring<T, kImplicit, LPC, 32>(s, p12, f12, o, st);
    }
    return fail(SPLITSART_ERR_ARG, "solve: kernels 7 and 8 take lanes_per_row 8, 16 or 32");
}

template <class T, bool kImplicit>
int launch_ring_lpc(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st) {
    switch (o.lanes_per_col > 0 ? o.lanes_per_col : 4) {
        case 4: return launch_ring_lpr<T, kImplicit, 4>(s, p12, f12, o, st);
        case 8: return launch_ring_lpr<T, kImplicit, 8>(s, p12, f12, o, st);
    }
    return fail(SPLITSART_ERR_ARG, "solve: kernels 7 and 8 take lanes_per_col 4 or 8");
}

}  // namespace

int run_solve_ring(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st) {
    const bool imp = o.kernel == 8;
    if (!imp && s->dtype == SPLITSART_BF16) return launch_ring_lpc<TBF16, false>(s, p12, f12, o, st);
    if (!imp && s->dtype == SPLITSART_F16) return launch_ring_lpc<TF16, false>(s, p12, f12, o, st);
    switch (s->dtype) {
        case SPLITSART_F64:
            return imp ? launch_ring_lpc<TF64, true>(s, p12, f12, o, st) : launch_ring_lpc<TF64, false>(s, p12, f12, o, st);
        case SPLITSART_F32:
            return imp ? launch_ring_lpc<TF32, true>(s, p12, f12, o, st) : launch_ring_lpc<TF32, false>(s, p12, f12, o, st);
    }
    return fail(SPLITSART_ERR_ARG, "solve: kernel 8 takes FP64 and FP32 systems (kernel 7 also BF16 and FP16)");
}

}  // namespace splitsart
