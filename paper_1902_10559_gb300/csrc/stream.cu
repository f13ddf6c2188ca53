// Row-streaming split-SART in compacted index order (solve kernels 5 and 6),
// for systems far larger than on-chip memory.
//
// The iteration is the simultaneous SART of sart.cu, on both split systems
// (Eqs. 3, 4; Section 1, reference [001]). What differs is how the matrix
// streams from HBM:
// - Compacted index space. Rows and columns with entries are renumbered in
//   order; p, u, f and the normalisers are held in that order for the launch
//   (p and f are gathered in at the start, f scattered back at the end). The
//   hot loop then indexes every vector directly, with no dependent index
//   load between a row's sum and its update.
// - Two storages. Kernel 5 streams the explicit fold (the pairs (a1, a2) of
//   the folded CSR and CSC, 12 bytes per entry and pass in FP32; 8 with
//   BF16/FP16 code pairs, whose row scale joins the row's data). Kernel 6
//   streams the implicit fold: each entry of the half rows of A is stored
//   once, as its compacted folded column with A1's sign in bit 31 and its
//   length w, so that a1 = +-w and a2 = w (8 bytes per entry and pass). Eq. (2)
//   makes the mirror row a reflection of the row itself, so the column index
//   alone says whether the length enters A1 with a plus or a minus sign. A ray
//   and its mirror through the same folded cell give two entries (+w, -w'),
//   which the explicit fold merges into one (w - w', w + w').
// - Chunks with their data loaded ahead. A warp takes chunks of 16 compacted
//   rows (32 columns) from a global counter, one chunk ahead, and loads the
//   next chunk's row pointers and row data (p, 1/R; or column pointers, 1/C
//   and f) while it works on the current one, one lane per row (column). A
//   step covers R rows (R columns per group of LPC lanes), U entries per lane
//   each; longer rows take more rounds.
// Per-row and per-column sums keep the lane-strided order and fixed shuffle
// tree of the other kernels, so f does not depend on the grid or the
// schedule, and kernel 5 returns kernel 3's f bit for bit at equal LPC.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <vector>

#include "stream_common.cuh"

namespace splitsart {

namespace {

constexpr int kSortCap = 512;  // column entries staged in shared memory by the sort (longer: global)

size_t st_align(size_t x) { return (x + 255) & ~size_t(255); }

// map[list[q]] = q.
__global__ void st_map_kernel(const int32_t* __restrict__ list, const int* __restrict__ n_ptr,
                              int32_t* __restrict__ map) {
    const int n = *n_ptr;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) map[list[q]] = q;
}

// out[e] = map[in[e] & mask] | (in[e] & sign): indices into compacted order, keeping the sign bit.
__global__ void st_remap_kernel(int64_t n, const int32_t* __restrict__ in, const int32_t* __restrict__ map,
                                int32_t* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)in[e];
        out[e] = (int32_t)((uint32_t)map[v & kIndexMask] | (v & kSignBit));
    }
}

// Implicit CSR row pointers in compacted order: half row nzr[q] starts at hrp[nzr[q]].
__global__ void st_implicit_rp_kernel(const int32_t* __restrict__ nzr, const int* __restrict__ n_ptr,
                                      const int64_t* __restrict__ hrp, int64_t nnz, int32_t* __restrict__ rp) {
    const int n = *n_ptr;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q <= n; q += gridDim.x * blockDim.x)
        rp[q] = q < n ? (int32_t)hrp[nzr[q]] : (int32_t)nnz;
}

__global__ void st_count_kernel(int64_t n, const int32_t* __restrict__ ci, int32_t* __restrict__ cnt) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[(uint32_t)ci[e] & kIndexMask], 1);
}

// Scatter the implicit CSR into column buckets; key = (compacted row << 1) | sign.
template <class V>
__global__ void st_place_kernel(const int32_t* __restrict__ rp, const int* __restrict__ n_ptr,
                                const int32_t* __restrict__ ci, const V* __restrict__ cv,
                                const int32_t* __restrict__ cp, int32_t* __restrict__ cnt,
                                int32_t* __restrict__ tkey, V* __restrict__ tval) {
    const int n = *n_ptr;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < n; q += nw) {
        for (int e = rp[q] + lane; e < rp[q + 1]; e += 32) {
            const uint32_t v = (uint32_t)ci[e];
            const int c = (int)(v & kIndexMask);
            const int pos = cp[c] + atomicAdd(&cnt[c], 1);
            tkey[pos] = (int32_t)(((uint32_t)q << 1) | (v >> 31));
            tval[pos] = cv[e];
        }
    }
}

// One warp per compacted column: order its entries by key (rank sort; keys are
// unique) and write them as (compacted row with the sign in bit 31, w).
template <class V>
__global__ void st_sort_kernel(const int32_t* __restrict__ cp, const int* __restrict__ n_ptr,
                               const int32_t* __restrict__ tkey, const V* __restrict__ tval,
                               int32_t* __restrict__ ri, V* __restrict__ rv) {
    __shared__ int32_t skey[8][kSortCap];
    const int n = *n_ptr;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n; c += nw) {
        const int e0 = cp[c], L = cp[c + 1] - e0;
        const bool staged = L <= kSortCap;
        if (staged)
            for (int t = lane; t < L; t += 32) skey[w][t] = tkey[e0 + t];
        __syncwarp();
        const int32_t* keys = staged ? skey[w] : tkey + e0;
        for (int t = lane; t < L; t += 32) {
            const int32_t k = keys[t];
            int rank = 0;
            for (int u = 0; u < L; ++u) rank += keys[u] < k;
            const uint32_t uk = (uint32_t)k;
            ri[e0 + rank] = (int32_t)((uk >> 1) | (uk << 31));
            rv[e0 + rank] = tval[e0 + t];
        }
        __syncwarp();
    }
}

// Compacted copies of the normalisers as the iteration applies them.
template <class N2>
__global__ void st_gather_norm_kernel(const int32_t* __restrict__ list, const int* __restrict__ n_ptr,
                                      const N2* __restrict__ in, N2* __restrict__ out) {
    const int n = *n_ptr;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) out[q] = in[list[q]];
}

// Batch maps: qs[s] = first compacted row of slice s (qs[ns] = n_nzr); cs[q] = slice of compacted column q.
__global__ void st_slice_maps_kernel(const int32_t* __restrict__ nzr, const int32_t* __restrict__ nzc,
                                     const FoldStats* __restrict__ stats, int ns, const long long* __restrict__ sl_rows,
                                     const long long* __restrict__ sl_cols, int32_t* __restrict__ qs,
                                     int32_t* __restrict__ cs) {
    const int n_nzr = stats->n_nzr, n_nzc = stats->n_nzc;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int sl = tid; sl <= ns; sl += nth) {
        const long long key = sl_rows[sl];
        int lo = 0, hi = n_nzr;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((long long)nzr[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        qs[sl] = lo;
    }
    for (int q = tid; q < n_nzc; q += nth) {
        const long long j = nzc[q];
        int lo = 0, hi = ns;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sl_cols[mid] <= j) lo = mid;
            else hi = mid;
        }
        cs[q] = lo;
    }
}

}  // namespace
}  // namespace splitsart

namespace splitsart {
namespace {

// Build format `kind` (0 explicit, 1 implicit) of system s, for value type T, once.
template <class T>
int build_stream_format(splitsart_system* s, int kind, const FoldStats& fs, cudaStream_t st) {
    StreamFmt& F = s->st[kind];
    if (F.built) return SPLITSART_OK;
    using V2 = typename T::Vec2;
    using N2 = typename T::KNorm2;
    using V = decltype(V2{}.x);
    const int64_t nnz = kind ? s->nnz_half : fs.S;
    const size_t nr = (size_t)fs.n_nzr, nc = (size_t)fs.n_nzc, ns = (size_t)s->ns;
    // Persistent arrays.
    size_t sz = 0;
    auto take = [&](size_t bytes) { const size_t at = sz; sz += st_align(bytes); return at; };
    const size_t o_rp = kind ? take(sizeof(int32_t) * (nr + 1)) : 0;
    const size_t o_ci = take(sizeof(int32_t) * (size_t)nnz);
    const size_t o_cv = kind ? take(sizeof(V) * (size_t)nnz) : 0;
    const size_t o_cp = kind ? take(sizeof(int32_t) * (nc + 1)) : 0;
    const size_t o_ri = take(sizeof(int32_t) * (size_t)nnz);
    const size_t o_rv = kind ? take(sizeof(V) * (size_t)nnz) : 0;
    const size_t o_ir = take(sizeof(N2) * (nr + 1));
    const size_t o_sc = T::kQuant ? take(sizeof(float2) * (nr + 1)) : 0;
    const size_t o_ic = take(sizeof(N2) * (nc + 1));
    const size_t o_pc = take(sizeof(V2) * (nr + 1));
    const size_t o_uc = take(sizeof(V2) * (nr + 1));
    const size_t o_fc = take(sizeof(V2) * (nc + 1));
    const size_t o_rr = take(sizeof(double) * (nr + 1));
    const size_t o_qs = take(sizeof(int32_t) * (ns + 1));
    const size_t o_cs = take(sizeof(int32_t) * (nc + 1));
    const size_t o_pz = take(sizeof(double) * (ns + 1));
    void* base = nullptr;
    cudaError_t e = cudaMalloc(&base, sz);
    if (e != cudaSuccess) return fail(SPLITSART_ERR_NOMEM, "solve: %zu bytes for the streaming format", sz);
    char* b = (char*)base;
    F.alloc = base;
    F.ci = (int32_t*)(b + o_ci);
    F.ri = (int32_t*)(b + o_ri);
    F.ir = b + o_ir;
    F.sc = T::kQuant ? (float2*)(b + o_sc) : nullptr;
    F.ic = b + o_ic;
    F.pc = b + o_pc;
    F.uc = b + o_uc;
    F.fc = b + o_fc;
    F.rr = (double*)(b + o_rr);
    F.qs = (int32_t*)(b + o_qs);
    F.cs = (int32_t*)(b + o_cs);
    F.pz = (double*)(b + o_pz);
    if (kind) {
        F.rp = (int32_t*)(b + o_rp);
        F.cv = b + o_cv;
        F.cp = (int32_t*)(b + o_cp);
        F.rv = b + o_rv;
    } else {
        F.rp = s->nzrp;
        F.cv = s->val;
        F.cp = s->nzcp;
        F.rv = s->valT;
    }
    auto fail_free = [&](int rc) {
        cudaStreamSynchronize(st);
        cudaFree(F.alloc);
        F = StreamFmt{};
        return rc;
    };
    const int G = 152 * 8, B = 256;
    // Index maps: compacted position of each row and column (scratch of the system: cnt, flags).
    int32_t* rmap = s->cnt;    // max(Mh, Nh) + 1 ints
    int32_t* cmap = s->flags;  // max(Mh, Nh) + 1 ints
    st_map_kernel<<<G, B, 0, st>>>(s->nzr, &s->stats->n_nzr, rmap);
    st_map_kernel<<<G, B, 0, st>>>(s->nzc, &s->stats->n_nzc, cmap);
    int rc = SPLITSART_OK;
    if (kind == 0) {
        st_remap_kernel<<<G, B, 0, st>>>(nnz, s->col, cmap, F.ci);
        st_remap_kernel<<<G, B, 0, st>>>(nnz, s->row, rmap, F.ri);
    } else {
        // CSR: the implicit fold of the half rows, then its columns renumbered.
        rc = run_implicit_rows(s, std::is_same<V, double>::value, F.ri /* scratch */, (void*)F.cv, st);
        if (rc) return fail_free(rc);
        st_remap_kernel<<<G, B, 0, st>>>(nnz, F.ri, cmap, F.ci);
        st_implicit_rp_kernel<<<G, B, 0, st>>>(s->nzr, &s->stats->n_nzr, s->hrp, nnz, F.rp);
        // CSC: count, scan, place into buckets, order each bucket by row.
        int32_t *cnt = nullptr, *tiles = nullptr, *tkey = nullptr;
        V* tval = nullptr;
        const size_t ntiles = nc / 4096 + 2;
        const size_t tmp = st_align(sizeof(int32_t) * (nc + 1)) + st_align(sizeof(int32_t) * ntiles) +
                           st_align(sizeof(int32_t) * (size_t)nnz) + st_align(sizeof(V) * (size_t)nnz);
        void* tb = nullptr;
        if ((e = cudaMalloc(&tb, tmp)) != cudaSuccess) return fail_free(fail(SPLITSART_ERR_NOMEM, "solve: %zu bytes of "
                                                                                                 "sort scratch", tmp));
        char* t = (char*)tb;
        cnt = (int32_t*)t;
        tiles = (int32_t*)(t + st_align(sizeof(int32_t) * (nc + 1)));
        tkey = (int32_t*)(t + st_align(sizeof(int32_t) * (nc + 1)) + st_align(sizeof(int32_t) * ntiles));
        tval = (V*)((char*)tkey + st_align(sizeof(int32_t) * (size_t)nnz));
        cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nc + 1), st);
        st_count_kernel<<<G, B, 0, st>>>(nnz, F.ci, cnt);
        rc = scan_exclusive(cnt, F.cp, tiles, (int64_t)nc, st);
        if (rc == SPLITSART_OK) {
            cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nc + 1), st);
            st_place_kernel<V><<<G, B, 0, st>>>(F.rp, &s->stats->n_nzr, F.ci, (const V*)F.cv, F.cp, cnt, tkey, tval);
            st_sort_kernel<V><<<G, B, 0, st>>>(F.cp, &s->stats->n_nzc, tkey, tval, F.ri, (V*)F.rv);
        }
        cudaStreamSynchronize(st);
        cudaFree(tb);
        if (rc) return fail_free(rc);
    }
    // Normalisers as applied, in compacted order.
    st_gather_norm_kernel<N2><<<G, B, 0, st>>>(s->nzr, &s->stats->n_nzr,
                                               (const N2*)(T::kQuant ? (const void*)s->wR : s->invR), (N2*)F.ir);
    st_gather_norm_kernel<N2><<<G, B, 0, st>>>(s->nzc, &s->stats->n_nzc,
                                               (const N2*)(T::kQuant ? (const void*)s->wC : s->invC), (N2*)F.ic);
    if (T::kQuant) st_gather_norm_kernel<float2><<<G, B, 0, st>>>(s->nzr, &s->stats->n_nzr, s->scale, F.sc);
    st_slice_maps_kernel<<<G, B, 0, st>>>(s->nzr, s->nzc, s->stats, s->ns, s->sl_rows, s->sl_cols, F.qs, F.cs);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail_free(cuda_fail(e, "solve: streaming format"));
    F.built = 1;
    return SPLITSART_OK;
}

// R: rows (columns per lane group) per step.
template <class T, bool kImplicit, bool kBatch, int LPC, int UF, int UB, int R>
__global__ void __launch_bounds__(512, 1) sart_compact_kernel(StArgs<T, kImplicit> a) {
    using Acc = typename T::Acc;
    using V2 = typename T::Vec2;
    using N2 = typename T::KNorm2;
    using St = Stor<T, kImplicit>;
    using Val = typename St::Val;
    constexpr int kGroups = 32 / LPC;
    constexpr int kRowChunk = 16;         // compacted rows per scheduled chunk (lanes 0..16 hold its pointers)
    constexpr int kColChunk = 32;         // compacted columns per chunk (lane k holds column k's data)
    constexpr int kColStep = R * kGroups; // columns per step: R per lane group
    static_assert(kColChunk % kColStep == 0, "a column chunk is a whole number of steps");
    __shared__ double s_red[32];
    __shared__ double s_tpp;
    __shared__ int s_stop;

    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const int sub = lane % LPC, grp = lane / LPC;
    const Acc lam = (Acc)a.lambda;
    const int n_nzr = a.stats->n_nzr, n_nzc = a.stats->n_nzc;

    const double ppz = st_prologue<T, kImplicit, kBatch>(a, s_red);  // thread 0: empty rows' ||p||^2
    unsigned nbar = 0;
    if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
    if (!kBatch && wib == 0) {
        const double t = grid_total(a.partials, gridDim.x, lane, 1);
        if (lane == 0) s_tpp = t;
    }

    // A step's loads (U entries per lane and item, lane-strided by W from `first`), then its use.
    auto load_step = [&](auto UC, auto& B, const int32_t* idx, const Val* val, const int (&lo)[R], const int (&hi)[R],
                         int off, int first, int W) {
        constexpr int U = decltype(UC)::value;
#pragma unroll
        for (int g = 0; g < R; ++g)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = lo[g] + off + first + u * W;
                if (e < hi[g]) {
                    B.ia[g][u] = st_ld(idx + e);
                    B.va[g][u] = st_ld(val + e);
                }
            }
    };
    auto use_step = [&](auto UC, const auto& B, const V2* src, const int (&lo)[R], const int (&hi)[R], int off,
                        int first, int W, Acc (&s1)[R], Acc (&s2)[R]) {
        constexpr int U = decltype(UC)::value;
        V2 gv[R][U];
#pragma unroll
        for (int g = 0; g < R; ++g)
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (lo[g] + off + first + u * W < hi[g]) gv[g][u] = ldca(src + St::col(B.ia[g][u]));
#pragma unroll
        for (int g = 0; g < R; ++g)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (lo[g] + off + first + u * W < hi[g]) {
                    int j;
                    Acc v1, v2;
                    St::get(B.ia[g][u], B.va[g][u], j, v1, v2);
                    s1[g] += v1 * gv[g][u].x;
                    s2[g] += v2 * gv[g][u].y;
                }
            }
    };
    constexpr std::integral_constant<int, UF> kUF{};
    constexpr std::integral_constant<int, UB> kUB{};
    constexpr int kRoundF = 32 * UF;   // entries of a row per forward round
    constexpr int kRoundB = LPC * UB;  // entries of a column per back round

    constexpr unsigned kFull = 0xffffffffu;
    const int nrc = (n_nzr + kRowChunk - 1) / kRowChunk;
    const int ncc = (n_nzc + kColChunk - 1) / kColChunk;
    // Row data of a chunk: lane l <= 16 holds rp[q0 + l]; lane l < 16 holds p and 1/R of row q0 + l.
    auto row_meta = [&](int ch, int& ptr, V2& pm, N2& irm, float2& scm) {
        const int q = ch * kRowChunk + lane;
        ptr = 0;
        pm = V2{};
        irm = N2{};
        scm = float2{1.f, 1.f};
        if (ch < nrc) {
            if (lane <= kRowChunk) ptr = __ldg(a.rp + min(q, n_nzr));
            if (lane < kRowChunk && q < n_nzr) {
                pm = ldcg(a.pc + q);
                irm = ldg(a.ir + q);
                if constexpr (T::kQuant) scm = ldg(a.sc + q);
            }
        }
    };
    // Column data of a chunk: lane k holds cp[c0 + k], 1/C and f of column c0 + k, and whether
    // its slice has stopped; every lane holds the chunk's end pointer.
    auto col_meta = [&](int ch, int& cpt, int& cend, N2& icm, V2& fm, int& skip) {
        const int c0 = ch * kColChunk, c = c0 + lane;
        cpt = 0;
        cend = 0;
        icm = N2{};
        fm = V2{};
        skip = 1;
        if (ch < ncc) {
            cpt = __ldg(a.cp + min(c, n_nzc));
            cend = __ldg(a.cp + min(c0 + kColChunk, n_nzc));
            if (c < n_nzc) {
                icm = ldg(a.ic + c);
                fm = ldcg(a.fc + c);
                skip = 0;
                if constexpr (kBatch) skip = __ldcg(&a.sl_solve[__ldg(a.cs + c)].done);
            }
        }
    };

    for (int k = 0;; ++k) {
        // ---- forward: r = p - A f and u = r / R per compacted row ----
        SqAcc<Acc> rr;
        if (blockIdx.x == 0 && tid == 0) a.ctl->work[1] = 0;  // the back pass's counter, idle until the barrier
        int grab = 0;
        if (lane == 0) grab = atomicAdd(&a.ctl->work[0], 1u);
        int chunk = __shfl_sync(kFull, grab, 0);
        int ptr;
        V2 pm;
        N2 irm;
        float2 scm;
        row_meta(chunk, ptr, pm, irm, scm);
        while (chunk < nrc) {
            if (lane == 0) grab = atomicAdd(&a.ctl->work[0], 1u);
            const int nchunk = __shfl_sync(kFull, grab, 0);
            int nptr;
            V2 npm;
            N2 nirm;
            float2 nscm;
            row_meta(nchunk, nptr, npm, nirm, nscm);  // the next chunk's row data loads while this one runs
            const int q0 = chunk * kRowChunk, nq = min(kRowChunk, n_nzr - q0);
            // Step (l, r): round r of chunk rows l .. l + R - 1 (warp-uniform bounds).
            auto row_bounds = [&](int l, int (&lo)[R], int (&hi)[R], int& len) {
                len = 0;
#pragma unroll
                for (int g = 0; g < R; ++g) {
                    const bool has = l + g < nq;
                    const int b0 = __shfl_sync(kFull, ptr, min(l + g, kRowChunk));
                    const int b1 = __shfl_sync(kFull, ptr, min(l + g + 1, kRowChunk));
                    lo[g] = has ? b0 : 0;
                    hi[g] = has ? b1 : 0;
                    len = max(len, hi[g] - lo[g]);
                }
            };
            int l = 0, r = 0, len;
            int lo[R], hi[R];
            row_bounds(0, lo, hi, len);
            StepBuf<Val, R, UF> cur;
            load_step(kUF, cur, a.ci, a.cv, lo, hi, 0, lane, 32);
            Acc s1[R], s2[R];
#pragma unroll
            for (int g = 0; g < R; ++g) s1[g] = s2[g] = 0;
            while (true) {
                const bool lastr = (r + 1) * kRoundF >= len;
                const int nl = lastr ? l + R : l, nr = lastr ? 0 : r + 1;
                const bool more = nl < nq;
                int nlo[R], nhi[R], nlen = len;
#pragma unroll
                for (int g = 0; g < R; ++g) {
                    nlo[g] = lo[g];
                    nhi[g] = hi[g];
                }
                if (more && lastr) row_bounds(nl, nlo, nhi, nlen);
                use_step(kUF, cur, a.fc, lo, hi, r * kRoundF, lane, 32, s1, s2);
                if (lastr) {
#pragma unroll
                    for (int g = 0; g < R; ++g) {
                        s1[g] = warp_sum(s1[g]);
                        s2[g] = warp_sum(s2[g]);
                    }
                    // Lane l + g finishes row q0 + l + g, with the p and 1/R it holds.
                    const int g = lane - l;
                    if (g >= 0 && g < R && lane < nq) {
                        Acc t1 = s1[0], t2 = s2[0];
#pragma unroll
                        for (int h = 1; h < R; ++h)
                            if (g == h) {
                                t1 = s1[h];
                                t2 = s2[h];
                            }
                        if constexpr (T::kQuant) {  // codes times the row's scale; 1/R already holds it for u
                            t1 *= scm.x;
                            t2 *= scm.y;
                        }
                        const Acc r1 = pm.x - t1, r2 = pm.y - t2;
                        stcg(a.uc + q0 + lane, V2{r1 * irm.x, r2 * irm.y});
                        if constexpr (kBatch) __stcg(a.rr + q0 + lane, (double)(r1 * r1 + r2 * r2));
                        else rr.add(r1, r2);
                    }
#pragma unroll
                    for (int h = 0; h < R; ++h) s1[h] = s2[h] = 0;
                }
                if (!more) break;
                load_step(kUF, cur, a.ci, a.cv, nlo, nhi, nr * kRoundF, lane, 32);
                l = nl;
                r = nr;
                len = nlen;
#pragma unroll
                for (int g = 0; g < R; ++g) {
                    lo[g] = nlo[g];
                    hi[g] = nhi[g];
                }
            }
            chunk = nchunk;
            ptr = nptr;
            pm = npm;
            irm = nirm;
            scm = nscm;
        }
        if constexpr (!kBatch) st_rr_partial(rr.sum(), ppz, a.partials, s_red);
        if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;

        const int stop = st_stop_test<T, kImplicit, kBatch>(a, k, s_red, s_tpp, &s_stop, nbar);
        if (stop != 0) return;  // stopped (f written back), or a barrier wait failed

        // ---- back-projection and update: f += lambda (A^T u) / C per compacted column ----
        if (blockIdx.x == 0 && tid == 0) a.ctl->work[0] = 0;  // the forward pass's counter, idle until the barrier
        if (lane == 0) grab = atomicAdd(&a.ctl->work[1], 1u);
        chunk = __shfl_sync(kFull, grab, 0);
        int cpt, cend, cskip;
        N2 icm;
        V2 fm;
        col_meta(chunk, cpt, cend, icm, fm, cskip);
        while (chunk < ncc) {
            if (lane == 0) grab = atomicAdd(&a.ctl->work[1], 1u);
            const int nchunk = __shfl_sync(kFull, grab, 0);
            int ncpt, ncend, ncskip;
            N2 nicm;
            V2 nfm;
            col_meta(nchunk, ncpt, ncend, nicm, nfm, ncskip);
            const int c0 = chunk * kColChunk, ncol = min(kColChunk, n_nzc - c0);
            const int nsteps = (ncol + kColStep - 1) / kColStep;
            // This lane group's columns in step st, and the step's rounds (warp-uniform).
            auto step_bounds = [&](int st, int (&lo)[R], int (&hi)[R], int& nrounds) {
                int len = 0;
#pragma unroll
                for (int g = 0; g < R; ++g) {
                    const int kc = st * kColStep + g * kGroups + grp;
                    const int v0 = __shfl_sync(kFull, cpt, kc & 31), v1 = __shfl_sync(kFull, cpt, (kc + 1) & 31);
                    lo[g] = v0;
                    hi[g] = kc + 1 >= kColChunk ? cend : v1;
                    len = max(len, hi[g] - lo[g]);
                }
                nrounds = max(1, (int)__reduce_max_sync(kFull, (unsigned)((len + kRoundB - 1) / kRoundB)));
            };
            int st = 0, r = 0, nrounds;
            int lo[R], hi[R];
            step_bounds(0, lo, hi, nrounds);
            StepBuf<Val, R, UB> cur;
            load_step(kUB, cur, a.ri, a.rv, lo, hi, 0, sub, LPC);
            Acc b1[R], b2[R];
#pragma unroll
            for (int g = 0; g < R; ++g) b1[g] = b2[g] = 0;
            while (true) {
                const bool lastr = r + 1 >= nrounds;
                const int nst = lastr ? st + 1 : st, nr = lastr ? 0 : r + 1;
                const bool more = nst < nsteps;
                int nlo[R], nhi[R], nR = nrounds;
#pragma unroll
                for (int g = 0; g < R; ++g) {
                    nlo[g] = lo[g];
                    nhi[g] = hi[g];
                }
                if (more && lastr) step_bounds(nst, nlo, nhi, nR);
                use_step(kUB, cur, a.uc, lo, hi, r * kRoundB, sub, LPC, b1, b2);
                if (lastr) {
#pragma unroll
                    for (int g = 0; g < R; ++g) {
                        b1[g] = warp_sum(b1[g], LPC);
                        b2[g] = warp_sum(b2[g], LPC);
                    }
                    // Lane k finishes column c0 + k with the data it holds; its sums come from
                    // lane (t mod groups) LPC, item t / groups, where t is k's place in the step.
                    const int t = lane - st * kColStep;
                    const bool in = t >= 0 && t < kColStep;
                    const int src = (in ? t % kGroups : 0) * LPC, item = in ? t / kGroups : 0;
                    Acc y1 = 0, y2 = 0;
#pragma unroll
                    for (int g = 0; g < R; ++g) {
                        const Acc z1 = __shfl_sync(kFull, b1[g], src), z2 = __shfl_sync(kFull, b2[g], src);
                        if (item == g) {
                            y1 = z1;
                            y2 = z2;
                        }
                    }
                    if (in && lane < ncol && !cskip) {
                        fm.x += lam * y1 * icm.x;
                        fm.y += lam * y2 * icm.y;
                        stcg(a.fc + c0 + lane, fm);
                    }
#pragma unroll
                    for (int g = 0; g < R; ++g) b1[g] = b2[g] = 0;
                }
                if (!more) break;
                load_step(kUB, cur, a.ri, a.rv, nlo, nhi, nr * kRoundB, sub, LPC);
                st = nst;
                r = nr;
                nrounds = nR;
#pragma unroll
                for (int g = 0; g < R; ++g) {
                    lo[g] = nlo[g];
                    hi[g] = nhi[g];
                }
            }
            chunk = nchunk;
            cpt = ncpt;
            cend = ncend;
            cskip = ncskip;
            icm = nicm;
            fm = nfm;
        }
        if (!grid_sync(a.ctl, (unsigned long long)a.expected * ++nbar, a.timeout_ns, (int)nbar)) return;
    }
}

}  // namespace
}  // namespace splitsart

namespace splitsart {
namespace {

// Step shape: items per step and entries in flight per lane and item. On the
// 256-slice batch (FP32, 200 iterations) two rows per step without a second
// register buffer for the next step's loads was the fastest of the shapes
// measured: 646 ms explicit (4 entries per lane forward, 3 back) and 574 ms
// implicit (5 and 4), against 817/682 ms for one row per step with the next
// step's loads issued ahead, 788/740 ms for two rows with them, 672/615 ms for
// one row with 8 entries per lane, and 1054/662 ms for two rows with 6 and 5.
// kNarrow: 4-byte values per entry (the implicit fold's FP32 lengths, or BF16/FP16
// code pairs); kWide: FP64 vectors.
template <bool kNarrow, bool kWide>
struct PipeShape {
    static constexpr int R = 2;
    static constexpr int UF = kWide ? 2 : (kNarrow ? 5 : 4);
    static constexpr int UB = kWide ? 2 : (kNarrow ? 4 : 3);
};

template <class T, bool kImplicit, int LPC>
int launch_pipe(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st) {
    using V2 = typename T::Vec2;
    constexpr bool kWide = sizeof(V2) == 16;
    using Shape = PipeShape<kImplicit || T::kQuant, kWide>;  // 2-byte codes take registers like the implicit fold
    constexpr int UF = Shape::UF, UB = Shape::UB, R = Shape::R;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "solve: cudaGetDevice");
    int nsm = 0, coop = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return fail(SPLITSART_ERR_CUDA, "solve: device lacks cooperative launch");
    int threads = o.block_threads > 0 ? o.block_threads : 512;
    if (threads % 32 != 0 || threads > 1024 || threads < 64)
        return fail(SPLITSART_ERR_ARG, "solve: block_threads must be a multiple of 32 in [64, 1024]");
    if (threads > 512) threads = 512;
    FoldStats fs;
    int rc = system_host_stats(s, &fs);
    if (rc) return rc;
    rc = build_stream_format<T>(s, kImplicit ? 1 : 0, fs, st);
    if (rc) return rc;
    const StreamFmt& F = s->st[kImplicit ? 1 : 0];
    const bool batch = s->ns > 1;
    void* kern = batch ? (void*)sart_compact_kernel<T, kImplicit, true, LPC, UF, UB, R>
                       : (void*)sart_compact_kernel<T, kImplicit, false, LPC, UF, UB, R>;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
    if (e != cudaSuccess) return cuda_fail(e, "solve: occupancy");
    if (per_sm < 1) return fail(SPLITSART_ERR_CUDA, "solve: kernel does not fit on an SM");
    if (o.ctas_per_sm > 0 && o.ctas_per_sm < per_sm) per_sm = o.ctas_per_sm;
    int grid = nsm * per_sm;
    if (grid > kMaxCtas) grid = kMaxCtas;

    StArgs<T, kImplicit> a = st_args<T, kImplicit>(s, F, p12, f12, o, grid);
    if ((rc = st_reset(s, st)) != SPLITSART_OK) return rc;
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(threads), args, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "solve: cooperative launch");
    return SPLITSART_OK;
}

template <class T, bool kImplicit>
int launch_pipe_lpc(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st) {
    switch (o.lanes_per_col > 0 ? o.lanes_per_col : 4) {
        case 4: return launch_pipe<T, kImplicit, 4>(s, p12, f12, o, st);
        case 8: return launch_pipe<T, kImplicit, 8>(s, p12, f12, o, st);
    }
    return fail(SPLITSART_ERR_ARG, "solve: kernels 5 and 6 take lanes_per_col 4 or 8");
}

}  // namespace

int stream_format(splitsart_system* s, int kind, cudaStream_t st) {
    FoldStats fs;
    const int rc = system_host_stats(s, &fs);
    if (rc) return rc;
    switch (s->dtype) {
        case SPLITSART_F64: return build_stream_format<TF64>(s, kind, fs, st);
        case SPLITSART_F32: return build_stream_format<TF32>(s, kind, fs, st);
        case SPLITSART_BF16: return build_stream_format<TBF16>(s, kind, fs, st);
        case SPLITSART_F16: return build_stream_format<TF16>(s, kind, fs, st);
    }
    return fail(SPLITSART_ERR_ARG, "solve: unknown value storage");
}

int run_solve_stream(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st) {
    const bool imp = o.kernel == 6;
    if (!imp && s->dtype == SPLITSART_BF16) return launch_pipe_lpc<TBF16, false>(s, p12, f12, o, st);
    if (!imp && s->dtype == SPLITSART_F16) return launch_pipe_lpc<TF16, false>(s, p12, f12, o, st);
    switch (s->dtype) {
        case SPLITSART_F64:
            return imp ? launch_pipe_lpc<TF64, true>(s, p12, f12, o, st) : launch_pipe_lpc<TF64, false>(s, p12, f12, o, st);
        case SPLITSART_F32:
            return imp ? launch_pipe_lpc<TF32, true>(s, p12, f12, o, st) : launch_pipe_lpc<TF32, false>(s, p12, f12, o, st);
    }
    return fail(SPLITSART_ERR_ARG, "solve: kernel 6 takes FP64 and FP32 systems (kernel 5 also BF16 and FP16)");
}

}  // namespace splitsart
