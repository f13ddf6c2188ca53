// Fold of the system and the small vector kernels around the solve.
//
// - Fold of A (formulas after Eq. 4): w1_ij = w_ij - w_{M-1-i,j},
//   w2_ij = w_ij + w_{M-1-i,j}, i < Mh, j < Nh. Eq. (2) gives
//   w_{M-1-i,j} = w_{i,N-1-j}, so folded row i needs row i of A alone.
//   Row i's columns are sorted. Its entries with j < Nh, read forward, and its
//   entries with j >= Nh, read backward and reflected to N-1-j, are then two
//   ascending lists. The folded row is their merge. Columns present in both
//   lists give one entry, (w_d - w_r, w_d + w_r).
// - Fold of p (after Eq. 4), fold of an image (proof of Theorem 1),
//   recombination (Theorem 1, Eq. 5), and forward projection through the
//   folded system.
// - A deterministic CSC transpose. Columns are counted, scanned and placed
//   with atomics, then each column is sorted by row. The absolute row and
//   column sums come last, in FP64, with 1/0 := 0.
// The per-row and per-column kernels run one warp per item. A half row is
// staged in shared memory with coalesced loads, and the union of its two
// sorted lists is formed by a merge path whose positions are split evenly
// over the lanes, so the FP64 work is spread over all 32 lanes.
#include <climits>
#include <cstdio>

#include "device_common.cuh"
#include "system.h"

namespace splitsart {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Warp-per-item kernels: warps per block, and the entries one warp stages in
// shared memory (longer items are read from global memory instead).
constexpr int kFoldWarps = 8;
constexpr int kRowCap = 1024;  // half-row entries
constexpr int kColCap = 256;   // CSC column entries

// The two ascending lists of half row i: L, its entries with column < N/2 in
// stored order, and R', its entries with column >= N/2 read backward and
// reflected to N-1-j. c and v point at the row's stored columns and values
// (in shared or in global memory); nL is the length of L.
struct HalfRow {
    const int32_t* c;
    const double* v;
    int n, nL, N;
    __device__ __forceinline__ int Lc(int a) const { return c[a]; }
    __device__ __forceinline__ int Rc(int b) const { return N - 1 - c[n - 1 - b]; }
    __device__ __forceinline__ double Lv(int a) const { return v[a]; }
    __device__ __forceinline__ double Rv(int b) const { return v[n - 1 - b]; }
};

// Merge path: the number of L items among the first d items of the merged
// order, in which L goes first on equal columns.
__device__ __forceinline__ int merge_split(const HalfRow& h, int d) {
    int lo = max(0, d - (h.n - h.nL)), hi = min(d, h.nL);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (h.Lc(mid) <= h.Rc(d - mid - 1)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Visit the merged positions [d0, d1) in ascending column order and call
// fn(col, w_direct, w_reflected) once per folded column, with 0.0 for an
// absent side. A column in both lists is visited at its L item; its R' twin,
// which comes next in the merged order, is skipped wherever it falls.
template <class F>
__device__ __forceinline__ void merge_walk(const HalfRow& h, int d0, int d1, F&& fn) {
    const int nR = h.n - h.nL;
    int a = merge_split(h, d0), b = d0 - a;
    for (int d = d0; d < d1; ++d) {
        if (a < h.nL && (b >= nR || h.Lc(a) <= h.Rc(b))) {
            const int c = h.Lc(a);
            const bool twin = b < nR && h.Rc(b) == c;
            fn(c, h.Lv(a), twin ? h.Rv(b) : 0.0);
            ++a;
        } else {
            const int c = h.Rc(b);
            if (!(a > 0 && h.Lc(a - 1) == c)) fn(c, 0.0, h.Rv(b));
            ++b;
        }
    }
}

__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The slice holding global index i: the largest s with off[s] <= i.
__device__ __forceinline__ int slice_of(const long long* off, int ns, long long i) {
    int lo = 0, hi = ns;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// One warp stages half row i (warp-uniform): returns the HalfRow view.
__device__ __forceinline__ HalfRow stage_half_row(const int64_t* __restrict__ hrp, const int32_t* __restrict__ hcol,
                                                  const double* __restrict__ hval, int64_t i, int N, int32_t* sc,
                                                  double* sv, int lane) {
    const int64_t e0 = hrp[i];
    const int n = (int)(hrp[i + 1] - e0);
    const bool staged = n <= kRowCap;
    const int Nh = N >> 1;
    int nL = 0;
    for (int t0 = 0; t0 < n; t0 += 32) {
        const int t = t0 + lane;
        int c = INT_MAX;
        if (t < n) {
            c = hcol[e0 + t];
            if (staged) {
                sc[t] = c;
                sv[t] = hval[e0 + t];
            }
        }
        nL += __popc(__ballot_sync(0xffffffffu, c < Nh));
    }
    __syncwarp();
    return staged ? HalfRow{sc, sv, n, nL, N} : HalfRow{hcol + e0, hval + e0, n, nL, N};
}

// Folded entries per row: one warp per row, the merged order split evenly over the lanes.
__global__ void __launch_bounds__(kFoldWarps * 32) fold_count_kernel(int64_t Mh, SliceMap sm,
                                                                     const int64_t* __restrict__ hrp,
                                                                     const int32_t* __restrict__ hcol,
                                                                     const double* __restrict__ hval,
                                                                     int32_t* __restrict__ cnt) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = blockIdx.x * (int64_t)kFoldWarps + w;
    if (i >= Mh) return;
    double* sv = reinterpret_cast<double*>(smem) + (size_t)w * kRowCap;
    int32_t* sc = reinterpret_cast<int32_t*>(smem + (size_t)kFoldWarps * kRowCap * 8) + (size_t)w * kRowCap;
    const int s = slice_of(sm.rows, sm.ns, i);
    const HalfRow h = stage_half_row(hrp, hcol, hval, i, (int)(sm.N[s + 1] - sm.N[s]), sc, sv, lane);
    int n = 0;
    merge_walk(h, (int)((long long)lane * h.n / 32), (int)((long long)(lane + 1) * h.n / 32),
               [&](int, double, double) { ++n; });
    n = warp_sum(n);
    if (lane == 0) cnt[i] = n;
}

// Exclusive scan of cnt[0..n) into out[0..n]; out[n] = total.
__global__ void scan_tiles_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                  int32_t* __restrict__ tile_sums, int64_t n) {
    __shared__ int32_t warp_tot[kScanThreads / 32];
    const int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * (int64_t)kScanItems;
    int32_t v[kScanItems];
    int32_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        run += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = run;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int32_t w = warp_tot[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        warp_tot[lane] = w;  // inclusive
    }
    __syncthreads();
    int32_t excl = incl - run + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = excl;
        excl += v[k];
    }
    if (threadIdx.x == kScanThreads - 1) tile_sums[blockIdx.x] = warp_tot[31];
}

__global__ void scan_tile_sums_kernel(int32_t* __restrict__ tile_sums, int ntiles) {
    // One CTA: exclusive scan of the tile sums, in chunks carried forward.
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b0 = 0; b0 < ntiles; b0 += blockDim.x) {
        const int idx = b0 + threadIdx.x;
        const int32_t v = idx < ntiles ? tile_sums[idx] : 0;
        int32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int32_t w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int32_t t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        const int32_t excl = carry + incl - v + (warp > 0 ? warp_tot[warp - 1] : 0);
        if (idx < ntiles) tile_sums[idx] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) tile_sums[ntiles] = carry;
}

__global__ void scan_add_kernel(int32_t* __restrict__ out, const int32_t* __restrict__ tile_sums, int64_t n,
                                int ntiles) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_sums[i / kScanTile];
    if (i == 0) out[n] = tile_sums[ntiles];
}

int exclusive_scan(const int32_t* in, int32_t* out, int32_t* tile_sums, int64_t n, cudaStream_t st) {
    const int ntiles = (int)((n + kScanTile - 1) / kScanTile);
    if (ntiles == 0) {
        cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int32_t), st);
        return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "scan");
    }
    scan_tiles_kernel<<<ntiles, kScanThreads, 0, st>>>(in, out, tile_sums, n);
    scan_tile_sums_kernel<<<1, 1024, 0, st>>>(tile_sums, ntiles);
    scan_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, tile_sums, n, ntiles);
    return SPLITSART_OK;
}

template <class T>
__device__ __forceinline__ void store_pair(typename T::Pair* p, double a1, double a2, float s1, float s2,
                                           double& d1, double& d2) {
    if constexpr (T::kDtype == SPLITSART_F64) {
        *p = make_double2(a1, a2);
        d1 = a1;
        d2 = a2;
    } else if constexpr (T::kDtype == SPLITSART_F32) {
        const float f1 = (float)a1, f2 = (float)a2;
        *p = make_float2(f1, f2);
        d1 = f1;
        d2 = f2;
    } else {
        // Codes q = round(a / s), with the division and the rounding in FP32.
        const float q1 = s1 > 0.f ? __fdiv_rn((float)a1, s1) : 0.f;
        const float q2 = s2 > 0.f ? __fdiv_rn((float)a2, s2) : 0.f;
        const typename T::Pair q = T::encode(q1, q2);
        *p = q;
        float c1, c2;
        T::decode(q, c1, c2);
        d1 = (double)s1 * (double)c1;  // exact: 24-bit x 11-bit mantissas
        d2 = (double)s2 * (double)c2;
    }
}

// Folded row i: columns, value pairs (quantised with the row's scales for
// BF16/FP16), and the FP64 absolute row sums of the stored values.
template <class T>
__global__ void __launch_bounds__(kFoldWarps * 32) fold_fill_kernel(
    int64_t Mh, SliceMap sm, const int64_t* __restrict__ hrp, const int32_t* __restrict__ hcol,
    const double* __restrict__ hval, const int32_t* __restrict__ frp, int32_t* __restrict__ col,
    typename T::Pair* __restrict__ val, double2* __restrict__ Rsum, typename T::Norm2* __restrict__ invR,
    float2* __restrict__ scale, float2* __restrict__ wR, FoldStats* __restrict__ stats) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = blockIdx.x * (int64_t)kFoldWarps + w;
    if (i >= Mh) return;
    double* sv = reinterpret_cast<double*>(smem) + (size_t)w * kRowCap;
    int32_t* sc = reinterpret_cast<int32_t*>(smem + (size_t)kFoldWarps * kRowCap * 8) + (size_t)w * kRowCap;
    const int sl = slice_of(sm.rows, sm.ns, i);
    const int col_base = (int)sm.cols[sl];  // folded columns of this slice start here
    const HalfRow h = stage_half_row(hrp, hcol, hval, i, (int)(sm.N[sl + 1] - sm.N[sl]), sc, sv, lane);
    const int d0 = (int)((long long)lane * h.n / 32), d1 = (int)((long long)(lane + 1) * h.n / 32);
    float s1 = 0.f, s2 = 0.f;
    if constexpr (T::kQuant) {
        double m1 = 0.0, m2 = 0.0;
        merge_walk(h, d0, d1, [&](int, double wd, double wr) {
            m1 = fmax(m1, fabs(wd - wr));
            m2 = fmax(m2, fabs(wd + wr));
        });
        s1 = (float)warp_max(m1);
        s2 = (float)warp_max(m2);
        if (lane == 0) scale[i] = make_float2(s1, s2);
    }
    // Output position of this lane's first column: an exclusive scan of the lanes' counts.
    int n = 0;
    merge_walk(h, d0, d1, [&](int, double, double) { ++n; });
    int incl = n;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int32_t first = frp[i];
    int32_t out = first + incl - n;
    double R1 = 0.0, R2 = 0.0;
    long long zeros = 0;
    merge_walk(h, d0, d1, [&](int c, double wd, double wr) {
        const double a1 = wd - wr, a2 = wd + wr;
        zeros += (a1 == 0.0);
        col[out] = col_base + c;
        double q1, q2;
        store_pair<T>(&val[out], a1, a2, s1, s2, q1, q2);
        R1 += fabs(q1);
        R2 += fabs(q2);
        ++out;
    });
    R1 = warp_sum(R1);
    R2 = warp_sum(R2);
    zeros = warp_sum(zeros);
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (lane == 0) {
        Rsum[i] = make_double2(R1, R2);
        using N2 = typename T::Norm2;
        using NS = decltype(N2{}.x);
        const double i1 = R1 > 0.0 ? 1.0 / R1 : 0.0, i2 = R2 > 0.0 ? 1.0 / R2 : 0.0;
        invR[i] = N2{(NS)i1, (NS)i2};
        // What the iteration applies: the row scale times 1/R, rounded once to FP32.
        if constexpr (T::kQuant) wR[i] = make_float2((float)(i1 * (double)s1), (float)(i2 * (double)s2));
        if (total == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&stats->empty_rows), 1ULL);
        else atomicMax(&stats->max_row, total);
        if (zeros) atomicAdd(reinterpret_cast<unsigned long long*>(&stats->exact_zeros), (unsigned long long)zeros);
        if (i == Mh - 1) stats->S = frp[Mh];
    }
}

__global__ void csc_count_kernel(const int32_t* __restrict__ frp, int64_t Mh, int64_t cap,
                                 const int32_t* __restrict__ col, int32_t* __restrict__ ccnt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= cap || e >= frp[Mh]) return;
    atomicAdd(&ccnt[col[e]], 1);
}

// Place each folded entry in its column: one warp per row, lanes over the row's
// entries. The order within a column is fixed afterwards by the sort.
template <class T>
__global__ void __launch_bounds__(kFoldWarps * 32) csc_place_kernel(
    int64_t Mh, const int32_t* __restrict__ frp, const int32_t* __restrict__ col,
    const typename T::Pair* __restrict__ val, const int32_t* __restrict__ cp, int32_t* __restrict__ cursor,
    int32_t* __restrict__ row, typename T::Pair* __restrict__ valT) {
    const int lane = threadIdx.x & 31;
    const int64_t i = blockIdx.x * (int64_t)kFoldWarps + (threadIdx.x >> 5);
    if (i >= Mh) return;
    for (int32_t e = frp[i] + lane; e < frp[i + 1]; e += 32) {
        const int32_t c = col[e];
        const int32_t pos = cp[c] + atomicAdd(&cursor[c], 1);
        row[pos] = (int32_t)i;
        valT[pos] = val[e];
    }
}

// Sort each column's entries by row, then take the FP64 absolute column sums
// in that order (lane-strided, fixed tree). One warp per column. A column of
// up to kColCap entries is ranked in shared memory (rows within a column are
// distinct, so an entry's rank is the number of smaller rows); a longer one is
// sorted in place by one lane.
template <class T>
__global__ void __launch_bounds__(kFoldWarps * 32) csc_sort_colsum_kernel(
    int64_t Nh, const int32_t* __restrict__ cp, int32_t* __restrict__ row, typename T::Pair* __restrict__ valT,
    const float2* __restrict__ scale, double2* __restrict__ Csum, typename T::Norm2* __restrict__ invC,
    float2* __restrict__ wC, FoldStats* __restrict__ stats) {
    using Pair = typename T::Pair;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t j = blockIdx.x * (int64_t)kFoldWarps + w;
    if (j >= Nh) return;
    Pair* sv = reinterpret_cast<Pair*>(smem) + (size_t)w * 2 * kColCap;                 // unsorted, then sorted
    int32_t* sr = reinterpret_cast<int32_t*>(smem + (size_t)kFoldWarps * 2 * kColCap * sizeof(Pair)) +
                  (size_t)w * 2 * kColCap;
    const int32_t b = cp[j], e = cp[j + 1];
    const int n = e - b;
    if (n <= kColCap) {
        for (int t = lane; t < n; t += 32) {
            sr[t] = row[b + t];
            sv[t] = valT[b + t];
        }
        __syncwarp();
        for (int t = lane; t < n; t += 32) {
            const int32_t r = sr[t];
            int rank = 0;
            for (int u = 0; u < n; ++u) rank += sr[u] < r;
            sr[kColCap + rank] = r;
            sv[kColCap + rank] = sv[t];
        }
        __syncwarp();
        for (int t = lane; t < n; t += 32) {
            row[b + t] = sr[kColCap + t];
            valT[b + t] = sv[kColCap + t];
        }
    } else if (lane == 0) {
        for (int32_t k = b + 1; k < e; ++k) {
            const int32_t r = row[k];
            const Pair v = valT[k];
            int32_t m = k - 1;
            while (m >= b && row[m] > r) {
                row[m + 1] = row[m];
                valT[m + 1] = valT[m];
                --m;
            }
            row[m + 1] = r;
            valT[m + 1] = v;
        }
    }
    __syncwarp();
    double C1 = 0.0, C2 = 0.0;
    for (int t = lane; t < n; t += 32) {
        const bool st = n <= kColCap;
        typename T::Acc a1, a2;
        T::decode(st ? sv[kColCap + t] : valT[b + t], a1, a2);
        double d1 = a1, d2 = a2;
        if constexpr (T::kQuant) {
            const float2 sc = scale[st ? sr[kColCap + t] : row[b + t]];
            d1 = (double)sc.x * d1;
            d2 = (double)sc.y * d2;
        }
        C1 += fabs(d1);
        C2 += fabs(d2);
    }
    C1 = warp_sum(C1);
    C2 = warp_sum(C2);
    if (lane == 0) {
        Csum[j] = make_double2(C1, C2);
        if (n > 0) atomicMax(&stats->max_col, n);
        using N2 = typename T::Norm2;
        using NS = decltype(N2{}.x);
        const double i1 = C1 > 0.0 ? 1.0 / C1 : 0.0, i2 = C2 > 0.0 ? 1.0 / C2 : 0.0;
        invC[j] = N2{(NS)i1, (NS)i2};
        if constexpr (T::kQuant) wC[j] = make_float2((float)i1, (float)i2);
    }
}

__global__ void nonempty_flags_kernel(int64_t n, const int32_t* __restrict__ ptr, int32_t* __restrict__ flags) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flags[i] = ptr[i + 1] > ptr[i];
}

// Split 0..n-1 into the indices with entries (nzlist, with their pointers
// nzptr) and those without (zlist). pos is the exclusive scan of the flags.
// The order is increasing in both lists, so the result is deterministic.
__global__ void compact_kernel(int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ pos,
                               int32_t* __restrict__ nzlist, int32_t* __restrict__ nzptr, int32_t* __restrict__ zlist,
                               int* __restrict__ n_nz, int* __restrict__ n_z) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (ptr[i + 1] > ptr[i]) {
        nzlist[pos[i]] = (int32_t)i;
        nzptr[pos[i]] = ptr[i];
    } else if (zlist) {
        zlist[i - pos[i]] = (int32_t)i;
    }
    if (i == 0) {
        const int total = pos[n];
        nzptr[total] = ptr[n];
        *n_nz = total;
        if (n_z) *n_z = (int)(n - total);
    }
}

int compact(const int32_t* ptr, int64_t n, int32_t* flags, int32_t* pos, int32_t* tile_sums, int32_t* nzlist,
            int32_t* nzptr, int32_t* zlist, int* n_nz, int* n_z, cudaStream_t st) {
    if (n == 0) return SPLITSART_OK;
    const unsigned g = (unsigned)((n + 255) / 256);
    nonempty_flags_kernel<<<g, 256, 0, st>>>(n, ptr, flags);
    int rc = exclusive_scan(flags, pos, tile_sums, n, st);
    if (rc) return rc;
    compact_kernel<<<g, 256, 0, st>>>(n, ptr, pos, nzlist, nzptr, zlist, n_nz, n_z);
    return SPLITSART_OK;
}

template <class T>
int fold_typed(splitsart_system* s, cudaStream_t st) {
    using Pair = typename T::Pair;
    using N2 = typename T::Norm2;
    const int64_t Mh = s->Mh, Nh = s->Nh;
    cudaError_t e;
    if ((e = cudaMemsetAsync(s->stats, 0, sizeof(FoldStats), st)) != cudaSuccess) return cuda_fail(e, "fold memset");
    const SliceMap sm = slice_map(s);
    const size_t row_smem = (size_t)kFoldWarps * kRowCap * (8 + 4);
    const size_t col_smem = (size_t)kFoldWarps * 2 * kColCap * (sizeof(Pair) + 4);
    cudaFuncSetAttribute((const void*)fold_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem);
    cudaFuncSetAttribute((const void*)fold_fill_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem);
    cudaFuncSetAttribute((const void*)csc_sort_colsum_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)col_smem);
    const unsigned row_blocks = (unsigned)((Mh + kFoldWarps - 1) / kFoldWarps);
    const unsigned col_blocks = (unsigned)((Nh + kFoldWarps - 1) / kFoldWarps);
    if (Mh > 0)
        fold_count_kernel<<<row_blocks, kFoldWarps * 32, row_smem, st>>>(Mh, sm, s->hrp, s->hcol, s->hval, s->cnt);
    int rc = exclusive_scan(s->cnt, s->rp, s->scan_tmp, Mh, st);
    if (rc) return rc;
    if (Mh > 0)
        fold_fill_kernel<T><<<row_blocks, kFoldWarps * 32, row_smem, st>>>(
            Mh, sm, s->hrp, s->hcol, s->hval, s->rp, s->col, (Pair*)s->val, s->Rsum, (N2*)s->invR, s->scale, s->wR,
            s->stats);
    rc = compact(s->rp, Mh, s->flags, s->cnt, s->scan_tmp, s->nzr, s->nzrp, s->zr, &s->stats->n_nzr,
                 &s->stats->n_zr, st);
    if (rc) return rc;
    // CSC.
    if ((e = cudaMemsetAsync(s->cnt, 0, sizeof(int32_t) * (Nh + 1), st)) != cudaSuccess)
        return cuda_fail(e, "fold memset");
    if (s->nnz_half > 0)
        csc_count_kernel<<<(unsigned)((s->nnz_half + 255) / 256), 256, 0, st>>>(s->rp, Mh, s->nnz_half, s->col,
                                                                                 s->cnt);
    rc = exclusive_scan(s->cnt, s->cp, s->scan_tmp, Nh, st);
    if (rc) return rc;
    if ((e = cudaMemsetAsync(s->cnt, 0, sizeof(int32_t) * (Nh + 1), st)) != cudaSuccess)
        return cuda_fail(e, "fold memset");
    if (Mh > 0)
        csc_place_kernel<T><<<row_blocks, kFoldWarps * 32, 0, st>>>(Mh, s->rp, s->col, (const Pair*)s->val, s->cp,
                                                                    s->cnt, s->row, (Pair*)s->valT);
    if (Nh > 0)
        csc_sort_colsum_kernel<T><<<col_blocks, kFoldWarps * 32, col_smem, st>>>(
            Nh, s->cp, s->row, (Pair*)s->valT, s->scale, s->Csum, (N2*)s->invC, s->wC, s->stats);
    rc = compact(s->cp, Nh, s->flags, s->cnt, s->scan_tmp, s->nzc, s->nzcp, nullptr, &s->stats->n_nzc, nullptr, st);
    if (rc) return rc;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fold launch");
    return SPLITSART_OK;
}

// ---- vector kernels (all slices at once; each index finds its slice) ----

__device__ __forceinline__ int64_t image_index(int64_t j, int nx, int nz) {
    const int64_t c = j / nz, q = j % nz;
    const int64_t r = (c & 1) ? (nz - 1 - q) : q;
    return r * nx + c;
}

// Positions in the full image vector of folded column j and of its mirror.
__device__ __forceinline__ void image_pair(const SliceMap& sm, int layout, int64_t j, int64_t& a_idx, int64_t& b_idx) {
    const int s = slice_of(sm.cols, sm.ns, j);
    const int64_t lj = j - sm.cols[s];
    const int64_t Ns = sm.N[s + 1] - sm.N[s], base = sm.N[s];
    const int64_t lm = Ns - 1 - lj;
    if (layout == SPLITSART_LAYOUT_IMAGE) {
        a_idx = base + image_index(lj, sm.nx[s], sm.nz[s]);
        b_idx = base + image_index(lm, sm.nx[s], sm.nz[s]);
    } else {
        a_idx = base + lj;
        b_idx = base + lm;
    }
}

// Positions in the full projection vector of folded row i and of its mirror ray.
__device__ __forceinline__ void ray_pair(const SliceMap& sm, int64_t i, int64_t& a_idx, int64_t& b_idx) {
    const int s = slice_of(sm.rows, sm.ns, i);
    const int64_t li = i - sm.rows[s];
    const int64_t Ms = sm.M[s + 1] - sm.M[s], base = sm.M[s];
    a_idx = base + li;
    b_idx = base + Ms - 1 - li;
}

template <class V, class V2>
__global__ void fold_rhs_kernel(int64_t Mh, SliceMap sm, const V* __restrict__ p, V2* __restrict__ p12) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= Mh) return;
    int64_t ia, ib;
    ray_pair(sm, i, ia, ib);
    const V a = p[ia], b = p[ib];
    p12[i] = V2{a - b, a + b};
}

template <class V, class V2>
__global__ void fold_image_kernel(int64_t Nh, SliceMap sm, int layout, const V* __restrict__ f, V2* __restrict__ f12) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= Nh) return;
    int64_t ia, ib;
    image_pair(sm, layout, j, ia, ib);
    const V a = f[ia], b = f[ib];
    f12[j] = V2{a - b, a + b};
}

// Theorem 1, Eq. (5).
template <class V, class V2>
__global__ void recombine_kernel(int64_t Nh, SliceMap sm, int layout, const V2* __restrict__ f12, V* __restrict__ f) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= Nh) return;
    const V2 v = f12[j];
    int64_t ia, ib;
    image_pair(sm, layout, j, ia, ib);
    f[ia] = (v.y + v.x) / V(2);
    f[ib] = (v.y - v.x) / V(2);
}

// q = (A1 f1, A2 f2): one warp per folded row.
template <class T>
__global__ void spmv_pairs_kernel(int64_t Mh, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                  const typename T::Pair* __restrict__ val, const float2* __restrict__ scale,
                                  const typename T::Vec2* __restrict__ f12, typename T::Vec2* __restrict__ q12) {
    using Acc = typename T::Acc;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= Mh) return;
    Acc s1 = 0, s2 = 0;
    for (int32_t e = rp[w] + lane; e < rp[w + 1]; e += 32) {
        Acc a1, a2;
        T::decode(val[e], a1, a2);
        const typename T::Vec2 fv = f12[col[e]];
        s1 += a1 * fv.x;
        s2 += a2 * fv.y;
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane == 0) {
        if constexpr (T::kQuant) {
            const float2 sc = scale[w];
            s1 *= sc.x;
            s2 *= sc.y;
        }
        q12[w] = typename T::Vec2{s1, s2};
    }
}

// p_i = (q2 + q1)/2, p_{M-1-i} = (q2 - q1)/2: the fold of p, inverted.
template <class V, class V2>
__global__ void unfold_rays_kernel(int64_t Mh, SliceMap sm, const V2* __restrict__ q12, V* __restrict__ p) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= Mh) return;
    const V2 q = q12[i];
    int64_t ia, ib;
    ray_pair(sm, i, ia, ib);
    p[ia] = (q.y + q.x) / V(2);
    p[ib] = (q.y - q.x) / V(2);
}

template <class T>
int project_typed(splitsart_system* s, const void* f, int layout, void* p, cudaStream_t st) {
    using V = typename T::Acc;
    using V2 = typename T::Vec2;
    const int64_t Nh = s->Nh, Mh = s->Mh;
    const SliceMap sm = slice_map(s);
    if (Nh > 0)
        fold_image_kernel<V, V2><<<(unsigned)((Nh + 255) / 256), 256, 0, st>>>(Nh, sm, layout, (const V*)f,
                                                                              (V2*)s->tmp_f12);
    if (Mh > 0) {
        spmv_pairs_kernel<T><<<(unsigned)((Mh * 32 + 255) / 256), 256, 0, st>>>(
            Mh, s->rp, s->col, (const typename T::Pair*)s->val, s->scale, (const V2*)s->tmp_f12, (V2*)s->tmp_q12);
        unfold_rays_kernel<V, V2><<<(unsigned)((Mh + 255) / 256), 256, 0, st>>>(Mh, sm, (const V2*)s->tmp_q12, (V*)p);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "project launch");
}

}  // namespace

namespace {

// The implicit fold of the half rows: folded row i lists every entry of half
// row i once, in the merged column order of the fold (L before its R' twin on
// equal columns), as (global folded column with A1's sign in bit 31, w). The
// entry at merged position d goes to hrp[i] + d. One warp per row.
template <class V>
__global__ void __launch_bounds__(kFoldWarps * 32) implicit_rows_kernel(int64_t Mh, SliceMap sm,
                                                                        const int64_t* __restrict__ hrp,
                                                                        const int32_t* __restrict__ hcol,
                                                                        const double* __restrict__ hval,
                                                                        int32_t* __restrict__ out_col,
                                                                        V* __restrict__ out_val) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = blockIdx.x * (int64_t)kFoldWarps + w;
    if (i >= Mh) return;
    double* sv = reinterpret_cast<double*>(smem) + (size_t)w * kRowCap;
    int32_t* sc = reinterpret_cast<int32_t*>(smem + (size_t)kFoldWarps * kRowCap * 8) + (size_t)w * kRowCap;
    const int s = slice_of(sm.rows, sm.ns, i);
    const HalfRow h = stage_half_row(hrp, hcol, hval, i, (int)(sm.N[s + 1] - sm.N[s]), sc, sv, lane);
    const long long col0 = sm.cols[s];
    const int64_t e0 = hrp[i];
    const int d0 = (int)((long long)lane * h.n / 32), d1 = (int)((long long)(lane + 1) * h.n / 32);
    const int nR = h.n - h.nL;
    int a = merge_split(h, d0), b = d0 - a;
    for (int d = d0; d < d1; ++d) {
        if (a < h.nL && (b >= nR || h.Lc(a) <= h.Rc(b))) {
            out_col[e0 + d] = (int32_t)(col0 + h.Lc(a));
            out_val[e0 + d] = (V)h.Lv(a);
            ++a;
        } else {
            out_col[e0 + d] = (int32_t)((uint32_t)(col0 + h.Rc(b)) | 0x80000000u);
            out_val[e0 + d] = (V)h.Rv(b);
            ++b;
        }
    }
}

}  // namespace

int run_implicit_rows(const splitsart_system* s, bool fp64, int32_t* col, void* val, cudaStream_t st) {
    if (s->Mh <= 0) return SPLITSART_OK;
    const size_t row_smem = (size_t)kFoldWarps * kRowCap * (8 + 4);
    const unsigned row_blocks = (unsigned)((s->Mh + kFoldWarps - 1) / kFoldWarps);
    const SliceMap sm = slice_map(s);
    if (fp64) {
        cudaFuncSetAttribute((const void*)implicit_rows_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)row_smem);
        implicit_rows_kernel<double><<<row_blocks, kFoldWarps * 32, row_smem, st>>>(s->Mh, sm, s->hrp, s->hcol,
                                                                                   s->hval, col, (double*)val);
    } else {
        cudaFuncSetAttribute((const void*)implicit_rows_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)row_smem);
        implicit_rows_kernel<float><<<row_blocks, kFoldWarps * 32, row_smem, st>>>(s->Mh, sm, s->hrp, s->hcol,
                                                                                  s->hval, col, (float*)val);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "implicit fold: rows");
}

int scan_exclusive(const int32_t* in, int32_t* out, int32_t* tile_sums, int64_t n, cudaStream_t st) {
    return exclusive_scan(in, out, tile_sums, n, st);
}

int run_fold(splitsart_system* s, cudaStream_t st) {
    switch (s->dtype) {
        case SPLITSART_F64: return fold_typed<TF64>(s, st);
        case SPLITSART_F32: return fold_typed<TF32>(s, st);
        case SPLITSART_BF16: return fold_typed<TBF16>(s, st);
        case SPLITSART_F16: return fold_typed<TF16>(s, st);
    }
    return fail(SPLITSART_ERR_ARG, "fold: unknown dtype %d", s->dtype);
}

int run_fold_rhs(const splitsart_system* s, const void* p, void* p12, cudaStream_t st) {
    const int64_t Mh = s->Mh;
    if (Mh == 0) return SPLITSART_OK;
    const unsigned g = (unsigned)((Mh + 255) / 256);
    const SliceMap sm = slice_map(s);
    if (s->dtype == SPLITSART_F64) fold_rhs_kernel<double, double2><<<g, 256, 0, st>>>(Mh, sm, (const double*)p, (double2*)p12);
    else fold_rhs_kernel<float, float2><<<g, 256, 0, st>>>(Mh, sm, (const float*)p, (float2*)p12);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "fold_rhs launch");
}

int run_fold_image(const splitsart_system* s, const void* f, int layout, void* f12, cudaStream_t st) {
    const int64_t Nh = s->Nh;
    if (Nh == 0) return SPLITSART_OK;
    const unsigned g = (unsigned)((Nh + 255) / 256);
    const SliceMap sm = slice_map(s);
    if (s->dtype == SPLITSART_F64)
        fold_image_kernel<double, double2><<<g, 256, 0, st>>>(Nh, sm, layout, (const double*)f, (double2*)f12);
    else
        fold_image_kernel<float, float2><<<g, 256, 0, st>>>(Nh, sm, layout, (const float*)f, (float2*)f12);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "fold_image launch");
}

int run_recombine(const splitsart_system* s, const void* f12, void* f, int layout, cudaStream_t st) {
    const int64_t Nh = s->Nh;
    if (Nh == 0) return SPLITSART_OK;
    const unsigned g = (unsigned)((Nh + 255) / 256);
    const SliceMap sm = slice_map(s);
    if (s->dtype == SPLITSART_F64)
        recombine_kernel<double, double2><<<g, 256, 0, st>>>(Nh, sm, layout, (const double2*)f12, (double*)f);
    else
        recombine_kernel<float, float2><<<g, 256, 0, st>>>(Nh, sm, layout, (const float2*)f12, (float*)f);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "recombine launch");
}

int run_project(splitsart_system* s, const void* f, int layout, void* p, cudaStream_t st) {
    switch (s->dtype) {
        case SPLITSART_F64: return project_typed<TF64>(s, f, layout, p, st);
        case SPLITSART_F32: return project_typed<TF32>(s, f, layout, p, st);
        case SPLITSART_BF16: return project_typed<TBF16>(s, f, layout, p, st);
        case SPLITSART_F16: return project_typed<TF16>(s, f, layout, p, st);
    }
    return fail(SPLITSART_ERR_ARG, "project: unknown dtype %d", s->dtype);
}

}  // namespace splitsart
