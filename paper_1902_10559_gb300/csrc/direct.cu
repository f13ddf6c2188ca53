// The direct method of Example 2 (Table 1), dense, in FP64 on the device:
// least squares A x = b through the normal equations.
//   1. B = A^T A (lower triangle), c = A^T b, from the CSR and the CSC of A.
//      Row j of B is sum_{i in column j} a_ij (row i of A), accumulated in
//      shared memory in the CSC's row order: deterministic, no atomics.
//   2. B = L L^T by a blocked right-looking Cholesky factorisation (blocks
//      of 64): the diagonal block is factored in shared memory by one CTA,
//      the panel below it is solved against it, and the trailing lower
//      triangle takes the rank-64 update, one CTA per 64 x 64 tile.
//   3. L y = c, then L^T x = y, block by block.
// The split form applies this to A1 and A2 (the normal matrices of the split
// systems are the folds of A^T A, text after Eq. 18) and recombines by
// Theorem 1; the full form applies it to A itself. A factorisation that meets
// a pivot <= 0 (B not positive definite: A lacks full column rank) records
// SPLITSART_ERR_NOT_SPD and the remaining steps do nothing.
#include <cmath>
#include <cstdio>
#include <algorithm>

#include "device_common.cuh"
#include "system.h"

namespace splitsart {

namespace {

constexpr int kNB = 64;  // Cholesky block size

// Strided views of value and vector arrays: element k at p[k * stride].
struct DView {
    const double* p;
    int stride;
    __device__ __forceinline__ double operator[](long long k) const { return p[k * stride]; }
};

// Row j of B = A^T A, lower part (k <= j), accumulated in shared memory.
__global__ void normal_rows_kernel(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col, DView val,
                                   const int32_t* __restrict__ cp, const int32_t* __restrict__ row, DView valT,
                                   double* __restrict__ B) {
    extern __shared__ double acc[];
    const int j = blockIdx.x;
    for (int k = threadIdx.x; k <= j; k += blockDim.x) acc[k] = 0.0;
    __syncthreads();
    for (int e = cp[j]; e < cp[j + 1]; ++e) {
        const int i = row[e];
        const double w = valT[e];
        for (int t = rp[i] + threadIdx.x; t < rp[i + 1]; t += blockDim.x) {
            const int k = col[t];
            if (k <= j) acc[k] += w * val[t];  // a row holds each column once: no two threads share k
        }
        __syncthreads();
    }
    double* out = B + (size_t)j * n;
    for (int k = threadIdx.x; k <= j; k += blockDim.x) out[k] = acc[k];
}

// c_j = sum_{i in column j} a_ij b_i; one warp per column.
__global__ void atb_kernel(int n, const int32_t* __restrict__ cp, const int32_t* __restrict__ row, DView valT, DView b,
                           double* __restrict__ c) {
    const int lane = threadIdx.x & 31;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += (gridDim.x * blockDim.x) >> 5) {
        double s = 0.0;
        for (int e = cp[j] + lane; e < cp[j + 1]; e += 32) s += valT[e] * b[row[e]];
        s = warp_sum(s);
        if (lane == 0) c[j] = s;
    }
}

// Factor the diagonal block kb in shared memory (lower Cholesky), one CTA.
__global__ void potrf_block_kernel(int n, int kb, double* __restrict__ B, int* __restrict__ status) {
    __shared__ double S[kNB][kNB + 1];
    if (*status) return;
    const int k0 = kb * kNB, bn = min(kNB, n - k0);
    for (int t = threadIdx.x; t < kNB * kNB; t += blockDim.x) {
        const int r = t / kNB, q = t % kNB;
        S[r][q] = (r < bn && q <= r) ? B[(size_t)(k0 + r) * n + k0 + q] : 0.0;
    }
    __syncthreads();
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int c = 0; c < bn; ++c) {
        if (threadIdx.x == 0) {
            const double d = S[c][c];
            if (!(d > 0.0) || !isfinite(d)) bad = 1;
            S[c][c] = sqrt(d > 0.0 ? d : 1.0);
        }
        __syncthreads();
        for (int r = c + 1 + threadIdx.x; r < bn; r += blockDim.x) S[r][c] /= S[c][c];
        __syncthreads();
        const int m = bn - c - 1;
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            const int r = c + 1 + t / m, q = c + 1 + t % m;
            if (q <= r) S[r][q] -= S[r][c] * S[q][c];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && bad) atomicCAS(status, 0, SPLITSART_ERR_NOT_SPD);
    for (int t = threadIdx.x; t < kNB * kNB; t += blockDim.x) {
        const int r = t / kNB, q = t % kNB;
        if (r < bn && q <= r) B[(size_t)(k0 + r) * n + k0 + q] = S[r][q];
    }
}

// Panel below block kb: X L_kk^T = A for each 64-row block ib > kb (one CTA each,
// one thread per row, forward substitution along the row).
__global__ void trsm_panel_kernel(int n, int kb, double* __restrict__ B, const int* __restrict__ status) {
    extern __shared__ double tsm[];  // two 64 x 65 tiles
    double(*L)[kNB + 1] = reinterpret_cast<double(*)[kNB + 1]>(tsm);
    double(*X)[kNB + 1] = reinterpret_cast<double(*)[kNB + 1]>(tsm + kNB * (kNB + 1));
    if (*status) return;
    const int k0 = kb * kNB, i0 = (kb + 1 + blockIdx.x) * kNB;
    const int bn = min(kNB, n - k0), rn = min(kNB, n - i0);
    for (int t = threadIdx.x; t < kNB * kNB; t += blockDim.x) {
        const int r = t / kNB, q = t % kNB;
        L[r][q] = (r < bn && q <= r) ? B[(size_t)(k0 + r) * n + k0 + q] : 0.0;
        X[r][q] = (r < rn && q < bn) ? B[(size_t)(i0 + r) * n + k0 + q] : 0.0;
    }
    __syncthreads();
    const int r = threadIdx.x;
    if (r < rn) {
        for (int c = 0; c < bn; ++c) {
            double s = X[r][c];
            for (int q = 0; q < c; ++q) s -= X[r][q] * L[c][q];
            X[r][c] = s / L[c][c];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kNB * kNB; t += blockDim.x) {
        const int rr = t / kNB, q = t % kNB;
        if (rr < rn && q < bn) B[(size_t)(i0 + rr) * n + k0 + q] = X[rr][q];
    }
}

// Trailing update after block kb: B[ib][jb] -= P_ib P_jb^T for kb < jb <= ib, one
// CTA per 64 x 64 tile of the lower triangle; 256 threads, 4 x 4 outputs each.
__global__ void __launch_bounds__(256) syrk_update_kernel(int n, int kb, double* __restrict__ B,
                                                           const int* __restrict__ status) {
    extern __shared__ double usm[];  // P: rows of block ib, Q: rows of block jb; columns of block kb
    double(*P)[kNB + 1] = reinterpret_cast<double(*)[kNB + 1]>(usm);
    double(*Q)[kNB + 1] = reinterpret_cast<double(*)[kNB + 1]>(usm + kNB * (kNB + 1));
    if (*status) return;
    // Tile t of the lower triangle of the trailing blocks: (ib, jb) with jb <= ib.
    const long long t = blockIdx.x;
    int a = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) / 2.0);
    while ((long long)(a + 1) * (a + 2) / 2 <= t) ++a;
    while ((long long)a * (a + 1) / 2 > t) --a;
    const int ib = kb + 1 + a, jb = kb + 1 + (int)(t - (long long)a * (a + 1) / 2);
    const int k0 = kb * kNB, i0 = ib * kNB, j0 = jb * kNB;
    const int kn = min(kNB, n - k0), in = min(kNB, n - i0), jn = min(kNB, n - j0);
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
        const int r = e / kNB, q = e % kNB;
        P[r][q] = (r < in && q < kn) ? B[(size_t)(i0 + r) * n + k0 + q] : 0.0;
        Q[r][q] = (r < jn && q < kn) ? B[(size_t)(j0 + r) * n + k0 + q] : 0.0;
    }
    __syncthreads();
    const int tr = (threadIdx.x / 16) * 4, tc = (threadIdx.x % 16) * 4;
    double acc[4][4] = {};
    for (int q = 0; q < kn; ++q) {
        double pr[4], qc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            pr[u] = P[tr + u][q];
            qc[u] = Q[tc + u][q];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += pr[u] * qc[v];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = tr + u, c = tc + v;
            if (r < in && c < jn && (ib != jb || c <= r)) B[(size_t)(i0 + r) * n + j0 + c] -= acc[u][v];
        }
}

}  // namespace
}  // namespace splitsart

namespace splitsart {
namespace {

// Forward substitution on block kb: y_kb = L_kk^{-1} c_kb (one warp; c is overwritten by y).
__global__ void trsv_lower_block_kernel(int n, int kb, const double* __restrict__ B, double* __restrict__ c,
                                        const int* __restrict__ status) {
    if (*status) return;
    const int k0 = kb * kNB, bn = min(kNB, n - k0), lane = threadIdx.x;
    for (int r = 0; r < bn; ++r) {
        double s = 0.0;
        for (int q = lane; q < r; q += 32) s += B[(size_t)(k0 + r) * n + k0 + q] * c[k0 + q];
        s = warp_sum(s);
        if (lane == 0) c[k0 + r] = (c[k0 + r] - s) / B[(size_t)(k0 + r) * n + k0 + r];
        __syncwarp();
    }
}

// c_i -= sum_{q in block kb} L_iq y_q for the rows i below block kb (one thread per row).
__global__ void trsv_lower_update_kernel(int n, int kb, const double* __restrict__ B, double* __restrict__ c,
                                         const int* __restrict__ status) {
    if (*status) return;
    const int k0 = kb * kNB, bn = min(kNB, n - k0);
    for (int i = k0 + bn + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < bn; ++q) s += B[(size_t)i * n + k0 + q] * c[k0 + q];
        c[i] -= s;
    }
}

// Back substitution on block kb: x_kb = L_kk^{-T} y_kb (one warp; y is overwritten by x).
__global__ void trsv_upper_block_kernel(int n, int kb, const double* __restrict__ B, double* __restrict__ y,
                                        const int* __restrict__ status) {
    if (*status) return;
    const int k0 = kb * kNB, bn = min(kNB, n - k0), lane = threadIdx.x;
    for (int r = bn - 1; r >= 0; --r) {
        double s = 0.0;
        for (int q = r + 1 + lane; q < bn; q += 32) s += B[(size_t)(k0 + q) * n + k0 + r] * y[k0 + q];
        s = warp_sum(s);
        if (lane == 0) y[k0 + r] = (y[k0 + r] - s) / B[(size_t)(k0 + r) * n + k0 + r];
        __syncwarp();
    }
}

// y_i -= sum_{q in block kb} L_qi x_q for the rows i above block kb (one thread per i; row q of L is contiguous in i).
__global__ void trsv_upper_update_kernel(int n, int kb, const double* __restrict__ B, double* __restrict__ y,
                                         const int* __restrict__ status) {
    if (*status) return;
    const int k0 = kb * kNB, bn = min(kNB, n - k0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k0; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < bn; ++q) s += B[(size_t)(k0 + q) * n + i] * y[k0 + q];
        y[i] -= s;
    }
}

// x (strided) = y.
__global__ void scatter_kernel(int n, const double* __restrict__ y, double* __restrict__ x, int stride) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[(size_t)i * stride] = y[i];
}

}  // namespace

// Bytes of the work buffer for n unknowns: B (n x n), c, the status word.
long long normal_work_bytes(long long n) { return 8LL * n * n + 8LL * n + 256; }

// The whole normal-equation solve, enqueued on st. status_dev receives 0 or SPLITSART_ERR_NOT_SPD.
int run_normal_solve(int m, int n, const int32_t* rp, const int32_t* col, const double* val, int vstride,
                     const int32_t* cp, const int32_t* row, const double* valT, const double* b, int bstride, double* x,
                     int xstride, void* work, int* status_dev, cudaStream_t st) {
    (void)m;
    if (n <= 0) return SPLITSART_OK;
    double* B = (double*)work;
    double* c = B + (size_t)n * n;
    cudaError_t e;
    const size_t smem = sizeof(double) * (size_t)n;
    int dev = 0, smax = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > (size_t)smax) return fail(SPLITSART_ERR_ARG, "normal solve: n = %d exceeds %d unknowns", n, smax / 8);
    if ((e = cudaFuncSetAttribute((const void*)normal_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return cuda_fail(e, "normal solve: shared memory attribute");
    const size_t tiles2 = sizeof(double) * 2 * kNB * (kNB + 1);
    if ((e = cudaFuncSetAttribute((const void*)trsm_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tiles2)) != cudaSuccess ||
        (e = cudaFuncSetAttribute((const void*)syrk_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tiles2)) != cudaSuccess)
        return cuda_fail(e, "normal solve: shared memory attribute");
    if ((e = cudaMemsetAsync(status_dev, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e, "normal solve: memset");
    normal_rows_kernel<<<n, 256, smem, st>>>(n, rp, col, DView{val, vstride}, cp, row, DView{valT, vstride}, B);
    atb_kernel<<<std::max(1, std::min((n + 7) / 8, 4096)), 256, 0, st>>>(n, cp, row, DView{valT, vstride},
                                                                        DView{b, bstride}, c);
    const int nb = (n + kNB - 1) / kNB;
    for (int kb = 0; kb < nb; ++kb) {
        potrf_block_kernel<<<1, 256, 0, st>>>(n, kb, B, status_dev);
        const int below = nb - kb - 1;
        if (below > 0) {
            trsm_panel_kernel<<<below, kNB, tiles2, st>>>(n, kb, B, status_dev);
            const long long tiles = (long long)below * (below + 1) / 2;
            syrk_update_kernel<<<(unsigned)tiles, 256, tiles2, st>>>(n, kb, B, status_dev);
        }
    }
    for (int kb = 0; kb < nb; ++kb) {
        trsv_lower_block_kernel<<<1, 32, 0, st>>>(n, kb, B, c, status_dev);
        if (kb + 1 < nb) trsv_lower_update_kernel<<<std::max(1, std::min((n + 255) / 256, 1024)), 256, 0, st>>>(
            n, kb, B, c, status_dev);
    }
    for (int kb = nb - 1; kb >= 0; --kb) {
        trsv_upper_block_kernel<<<1, 32, 0, st>>>(n, kb, B, c, status_dev);
        if (kb > 0) trsv_upper_update_kernel<<<std::max(1, std::min((kb * kNB + 255) / 256, 1024)), 256, 0, st>>>(
            n, kb, B, c, status_dev);
    }
    scatter_kernel<<<std::max(1, std::min((n + 255) / 256, 1024)), 256, 0, st>>>(n, c, x, xstride);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "normal solve: launch");
    return SPLITSART_OK;
}

}  // namespace splitsart

using namespace splitsart;

extern "C" int splitsart_normal_solve_bytes(int64_t n, int64_t* bytes) {
    if (!bytes || n < 0) return fail(SPLITSART_ERR_ARG, "normal_solve_bytes: bad argument");
    *bytes = normal_work_bytes(n);
    return SPLITSART_OK;
}

extern "C" int splitsart_normal_solve(int64_t m, int64_t n, const int32_t* rp_dev, const int32_t* col_dev,
                                      const double* val_dev, const int32_t* cp_dev, const int32_t* row_dev,
                                      const double* valT_dev, int32_t val_stride, const double* b_dev, int32_t b_stride,
                                      double* x_dev, int32_t x_stride, void* work_dev, int32_t* status_dev,
                                      void* stream) {
    splitsart::NvtxRange nvtx_range("splitsart_normal_solve");
    if (m < 0 || n < 0 || m > INT32_MAX || n > 65536) return fail(SPLITSART_ERR_ARG, "normal_solve: bad sizes");
    if (!rp_dev || !col_dev || !val_dev || !cp_dev || !row_dev || !valT_dev || !b_dev || !x_dev || !work_dev ||
        !status_dev)
        return fail(SPLITSART_ERR_ARG, "normal_solve: NULL argument");
    if (val_stride < 1 || b_stride < 1 || x_stride < 1) return fail(SPLITSART_ERR_ARG, "normal_solve: strides must be >= 1");
    return run_normal_solve((int)m, (int)n, rp_dev, col_dev, val_dev, val_stride, cp_dev, row_dev, valT_dev, b_dev,
                            b_stride, x_dev, x_stride, work_dev, status_dev, (cudaStream_t)stream);
}

extern "C" int splitsart_direct_split(splitsart_system* s, const double* p_dev, double* f_dev, void* work_dev,
                                      int32_t* status_dev, void* stream) {
    splitsart::NvtxRange nvtx_range("splitsart_direct_split");
    if (!s || !p_dev || !f_dev || !work_dev || !status_dev) return fail(SPLITSART_ERR_ARG, "direct_split: NULL argument");
    if (s->dtype != SPLITSART_F64) return fail(SPLITSART_ERR_ARG, "direct_split: the system must be FP64");
    if (s->ns != 1) return fail(SPLITSART_ERR_ARG, "direct_split: single-slice systems only");
    if (s->Nh > 65536) return fail(SPLITSART_ERR_ARG, "direct_split: too many unknowns");
    cudaStream_t st = (cudaStream_t)stream;
    s->last = st;
    double* p12 = (double*)s->tmp_q12;  // Mh pairs
    double* f12 = (double*)s->tmp_f12;  // Nh pairs
    int rc = run_fold_rhs(s, p_dev, p12, st);
    if (rc) return rc;
    const double* val = (const double*)s->val;
    const double* valT = (const double*)s->valT;
    for (int k = 0; k < 2; ++k) {
        rc = run_normal_solve((int)s->Mh, (int)s->Nh, s->rp, s->col, val + k, 2, s->cp, s->row, valT + k, p12 + k, 2,
                              f12 + k, 2, work_dev, status_dev + 0, st);
        if (rc) return rc;
    }
    return run_recombine(s, f12, f_dev, SPLITSART_LAYOUT_SNAKE, st);
}
