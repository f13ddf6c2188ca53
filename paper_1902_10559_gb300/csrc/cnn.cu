// Warm-start network: a 4-layer residual CNN that maps an early split-SART
// image to an initial guess for the solve. The paper has no network; this
// supports the library's warm-start path.
//
//   a1 = relu(conv(x, W1) + b1)      1 -> 32
//   a2 = relu(conv(a1, W2) + b2)    32 -> 32
//   a3 = relu(conv(a2, W3) + b3)    32 -> 32
//   y  = x + conv(a3, W4) + b4      32 -> 1
//
// conv is a 3x3 cross-correlation with zero padding 1; tap (dy, dx) reads
// input pixel (r + dy - 1, c + dx - 1). Weights are [out][in][3][3].
// Activations are channels-last ([B][H][W][C]) so a pixel's channels are
// contiguous. Training minimises the mean squared error with Adam.
//
// Two arithmetic modes for the 32 -> 32 layers:
// - mode 0: FP32 on CUDA cores (this file);
// - mode 1: BF16 on the tensor cores with FP32 accumulation (cnn_mma.cu).
// Layers 1 and 4, the weight gradients and Adam always run in FP32.
// Every reduction has a fixed order, so results are deterministic.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "cnn.h"
#include "device_common.cuh"
#include "system.h"

namespace splitsart {

namespace {

constexpr int C = kCnnChannels;
constexpr int kWB = 8;  // pixel rows per weight-gradient block

// ---- forward convolution, FP32 on CUDA cores ----
// Block: one output row (b, y). Thread: CO_T consecutive output channels of one pixel.
template <int CI, int CO, bool RELU, bool RESID>
__global__ void __launch_bounds__(256) conv3_fwd_kernel(const float* __restrict__ in, const float* __restrict__ Wt,
                                                        const float* __restrict__ bias, const float* __restrict__ resid,
                                                        float* __restrict__ out, int H, int Wd) {
    constexpr int CO_T = CO >= 4 ? 4 : 1;
    extern __shared__ float sm[];
    float* s_in = sm;                      // [3][Wd+2][CI]
    float* s_w = sm + 3 * (Wd + 2) * CI;   // [9*CI][CO]
    const int b = blockIdx.x / H, y = blockIdx.x % H;
    for (int t = threadIdx.x; t < 3 * (Wd + 2) * CI; t += blockDim.x) {
        const int ci = t % CI, xx = (t / CI) % (Wd + 2), ry = t / (CI * (Wd + 2));
        const int iy = y + ry - 1, ix = xx - 1;
        s_in[t] = (iy >= 0 && iy < H && ix >= 0 && ix < Wd) ? in[(((size_t)b * H + iy) * Wd + ix) * CI + ci] : 0.f;
    }
    for (int t = threadIdx.x; t < 9 * CI * CO; t += blockDim.x) {
        const int co = t % CO, k = t / CO;  // k = tap * CI + ci
        const int tap = k / CI, ci = k % CI;
        s_w[t] = Wt[(co * CI + ci) * 9 + tap];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < Wd * (CO / CO_T); o += blockDim.x) {
        const int x = o / (CO / CO_T), c0 = (o % (CO / CO_T)) * CO_T;
        float acc[CO_T];
#pragma unroll
        for (int j = 0; j < CO_T; ++j) acc[j] = bias[c0 + j];
        for (int tap = 0; tap < 9; ++tap) {
            const float* ip = s_in + ((tap / 3) * (Wd + 2) + x + tap % 3) * CI;
            const float* wp = s_w + tap * CI * CO + c0;
#pragma unroll 8
            for (int ci = 0; ci < CI; ++ci) {
                const float v = ip[ci];
#pragma unroll
                for (int j = 0; j < CO_T; ++j) acc[j] += v * wp[ci * CO + j];
            }
        }
        const size_t base = (((size_t)b * H + y) * Wd + x) * CO + c0;
#pragma unroll
        for (int j = 0; j < CO_T; ++j) {
            float v = acc[j];
            if (RELU) v = fmaxf(v, 0.f);
            if (RESID) v += resid[base + j];
            out[base + j] = v;
        }
    }
}

// ---- input gradient, FP32: gx = conv^T(gz, W), then times the ReLU mask of the input ----
// gx[b][y][x][ci] = sum_{co,dy,dx} gz[b][y+1-dy][x+1-dx][co] W[co][ci][dy][dx]
template <int CI, int CO>
__global__ void __launch_bounds__(256) conv3_bwd_data_kernel(const float* __restrict__ gz, const float* __restrict__ Wt,
                                                             const float* __restrict__ act, float* __restrict__ gx,
                                                             int H, int Wd) {
    constexpr int CI_T = CI >= 4 ? 4 : 1;
    extern __shared__ float sm[];
    float* s_g = sm;                      // [3][Wd+2][CO]: gz rows y+1, y, y-1 (by dy = 0, 1, 2)
    float* s_w = sm + 3 * (Wd + 2) * CO;  // [9*CO][CI]
    const int b = blockIdx.x / H, y = blockIdx.x % H;
    for (int t = threadIdx.x; t < 3 * (Wd + 2) * CO; t += blockDim.x) {
        const int co = t % CO, xx = (t / CO) % (Wd + 2), dy = t / (CO * (Wd + 2));
        const int gy = y + 1 - dy, gxx = xx - 1;
        s_g[t] = (gy >= 0 && gy < H && gxx >= 0 && gxx < Wd) ? gz[(((size_t)b * H + gy) * Wd + gxx) * CO + co] : 0.f;
    }
    for (int t = threadIdx.x; t < 9 * CO * CI; t += blockDim.x) {
        const int ci = t % CI, k = t / CI;  // k = tap * CO + co
        const int tap = k / CO, co = k % CO;
        s_w[t] = Wt[(co * CI + ci) * 9 + tap];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < Wd * (CI / CI_T); o += blockDim.x) {
        const int x = o / (CI / CI_T), c0 = (o % (CI / CI_T)) * CI_T;
        float acc[CI_T] = {};
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap % 3;
            // gz pixel x + 1 - dx sits at column x + 2 - dx of the padded row.
            const float* gp = s_g + (dy * (Wd + 2) + x + 2 - dx) * CO;
            const float* wp = s_w + tap * CO * CI + c0;
#pragma unroll 8
            for (int co = 0; co < CO; ++co) {
                const float v = gp[co];
#pragma unroll
                for (int j = 0; j < CI_T; ++j) acc[j] += v * wp[co * CI + j];
            }
        }
        const size_t base = (((size_t)b * H + y) * Wd + x) * CI + c0;
#pragma unroll
        for (int j = 0; j < CI_T; ++j) gx[base + j] = (act == nullptr || act[base + j] > 0.f) ? acc[j] : 0.f;
    }
}

// ---- weight gradient, FP32, deterministic two-pass reduction ----
// Pass 1: block k sums pixel rows [k*kWB, (k+1)*kWB) of the batch into part[k][CO*CI*9 + CO].
template <int CI, int CO>
__global__ void __launch_bounds__(256) conv3_bwd_w_kernel(const float* __restrict__ gz, const float* __restrict__ in,
                                                          float* __restrict__ part, int rows, int H, int Wd) {
    constexpr int NW = CO * CI * 9;
    extern __shared__ float sm[];
    float* s_g = sm;                      // [Wd][CO]
    float* s_in = sm + Wd * CO;           // [3][Wd+2][CI]
    const int r0 = blockIdx.x * kWB, r1 = min(r0 + kWB, rows);
    constexpr int PER = (NW + CO + 255) / 256;
    float acc[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) acc[j] = 0.f;
    for (int r = r0; r < r1; ++r) {
        const int b = r / H, y = r % H;
        __syncthreads();
        for (int t = threadIdx.x; t < Wd * CO; t += blockDim.x) s_g[t] = gz[((size_t)r * Wd) * CO + t];
        for (int t = threadIdx.x; t < 3 * (Wd + 2) * CI; t += blockDim.x) {
            const int ci = t % CI, xx = (t / CI) % (Wd + 2), ry = t / (CI * (Wd + 2));
            const int iy = y + ry - 1, ix = xx - 1;
            s_in[t] = (iy >= 0 && iy < H && ix >= 0 && ix < Wd) ? in[(((size_t)b * H + iy) * Wd + ix) * CI + ci] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int w = threadIdx.x + j * 256;
            if (w < NW) {
                const int tap = w % 9, ci = (w / 9) % CI, co = w / (9 * CI);
                const float* ip = s_in + ((tap / 3) * (Wd + 2) + tap % 3) * CI + ci;
                float s = 0.f;
                for (int x = 0; x < Wd; ++x) s += s_g[x * CO + co] * ip[x * CI];
                acc[j] += s;
            } else if (w < NW + CO) {
                const int co = w - NW;
                float s = 0.f;
                for (int x = 0; x < Wd; ++x) s += s_g[x * CO + co];
                acc[j] += s;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int w = threadIdx.x + j * 256;
        if (w < NW + CO) part[(size_t)blockIdx.x * (NW + CO) + w] = acc[j];
    }
}

// Pass 2: grad[w] = sum over blocks k = 0..nblk-1 of part[k][w], in order.
__global__ void sum_parts_kernel(const float* __restrict__ part, int nblk, int nw, float* __restrict__ gW,
                                 float* __restrict__ gb, int nwts) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    float s = 0.f;
    for (int k = 0; k < nblk; ++k) s += part[(size_t)k * nw + w];
    if (w < nwts) gW[w] = s;
    else gb[w - nwts] = s;
}

// d = y - t; per-block sums of d^2 (FP64); gy = 2 d / count.
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ gy,
                           double* __restrict__ part, long long n) {
    __shared__ double s[256];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        gy[i] = 2.f * d / (float)n;
        acc += (double)d * (double)d;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void mse_final_kernel(const double* __restrict__ part, int nblk, long long n, float* __restrict__ loss) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += part[k];
    *loss = (float)(s / (double)n);
}

// Adam with bias correction: c1 = 1 - b1^k, c2 = 1 - b2^k.
__global__ void adam_kernel(float* __restrict__ th, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

template <int CI, int CO, bool RELU, bool RESID>
void launch_fwd(const float* in, const float* W, const float* b, const float* resid, float* out, int B, int H, int Wd,
                cudaStream_t st) {
    const size_t smem = sizeof(float) * (3 * (Wd + 2) * CI + 9 * CI * CO);
    auto k = conv3_fwd_kernel<CI, CO, RELU, RESID>;
    cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<B * H, 256, smem, st>>>(in, W, b, resid, out, H, Wd);
}

template <int CI, int CO>
void launch_bwd_data(const float* gz, const float* W, const float* act, float* gx, int B, int H, int Wd,
                     cudaStream_t st) {
    const size_t smem = sizeof(float) * (3 * (Wd + 2) * CO + 9 * CI * CO);
    auto k = conv3_bwd_data_kernel<CI, CO>;
    cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<B * H, 256, smem, st>>>(gz, W, act, gx, H, Wd);
}

template <int CI, int CO>
void launch_bwd_w(const float* gz, const float* in, float* part, float* gW, float* gb, int B, int H, int Wd,
                  cudaStream_t st) {
    const int rows = B * H, nblk = (rows + kWB - 1) / kWB;
    const size_t smem = sizeof(float) * (Wd * CO + 3 * (Wd + 2) * CI);
    conv3_bwd_w_kernel<CI, CO><<<nblk, 256, smem, st>>>(gz, in, part, rows, H, Wd);
    const int nw = CO * CI * 9 + CO;
    sum_parts_kernel<<<(nw + 255) / 256, 256, 0, st>>>(part, nblk, nw, gW, gb, CO * CI * 9);
}

}  // namespace

// Parameter offsets in the flat vector: W1, b1, W2, b2, W3, b3, W4, b4.
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + C * 9, kOffW2 = kOffB1 + C, kOffB2 = kOffW2 + C * C * 9,
              kOffW3 = kOffB2 + C, kOffB3 = kOffW3 + C * C * 9, kOffW4 = kOffB3 + C, kOffB4 = kOffW4 + C * 9;
static_assert(kOffB4 + 1 == kCnnParams, "parameter layout");

int cnn_forward_impl(splitsart_cnn* n, const float* x, int B, float* y, bool keep, cudaStream_t st) {
    const int H = n->H, Wd = n->W;
    const float* P = n->params;
    launch_fwd<1, C, true, false>(x, P + kOffW1, P + kOffB1, nullptr, n->a1, B, H, Wd, st);
    if (n->mode == 1) {
        int rc = cnn_mma_conv_fwd(n, n->a1, P + kOffW2, P + kOffB2, n->a2, B, st);
        if (rc) return rc;
        rc = cnn_mma_conv_fwd(n, n->a2, P + kOffW3, P + kOffB3, n->a3, B, st);
        if (rc) return rc;
    } else {
        launch_fwd<C, C, true, false>(n->a1, P + kOffW2, P + kOffB2, nullptr, n->a2, B, H, Wd, st);
        launch_fwd<C, C, true, false>(n->a2, P + kOffW3, P + kOffB3, nullptr, n->a3, B, H, Wd, st);
    }
    launch_fwd<C, 1, false, true>(n->a3, P + kOffW4, P + kOffB4, x, y, B, H, Wd, st);
    (void)keep;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "cnn forward");
}

int cnn_backward_impl(splitsart_cnn* n, const float* x, const float* t, int B, float* loss, cudaStream_t st) {
    const int H = n->H, Wd = n->W;
    const long long npx = (long long)B * H * Wd;
    int rc = cnn_forward_impl(n, x, B, n->y, true, st);
    if (rc) return rc;
    const int mblk = 128;
    mse_kernel<<<mblk, 256, 0, st>>>(n->y, t, n->gy, n->lpart, npx);
    if (loss) mse_final_kernel<<<1, 32, 0, st>>>(n->lpart, mblk, npx, loss);
    const float* P = n->params;
    float* G = n->grads;
    // Layer 4: y = x + conv(a3) + b4, so dL/d(conv out) = gy.
    launch_bwd_w<C, 1>(n->gy, n->a3, n->wpart, G + kOffW4, G + kOffB4, B, H, Wd, st);
    launch_bwd_data<C, 1>(n->gy, P + kOffW4, n->a3, n->g3, B, H, Wd, st);
    // Layer 3.
    launch_bwd_w<C, C>(n->g3, n->a2, n->wpart, G + kOffW3, G + kOffB3, B, H, Wd, st);
    if (n->mode == 1) {
        rc = cnn_mma_conv_bwd_data(n, n->g3, P + kOffW3, n->a2, n->g2, B, st);
        if (rc) return rc;
    } else {
        launch_bwd_data<C, C>(n->g3, P + kOffW3, n->a2, n->g2, B, H, Wd, st);
    }
    // Layer 2.
    launch_bwd_w<C, C>(n->g2, n->a1, n->wpart, G + kOffW2, G + kOffB2, B, H, Wd, st);
    if (n->mode == 1) {
        rc = cnn_mma_conv_bwd_data(n, n->g2, P + kOffW2, n->a1, n->g1, B, st);
        if (rc) return rc;
    } else {
        launch_bwd_data<C, C>(n->g2, P + kOffW2, n->a1, n->g1, B, H, Wd, st);
    }
    // Layer 1 (its input gradient is not needed).
    launch_bwd_w<1, C>(n->g1, x, n->wpart, G + kOffW1, G + kOffB1, B, H, Wd, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "cnn backward");
}

}  // namespace splitsart

using namespace splitsart;

extern "C" int splitsart_cnn_create(int nz, int nx, int max_batch, const float* params_host, splitsart_cnn** out) {
    if (!out || nz <= 0 || nx <= 0 || max_batch <= 0 || !params_host)
        return fail(SPLITSART_ERR_ARG, "cnn_create: bad argument");
    if (nx > 256) return fail(SPLITSART_ERR_ARG, "cnn_create: nx must be <= 256");
    *out = nullptr;
    auto* n = new (std::nothrow) splitsart_cnn();
    if (!n) return fail(SPLITSART_ERR_NOMEM, "cnn_create: out of host memory");
    n->H = nz;
    n->W = nx;
    n->maxB = max_batch;
    const size_t px = (size_t)max_batch * nz * nx;
    const int rows = max_batch * nz, nblk = (rows + kWB - 1) / kWB;
    const size_t sizes[] = {
        sizeof(float) * kCnnParams * 4,      // params, grads, m, v
        sizeof(float) * px * C * 6,          // a1, a2, a3, g1, g2, g3
        sizeof(float) * px * 2,              // y, gy
        sizeof(float) * (size_t)nblk * (C * C * 9 + C),  // weight-gradient partials
        sizeof(double) * 128,                // loss partials
        cnn_mma_scratch_bytes(max_batch, nz, nx),
    };
    size_t total = 0;
    for (size_t s : sizes) total += (s + 255) & ~size_t(255);
    cudaError_t e = cudaMalloc(&n->base, total);
    if (e != cudaSuccess) {
        delete n;
        cudaGetLastError();
        return fail(SPLITSART_ERR_NOMEM, "cnn_create: cudaMalloc of %zu bytes failed", total);
    }
    char* p = (char*)n->base;
    auto take = [&](size_t s) {
        char* q = p;
        p += (s + 255) & ~size_t(255);
        return q;
    };
    float* pv = (float*)take(sizes[0]);
    n->params = pv;
    n->grads = pv + kCnnParams;
    n->m = pv + 2 * kCnnParams;
    n->v = pv + 3 * kCnnParams;
    float* act = (float*)take(sizes[1]);
    n->a1 = act;
    n->a2 = act + px * C;
    n->a3 = act + 2 * px * C;
    n->g1 = act + 3 * px * C;
    n->g2 = act + 4 * px * C;
    n->g3 = act + 5 * px * C;
    float* yy = (float*)take(sizes[2]);
    n->y = yy;
    n->gy = yy + px;
    n->wpart = (float*)take(sizes[3]);
    n->lpart = (double*)take(sizes[4]);
    n->mma_scratch = take(sizes[5]);
    n->device_bytes = total;
    if ((e = cudaMemcpy(n->params, params_host, sizeof(float) * kCnnParams, cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(n->m, 0, sizeof(float) * kCnnParams * 2)) ||
        (e = cudaMemset(n->mma_scratch, 0, sizes[5]))) {
        splitsart_cnn_destroy(n);
        return cuda_fail(e, "cnn_create: upload");
    }
    *out = n;
    return SPLITSART_OK;
}

extern "C" void splitsart_cnn_destroy(splitsart_cnn* n) {
    if (!n) return;
    if (n->base) {
        cudaDeviceSynchronize();
        cudaFree(n->base);
    }
    delete n;
}

extern "C" int splitsart_cnn_set_mode(splitsart_cnn* n, int mode) {
    if (!n || mode < 0 || mode > 1) return fail(SPLITSART_ERR_ARG, "cnn_set_mode: mode must be 0 or 1");
    if (mode == 1 && !cnn_mma_supported(n)) return fail(SPLITSART_ERR_ARG, "cnn_set_mode: tensor-core mode needs a non-empty image");
    n->mode = mode;
    return SPLITSART_OK;
}

extern "C" int splitsart_cnn_params(splitsart_cnn* n, float* out_host, float* moments_host) {
    if (!n || !out_host) return fail(SPLITSART_ERR_ARG, "cnn_params: NULL argument");
    int err = 0;
    cudaError_t e = cudaMemcpy(&err, n->mma_scratch, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cnn_params");
    if (err != 0) return fail(err, "cnn: a tensor-core wait ran out; results since are invalid");
    e = cudaMemcpy(out_host, n->params, sizeof(float) * kCnnParams, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && moments_host)
        e = cudaMemcpy(moments_host, n->m, sizeof(float) * kCnnParams * 2, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "cnn_params");
}

extern "C" int splitsart_cnn_set_params(splitsart_cnn* n, const float* in_host, const float* moments_host, int step) {
    if (!n || !in_host || step < 0) return fail(SPLITSART_ERR_ARG, "cnn_set_params: bad argument");
    cudaError_t e = cudaMemcpy(n->params, in_host, sizeof(float) * kCnnParams, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        if (moments_host) e = cudaMemcpy(n->m, moments_host, sizeof(float) * kCnnParams * 2, cudaMemcpyHostToDevice);
        else e = cudaMemset(n->m, 0, sizeof(float) * kCnnParams * 2);
    }
    n->step = step;
    return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "cnn_set_params");
}

extern "C" int splitsart_cnn_forward(splitsart_cnn* n, const float* x_dev, int B, float* y_dev, void* stream) {
    if (!n || !x_dev || !y_dev || B <= 0 || B > n->maxB) return fail(SPLITSART_ERR_ARG, "cnn_forward: bad argument");
    return cnn_forward_impl(n, x_dev, B, y_dev, false, (cudaStream_t)stream);
}

extern "C" int splitsart_cnn_loss_grad(splitsart_cnn* n, const float* x_dev, const float* t_dev, int B, float* loss_dev,
                                       float* grad_dev, void* stream) {
    if (!n || !x_dev || !t_dev || B <= 0 || B > n->maxB) return fail(SPLITSART_ERR_ARG, "cnn_loss_grad: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = cnn_backward_impl(n, x_dev, t_dev, B, loss_dev, st);
    if (rc) return rc;
    if (grad_dev) {
        cudaError_t e = cudaMemcpyAsync(grad_dev, n->grads, sizeof(float) * kCnnParams, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "cnn_loss_grad: copy");
    }
    return SPLITSART_OK;
}

extern "C" int splitsart_cnn_train_step(splitsart_cnn* n, const float* x_dev, const float* t_dev, int B, double lr,
                                        double beta1, double beta2, double eps, float* loss_dev, void* stream) {
    if (!n || !x_dev || !t_dev || B <= 0 || B > n->maxB || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) ||
        !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
        return fail(SPLITSART_ERR_ARG, "cnn_train_step: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = cnn_backward_impl(n, x_dev, t_dev, B, loss_dev, st);
    if (rc) return rc;
    n->step += 1;
    const double c1 = 1.0 - std::pow(beta1, n->step), c2 = 1.0 - std::pow(beta2, n->step);
    adam_kernel<<<(kCnnParams + 255) / 256, 256, 0, st>>>(n->params, n->m, n->v, n->grads, kCnnParams, (float)lr,
                                                          (float)beta1, (float)beta2, (float)eps, (float)c1, (float)c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "cnn_train_step");
}
