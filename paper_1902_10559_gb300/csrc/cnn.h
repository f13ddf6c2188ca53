// Internal state of the warm-start network. Shared by cnn.cu (CUDA-core
// layers, training) and cnn_mma.cu (tensor-core layers); not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "host_common.h"

namespace splitsart {
constexpr int kCnnChannels = 32;
// W1 (32*1*9) + b1 (32) + W2 (32*32*9) + b2 (32) + W3 (32*32*9) + b3 (32) + W4 (1*32*9) + b4 (1)
constexpr int kCnnParams = 19105;
}  // namespace splitsart

struct splitsart_cnn {
    int H = 0, W = 0, maxB = 0;
    int mode = 0;  // 0: FP32 CUDA cores; 1: BF16 tensor cores for the 32 -> 32 layers
    int step = 0;  // Adam steps taken
    size_t device_bytes = 0;
    void* base = nullptr;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    float *a1 = nullptr, *a2 = nullptr, *a3 = nullptr;  // activations [B][H][W][32]
    float *g1 = nullptr, *g2 = nullptr, *g3 = nullptr;  // gradients w.r.t. the layers' pre-activations
    float *y = nullptr, *gy = nullptr;                  // output [B][H][W] and dL/dy
    float* wpart = nullptr;                             // weight-gradient partials
    double* lpart = nullptr;                            // loss partials
    void* mma_scratch = nullptr;                        // BF16 operands of the tensor-core layers
};

namespace splitsart {
int cuda_fail(cudaError_t e, const char* what);
// Defined in cnn_mma.cu.
size_t cnn_mma_scratch_bytes(int max_batch, int H, int W);
bool cnn_mma_supported(const splitsart_cnn* n);
int cnn_mma_conv_fwd(splitsart_cnn* n, const float* in, const float* W, const float* b, float* out, int B,
                     cudaStream_t st);
int cnn_mma_conv_bwd_data(splitsart_cnn* n, const float* gz, const float* W, const float* act, float* gx, int B,
                          cudaStream_t st);
}  // namespace splitsart
