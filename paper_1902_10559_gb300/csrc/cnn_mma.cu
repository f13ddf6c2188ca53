// Tensor-core path of the warm-start network's 32 -> 32 convolutions.
//
// A 3x3 convolution with 32 input and 32 output channels is an implicit GEMM:
//   forward: out[p][co] = sum_k A[p][k] B[co][k],
//            A[p][k = tap*32 + ci] = in[p shifted by tap][ci]
//            B[co][k] = W[co][ci][tap]
//   input gradient: the same GEMM with the taps flipped (p - tap + 1) and
//            B[ci][k = tap*32 + co] = W[co][ci][tap].
// One CTA computes a tile of 128 consecutive pixels of the batch (in
// [image][y][x] order, any image size; the last tile is padded) for all 32
// channels: M = 128, N = 32, K = 288.
//
// sm_100-family tensor cores (tcgen05), BF16 x BF16 -> FP32:
// - Operands: the CTA converts its FP32 inputs to BF16 and writes A and B
//   into shared memory in the canonical K-major layout without swizzle.
//   8-row x 16-byte core matrices: along K 128 bytes apart (LBO), row groups
//   (K/8)*128 bytes apart (SBO).
// - MMA: one thread issues 18 tcgen05.mma (K = 16 each) that accumulate into
//   32 columns of tensor memory (TMEM), then commits to an mbarrier.
// - Epilogue: four warps read the accumulator with tcgen05.ld (one pixel per
//   thread, 32 channels) and apply the bias and ReLU (forward) or the ReLU
//   mask (input gradient).
// The wait on the mbarrier is bounded. If it runs out, the kernel records
// SPLITSART_ERR_TIMEOUT and skips its epilogue.
#include <cuda_bf16.h>

#include "cnn.h"
#include "device_common.cuh"

namespace splitsart {

namespace {

constexpr int kM = 128, kN = 32, kK = 288;
constexpr int kA_bytes = kM * kK * 2;  // 73728
constexpr int kB_bytes = kN * kK * 2;  // 18432
constexpr int kLBO = 128;              // bytes between core matrices along K
constexpr int kSBO = (kK / 8) * 128;   // bytes between 8-row groups

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor for tcgen05.mma (no swizzle, K-major).
// Fields: start address >> 4 in bits 0-13, LBO >> 4 in bits 16-29, SBO >> 4
// in bits 32-45, descriptor version 1 in bits 46-47. Base offset, LBO mode
// and swizzle (bits 49-63) are 0.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16.
// Fields: D format F32 (1) in bits 4-5; A and B format BF16 (1) in bits 7-9
// and 10-12; both K-major (bits 15, 16 = 0); N >> 3 in bits 17-22; M >> 4 in
// bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);

// Byte offset of element (row, k) in the core-matrix layout.
__device__ __forceinline__ int core_off(int row, int k) {
    return (row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, unsigned long long timeout_ns) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > timeout_ns) return false;
    }
}

// BWD = false: forward (bias + ReLU). BWD = true: input gradient (ReLU mask of `act`).
template <bool BWD>
__global__ void __launch_bounds__(256) conv32_mma_kernel(const float* __restrict__ in, const float* __restrict__ Wt,
                                                         const float* __restrict__ bias, const float* __restrict__ act,
                                                         float* __restrict__ out, int B, int H, int Wd,
                                                         int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB = smem + kA_bytes;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_ok;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long HW = (long long)H * Wd, total = (long long)B * HW;
    const long long P0 = (long long)blockIdx.x * kM;  // the tile's first pixel

    // TMEM: 32 columns (the minimum allocation), by warp 0.
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(32)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }

    // A: 128 pixels x 36 chunks of 8 channels (one tap each), converted to BF16;
    // zero rows past the batch's last pixel.
    for (int c = tid; c < kM * (kK / 8); c += blockDim.x) {
        const int m = c / (kK / 8), kc = c % (kK / 8);
        const int tap = kc / 4, ci0 = (kc % 4) * 8;
        const int dy = tap / 3, dx = tap % 3;
        const long long P = P0 + m;
        const int b = (int)(P / HW), rem = (int)(P - (long long)b * HW);
        const int py = rem / Wd, px = rem - py * Wd;
        const int iy = BWD ? py + 1 - dy : py + dy - 1;
        const int ix = BWD ? px + 1 - dx : px + dx - 1;
        uint4 pack = make_uint4(0, 0, 0, 0);
        if (P < total && iy >= 0 && iy < H && ix >= 0 && ix < Wd) {
            const float4* src = reinterpret_cast<const float4*>(in + (((size_t)b * H + iy) * Wd + ix) * 32 + ci0);
            const float4 v0 = src[0], v1 = src[1];
            __nv_bfloat162 h0 = __floats2bfloat162_rn(v0.x, v0.y), h1 = __floats2bfloat162_rn(v0.z, v0.w);
            __nv_bfloat162 h2 = __floats2bfloat162_rn(v1.x, v1.y), h3 = __floats2bfloat162_rn(v1.z, v1.w);
            pack.x = *reinterpret_cast<uint32_t*>(&h0);
            pack.y = *reinterpret_cast<uint32_t*>(&h1);
            pack.z = *reinterpret_cast<uint32_t*>(&h2);
            pack.w = *reinterpret_cast<uint32_t*>(&h3);
        }
        *reinterpret_cast<uint4*>(sA + core_off(m, kc * 8)) = pack;
    }
    // B: 32 rows (forward: co; gradient: ci) x 288 (tap * 32 + the other channel).
    for (int e = tid; e < kN * kK; e += blockDim.x) {
        const int n = e / kK, k = e % kK;
        const int tap = k / 32, j = k % 32;
        const float w = BWD ? Wt[(j * 32 + n) * 9 + tap] : Wt[(n * 32 + j) * 9 + tap];
        *reinterpret_cast<__nv_bfloat16*>(sB + core_off(n, k)) = __float2bfloat16_rn(w);
    }
    // Make the generic-proxy shared-memory writes visible to the tensor core.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    if (tid == 0) {
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll 1
        for (int kk = 0; kk < kK / 16; ++kk) {
            const uint64_t ad = make_desc(a0 + kk * 2 * kLBO);
            const uint64_t bd = make_desc(b0 + kk * 2 * kLBO);
            const uint32_t accum = kk > 0 ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                ::"r"(tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(accum)
                : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&s_mbar))
                     : "memory");
    }
    if (tid == 0 && !mbar_wait(smem_u32(&s_mbar), 0, 2000000000ull)) {
        atomicCAS(err, 0, SPLITSART_ERR_TIMEOUT);
        s_ok = 0;
    }
    __syncthreads();
    if (s_ok) {
        // Threads other than 0 still need the mbarrier's completion for ordering.
        mbar_wait(smem_u32(&s_mbar), 0, 2000000000ull);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (warp < 4) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const long long P = P0 + warp * 32 + lane;  // this thread's pixel; [image][y][x] is P itself
            const size_t base = (size_t)P * 32;
#pragma unroll
            for (int c = 0; c < 32 && P < total; c += 4) {
                float4 o;
                float* po = &o.x;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float v = __uint_as_float(r[c + j]);
                    if (BWD) {
                        if (!(act[base + c + j] > 0.f)) v = 0.f;
                    } else {
                        v = fmaxf(v + bias[c + j], 0.f);
                    }
                    po[j] = v;
                }
                *reinterpret_cast<float4*>(out + base + c) = o;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
}

template <bool BWD>
int launch_mma(splitsart_cnn* n, const float* in, const float* W, const float* b, const float* act, float* out, int B,
               cudaStream_t st) {
    auto k = conv32_mma_kernel<BWD>;
    const size_t smem = kA_bytes + kB_bytes;
    cudaError_t e = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cnn mma: shared memory attribute");
    const long long pixels = (long long)B * n->H * n->W;
    const unsigned tiles = (unsigned)((pixels + kM - 1) / kM);
    k<<<tiles, 256, smem, st>>>(in, W, b, act, out, B, n->H, n->W, reinterpret_cast<int*>(n->mma_scratch));
    e = cudaGetLastError();
    return e == cudaSuccess ? SPLITSART_OK : cuda_fail(e, "cnn mma: launch");
}

}  // namespace

size_t cnn_mma_scratch_bytes(int, int, int) { return 256; }  // one error word

bool cnn_mma_supported(const splitsart_cnn* n) { return n->W > 0 && n->H > 0; }

int cnn_mma_conv_fwd(splitsart_cnn* n, const float* in, const float* W, const float* b, float* out, int B,
                     cudaStream_t st) {
    return launch_mma<false>(n, in, W, b, nullptr, out, B, st);
}

int cnn_mma_conv_bwd_data(splitsart_cnn* n, const float* gz, const float* W, const float* act, float* gx, int B,
                          cudaStream_t st) {
    return launch_mma<true>(n, gz, W, nullptr, act, gx, B, st);
}

}  // namespace splitsart
