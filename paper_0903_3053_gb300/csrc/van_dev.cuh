// van_dev.cuh -- device building blocks of the learned proposal: a masked
// autoregressive convolutional network over Ising spins (variational
// autoregressive network, Wu, Wang & Zhang, PRL 122 (2019) 080602), used as an
// independence proposal corrected by Metropolis-Hastings.  The paper has no
// learned component.
//
// Network (raster order k = y L + x, zero padding): layer 1 is a 5x5
// convolution 1 -> 32 channels with mask A (taps strictly before the centre),
// layers 2..D-1 are 5x5 convolutions 32 -> 32 with mask B (mask A plus the
// centre), each followed by bias and ReLU; layer D is 5x5, 32 -> 1, mask B,
// giving the logit f_k with p(s_k = +1 | s_<k) = sigmoid(f_k).
// Activations are BF16, channels innermost ([n][y][x][32]).  Every layer of
// the forward pass and the 32 -> 32 layers' data and weight gradients run on
// the fifth-generation tensor cores (tcgen05.mma with a tensor-memory
// accumulator); the sampler's per-position 32-sample tiles use mma.sync
// m16n8k16 (M = 32 is below a tcgen05 tile); BF16 in, FP32 accumulate; log q
// is accumulated in FP64.  The edge layers' gradients run on the CUDA cores.
#pragma once
#include <cuda_bf16.h>

#include "mc_internal.cuh"

namespace mc {
namespace van {

constexpr int kCh = 32;         // channels of the hidden layers
constexpr int kTapsB = 13;      // mask B taps (mask A = first 12 of them)
constexpr int kTapsA = 12;
constexpr int kMaxL = 128;      // largest lattice side
constexpr int kMaxDepth = 7;    // layers (>= 3)

// Tap t of mask B in raster order: dy = -2..0, dx = -2..2; the last (t = 12)
// is the centre (0, 0).
__host__ __device__ __forceinline__ int tap_dy(int t) { return t < 10 ? t / 5 - 2 : 0; }
__host__ __device__ __forceinline__ int tap_dx(int t) { return t < 10 ? t % 5 - 2 : t - 12; }

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// D += A B: A 16x16 bf16 (row-major fragments a0..a3), B 16x8 bf16 (b0, b1), D 16x8 fp32.
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ float log_sigmoid(float t)
{
    // log(1 / (1 + e^{-t})) = -softplus(-t), written to stay finite for large |t|
    return t >= 0.f ? -log1pf(expf(-t)) : t - log1pf(expf(t));
}

__device__ __forceinline__ float sigmoid(float t) { return 1.0f / (1.0f + expf(-t)); }

}  // namespace van
}  // namespace mc

namespace mc {
namespace van {
__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t &r0, uint32_t &r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}
}  // namespace van
}  // namespace mc
