// The tcgen05 kernels' completion wait (mc::tc::mbar_wait) gives up after a
// bounded number of polls.  Here nothing ever arrives on the barrier (no MMA is
// issued), so the wait must return false after `polls` polls, and a barrier
// that does get its arrival must return true.  Nothing is left in flight.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#include "../../paper_0903_3053_gb300/csrc/tc_dev.cuh"

__global__ void k_wait(int polls, int *out)
{
    __shared__ __align__(8) uint64_t bar[2];
    const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(&bar[0]), b1 = (uint32_t)__cvta_generic_to_shared(&bar[1]);
    if (threadIdx.x == 0) {
        mc::tc::mbar_init(b0, 1);
        mc::tc::mbar_init(b1, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) // arrive on barrier 1 only
        asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(b1) : "memory");
    __syncthreads();
    const bool never = mc::tc::mbar_wait(b0, 0u, polls);
    const bool done = mc::tc::mbar_wait(b1, 0u, polls);
    if (threadIdx.x == 0) {
        out[0] = never ? 1 : 0;
        out[1] = done ? 1 : 0;
    }
}

int main()
{
    int *d, h[2] = {-1, -1};
    if (cudaMalloc(&d, 8) != cudaSuccess) return 2;
    k_wait<<<1, 32>>>(1000, d);
    if (cudaDeviceSynchronize() != cudaSuccess) return 3;
    cudaMemcpy(h, d, 8, cudaMemcpyDeviceToHost);
    printf("never-arrived wait returned %d, arrived wait returned %d\n", h[0], h[1]);
    return (h[0] == 0 && h[1] == 1) ? 0 : 1;
}
