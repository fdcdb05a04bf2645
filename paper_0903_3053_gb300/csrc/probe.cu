// probe.cu -- the multiply ceiling that the Ising sweep's roofline divides by.
//
// Every attempted spin flip consumes one 32-bit word of a Philox4x32-10 block
// (Salmon et al., SC'11; the counter-based generator that replaces the
// paper's RANMAR, Sec. 2.2): ten rounds of two 32 x 32 -> 64-bit products, 40
// 32-bit multiplies (high and low halves) per block.  k_philox_rate generates
// blocks back to back and does nothing else -- one xor chain per thread keeps
// the results alive -- so its multiplies per second, timed by the caller, are
// the rate this GPU sustains on the generator's own instruction mix, the
// measured peak of the sweep's multiply roofline.
#include <string>

#include "mc_internal.cuh"

namespace {

constexpr uint32_t kTagProbe = 0x7F000000u;

// Thread id draws blocks (id, i, TAG_PROBE, 0), i = 0 .. iters - 1, and
// writes the xor of all their words to out[id].
__global__ void __launch_bounds__(256) k_philox_rate(mc::PhiloxKey key, uint32_t iters, uint32_t *out)
{
    const mc::PhiloxSchedule ks = mc::philox_schedule(key);
    const uint32_t id = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0u;
#pragma unroll 4
    for (uint32_t i = 0; i < iters; ++i) {
        const uint4 r = mc::philox4x32_10(make_uint4(id, i, kTagProbe, 0u), ks);
        acc ^= r.x ^ r.y ^ r.z ^ r.w;
    }
    out[id] = acc;
}

}  // namespace

extern "C" mc_status mc_philox_rate(int32_t blocks, int32_t threads, uint32_t iters, uint64_t seed, uint32_t *dev_out,
                                    void *cuda_stream)
{
    if (blocks < 1 || threads < 32 || threads > 256 || threads % 32 != 0 || !dev_out) {
        mc::set_last_error("mc_philox_rate: need blocks >= 1, threads a multiple of 32 in [32, 256], dev_out");
        return MC_EINVAL;
    }
    const mc::PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
    k_philox_rate<<<blocks, threads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(key, iters, dev_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        mc::set_last_error(std::string("mc_philox_rate: ") + cudaGetErrorString(e));
        return MC_ECUDA;
    }
    return MC_OK;
}
