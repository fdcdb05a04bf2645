// noalloc.cu -- SU(2) plaquette measurement that allocates no device memory.
//
// The regular measurement (mc_measure on a context) keeps its per-block
// partial sums in the workspace the caller allocated for the context.  Some
// callers cannot provide that memory: a host program whose device memory is
// entirely reserved by another allocator (a framework's memory pool, a fixed
// arena sized at start-up), or a monitoring loop that must never enter the
// CUDA allocator while a simulation runs.  For them
// mc_su2_plaquette_noalloc takes the links and the output in memory they
// already own and keeps its partial sums in a file-scope __device__ array of
// fixed size, which every GPU that loads libmc.so holds until the process
// exits.
#include <mutex>
#include <string>

#include "mc_internal.cuh"

namespace {

constexpr int kThreads = 256;
// Largest lattice the fixed scratch serves: kMaxBlocks CTAs of kThreads sites.
constexpr uint32_t kMaxBlocks = 16384;                     // 4,194,304 sites (e.g. 32^4 x 4, 44^4)
constexpr size_t kMaxSites = (size_t)kMaxBlocks * kThreads;

// Two doubles (spatial, temporal partial sum) per CTA: 256 KiB per device.
static __device__ __align__(256) double g_plaquette_scratch[2 * kMaxBlocks];

// Device address of g_plaquette_scratch, looked up once per device and kept
// for the life of the process (a device reset would invalidate it).  In host
// code the symbol itself is only a host-side stand-in and must never be handed
// to a kernel.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices] = {};

__device__ __forceinline__ float4 quat_mul(float4 a, float4 b)
{
    return make_float4(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w,
                       a.x * b.y + b.x * a.y - (a.z * b.w - a.w * b.z),
                       a.x * b.z + b.x * a.z - (a.w * b.y - a.y * b.w),
                       a.x * b.w + b.x * a.w - (a.y * b.z - a.z * b.y));
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct Dims {
    int L[4];
};

// One thread per site of a link field in the canonical order of include/mc.h,
// q[s][mu][4] with s = x1 + L1 (x2 + L2 (x3 + L3 x0)).  Each CTA writes its
// spatial and temporal sums of (1/2) Tr U_munu(x) (Eq. (3); FP32 products,
// FP64 sums) to scratch[2 b], scratch[2 b + 1]; every entry the final pass reads
// is written by this call, so nothing needs clearing first.
__global__ void __launch_bounds__(kThreads) k_plaquette_canonical(const float4 *__restrict__ q, Dims d,
                                                                  double *scratch)
{
    __shared__ double ss[kThreads / 32], st[kThreads / 32];
    const uint32_t n = (uint32_t)(d.L[0] * d.L[1] * d.L[2] * d.L[3]);
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    double ps = 0.0, pt = 0.0;
    if (s < n) {
        int x[4];
        uint32_t r = s;
        x[1] = (int)(r % (uint32_t)d.L[1]);
        r /= (uint32_t)d.L[1];
        x[2] = (int)(r % (uint32_t)d.L[2]);
        r /= (uint32_t)d.L[2];
        x[3] = (int)(r % (uint32_t)d.L[3]);
        x[0] = (int)(r / (uint32_t)d.L[3]);
        uint32_t fwd[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            int y[4] = {x[0], x[1], x[2], x[3]};
            y[m] = y[m] + 1 == d.L[m] ? 0 : y[m] + 1;
            fwd[m] = (uint32_t)(y[1] + d.L[1] * (y[2] + d.L[2] * (y[3] + d.L[3] * y[0])));
        }
        float fs = 0.f, ft = 0.f;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu)
#pragma unroll
            for (int nu = mu + 1; nu < 4; ++nu) {
                // (1/2) Tr[U_mu(x) U_nu(x+mu) (U_nu(x) U_mu(x+nu))^+] = A . B
                const float4 A = quat_mul(__ldg(&q[(size_t)s * 4 + mu]), __ldg(&q[(size_t)fwd[mu] * 4 + nu]));
                const float4 B = quat_mul(__ldg(&q[(size_t)s * 4 + nu]), __ldg(&q[(size_t)fwd[nu] * 4 + mu]));
                const float h = A.x * B.x + A.y * B.y + A.z * B.z + A.w * B.w;
                if (mu == 0)
                    ft += h;
                else
                    fs += h;
            }
        ps = (double)fs;
        pt = (double)ft;
    }
    ps = warp_sum_d(ps);
    pt = warp_sum_d(pt);
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = ps;
        st[threadIdx.x >> 5] = pt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            a += ss[w];
            b += st[w];
        }
        scratch[2 * blockIdx.x] = a;
        scratch[2 * blockIdx.x + 1] = b;
    }
}

// Fixed-order sum of the nblocks partials; out = {P, P_s, P_t}.
__global__ void __launch_bounds__(kThreads) k_plaquette_canonical_final(const double *scratch, uint32_t nblocks,
                                                                        double nsites, double *out)
{
    __shared__ double ss[kThreads / 32], st[kThreads / 32];
    double a = 0.0, b = 0.0;
    for (uint32_t i = threadIdx.x; i < nblocks; i += blockDim.x) {
        a += scratch[2 * i];
        b += scratch[2 * i + 1];
    }
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = a;
        st[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, B = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            A += ss[w];
            B += st[w];
        }
        out[0] = (A + B) / (6.0 * nsites);
        out[1] = A / (3.0 * nsites);
        out[2] = B / (3.0 * nsites);
    }
}

mc_status fail(mc_status s, const std::string &msg)
{
    mc::set_last_error(msg);
    return s;
}

}  // namespace

extern "C" mc_status mc_su2_plaquette_noalloc(const float *links, const int32_t L[4], double *out, void *cuda_stream)
{
    if (!links || !L || !out)
        return fail(MC_EINVAL, "mc_su2_plaquette_noalloc: NULL argument");
    if ((reinterpret_cast<uintptr_t>(links) & 15u) != 0 || (reinterpret_cast<uintptr_t>(out) & 7u) != 0)
        return fail(MC_EINVAL, "mc_su2_plaquette_noalloc: links must be 16-byte and out 8-byte aligned");
    double sites = 1.0;
    for (int m = 0; m < 4; ++m) {
        if (L[m] < 2)
            return fail(MC_EINVAL, "mc_su2_plaquette_noalloc: every extent must be >= 2");
        sites *= (double)L[m];
    }
    if (sites > (double)kMaxSites)
        return fail(MC_EINVAL, "mc_su2_plaquette_noalloc: lattice has " + std::to_string((long long)sites) +
                                   " sites, more than the fixed scratch serves (" + std::to_string(kMaxSites) + ")");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return fail(MC_ECUDA, std::string("mc_su2_plaquette_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(MC_EINVAL, "mc_su2_plaquette_noalloc: device index beyond the supported range");
    double *scratch = nullptr;
    {
        // First call on this device (which must be current): look up the
        // device address of the scratch array once.
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_plaquette_scratch);
            if (e != cudaSuccess)
                return fail(MC_ECUDA,
                            std::string("mc_su2_plaquette_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    const uint32_t n = (uint32_t)sites;
    const uint32_t nblocks = (n + kThreads - 1) / kThreads;
    Dims d{{L[0], L[1], L[2], L[3]}};
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    k_plaquette_canonical<<<nblocks, kThreads, 0, st>>>(reinterpret_cast<const float4 *>(links), d, scratch);
    k_plaquette_canonical_final<<<1, kThreads, 0, st>>>(scratch, nblocks, sites, out);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(MC_ECUDA, std::string("mc_su2_plaquette_noalloc: launch: ") + cudaGetErrorString(e));
    return MC_OK;
}
