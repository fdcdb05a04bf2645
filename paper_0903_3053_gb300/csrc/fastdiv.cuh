// fastdiv.cuh -- division by a run-time invariant divisor with one high
// multiply, after Granlund & Montgomery, "Division by invariant integers using
// multiplication" (PLDI 1994), Sec. 4: for d >= 1 let l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1 (< 2^32); then for every n < 2^31
//   floor(n / d) = (umulhi(m, n) + n) >> l,
// the sum staying below 2^32.  Lattice site indices are below 2^31.
// Usable from host code (no CUDA needed) so that it can be checked on the CPU.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define MC_HD __host__ __device__ __forceinline__
#else
#define MC_HD inline
#endif

namespace mc {

struct FastDiv {
    uint32_t d; // divisor
    uint32_t m; // magic multiplier
    uint32_t l; // shift
    uint32_t pad;
};

// 1 <= d <= 2^31.
inline FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f{d, 1u, 0u, 0u};
    while ((1ull << f.l) < d)
        ++f.l;
    f.m = (uint32_t)((((1ull << 32) * ((1ull << f.l) - d)) / d) + 1ull);
    return f;
}

MC_HD uint32_t fast_div(uint32_t n, const FastDiv &f)
{
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(f.m, n);
#else
    const uint32_t t = (uint32_t)(((uint64_t)f.m * n) >> 32);
#endif
    return (t + n) >> f.l;
}

// q = n / d, r = n - q d.
MC_HD void fast_divmod(uint32_t n, const FastDiv &f, uint32_t &q, uint32_t &r)
{
    q = fast_div(n, f);
    r = n - q * f.d;
}

}  // namespace mc
