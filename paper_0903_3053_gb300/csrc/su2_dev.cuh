// su2_dev.cuh -- per-link device code of the 4D SU(2) heat-bath (Sec. 2.4,
// Eqs. (2)-(7)), shared by the per-phase kernels of su2.cu, the persistent
// batch kernel of batch.cu and the resident kernel of su2_resident.cu.
// Quaternion links (U0, U1, U2, U3) of Eq. (4) in FP32, stored per chain as
// float4 [parity][mu][site-within-parity].
//
// Every floating-point sum of products on the update path is written with
// explicit rounding intrinsics (__fmaf_rn, __fmul_rn, __fadd_rn, ...), which
// the compiler neither contracts nor reorders: how it would otherwise fuse
// a*b - c*d into an FMA depends on the surrounding code, and the kernels that
// share these functions must produce bit-identical links.
#pragma once
#include "mc_internal.cuh"

namespace mc {
namespace {

// (a0 + i a.sigma)(b0 + i b.sigma) = (a0 b0 - a.b) + i (a0 b + b0 a - a x b).sigma,
// each component one product and three fused multiply-adds in a fixed order.
__device__ __forceinline__ float4 qmul(float4 a, float4 b)
{
    return make_float4(__fmaf_rn(-a.w, b.w, __fmaf_rn(-a.z, b.z, __fmaf_rn(-a.y, b.y, __fmul_rn(a.x, b.x)))),
                       __fmaf_rn(a.w, b.z, __fmaf_rn(-a.z, b.w, __fmaf_rn(b.x, a.y, __fmul_rn(a.x, b.y)))),
                       __fmaf_rn(a.y, b.w, __fmaf_rn(-a.w, b.y, __fmaf_rn(b.x, a.z, __fmul_rn(a.x, b.z)))),
                       __fmaf_rn(a.z, b.y, __fmaf_rn(-a.y, b.z, __fmaf_rn(b.x, a.w, __fmul_rn(a.x, b.w)))));
}
__device__ __forceinline__ float4 qdag(float4 a) { return make_float4(a.x, -a.y, -a.z, -a.w); }
__device__ __forceinline__ float4 qadd(float4 a, float4 b)
{
    return make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w));
}
__device__ __forceinline__ float qdot(float4 a, float4 b)
{
    return __fmaf_rn(a.w, b.w, __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x))));
}
__device__ __forceinline__ float4 qscale(float4 a, float s)
{
    return make_float4(__fmul_rn(a.x, s), __fmul_rn(a.y, s), __fmul_rn(a.z, s), __fmul_rn(a.w, s));
}

struct Site {
    int x[4];
};

__device__ __forceinline__ Site site_from_parity_index(const Su2Chain &ch, int p, uint32_t e)
{
    // e = x1/2 + (L1/2) (x2 + L2 (x3 + L3 x0)); magic-number divisions (fastdiv.cuh)
    uint32_t q1, x1h, q2, x2, x0, x3;
    fast_divmod(e, ch.div1h, q1, x1h);
    fast_divmod(q1, ch.div2, q2, x2);
    fast_divmod(q2, ch.div3, x0, x3);
    Site s;
    s.x[0] = (int)x0;
    s.x[2] = (int)x2;
    s.x[3] = (int)x3;
    s.x[1] = 2 * (int)x1h + ((p + s.x[0] + s.x[2] + s.x[3]) & 1);
    return s;
}

__device__ __forceinline__ uint32_t canonical(const Su2Chain &ch, const Site &s)
{
    return (uint32_t)(s.x[1] + ch.L[1] * (s.x[2] + ch.L[2] * (s.x[3] + ch.L[3] * s.x[0])));
}

template <int D>
__device__ __forceinline__ Site step(const Su2Chain &ch, Site s, int dir)
{
    s.x[D] += dir;
    if (s.x[D] == ch.L[D])
        s.x[D] = 0;
    else if (s.x[D] < 0)
        s.x[D] = ch.L[D] - 1;
    return s;
}

template <int LD>
__device__ __forceinline__ float4 load_link(const float4 *U, uint32_t nh, int par, int dir, uint32_t e)
{
    return lat_load<LD>(&U[(size_t)(par * 4 + dir) * nh + e]);
}

// Canonical index strides: direction mu moves the canonical index by st[mu].
struct Strides {
    uint32_t st[4];
};

__device__ __forceinline__ Strides strides_of(const Su2Chain &ch)
{
    Strides g;
    g.st[1] = 1u;
    g.st[2] = (uint32_t)ch.L[1];
    g.st[3] = (uint32_t)(ch.L[1] * ch.L[2]);
    g.st[0] = (uint32_t)(ch.L[1] * ch.L[2] * ch.L[3]);
    return g;
}

// Canonical index of x + e_D / x - e_D, given x's coordinate along D.
template <int D>
__device__ __forceinline__ uint32_t fwd(const Su2Chain &ch, const Strides &g, int xd, uint32_t s)
{
    return xd + 1 == ch.L[D] ? s - (uint32_t)(ch.L[D] - 1) * g.st[D] : s + g.st[D];
}
template <int D>
__device__ __forceinline__ uint32_t bwd(const Su2Chain &ch, const Strides &g, int xd, uint32_t s)
{
    return xd == 0 ? s + (uint32_t)(ch.L[D] - 1) * g.st[D] : s - g.st[D];
}

// The two staples of Eq. (6) in the (MU, NU) plane:
//   U_nu(x) U_mu(x+nu) U_nu(x+mu)^+  +  U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu).
// x + nu, x + mu and x - nu have parity 1 - P; x - nu + mu has parity P.
template <int MU, int NU, int P, int LD>
__device__ __forceinline__ float4 staple_pair(const float4 *__restrict__ U, const Su2Chain &ch, const Strides &g,
                                              const Site &x, uint32_t s, uint32_t spm, uint32_t e)
{
    constexpr int Q = 1 - P;
    const uint32_t nh = ch.nh;
    const uint32_t spn = fwd<NU>(ch, g, x.x[NU], s);
    const uint32_t smn = bwd<NU>(ch, g, x.x[NU], s);
    const uint32_t smnpm = fwd<MU>(ch, g, x.x[MU], smn); // x - nu has the same MU coordinate as x
    const float4 a = load_link<LD>(U, nh, P, NU, e);
    const float4 b = load_link<LD>(U, nh, Q, MU, spn >> 1);
    const float4 c = load_link<LD>(U, nh, Q, NU, spm >> 1);
    const float4 d = load_link<LD>(U, nh, Q, NU, smn >> 1);
    const float4 f = load_link<LD>(U, nh, Q, MU, smn >> 1);
    const float4 h = load_link<LD>(U, nh, P, NU, smnpm >> 1);
    return qadd(qmul(qmul(a, b), qdag(c)), qmul(qmul(qdag(d), f), h));
}

template <int MU, int P, int LD>
__device__ __forceinline__ float4 staple(const float4 *__restrict__ U, const Su2Chain &ch, const Site &x, uint32_t s,
                                         uint32_t e)
{
    const Strides g = strides_of(ch);
    const uint32_t spm = fwd<MU>(ch, g, x.x[MU], s);
    float4 W = make_float4(0.f, 0.f, 0.f, 0.f);
    if (MU != 0) W = qadd(W, staple_pair<MU, 0, P, LD>(U, ch, g, x, s, spm, e));
    if (MU != 1) W = qadd(W, staple_pair<MU, 1, P, LD>(U, ch, g, x, s, spm, e));
    if (MU != 2) W = qadd(W, staple_pair<MU, 2, P, LD>(U, ch, g, x, s, spm, e));
    if (MU != 3) W = qadd(W, staple_pair<MU, 3, P, LD>(U, ch, g, x, s, spm, e));
    return W;
}

// Counts a link update whose every try was rejected.  Out of line on purpose:
// with the atomic inlined, the phase kernel ran 11% slower on 4 x 32^4
// although the branch is essentially never taken.
__device__ __noinline__ void count_heatbath_failure(DevState *state) { atomicAdd(&state->hb_failures, 1ull); }

constexpr int kKpTries = 8;
constexpr int kCreutzTries = 64;
constexpr uint8_t kFailed = 255;

// The part of a Kennedy-Pendleton try that does not depend on alpha:
// q = -(log u1 + cos^2(2 pi u2) log u3), so that lambda^2 = q / (2 alpha), and
// u4^2 for the acceptance test.
struct KpFirstTry {
    float q, u4sq;
};

__device__ __forceinline__ KpFirstTry kp_parts(uint4 r)
{
    const float u1 = uniform_open0(r.x), u2 = uniform_open0(r.y);
    const float u3 = uniform_open0(r.z), u4 = uniform_open0(r.w);
    const float cs = cospif(2.0f * u2);
    return KpFirstTry{-__fmaf_rn(__fmul_rn(cs, cs), logf(u3), logf(u1)), __fmul_rn(u4, u4)};
}

// Acceptance of a Kennedy-Pendleton try at alpha > 0: lambda^2 = q / (2 alpha),
// accepted iff u4^2 <= 1 - lambda^2; a0 = 1 - 2 lambda^2 either way.
__device__ __forceinline__ bool kp_accept(const KpFirstTry &f, float alpha, float &a0)
{
    const float lam2 = __fmul_rn(f.q, __fdividef(0.5f, alpha));
    a0 = __fmaf_rn(-2.0f, lam2, 1.0f);
    return f.u4sq <= __fsub_rn(1.0f, lam2);
}

// One heat-bath try t for a0 ~ sqrt(1-a0^2) exp(alpha a0): Kennedy-Pendleton
// for t < kKpTries (alpha > 0), Creutz after; a0 is set whether or not the try
// is accepted.
__device__ __forceinline__ bool heatbath_try(int t, float alpha, uint32_t e, uint32_t sweep, uint32_t sel,
                                             const Su2Chain &ch, const PhiloxSchedule &ks, float &a0)
{
    const uint4 r = philox4x32_10(make_uint4(e, sweep, kTagSu2Heatbath | sel | (uint32_t)t, ch.chain_id), ks);
    if (t < kKpTries)
        return kp_accept(kp_parts(r), alpha, a0);
    const float cexp = alpha > 0.f ? -expm1f(-2.0f * alpha) : 0.f; // 1 - e^{-2 alpha}
    const float u1 = uniform_open0(r.x), u2 = uniform_open0(r.y);
    const float c = alpha > 0.f ? __fadd_rn(1.0f, log1pf(__fmul_rn(-__fsub_rn(1.0f, u1), cexp)) / alpha)
                                : __fmaf_rn(2.0f, u1, -1.0f);
    a0 = c;
    return __fmul_rn(u2, u2) <= __fmaf_rn(-c, c, 1.0f);
}

// The alpha-free part of Kennedy-Pendleton try t of a link (t = 0 for the
// first try; `sel` carries parity and direction).  The grid kernel computes
// try 0's part before the staple, so that it fills the wait for the staple's
// loads; the resident kernel computes several tries' parts at once.
__device__ __forceinline__ KpFirstTry kp_first_try(uint32_t e, uint32_t sweep, uint32_t sel, const Su2Chain &ch,
                                                   const PhiloxSchedule &ks)
{
    return kp_parts(philox4x32_10(make_uint4(e, sweep, kTagSu2Heatbath | sel, ch.chain_id), ks));
}

// Heat-bath draw of a0: tries 0 .. kKpTries - 1 by Kennedy-Pendleton (skipped
// when alpha = 0; try 0 from its precomputed part f), then Creutz up to
// kKpTries + kCreutzTries - 1; returns the try taken, or kFailed.  One loop
// over both samplers (measured ~2% faster on 4 x 32^4 than a loop per
// sampler); the same draws as heatbath_try for every t.
__device__ __forceinline__ int draw_a0(float alpha, uint32_t e, uint32_t sweep, uint32_t sel, const Su2Chain &ch,
                                       const PhiloxSchedule &ks, const KpFirstTry &f, float &a0)
{
    if (alpha > 0.f) {
        float a;
        if (kp_accept(f, alpha, a)) {
            a0 = a;
            return 0;
        }
    }
    for (int t = alpha > 0.f ? 1 : kKpTries; t < kKpTries + kCreutzTries; ++t) {
        float a;
        if (heatbath_try(t, alpha, e, sweep, sel, ch, ks, a)) {
            a0 = a;
            return t;
        }
    }
    return kFailed;
}

// Staple of the link U_MU(x) at site e of parity P (Eq. (6)) as V = W / |W| and
// alpha = beta |W| (V = 1 for a vanishing staple); sc = canonical site index.
// V = W / |W| and alpha = beta |W| of a staple W (V = 1 for a vanishing staple);
// one reciprocal square root serves both.
__device__ __forceinline__ void staple_to_heatbath(const float4 &W, float beta, float4 &V, float &alpha)
{
    const float k2 = qdot(W, W);
    V = make_float4(1.f, 0.f, 0.f, 0.f);
    float kn = 0.f;
    if (k2 > 0.f) {
        const float inv = rsqrtf(k2);
        V = qscale(W, inv);
        kn = __fmul_rn(k2, inv);
    }
    alpha = __fmul_rn(beta, kn);
}

template <int P, int MU, int LD>
__device__ __forceinline__ void su2_link_staple(const float4 *U, const Su2Chain &ch, uint32_t e, float4 &V,
                                                float &alpha, uint32_t &sc)
{
    const Site x = site_from_parity_index(ch, P, e);
    sc = canonical(ch, x);
    const float4 W = staple<MU, P, LD>(U, ch, x, sc, e);
    staple_to_heatbath(W, ch.beta, V, alpha);
}

// Uniform direction on S^2 for the vector part of X in Eq. (5): cos theta =
// 2 u1 - 1, phi = 2 pi u2 from the link's direction Philox block.
struct S2Direction {
    float ct, st, sphi, cphi;
};

template <int P, int MU>
__device__ __forceinline__ S2Direction su2_direction(const Su2Chain &ch, const PhiloxSchedule &ks, uint32_t e,
                                                     uint32_t sweep)
{
    const uint32_t sel = ((uint32_t)P << 12) | ((uint32_t)MU << 8);
    const uint4 r = philox4x32_10(make_uint4(e, sweep, kTagSu2Direction | sel, ch.chain_id), ks);
    S2Direction d;
    d.ct = __fmaf_rn(2.0f, uniform_open0(r.x), -1.0f);
    // phi = 2 pi u2 reduced to (-pi, pi]: u2 - 1 for u2 > 1/2 (exact in FP32)
    const float u2 = uniform_open0(r.y), v = u2 > 0.5f ? u2 - 1.0f : u2;
    __sincosf(6.2831853f * v, &d.sphi, &d.cphi);
    const float s2 = fmaxf(0.f, __fmaf_rn(-d.ct, d.ct, 1.0f));
    d.st = s2 > 0.f ? __fmul_rn(s2, rsqrtf(s2)) : 0.f;
    return d;
}

// The new link X V of Eq. (5) for the drawn a0 and direction d, X = a0 +
// i sqrt(1 - a0^2) d.sigma, reprojected onto SU(2) (Eq. (7)).
__device__ __forceinline__ float4 heatbath_link(float a0, const float4 &V, const S2Direction &d)
{
    const float r2 = fmaxf(0.f, __fmaf_rn(-a0, a0, 1.0f));
    const float rad = r2 > 0.f ? __fmul_rn(r2, rsqrtf(r2)) : 0.f;
    const float rs = __fmul_rn(rad, d.st);
    const float4 X = make_float4(a0, __fmul_rn(rs, d.cphi), __fmul_rn(rs, d.sphi), __fmul_rn(rad, d.ct));
    const float4 Un = qmul(X, V);
    return qscale(Un, rsqrtf(qdot(Un, Un)));
}

// Heat-bath draw and store for a link whose staple is (V, alpha) and whose
// direction is d: a0 by Kennedy-Pendleton / Creutz, U = X V, reprojection
// (Eqs. (5), (7)).  Returns the try taken (kFailed: link unchanged, counted).
template <int P, int MU, bool INLINE_FAIL>
__device__ __forceinline__ int su2_link_draw(float4 *U, const Su2Chain &ch, const PhiloxSchedule &ks, uint32_t e,
                                             uint32_t sweep, float4 V, float alpha, const S2Direction &d,
                                             const KpFirstTry &f, DevState *state)
{
    const uint32_t sel = ((uint32_t)P << 12) | ((uint32_t)MU << 8);
    float a0 = 0.f;
    const int t = draw_a0(alpha, e, sweep, sel, ch, ks, f, a0);
    if (t == kFailed) {
        if (INLINE_FAIL)
            atomicAdd(&state->hb_failures, 1ull);
        else
            count_heatbath_failure(state);
        return t;
    }
    U[(size_t)(P * 4 + MU) * ch.nh + e] = heatbath_link(a0, V, d);
    return t;
}

// Heat-bath update of the link U_MU(x) at site e of parity P (Eqs. (5)-(7)):
// staple, a0 by Kennedy-Pendleton / Creutz, direction on S^2, U = X V,
// reprojection.  REC: store the try taken at tries[2 e + b][MU] (canonical
// site 2 e + b, b the parity bit of x1); a separate instantiation so that the
// sweeps that do not record keep no extra state live across the heat-bath loop.
// INLINE_FAIL: count a failed update with an inlined atomic (the persistent
// batch kernel, where the out-of-line call costs a stack frame) instead of
// count_heatbath_failure.
template <int P, int MU, int LD, bool REC, bool INLINE_FAIL = false, int EARLY = 2>
__device__ __forceinline__ void su2_update_link(float4 *U, const Su2Chain &ch, const PhiloxSchedule &ks, uint32_t e,
                                                uint32_t sweep, uint8_t *tries, DevState *state)
{
    // The direction and the alpha-free part of the first heat-bath try do not
    // depend on the staple: computed first (EARLY = 2), their Philox blocks,
    // logarithms and trigonometry fill the wait for the staple's 18 link loads
    // (0.609 against 0.650 ms per sweep of 4 x 32^4, identical links).  EARLY
    // = 1 moves only the direction, 0 neither; the draws are the same.
    const uint32_t sel = ((uint32_t)P << 12) | ((uint32_t)MU << 8);
    S2Direction d;
    KpFirstTry f;
    if (EARLY >= 1)
        d = su2_direction<P, MU>(ch, ks, e, sweep);
    if (EARLY >= 2)
        f = kp_first_try(e, sweep, sel, ch, ks);
    float4 V;
    float alpha;
    uint32_t sc;
    su2_link_staple<P, MU, LD>(U, ch, e, V, alpha, sc);
    if (EARLY < 2)
        f = kp_first_try(e, sweep, sel, ch, ks);
    if (EARLY < 1)
        d = su2_direction<P, MU>(ch, ks, e, sweep);
    const int t = su2_link_draw<P, MU, INLINE_FAIL>(U, ch, ks, e, sweep, V, alpha, d, f, state);
    if (REC)
        tries[ch.tries_off + (size_t)sc * 4 + MU] = (uint8_t)t;
}

// Overrelaxation of the link U_MU(x) at site e of parity P (the
// "overrelaxation" of Sec. 2.4's heat-bath with overrelaxation): the
// reflection U' = V U^dag V, V = W / |W|, keeps Re Tr(U W^dag) and so the
// action; deterministic, no random numbers.  A vanishing staple leaves the link
// as it is.  The result is reprojected onto SU(2).
template <int P, int MU, int LD>
__device__ __forceinline__ void su2_overrelax_link(float4 *U, const Su2Chain &ch, uint32_t e)
{
    float4 V;
    {
        const Site x = site_from_parity_index(ch, P, e);
        const uint32_t sc = canonical(ch, x);
        const float4 W = staple<MU, P, LD>(U, ch, x, sc, e);
        const float k2 = qdot(W, W);
        if (!(k2 > 0.f))
            return;
        V = qscale(W, 1.0f / sqrtf(k2));
    }
    float4 *dst = &U[(size_t)(P * 4 + MU) * ch.nh + e];
    const float4 u = lat_load<LD>(dst);
    float4 Un = qmul(qmul(V, qdag(u)), V);
    *dst = qscale(Un, rsqrtf(qdot(Un, Un)));
}

template <int LD>
__device__ __forceinline__ void su2_overrelax_link_rt(int phase, float4 *U, const Su2Chain &ch, uint32_t e)
{
    switch (phase) {
    case 0: su2_overrelax_link<1, 0, LD>(U, ch, e); break;
    case 1: su2_overrelax_link<1, 1, LD>(U, ch, e); break;
    case 2: su2_overrelax_link<1, 2, LD>(U, ch, e); break;
    case 3: su2_overrelax_link<1, 3, LD>(U, ch, e); break;
    case 4: su2_overrelax_link<0, 0, LD>(U, ch, e); break;
    case 5: su2_overrelax_link<0, 1, LD>(U, ch, e); break;
    case 6: su2_overrelax_link<0, 2, LD>(U, ch, e); break;
    default: su2_overrelax_link<0, 3, LD>(U, ch, e); break;
    }
}

// How much of the RNG-only work the persistent batch kernel moves ahead of the
// staple (the EARLY argument of su2_update_link).  With its 128-register
// budget the direction alone measured best on the batched workload: 0.459 ms
// per sweep against 0.475-0.491 (direction and first try) and 0.487 (neither).
#ifndef MC_GROUP_EARLY
#define MC_GROUP_EARLY 1
#endif

// Runtime (P, MU) dispatch of su2_update_link for the persistent batch kernel
// (no try record, inlined failure count).
template <int LD>
__device__ __forceinline__ void su2_update_link_rt(int phase, float4 *U, const Su2Chain &ch, const PhiloxSchedule &ks,
                                                   uint32_t e, uint32_t sweep, DevState *state)
{
    switch (phase) { // phase = position in the sweep: (odd, mu = 0..3), then (even, mu = 0..3)
    case 0: su2_update_link<1, 0, LD, false, true, MC_GROUP_EARLY>(U, ch, ks, e, sweep, nullptr, state); break;
    case 1: su2_update_link<1, 1, LD, false, true, MC_GROUP_EARLY>(U, ch, ks, e, sweep, nullptr, state); break;
    case 2: su2_update_link<1, 2, LD, false, true, MC_GROUP_EARLY>(U, ch, ks, e, sweep, nullptr, state); break;
    case 3: su2_update_link<1, 3, LD, false, true, MC_GROUP_EARLY>(U, ch, ks, e, sweep, nullptr, state); break;
    case 4: su2_update_link<0, 0, LD, false, true, MC_GROUP_EARLY>(U, ch, ks, e, sweep, nullptr, state); break;
    case 5: su2_update_link<0, 1, LD, false, true, MC_GROUP_EARLY>(U, ch, ks, e, sweep, nullptr, state); break;
    case 6: su2_update_link<0, 2, LD, false, true, MC_GROUP_EARLY>(U, ch, ks, e, sweep, nullptr, state); break;
    default: su2_update_link<0, 3, LD, false, true, MC_GROUP_EARLY>(U, ch, ks, e, sweep, nullptr, state); break;
    }
}

// Plaquette sums in exact fixed point: each plaquette's FP32 value h (|h| <= 1)
// is rounded to a multiple of 2^-29 (an int32) and summed in int64.  The sum is
// exact, hence independent of the order, of the launch shape and of how the
// plaquettes are shared out among threads, for up to 2.8e9 sites, and it stays
// off the GB300's FP64 pipe, which made an FP64 shuffle reduction the larger
// part of the measurement's cost.
constexpr float kPlaqFix = 536870912.0f; // 2^29 (kPlaqUnfix, its inverse, is in mc_internal.cuh)
__device__ __forceinline__ long long plaq_fixed(float v) { return (long long)__float2int_rn(v * kPlaqFix); }

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// (1/2) Tr U_munu(x) of Eq. (3): (1/2) Tr[U_mu(x) U_nu(x+mu) (U_nu(x) U_mu(x+nu))^+]
// = A . B with A = U_mu(x) U_nu(x+mu), B = U_nu(x) U_mu(x+nu).
__device__ __forceinline__ float plaquette_value(float4 umu_x, float4 unu_xmu, float4 unu_x, float4 umu_xnu)
{
    return qdot(qmul(umu_x, unu_xmu), qmul(unu_x, umu_xnu));
}

// The six plaquettes at a site, from its own links Ux[mu] and the forward
// links Uf[mu][nu] = U_nu(x + mu), added in fixed point: spatial planes to ps,
// temporal (mu = 0) to pt.
__device__ __forceinline__ void plaquettes_of(const float4 (&Ux)[4], const float4 (&Uf)[4][4], long long &ps,
                                              long long &pt)
{
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
#pragma unroll
        for (int nu = mu + 1; nu < 4; ++nu) {
            const long long h = plaq_fixed(plaquette_value(Ux[mu], Uf[mu][nu], Ux[nu], Uf[nu][mu]));
            if (mu == 0)
                pt += h;
            else
                ps += h;
        }
}

__device__ __forceinline__ Site site_of_canonical(const Su2Chain &ch, uint32_t s)
{
    uint32_t q1, q2, c[4];
    fast_divmod(s, ch.div1, q1, c[1]);
    fast_divmod(q1, ch.div2, q2, c[2]);
    fast_divmod(q2, ch.div3, c[0], c[3]);
    Site x;
    for (int m = 0; m < 4; ++m)
        x.x[m] = (int)c[m];
    return x;
}

// Spatial and temporal fixed-point sums of (1/2) Tr U_munu(x) over the six
// plaquettes with corner at canonical site s, added to ps and pt; FP32 products.
template <int LD>
__device__ __forceinline__ void su2_site_plaquettes(const float4 *U, const Su2Chain &ch, uint32_t s, long long &ps,
                                                    long long &pt)
{
    const Site x = site_of_canonical(ch, s);
    const int p = (x.x[0] + x.x[1] + x.x[2] + x.x[3]) & 1, q = 1 - p;
    const uint32_t e = s >> 1;
    float4 Ux[4], Uf[4][4]; // Uf[mu][nu] = U_nu(x + mu)
    Site xf[4];
    xf[0] = step<0>(ch, x, +1);
    xf[1] = step<1>(ch, x, +1);
    xf[2] = step<2>(ch, x, +1);
    xf[3] = step<3>(ch, x, +1);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
        Ux[mu] = load_link<LD>(U, ch.nh, p, mu, e);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const uint32_t ef = canonical(ch, xf[mu]) >> 1;
#pragma unroll
        for (int nu = 0; nu < 4; ++nu)
            if (nu != mu)
                Uf[mu][nu] = load_link<LD>(U, ch.nh, q, nu, ef);
    }
    plaquettes_of(Ux, Uf, ps, pt);
}

// The same sums for the two sites of an x1 pair, canonical 2j and 2j + 1 (L1 is
// even, so both lie in one row and have opposite parities; both have index j
// within their parity).  The second site's own links are the first site's
// forward links along x1, so the pair takes 29 link loads instead of 32, and
// one thread carries two independent products chains.
template <int LD>
__device__ __forceinline__ void su2_pair_plaquettes(const float4 *U, const Su2Chain &ch, uint32_t j, long long &ps,
                                                    long long &pt)
{
    const Site x = site_of_canonical(ch, 2 * j);
    Site y = x;
    y.x[1] += 1;
    const int p0 = (x.x[0] + x.x[1] + x.x[2] + x.x[3]) & 1, p1 = 1 - p0;
    const uint32_t nh = ch.nh;
    float4 U0[4], U1[4], F0[4][4], F1[4][4]; // F0[mu][nu] = U_nu(x + mu), F1[mu][nu] = U_nu(y + mu)
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        U0[mu] = load_link<LD>(U, nh, p0, mu, j);
        U1[mu] = load_link<LD>(U, nh, p1, mu, j);
    }
#pragma unroll
    for (int nu = 0; nu < 4; ++nu)
        F0[1][nu] = U1[nu];
    const uint32_t e00 = canonical(ch, step<0>(ch, x, +1)) >> 1, e02 = canonical(ch, step<2>(ch, x, +1)) >> 1,
                   e03 = canonical(ch, step<3>(ch, x, +1)) >> 1;
    const uint32_t e10 = canonical(ch, step<0>(ch, y, +1)) >> 1, e11 = canonical(ch, step<1>(ch, y, +1)) >> 1,
                   e12 = canonical(ch, step<2>(ch, y, +1)) >> 1, e13 = canonical(ch, step<3>(ch, y, +1)) >> 1;
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
        if (nu != 0) F0[0][nu] = load_link<LD>(U, nh, p1, nu, e00);
        if (nu != 2) F0[2][nu] = load_link<LD>(U, nh, p1, nu, e02);
        if (nu != 3) F0[3][nu] = load_link<LD>(U, nh, p1, nu, e03);
        if (nu != 0) F1[0][nu] = load_link<LD>(U, nh, p0, nu, e10);
        if (nu != 1) F1[1][nu] = load_link<LD>(U, nh, p0, nu, e11);
        if (nu != 2) F1[2][nu] = load_link<LD>(U, nh, p0, nu, e12);
        if (nu != 3) F1[3][nu] = load_link<LD>(U, nh, p0, nu, e13);
    }
    plaquettes_of(U0, F0, ps, pt);
    plaquettes_of(U1, F1, ps, pt);
}

// Canonical index of the neighbour x + e_D of site x (canonical index s).
template <int D>
__device__ __forceinline__ uint32_t canonical_fwd(const Su2Chain &ch, const Site &x, uint32_t s)
{
    return fwd<D>(ch, strides_of(ch), x.x[D], s);
}

// One plaquette, plane (MU, NU) at canonical site s, added in fixed point to pt
// (MU = 0) or ps: the value plaquettes_of computes for that plane.
template <int MU, int NU, int LD>
__device__ __forceinline__ void su2_plane_plaquette(const float4 *U, const Su2Chain &ch, const Site &x, uint32_t s,
                                                    long long &ps, long long &pt)
{
    const int p = (x.x[0] + x.x[1] + x.x[2] + x.x[3]) & 1;
    const uint32_t nh = ch.nh, e = s >> 1;
    const float4 umu = load_link<LD>(U, nh, p, MU, e);
    const float4 unu = load_link<LD>(U, nh, p, NU, e);
    const float4 unu_f = load_link<LD>(U, nh, 1 - p, NU, canonical_fwd<MU>(ch, x, s) >> 1);
    const float4 umu_f = load_link<LD>(U, nh, 1 - p, MU, canonical_fwd<NU>(ch, x, s) >> 1);
    const long long h = plaq_fixed(plaquette_value(umu, unu_f, unu, umu_f));
    if (MU == 0)
        pt += h;
    else
        ps += h;
}

// Plaquette number u of a chain, u = plane N + s (N = 2 nh sites; planes in
// the order (0,1), (0,2), (0,3), (1,2), (1,3), (2,3)), so that consecutive
// threads take consecutive sites of one plane; added in fixed point to ps / pt.
template <int LD>
__device__ __forceinline__ void su2_plaquette_unit(const float4 *U, const Su2Chain &ch, uint32_t u, long long &ps,
                                                   long long &pt)
{
    const uint32_t n = 2u * ch.nh, plane = u / n, s = u - plane * n;
    const Site x = site_of_canonical(ch, s);
    switch (plane) {
    case 0: su2_plane_plaquette<0, 1, LD>(U, ch, x, s, ps, pt); break;
    case 1: su2_plane_plaquette<0, 2, LD>(U, ch, x, s, ps, pt); break;
    case 2: su2_plane_plaquette<0, 3, LD>(U, ch, x, s, ps, pt); break;
    case 3: su2_plane_plaquette<1, 2, LD>(U, ch, x, s, ps, pt); break;
    case 4: su2_plane_plaquette<1, 3, LD>(U, ch, x, s, ps, pt); break;
    default: su2_plane_plaquette<2, 3, LD>(U, ch, x, s, ps, pt); break;
    }
}

}  // namespace
}  // namespace mc
