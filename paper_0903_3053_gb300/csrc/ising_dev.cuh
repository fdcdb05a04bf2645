// ising_dev.cuh -- per-site and per-word device code of the 2D Ising
// Metropolis update (Eq. (1), Sec. 2.3), shared by the grid-mode and resident
// kernels of ising.cu and the persistent batch kernel of batch.cu.
//
// Random numbers: site i = y*(Lx/2) + j of colour c uses word (i & 3) of the
// Philox block with counter (i >> 2, sweep, TAG_METRO | c, chain_id).  A spin
// flips when dE = 2 s h <= 0, or when its word is below
// T[dE] = floor(e^{-beta dE} 2^32).
#pragma once
#include "mc_internal.cuh"

namespace mc {
namespace {

__device__ __forceinline__ uint32_t inc_wrap(uint32_t v, uint32_t n) { return v + 1 == n ? 0u : v + 1; }
__device__ __forceinline__ uint32_t dec_wrap(uint32_t v, uint32_t n) { return v == 0 ? n - 1 : v - 1; }

// Sum two per-thread counters over the CTA; thread 0 receives the totals.
// Every thread of the CTA must call it.
__device__ __forceinline__ void block_sum2(uint32_t &a, uint32_t &b)
{
    __shared__ uint32_t sa[32], sb[32];
    a = __reduce_add_sync(0xffffffffu, a);
    b = __reduce_add_sync(0xffffffffu, b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t ta = 0, tb = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ta += sa[w];
            tb += sb[w];
        }
        a = ta;
        b = tb;
    }
}

// ------------------------------------------------------------------ int8 layout
// Update the (up to four) sites of colour C that share Philox block g.
template <int C, bool MEASURE, int LD = kLdPlain>
__device__ __forceinline__ void int8_group(int8_t *s, const IsingChain &ch, const PhiloxSchedule &ks, uint32_t g,
                                           uint32_t sweep, uint32_t &anti, uint32_t &up)
{
    const uint32_t Lx = ch.Lx, Ly = ch.Ly, half = Lx >> 1, nc = (Lx * Ly) >> 1;
    const uint4 r4 = philox4x32_10(make_uint4(g, sweep, kTagIsingMetro | (uint32_t)C, ch.chain_id), ks);
    const uint32_t rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t i = 4 * g + q;
        if (i >= nc)
            break;
        const uint32_t y = i / half, j = i - y * half;
        const uint32_t x = 2 * j + ((y + C) & 1u);
        const uint32_t row = y * Lx, rowp = inc_wrap(y, Ly) * Lx, rowm = dec_wrap(y, Ly) * Lx;
        const int sv = lat_load<LD>(&s[row + x]);
        const int ne = lat_load<LD>(&s[row + inc_wrap(x, Lx)]), nw = lat_load<LD>(&s[row + dec_wrap(x, Lx)]);
        const int nn = lat_load<LD>(&s[rowm + x]), ns = lat_load<LD>(&s[rowp + x]);
        const int local = sv * (ne + nw + nn + ns); // dE / 2
        const bool flip = local <= 0 || rr[q] < (local == 2 ? ch.T2 : ch.T4);
        const int nv = flip ? -sv : sv;
        if (flip)
            s[row + x] = (int8_t)nv;
        if (MEASURE) {
            anti += (uint32_t)(ne != nv) + (uint32_t)(nw != nv) + (uint32_t)(nn != nv) + (uint32_t)(ns != nv);
            const int partner = (x & 1u) ? nw : ne; // colour-0 site (x ^ 1, y)
            up += (uint32_t)(nv > 0) + (uint32_t)(partner > 0);
        }
    }
}

// ------------------------------------------------------------------ MSC layout
// Comparison of one random word with a threshold, appended to a bit mask: the
// carry out of r + (2^32 - T) is (r >= T) for T >= 1 and is shifted into `g`
// (g <- 2 g + carry), two integer adds per site and no predicate.  T = 0 (no
// site accepted) is fixed up by the caller.
__device__ __forceinline__ void ge_chain2(uint32_t &g2, uint32_t &g4, uint32_t r, uint32_t nT2, uint32_t nT4)
{
    asm("{\n\t.reg .u32 t;\n\t"
        "add.cc.u32 t, %2, %3;\n\t"
        "addc.u32 %0, %0, %0;\n\t"
        "add.cc.u32 t, %2, %4;\n\t"
        "addc.u32 %1, %1, %1;\n\t}"
        : "+r"(g2), "+r"(g4)
        : "r"(r), "r"(nT2), "r"(nT4));
}

// New value of one colour-C word given its four neighbour words.  Every 4-site
// Philox block is drawn (a per-block skip branch costs more than it saves).
// Every site is compared with both thresholds, as two carry chains that build
// the masks g2 = (r >= T2) and g4 = (r >= T4) with site b at bit b (sites are
// visited from 31 down to 0); a site with one anti-aligned neighbour (dE = 4)
// flips iff r < T2, one with none (dE = 8) iff r < T4, and since T4 <= T2
// the flip mask is ge2 | ~g4 | (eq1 & ~g2).  (A per-site select of the
// threshold followed by one compare measured 12% slower.)
template <int C>
__device__ __forceinline__ uint32_t msc_word(uint32_t s, uint32_t nu, uint32_t nd, uint32_t ns, uint32_t side,
                                             uint32_t blk0, uint32_t sweep, const IsingChain &ch,
                                             const PhiloxSchedule &ks)
{
    const uint32_t a1 = s ^ nu, a2 = s ^ nd, a3 = s ^ ns, a4 = s ^ side; // 1 = anti-aligned
    const uint32_t s12 = a1 ^ a2, c12 = a1 & a2, s34 = a3 ^ a4, c34 = a3 & a4;
    const uint32_t ge2 = c12 | c34 | (s12 & s34); // >= 2 anti-aligned: dE <= 0, always flip
    const uint32_t eq0 = ~(a1 | a2 | a3 | a4);    // dE = 8
    const uint32_t eq1 = ~(ge2 | eq0);            // dE = 4
    const uint32_t nT2 = 0u - ch.T2, nT4 = 0u - ch.T4;
    uint32_t g2 = 0, g4 = 0;
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        const uint4 r = philox4x32_10(make_uint4(blk0 + k, sweep, kTagIsingMetro | (uint32_t)C, ch.chain_id), ks);
        ge_chain2(g2, g4, r.w, nT2, nT4);
        ge_chain2(g2, g4, r.z, nT2, nT4);
        ge_chain2(g2, g4, r.y, nT2, nT4);
        ge_chain2(g2, g4, r.x, nT2, nT4);
    }
    if (ch.T2 == 0)
        g2 = ~0u;
    if (ch.T4 == 0)
        g4 = ~0u;
    return s ^ (ge2 | ~g4 | (eq1 & ~g2));
}

// Update words (2 yy, w) and (2 yy + 1, w) of plane C.  The two rows share the
// other plane's rows 2 yy and 2 yy + 1 as neighbours, so six loads serve both
// words.  Row y holds sites x = 2 j + ((y + C) & 1): offset C on the even row,
// 1 - C on the odd one, which decides the side (j - 1 or j + 1) neighbour.
template <int C, bool MEASURE, int LD = kLdPlain>
__device__ __forceinline__ void msc_row_pair(uint32_t *pc, const uint32_t *po, uint32_t yy, uint32_t w,
                                             const IsingChain &ch, const PhiloxSchedule &ks, uint32_t sweep,
                                             uint32_t &anti, uint32_t &up)
{
    const uint32_t W = ch.W, Ly = ch.Ly, y0 = 2 * yy, y1 = y0 + 1;
    const uint32_t om = lat_load<LD>(&po[dec_wrap(y0, Ly) * W + w]);
    const uint32_t o0 = lat_load<LD>(&po[y0 * W + w]);
    const uint32_t o1 = lat_load<LD>(&po[y1 * W + w]);
    const uint32_t op = lat_load<LD>(&po[inc_wrap(y1, Ly) * W + w]);
    uint32_t side0, side1;
    if (C == 0) {
        side0 = (o0 << 1) | (lat_load<LD>(&po[y0 * W + dec_wrap(w, W)]) >> 31);
        side1 = (o1 >> 1) | (lat_load<LD>(&po[y1 * W + inc_wrap(w, W)]) << 31);
    } else {
        side0 = (o0 >> 1) | (lat_load<LD>(&po[y0 * W + inc_wrap(w, W)]) << 31);
        side1 = (o1 << 1) | (lat_load<LD>(&po[y1 * W + dec_wrap(w, W)]) >> 31);
    }
    const uint32_t s0 = lat_load<LD>(&pc[y0 * W + w]), s1 = lat_load<LD>(&pc[y1 * W + w]);
    const uint32_t bpr = ch.Lx >> 3; // Philox blocks per row of one colour
    const uint32_t n0 = msc_word<C>(s0, om, o1, o0, side0, y0 * bpr + 8 * w, sweep, ch, ks);
    const uint32_t n1 = msc_word<C>(s1, o0, op, o1, side1, y1 * bpr + 8 * w, sweep, ch, ks);
    if (n0 != s0)
        pc[y0 * W + w] = n0;
    if (n1 != s1)
        pc[y1 * W + w] = n1;
    if (MEASURE) {
        anti += __popc(n0 ^ om) + __popc(n0 ^ o1) + __popc(n0 ^ o0) + __popc(n0 ^ side0) + __popc(n1 ^ o0) +
                __popc(n1 ^ op) + __popc(n1 ^ o1) + __popc(n1 ^ side1);
        up += __popc(n0) + __popc(o0) + __popc(n1) + __popc(o1);
    }
}

// Gather the neighbours of word (y, w) of plane C from the other plane `po`.
template <int C>
__device__ __forceinline__ void msc_neighbours(const uint32_t *po, uint32_t y, uint32_t w, uint32_t W, uint32_t Ly,
                                               uint32_t &nu, uint32_t &nd, uint32_t &ns, uint32_t &side)
{
    const uint32_t row = y * W;
    nu = po[dec_wrap(y, Ly) * W + w];
    nd = po[inc_wrap(y, Ly) * W + w];
    ns = po[row + w];
    if (((y + C) & 1u) == 0) { // x = 2j: other colour at j-1 and j
        const uint32_t prev = po[row + dec_wrap(w, W)];
        side = (ns << 1) | (prev >> 31);
    } else { // x = 2j+1: other colour at j and j+1
        const uint32_t next = po[row + inc_wrap(w, W)];
        side = (ns >> 1) | (next << 31);
    }
}

}  // namespace
}  // namespace mc
