// su2.cu -- 4D SU(2) pure-gauge heat-bath (Sec. 2.4).
//
// Links are the quaternions (U0, U1, U2, U3) of Eq. (4), one float4 per link,
// stored per chain as [parity][mu][site-within-parity] so that the 32 links a
// warp reads for one neighbour direction are 512 contiguous bytes.  Canonical
// site index s = x1 + L1 (x2 + L2 (x3 + L3 x0)) (mu = 0 is time); with L1 even,
// the index of s within its parity class is s >> 1.
//
// One kernel per (parity p, direction mu) phase, in the order of Sec. 2.4
// (mu = 0..3 on odd sites, then on even sites), one thread per site of parity p:
//   1. staple W of Eq. (6), summed over the six nu != mu (the paper's separate
//      staple kernel and its N_vect staple buffer are fused away: W lives in
//      registers only);
//   2. k = |W|, V = W / k, alpha = beta k;
//   3. a0 from Kennedy-Pendleton (up to 8 tries, the "8 attempts per start" of
//      Sec. 2.4), then Creutz (up to 64 tries); a link whose every try fails is
//      left unchanged and counted (still exact: the failure probability depends
//      on alpha only);
//   4. a uniform direction on S^2 for the remaining components;
//   5. U = X V (Eq. (5) with w = X/k) and reprojection onto SU(2) (U / |U|).
// Try t of the link at parity index e uses the Philox block
// (e, sweep, TAG_HB | p<<12 | mu<<8 | t, chain); the direction uses
// (e, sweep, TAG_DIR | p<<12 | mu<<8, chain).  Uniforms are ((r>>8)+1) 2^-24.
// FP32 throughout.  The heat-bath draw keeps the correctly rounded library
// functions (logf, cospif, expm1f, log1pf): a0 = 1 - 2 lambda^2 amplifies their
// error near a0 = 1, and __logf / __cosf there moved single links by more than
// 1e-5.  The normalisations (1 / |W|, |W|, sqrt(1 - a0^2), sin theta) use
// rsqrtf, 1 / (2 alpha) uses __fdividef, and the direction's angle uses
// __sincosf on an argument reduced to (-pi, pi] -- errors of a few 1e-7 per
// link, 5% less time per phase.  Lattice-wide plaquette and Polyakov sums in
// exact int64 fixed point, FP64 only for the final averages.  Site coordinates
// come from magic-number divisions.
#include "su2_dev.cuh"

namespace mc {
namespace {

// 256 threads, at least 6 blocks per SM (40 registers; ptxas spills 12-48
// bytes per thread, about 1% of the kernel's load requests): the phase is bound
// by the latency of the 18 neighbour-link loads, and 48 resident warps hide it
// better than the 40 an unconstrained build allows (+14% measured on 4 x 32^4).
template <int P, int MU, bool REC>
__global__ void __launch_bounds__(256, 6) k_phase(SweepArgs a)
{
    const uint32_t b = blockIdx.x + a.block_base;
    const int k = find_chain(a.block_start, a.n_chains, b);
    const Su2Chain ch = static_cast<const Su2Chain *>(a.chains)[k];
    const uint32_t e = (b - a.block_start[k]) * blockDim.x + threadIdx.x;
    if (e >= ch.nh)
        return;
    float4 *U = reinterpret_cast<float4 *>(a.lattice + ch.link_off);
    const PhiloxSchedule ks = philox_schedule(ch.key);
    su2_update_link<P, MU, kLdReadOnly, REC>(U, ch, ks, e, (uint32_t)(a.state->sweep_base + a.k), a.tries, a.state);
}

// Overrelaxation phase: same thread layout as k_phase, no random numbers.
template <int P, int MU>
__global__ void __launch_bounds__(256, 6) k_or_phase(SweepArgs a)
{
    const uint32_t b = blockIdx.x + a.block_base;
    const int k = find_chain(a.block_start, a.n_chains, b);
    const Su2Chain ch = static_cast<const Su2Chain *>(a.chains)[k];
    const uint32_t e = (b - a.block_start[k]) * blockDim.x + threadIdx.x;
    if (e >= ch.nh)
        return;
    float4 *U = reinterpret_cast<float4 *>(a.lattice + ch.link_off);
    su2_overrelax_link<P, MU, kLdReadOnly>(U, ch, e);
}

// ------------------------------------------------------------------ plaquette
// Per-block partial sums of (1/2) Tr U_munu(x) of Eq. (3), spatial and temporal
// separately (the two values per measuring thread of Sec. 2.4).  One thread per
// x1 pair of sites (su2_pair_plaquettes), kPlaqThreads pairs per block, at
// least 8 blocks per SM: 74 us instead of 96 us for one site per thread on
// 4 x 32^4, where the kernel is bound by the latency of its link loads.
// Products in FP32, sums in exact int64 fixed point (plaq_fixed);
// partial[2 b], partial[2 b + 1].
__global__ void __launch_bounds__(kPlaqThreads, 8) k_plaquette(const Su2Chain *chains, const uint32_t *meas_start,
                                                               int n_chains, const char *lattice, long long *partial,
                                                               uint32_t block_base)
{
    __shared__ long long ss[kPlaqThreads / 32], st[kPlaqThreads / 32];
    const uint32_t blk = blockIdx.x + block_base;
    const int k = find_chain(meas_start, n_chains, blk);
    const Su2Chain ch = chains[k];
    const uint32_t j = (blk - meas_start[k]) * kPlaqThreads + threadIdx.x;
    long long ps = 0, pt = 0;
    if (j < ch.nh)
        su2_pair_plaquettes<kLdReadOnly>(reinterpret_cast<const float4 *>(lattice + ch.link_off), ch, j, ps, pt);
    ps = warp_sum_ll(ps);
    pt = warp_sum_ll(pt);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        ss[w] = ps;
        st[w] = pt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0, b = 0;
        for (int i = 0; i < kPlaqThreads / 32; ++i) {
            a += ss[i];
            b += st[i];
        }
        partial[2 * blk] = a;
        partial[2 * blk + 1] = b;
    }
}

// One block per chain (blockIdx.x = chain index, or `only` when >= 0): exact sum
// of the chain's partials, written as P, P_s, P_t.
__global__ void __launch_bounds__(256) k_plaquette_final(const Su2Chain *chains, const uint32_t *meas_start,
                                                         const long long *partial, DevRecord *series, long long cap,
                                                         const DevState *state, uint32_t ksweep, uint32_t rec_k,
                                                         int only, DevRecord *out)
{
    __shared__ long long ss[8], st[8];
    const int k = only >= 0 ? only : (int)blockIdx.x;
    const uint32_t b0 = meas_start[k], b1 = meas_start[k + 1];
    long long a = 0, b = 0;
    for (uint32_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        a += partial[2 * i];
        b += partial[2 * i + 1];
    }
    a = warp_sum_ll(a);
    b = warp_sum_ll(b);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        ss[w] = a;
        st[w] = b;
    }
    __syncthreads();
    if (threadIdx.x != 0)
        return;
    long long A = 0, B = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
        A += ss[i];
        B += st[i];
    }
    DevRecord *rec = out;
    long long sweep = (long long)(state->sweep_base + ksweep);
    if (!rec) {
        const unsigned long long slot = (state->rec_head + rec_k) % (unsigned long long)cap;
        rec = &series[(long long)k * cap + (long long)slot];
    } else {
        sweep = (long long)state->sweep_base - 1;
    }
    rec->sweep = sweep;
    rec->a = (unsigned long long)A; // the exact sums; P, P_s, P_t are formed on the host
    rec->b = (unsigned long long)B;
    rec->d0 = rec->d1 = rec->d2 = 0.0;
}

// ------------------------------------------------------------------ Polyakov loop
// One thread per spatial site xs = x1 + L1 (x2 + L2 x3): the time-ordered
// product U_0(0, xs) ... U_0(L0 - 1, xs) of FP32 quaternions; (1/2) Tr of an
// SU(2) quaternion is its first component.  Exact fixed-point sums as for the
// plaquette; partial[b] per block, then one block for the chain.
__global__ void __launch_bounds__(256) k_polyakov(Su2Chain ch, const float4 *__restrict__ U, long long *partial)
{
    __shared__ long long sp[8];
    const uint32_t nspace = (uint32_t)ch.L[1] * ch.L[2] * ch.L[3];
    const uint32_t xs = blockIdx.x * blockDim.x + threadIdx.x;
    long long v = 0;
    if (xs < nspace) {
        uint32_t q1, q2, x1, x2, x3;
        fast_divmod(xs, ch.div1, q1, x1);
        fast_divmod(q1, ch.div2, q2, x2);
        x3 = q2;
        const uint32_t sp0 = (x1 + x2 + x3) & 1u;
        float4 P = make_float4(1.f, 0.f, 0.f, 0.f);
        for (int t = 0; t < ch.L[0]; ++t) {
            const uint32_t s = xs + (uint32_t)t * nspace, p = (sp0 + (uint32_t)t) & 1u;
            P = qmul(P, __ldg(&U[(size_t)(p * 4 + 0) * ch.nh + (s >> 1)]));
        }
        v = plaq_fixed(P.x);
    }
    v = warp_sum_ll(v);
    if ((threadIdx.x & 31) == 0)
        sp[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i)
            a += sp[i];
        partial[blockIdx.x] = a;
    }
}

__global__ void __launch_bounds__(256) k_polyakov_final(const long long *partial, uint32_t nb, uint32_t nspace,
                                                        DevRecord *out)
{
    __shared__ long long sp[8];
    long long a = 0;
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x)
        a += partial[i];
    a = warp_sum_ll(a);
    if ((threadIdx.x & 31) == 0)
        sp[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long A = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i)
            A += sp[i];
        out->a = out->b = 0;
        out->d0 = (double)A * kPlaqUnfix / (double)nspace;
        out->d1 = out->d2 = 0.0;
    }
}

// ------------------------------------------------------------------ init / I/O
// Hot start: Haar-random link = normalised 4-vector of four Box-Muller normals
// from the Philox block (s, 0, TAG_INIT | mu, chain); cold start: identity.
__global__ void k_su2_init(Su2Chain ch, float4 *U, int hot)
{
    const uint32_t n = 2 * ch.nh;
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4 * n)
        return;
    const uint32_t s = idx >> 2, mu = idx & 3u;
    float4 v = make_float4(1.f, 0.f, 0.f, 0.f);
    if (hot) {
        const uint4 r = philox4x32_10(make_uint4(s, 0u, kTagSu2Init | mu, ch.chain_id), ch.key);
        const float ra = sqrtf(-2.0f * logf(uniform_open0(r.x)));
        const float rb = sqrtf(-2.0f * logf(uniform_open0(r.z)));
        float sa, ca, sb, cb;
        sincospif(2.0f * uniform_open0(r.y), &sa, &ca);
        sincospif(2.0f * uniform_open0(r.w), &sb, &cb);
        v = make_float4(ra * ca, ra * sa, rb * cb, rb * sb);
        const float inv = rsqrtf(qdot(v, v));
        v = make_float4(v.x * inv, v.y * inv, v.z * inv, v.w * inv);
    }
    // parity of s from its coordinates
    uint32_t r = s;
    int x1 = (int)(r % (uint32_t)ch.L[1]);
    r /= (uint32_t)ch.L[1];
    int x2 = (int)(r % (uint32_t)ch.L[2]);
    r /= (uint32_t)ch.L[2];
    int x3 = (int)(r % (uint32_t)ch.L[3]);
    int x0 = (int)(r / (uint32_t)ch.L[3]);
    const int p = (x0 + x1 + x2 + x3) & 1;
    U[(size_t)(p * 4 + mu) * ch.nh + (s >> 1)] = v;
}

// canonical float q[s][mu][4] <-> internal [parity][mu][s >> 1]
__global__ void k_su2_io(Su2Chain ch, float4 *U, float4 *canon, int to_lattice)
{
    const uint32_t n = 2 * ch.nh;
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4 * n)
        return;
    const uint32_t s = idx >> 2, mu = idx & 3u;
    uint32_t r = s;
    int x1 = (int)(r % (uint32_t)ch.L[1]);
    r /= (uint32_t)ch.L[1];
    int x2 = (int)(r % (uint32_t)ch.L[2]);
    r /= (uint32_t)ch.L[2];
    int x3 = (int)(r % (uint32_t)ch.L[3]);
    int x0 = (int)(r / (uint32_t)ch.L[3]);
    const int p = (x0 + x1 + x2 + x3) & 1;
    float4 *in = &U[(size_t)(p * 4 + mu) * ch.nh + (s >> 1)];
    if (to_lattice)
        *in = canon[idx];
    else
        canon[idx] = *in;
}

inline unsigned blocks_for(size_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <int P>
void launch_phase(mc_ctx *c, const SweepArgs &a, int mu, unsigned nblocks)
{
    if (prof_begin(c) != cudaSuccess)
        return;
    const bool rec = a.tries != nullptr;
    switch (mu * 2 + (rec ? 1 : 0)) {
    case 0: k_phase<P, 0, false><<<nblocks, c->threads, 0, c->ls>>>(a); break;
    case 1: k_phase<P, 0, true><<<nblocks, c->threads, 0, c->ls>>>(a); break;
    case 2: k_phase<P, 1, false><<<nblocks, c->threads, 0, c->ls>>>(a); break;
    case 3: k_phase<P, 1, true><<<nblocks, c->threads, 0, c->ls>>>(a); break;
    case 4: k_phase<P, 2, false><<<nblocks, c->threads, 0, c->ls>>>(a); break;
    case 5: k_phase<P, 2, true><<<nblocks, c->threads, 0, c->ls>>>(a); break;
    case 6: k_phase<P, 3, false><<<nblocks, c->threads, 0, c->ls>>>(a); break;
    default: k_phase<P, 3, true><<<nblocks, c->threads, 0, c->ls>>>(a); break;
    }
    prof_end(c);
}

template <int P>
void launch_or_phase(mc_ctx *c, const SweepArgs &a, int mu, unsigned nblocks)
{
    if (prof_begin(c) != cudaSuccess)
        return;
    switch (mu) {
    case 0: k_or_phase<P, 0><<<nblocks, c->threads, 0, c->ls>>>(a); break;
    case 1: k_or_phase<P, 1><<<nblocks, c->threads, 0, c->ls>>>(a); break;
    case 2: k_or_phase<P, 2><<<nblocks, c->threads, 0, c->ls>>>(a); break;
    default: k_or_phase<P, 3><<<nblocks, c->threads, 0, c->ls>>>(a); break;
    }
    prof_end(c);
}

}  // namespace

// =========================================================================== host
size_t su2_config_bytes(const Su2Chain &ch) { return (size_t)2 * ch.nh * 4 * sizeof(float4); }

// Block tables.  All chains of the batch form one launch group: sweeping
// L2-sized groups of chains one after another (to keep each group's links
// L2-resident across its eight phases) was measured slower on 4 x 32^4 -- the
// phase kernel is issue-bound, and four one-chain launches per phase add tail
// waves -- so the group list holds a single entry.
void su2_plan_grid(mc_ctx *c)
{
    c->block_start.assign(c->n_chains + 1, 0);
    c->meas_start.assign(c->n_chains + 1, 0);
    uint32_t acc = 0, macc = 0;
    for (int k = 0; k < c->n_chains; ++k) {
        c->block_start[k] = acc;
        c->meas_start[k] = macc;
        acc += blocks_for(c->su2[k].nh, c->threads);
        macc += blocks_for(c->su2[k].nh, kPlaqThreads);
    }
    c->block_start[c->n_chains] = acc;
    c->meas_start[c->n_chains] = macc;
    c->grid_blocks = acc;
    c->meas_blocks = macc;
    c->groups.assign(1, std::make_pair(0, c->n_chains));
}

cudaError_t su2_init_launch(mc_ctx *c, const mc_chain_desc *desc)
{
    for (int k = 0; k < c->n_chains; ++k) {
        const Su2Chain &ch = c->su2[k];
        k_su2_init<<<blocks_for((size_t)8 * ch.nh, 256), 256, 0, c->ls>>>(
            ch, reinterpret_cast<float4 *>(c->d_lattice + ch.link_off), desc[k].start == MC_HOT);
    }
    return cudaGetLastError();
}

// Per-block plaquette partial sums for chains [k0, k1).
static void plaquette_partials(mc_ctx *c, int k0, int k1)
{
    const uint32_t b0 = c->meas_start[k0], b1 = c->meas_start[k1];
    k_plaquette<<<b1 - b0, kPlaqThreads, 0, c->ls>>>(static_cast<const Su2Chain *>(c->d_chains), c->d_meas_start, c->n_chains,
                                            c->d_lattice, c->d_partials, b0);
}

static void plaquette_final(mc_ctx *c, uint32_t ksweep, uint32_t rec_k, int only, DevRecord *out)
{
    const unsigned nb = only >= 0 ? 1u : (unsigned)c->n_chains;
    k_plaquette_final<<<nb, 256, 0, c->ls>>>(static_cast<const Su2Chain *>(c->d_chains), c->d_meas_start,
                                             c->d_partials, c->d_series, c->cap, c->d_state, ksweep, rec_k, only, out);
}

cudaError_t su2_sweep_enqueue(mc_ctx *c, long long n, int every)
{
    SweepArgs a{};
    a.chains = c->d_chains;
    a.block_start = c->d_block_start;
    a.n_chains = c->n_chains;
    a.lattice = c->d_lattice;
    a.series = c->d_series;
    a.state = c->d_state;
    a.cap = c->cap;
    a.tries = c->record_tries ? c->d_tries : nullptr;
    for (long long t = 0; t < n; ++t) {
        a.k = (uint32_t)t;
        const bool measure = every > 0 && ((t + 1) % every) == 0;
        for (const auto &g : c->groups) {
            a.block_base = c->block_start[g.first];
            const unsigned nb = c->block_start[g.second] - c->block_start[g.first];
            for (int mu = 0; mu < 4; ++mu)
                launch_phase<1>(c, a, mu, nb); // odd sites first (Sec. 2.4)
            for (int mu = 0; mu < 4; ++mu)
                launch_phase<0>(c, a, mu, nb);
            for (int r = 0; r < c->n_or; ++r) { // overrelaxation sweeps, same phase order
                for (int mu = 0; mu < 4; ++mu)
                    launch_or_phase<1>(c, a, mu, nb);
                for (int mu = 0; mu < 4; ++mu)
                    launch_or_phase<0>(c, a, mu, nb);
            }
            if (measure)
                plaquette_partials(c, g.first, g.second);
        }
        if (measure)
            plaquette_final(c, (uint32_t)t, (uint32_t)((t + 1) / every - 1), -1, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t su2_polyakov_launch(mc_ctx *c, int chain, DevRecord *out)
{
    const Su2Chain &ch = c->su2[chain];
    const uint32_t nspace = (uint32_t)ch.L[1] * ch.L[2] * ch.L[3];
    const unsigned nb = (nspace + 255) / 256;
    const float4 *U = reinterpret_cast<const float4 *>(c->d_lattice + ch.link_off);
    k_polyakov<<<nb, 256, 0, c->ls>>>(ch, U, c->d_partials);
    k_polyakov_final<<<1, 256, 0, c->ls>>>(c->d_partials, nb, nspace, out);
    return cudaGetLastError();
}

cudaError_t su2_measure_launch(mc_ctx *c, int chain, DevRecord *out)
{
    plaquette_partials(c, chain, chain + 1);
    plaquette_final(c, 0, 0, chain, out);
    return cudaGetLastError();
}

cudaError_t su2_config_io(mc_ctx *c, int chain, void *dev_buf, bool to_lattice)
{
    const Su2Chain &ch = c->su2[chain];
    k_su2_io<<<blocks_for((size_t)8 * ch.nh, 256), 256, 0, c->ls>>>(
        ch, reinterpret_cast<float4 *>(c->d_lattice + ch.link_off), static_cast<float4 *>(dev_buf), to_lattice);
    return cudaGetLastError();
}

}  // namespace mc
