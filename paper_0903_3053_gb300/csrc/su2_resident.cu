// su2_resident.cu -- SU(2) heat-bath for small lattices in ONE launch per call
// (the SU(2) counterpart of the Ising resident mode; Sec. 2.4 phase order,
// Eqs. (5)-(7)).
//
// On a small lattice (the 4 x 8^3 .. 8 x 8^3 lattices of Table 1, the 8^4
// workload) a phase has only ~1-2 thousand links: a grid-mode sweep is ten
// graph-replayed launches each lasting one link update's latency, and within a
// phase the slowest link -- the one whose Kennedy-Pendleton draw needs the
// most tries -- sets the time.  Here one thread-block cluster of C CTAs
// (C <= 16) owns one chain for the whole call: every phase of every sweep,
// the overrelaxation sweeps and the plaquette measurement run inside the
// launch, separated by the hardware cluster barrier (no spin-waits).  A phase
// is computed in passes of 128 links per CTA, each pass in two stages with
// roles assigned per warp, so that no warp diverges:
//   stage 1 (all 32 warps, one link per lane)
//     warps  0-11  the three staple pairs of Eq. (6) (nu != mu, in nu order),
//     warps 12-15  the direction on S^2,
//     warps 16-31  the alpha-free parts of Kennedy-Pendleton tries 0-7, two
//                  per lane (a counter-based stream lets later tries be drawn
//                  before earlier ones are rejected: at beta = 1.5 one link in
//                  ~2000 needs a fourth try, and a phase waits for its slowest
//                  link);
//   stage 2 (warps 0-3)  W = sum of the pairs, V and alpha, the first accepted
//                  of tries 0-7 (the rare link that rejects all eight continues
//                  sequentially with the Creutz tries 8..71), X V,
//                  reprojection, store.
// The arithmetic is the grid kernel's, function for function (su2_dev.cuh),
// with the staple summed in the same order, so the links are bit-identical to
// a grid-mode sweep.  The plaquette measurement gives each thread single
// plaquettes (four link loads, two plaquettes' loads issued together) rather
// than a site pair (29 loads in a dependent chain); the fixed-point sums are
// exact, so the records equal the grid kernels' too.
#include <cooperative_groups.h>

#include <algorithm>

#include "su2_dev.cuh"

namespace cg = cooperative_groups;

namespace mc {
namespace {

constexpr int kResThreads = 1024;
constexpr int kResLinks = 128; // links per CTA pass (4 warps)
constexpr int kResSpec = 8;    // Kennedy-Pendleton tries drawn at once (two per lane of warps 16-31)

struct ResidentArgs {
    const Su2Chain *chains;
    char *lattice;
    DevRecord *series;
    DevState *state;
    long long cap;
    uint32_t n_sweeps, every;
    int n_or;
};

struct ResidentStage {
    float4 pair[3][kResLinks];
    S2Direction dir[2][kResLinks];        // double buffered: this pass, next pass
    KpFirstTry kp[2][kResSpec][kResLinks];
    long long red[2 * kSu2ResidentMaxCluster]; // rank 0: the plaquette partials of the cluster
};

__device__ __forceinline__ void cluster_barrier(int C, cg::cluster_group &cluster)
{
    if (C > 1)
        cluster.sync(); // arrive.release / wait.acquire at cluster scope: orders global and shared memory
    else
        __syncthreads();
}

// Barrier 1: the 12 staple warps only (stage 2 needs their pairs, not the
// random-number warps, which may still be drawing the next pass's numbers).
__device__ __forceinline__ void staple_warps_barrier()
{
    asm volatile("bar.sync 1, 384;" ::: "memory");
}

// The r-th staple pair (nu = r-th direction other than MU) of the link at
// parity index e.
template <int P, int MU>
__device__ __forceinline__ float4 staple_pair_nth(const float4 *U, const Su2Chain &ch, uint32_t e, int r)
{
    const Site x = site_from_parity_index(ch, P, e);
    const uint32_t s = canonical(ch, x);
    const Strides g = strides_of(ch);
    const uint32_t spm = fwd<MU>(ch, g, x.x[MU], s);
    constexpr int N0 = MU == 0 ? 1 : 0, N1 = MU <= 1 ? 2 : 1, N2 = MU <= 2 ? 3 : 2;
    if (r == 0)
        return staple_pair<MU, N0, P, kLdCoherent>(U, ch, g, x, s, spm, e);
    if (r == 1)
        return staple_pair<MU, N1, P, kLdCoherent>(U, ch, g, x, s, spm, e);
    return staple_pair<MU, N2, P, kLdCoherent>(U, ch, g, x, s, spm, e);
}

// Random numbers of one pass (phase (P, MU), links e0 .. e0 + 127, sweep) into
// buffer b, by warps 12-31: the direction on S^2 (warps 12-15) and the
// alpha-free parts of Kennedy-Pendleton tries 0-7 (warps 16-31, two tries per
// lane).  They depend on no link, so they are drawn one pass ahead.
template <int P, int MU>
__device__ __forceinline__ void pass_randoms(const Su2Chain &ch, const PhiloxSchedule &ks, uint32_t e0, uint32_t sweep,
                                             ResidentStage &st, int b)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sel = ((uint32_t)P << 12) | ((uint32_t)MU << 8);
    if (warp < 16) {
        const int l = (warp - 12) * 32 + lane;
        const uint32_t e = e0 + l;
        if (e < ch.nh)
            st.dir[b][l] = su2_direction<P, MU>(ch, ks, e, sweep);
    } else {
        const int t = (warp - 16) >> 2, l = (warp & 3) * 32 + lane;
        const uint32_t e = e0 + l;
        if (e < ch.nh) {
            st.kp[b][t][l] = kp_first_try(e, sweep, sel | (uint32_t)t, ch, ks);
            st.kp[b][t + 4][l] = kp_first_try(e, sweep, sel | (uint32_t)(t + 4), ch, ks);
        }
    }
}

__device__ __forceinline__ void pass_randoms_rt(int phase, const Su2Chain &ch, const PhiloxSchedule &ks, uint32_t e0,
                                                uint32_t sweep, ResidentStage &st, int b)
{
    switch (phase) { // (odd, mu = 0..3), then (even, mu = 0..3)
    case 0: pass_randoms<1, 0>(ch, ks, e0, sweep, st, b); break;
    case 1: pass_randoms<1, 1>(ch, ks, e0, sweep, st, b); break;
    case 2: pass_randoms<1, 2>(ch, ks, e0, sweep, st, b); break;
    case 3: pass_randoms<1, 3>(ch, ks, e0, sweep, st, b); break;
    case 4: pass_randoms<0, 0>(ch, ks, e0, sweep, st, b); break;
    case 5: pass_randoms<0, 1>(ch, ks, e0, sweep, st, b); break;
    case 6: pass_randoms<0, 2>(ch, ks, e0, sweep, st, b); break;
    default: pass_randoms<0, 3>(ch, ks, e0, sweep, st, b); break;
    }
}

// The link updates of one pass (phase (P, MU), links e0 .. e0 + 127) whose
// random numbers are in buffer b: warps 0-11 the staple pairs, then warps 0-3
// the heat-bath draw and the store.  Warps 12-31 meanwhile draw the next
// pass's random numbers (phase nphase at nsweep, links ne0, into buffer 1 - b;
// nphase < 0: none).  Ends with the whole CTA synchronised.
template <int P, int MU>
__device__ __forceinline__ void resident_pass(float4 *U, const Su2Chain &ch, const PhiloxSchedule &ks, uint32_t e0,
                                              uint32_t sweep, DevState *state, ResidentStage &st, int b, int nphase,
                                              uint32_t ne0, uint32_t nsweep)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sel = ((uint32_t)P << 12) | ((uint32_t)MU << 8);
    if (warp < 12) {
        const int l = (warp & 3) * 32 + lane;
        const uint32_t e = e0 + l;
        if (e < ch.nh)
            st.pair[warp >> 2][l] = staple_pair_nth<P, MU>(U, ch, e, warp >> 2);
        staple_warps_barrier();
        if (warp < 4 && e < ch.nh) {
            // the grid kernel's staple: 0 + pair(nu_0) + pair(nu_1) + pair(nu_2), in that order
            float4 W = make_float4(0.f, 0.f, 0.f, 0.f);
            W = qadd(W, st.pair[0][l]);
            W = qadd(W, st.pair[1][l]);
            W = qadd(W, st.pair[2][l]);
            float4 V;
            float alpha;
            staple_to_heatbath(W, ch.beta, V, alpha);
            int t = kFailed;
            float a0 = 0.f;
            if (alpha > 0.f)
                for (int k = 0; k < kResSpec; ++k) {
                    float a;
                    if (kp_accept(st.kp[b][k][l], alpha, a)) {
                        a0 = a;
                        t = k;
                        break;
                    }
                }
            if (t == kFailed) // the same draws draw_a0 takes after the first kResSpec
                for (int k = alpha > 0.f ? kResSpec : kKpTries; k < kKpTries + kCreutzTries; ++k) {
                    float a;
                    if (heatbath_try(k, alpha, e, sweep, sel, ch, ks, a)) {
                        a0 = a;
                        t = k;
                        break;
                    }
                }
            if (t == kFailed)
                atomicAdd(&state->hb_failures, 1ull);
            else
                U[(size_t)(P * 4 + MU) * ch.nh + e] = heatbath_link(a0, V, st.dir[b][l]);
        }
    } else if (nphase >= 0) {
        pass_randoms_rt(nphase, ch, ks, ne0, nsweep, st, 1 - b);
    }
    __syncthreads();
}

__device__ __forceinline__ void resident_pass_rt(int phase, float4 *U, const Su2Chain &ch, const PhiloxSchedule &ks,
                                                 uint32_t e0, uint32_t sweep, DevState *state, ResidentStage &st,
                                                 int b, int nphase, uint32_t ne0, uint32_t nsweep)
{
    switch (phase) {
    case 0: resident_pass<1, 0>(U, ch, ks, e0, sweep, state, st, b, nphase, ne0, nsweep); break;
    case 1: resident_pass<1, 1>(U, ch, ks, e0, sweep, state, st, b, nphase, ne0, nsweep); break;
    case 2: resident_pass<1, 2>(U, ch, ks, e0, sweep, state, st, b, nphase, ne0, nsweep); break;
    case 3: resident_pass<1, 3>(U, ch, ks, e0, sweep, state, st, b, nphase, ne0, nsweep); break;
    case 4: resident_pass<0, 0>(U, ch, ks, e0, sweep, state, st, b, nphase, ne0, nsweep); break;
    case 5: resident_pass<0, 1>(U, ch, ks, e0, sweep, state, st, b, nphase, ne0, nsweep); break;
    case 6: resident_pass<0, 2>(U, ch, ks, e0, sweep, state, st, b, nphase, ne0, nsweep); break;
    default: resident_pass<0, 3>(U, ch, ks, e0, sweep, state, st, b, nphase, ne0, nsweep); break;
    }
}

// The four links of plaquette unit u (u = plane N + s, as su2_plaquette_unit),
// in the order plaquette_value takes them; temporal: the plane contains mu = 0.
template <int MU, int NU>
__device__ __forceinline__ void plane_links(const float4 *U, const Su2Chain &ch, const Site &x, uint32_t s,
                                            float4 (&q)[4])
{
    const int p = (x.x[0] + x.x[1] + x.x[2] + x.x[3]) & 1;
    const uint32_t nh = ch.nh, e = s >> 1;
    q[0] = load_link<kLdCoherent>(U, nh, p, MU, e);
    q[1] = load_link<kLdCoherent>(U, nh, 1 - p, NU, canonical_fwd<MU>(ch, x, s) >> 1);
    q[2] = load_link<kLdCoherent>(U, nh, p, NU, e);
    q[3] = load_link<kLdCoherent>(U, nh, 1 - p, MU, canonical_fwd<NU>(ch, x, s) >> 1);
}
__device__ __forceinline__ bool unit_links(const float4 *U, const Su2Chain &ch, uint32_t u, float4 (&q)[4])
{
    const uint32_t n = 2u * ch.nh, plane = u / n, s = u - plane * n;
    const Site x = site_of_canonical(ch, s);
    switch (plane) {
    case 0: plane_links<0, 1>(U, ch, x, s, q); break;
    case 1: plane_links<0, 2>(U, ch, x, s, q); break;
    case 2: plane_links<0, 3>(U, ch, x, s, q); break;
    case 3: plane_links<1, 2>(U, ch, x, s, q); break;
    case 4: plane_links<1, 3>(U, ch, x, s, q); break;
    default: plane_links<2, 3>(U, ch, x, s, q); break;
    }
    return plane < 3;
}

__device__ __forceinline__ void block_sum2ll(long long &a, long long &b)
{
    __shared__ long long sa[32], sb[32];
    a = warp_sum_ll(a);
    b = warp_sum_ll(b);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long ta = 0, tb = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            ta += sa[i];
            tb += sb[i];
        }
        a = ta;
        b = tb;
    }
    __syncthreads();
}

// One cluster of C CTAs per chain (chain = cluster index); all n_sweeps of
// the call, with the overrelaxation sweeps and the measurements.  A sweep is
// 8 phases x np passes per CTA (pass k of phase f: links rank * 128 +
// k * C * 128); pass i's random numbers are in buffer i & 1, drawn during pass
// i - 1 (the first before the loop).
__global__ void __launch_bounds__(kResThreads, 1) k_su2_resident(ResidentArgs a, int C)
{
    __shared__ ResidentStage st;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = C > 1 ? (int)cluster.block_rank() : 0;
    const int chain = (int)(blockIdx.x / (unsigned)C);
    const Su2Chain ch = a.chains[chain];
    const PhiloxSchedule ks = philox_schedule(ch.key);
    float4 *U = reinterpret_cast<float4 *>(a.lattice + ch.link_off);
    const unsigned long long base = a.state->sweep_base;
    const uint32_t stride = (uint32_t)C * kResThreads, start = (uint32_t)rank * kResThreads + threadIdx.x;
    const uint32_t first = (uint32_t)rank * kResLinks, step = (uint32_t)C * kResLinks;
    const int np = first < ch.nh ? (int)((ch.nh - first + step - 1) / step) : 0; // passes per phase
    const int units = 8 * np;
    if (np > 0 && (threadIdx.x >> 5) >= 12)
        pass_randoms_rt(0, ch, ks, first, (uint32_t)base, st, 0);
    __syncthreads();
    int buf = 0;
    for (uint32_t t = 0; t < a.n_sweeps; ++t) {
        const uint32_t sweep = (uint32_t)(base + t);
        for (int f = 0; f < 8; ++f) {
            for (int k = 0; k < np; ++k) {
                const int i = f * np + k;
                int nphase = -1;
                uint32_t ne0 = 0, nsweep = sweep;
                if (i + 1 < units) {
                    nphase = (i + 1) / np;
                    ne0 = first + (uint32_t)((i + 1) % np) * step;
                } else if (t + 1 < a.n_sweeps) {
                    nphase = 0;
                    ne0 = first;
                    nsweep = sweep + 1;
                }
                resident_pass_rt(f, U, ch, ks, first + (uint32_t)k * step, sweep, a.state, st, buf, nphase, ne0,
                                 nsweep);
                buf ^= 1;
            }
            cluster_barrier(C, cluster);
        }
        for (int r = 0; r < a.n_or; ++r) // overrelaxation sweeps, same phase order
            for (int phase = 0; phase < 8; ++phase) {
                for (uint32_t e = start; e < ch.nh; e += stride)
                    su2_overrelax_link_rt<kLdCoherent>(phase, U, ch, e);
                cluster_barrier(C, cluster);
            }
        if (a.every != 0 && ((t + 1) % a.every) == 0) {
            // two plaquettes per thread step, the loads of both issued before either product
            long long ps = 0, pt = 0;
            const uint32_t units = 12u * ch.nh;
            for (uint32_t u = start; u < units; u += 2 * stride) {
                float4 qa[4], qb[4];
                const bool ta = unit_links(U, ch, u, qa);
                const bool two = u + stride < units;
                bool tb = false;
                if (two)
                    tb = unit_links(U, ch, u + stride, qb);
                const long long ha = plaq_fixed(plaquette_value(qa[0], qa[1], qa[2], qa[3]));
                (ta ? pt : ps) += ha;
                if (two) {
                    const long long hb = plaq_fixed(plaquette_value(qb[0], qb[1], qb[2], qb[3]));
                    (tb ? pt : ps) += hb;
                }
            }
            block_sum2ll(ps, pt);
            if (threadIdx.x == 0) { // into rank 0's shared memory
                long long *red = C > 1 ? cluster.map_shared_rank(st.red, 0) : st.red;
                red[2 * rank] = ps;
                red[2 * rank + 1] = pt;
            }
            cluster_barrier(C, cluster);
            // exact fixed-point sum, the grid kernels' value, by the last thread of rank 0: a warp that
            // draws random numbers one pass ahead, not one of the heat-bath warps of the next pass
            if (rank == 0 && threadIdx.x == kResThreads - 1) {
                long long A = 0, B = 0;
                for (int r = 0; r < C; ++r) {
                    A += st.red[2 * r];
                    B += st.red[2 * r + 1];
                }
                const unsigned long long ri = a.state->rec_head + (t + 1) / a.every - 1;
                DevRecord *rec = &a.series[(long long)chain * a.cap + (long long)(ri % (unsigned long long)a.cap)];
                rec->sweep = (long long)sweep;
                rec->a = (unsigned long long)A; // the exact sums; P, P_s, P_t are formed on the host
                rec->b = (unsigned long long)B;
                rec->d0 = rec->d1 = rec->d2 = 0.0;
            }
        }
    }
    // rank 0's partials are read above before any CTA can write the next ones:
    // at least eight cluster barriers separate two measurements.
}

// CTAs per chain: enough for one pass per phase, a power of two <= 16.
int resident_cluster(const mc_ctx *c)
{
    uint32_t nh = 0;
    for (const auto &ch : c->su2)
        nh = std::max(nh, ch.nh);
    int C = 1;
    while (C < kSu2ResidentMaxCluster && (uint32_t)C * kResLinks < nh)
        C *= 2;
    return C;
}

}  // namespace

// Automatic choice: one pass per phase (<= 2048 links per phase and chain:
// 8^4 and the 4 x 8^3, 8 x 8^3 lattices of Table 1; measured 1.2-1.35x faster
// than the grid launches there, and slower from two passes on) and no
// per-link try record.
bool su2_resident_auto(const mc_ctx *c)
{
    if (c->kind != MC_KIND_SU2 || c->record_tries)
        return false;
    for (const auto &ch : c->su2)
        if (ch.nh > (uint32_t)kSu2ResidentMaxCluster * kResLinks)
            return false;
    return true;
}

// Cluster size for this context: the smallest power of two giving one pass
// per phase (at most 16), lowered until the device can place such a cluster of
// 1024-thread CTAs.
cudaError_t su2_prepare_resident(mc_ctx *c)
{
    cudaError_t e = cudaFuncSetAttribute(k_su2_resident, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess)
        return e;
    for (int C = resident_cluster(c); C >= 1; C /= 2) {
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)C);
        cfg.blockDim = dim3(kResThreads);
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, k_su2_resident, &cfg);
        if (e != cudaSuccess)
            return e;
        if (n >= 1) {
            c->su2_res_cluster = C;
            return cudaSuccess;
        }
    }
    return cudaErrorLaunchOutOfResources;
}

cudaError_t su2_resident_enqueue(mc_ctx *c, long long n, int every)
{
    ResidentArgs a{};
    a.chains = static_cast<const Su2Chain *>(c->d_chains);
    a.lattice = c->d_lattice;
    a.series = c->d_series;
    a.state = c->d_state;
    a.cap = c->cap;
    a.n_sweeps = (uint32_t)n;
    a.every = (uint32_t)std::max(every, 0);
    a.n_or = c->n_or;
    const int C = c->su2_res_cluster > 0 ? c->su2_res_cluster : 1;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(c->n_chains * C));
    cfg.blockDim = dim3(kResThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = c->ls;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = prof_begin(c);
    if (e != cudaSuccess)
        return e;
    e = cudaLaunchKernelEx(&cfg, k_su2_resident, a, C);
    if (e != cudaSuccess)
        return e;
    return prof_end(c);
}

}  // namespace mc
