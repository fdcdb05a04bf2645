// batch.cu -- many uneven chains (Ising in either layout, SU(2)) advanced by
// ONE persistent kernel launch per call, captured in a CUDA graph.
//
// A group borrows the chains of several contexts.  The host computes a
// schedule once (longest-processing-time first): the grid is a set of
// thread-block clusters of C CTAs, and each cluster walks a list of rounds.  A
// round is either
//   * shared: one large chain whose sites are split over the C CTAs of the
//     cluster; its half-sweeps / heat-bath phases are separated by the
//     hardware cluster barrier (no spin-waits), or
//   * a lane round: up to C small chains, one per CTA, each separated only by
//     __syncthreads; CTAs walk their lanes independently.
// Every chain runs all sweeps of the call inside its round, so the launch
// carries the whole call.  Lattices stay where their contexts keep them
// (global memory, L2-resident for batches that fit); the per-site work is the
// same device code as the grid-mode kernels (ising_dev.cuh, su2_dev.cuh), so
// results are bit-identical to those of the contexts' own sweeps.
#include <cooperative_groups.h>

#include <algorithm>
#include <numeric>
#include <string>

#include "ising_dev.cuh"
#include "su2_dev.cuh"

namespace cg = cooperative_groups;

struct mc_group;

namespace mc {
namespace {

constexpr int kMaxCluster = 16; // 16 is a non-portable cluster size (opted into at group creation)
constexpr int kMaxMembers = 16;

struct GroupMember {
    const void *chains;
    char *lattice;
    DevRecord *series;
    DevState *state;
    long long cap;
    int kind;
    int layout;
    int n_or; // SU(2): overrelaxation sweeps after each heat-bath sweep (from the context)
    int pad;
};

struct GroupArgs {
    const GroupMember *members;
    const int2 *items;           // {member, chain}
    const uint32_t *round_start; // per cluster, into `rounds` (n_clusters + 1 entries)
    const int32_t *rounds;       // [round][C] item per CTA rank, -1 = idle
    const uint8_t *round_shared; // per round: 1 = all ranks share the item
    long long *partials;         // [item][kMaxCluster][2] SU(2) plaquette partials (fixed point)
    int C;
    uint32_t n_sweeps, every;
};

// Lattice loads of the batch kernel: plain (L1-cacheable) loads.  A phase reads
// links or spins that other CTAs of the cluster (or other threads of the CTA)
// wrote in the previous phase; the barrier between the two -- the cluster
// barrier's arrive.release / wait.acquire, or __syncthreads in a lane round --
// orders those writes before every later load of the waiting threads, plain
// ones included.  Against loads through L2 only: 0.372 against 0.394 ms per
// sweep of the batched workload, identical records and configurations.
constexpr int kLdBatch = kLdPlain;

__device__ __forceinline__ void group_barrier(int G, cg::cluster_group &cluster)
{
    if (G > 1)
        cluster.sync(); // barrier.cluster arrive.release / wait.acquire: orders global memory too
    else
        __syncthreads();
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

template <int LAYOUT>
__device__ void run_ising(const GroupMember &m, int chain, int G, int rank, const GroupArgs &g,
                          cg::cluster_group &cluster)
{
    const IsingChain ch = static_cast<const IsingChain *>(m.chains)[chain];
    const PhiloxSchedule ks = philox_schedule(ch.key);
    const unsigned long long base = m.state->sweep_base;
    const uint32_t stride = (uint32_t)G * blockDim.x, start = (uint32_t)rank * blockDim.x + threadIdx.x;
    char *lat = m.lattice + ch.spin_off;
    const uint32_t units = LAYOUT == MC_LAYOUT_INT8 ? ((((ch.Lx * ch.Ly) >> 1) + 3) >> 2) : ch.W * (ch.Ly >> 1);
    const uint32_t nw = ch.W * ch.Ly;
    for (uint32_t t = 0; t < g.n_sweeps; ++t) {
        const uint32_t sweep = (uint32_t)(base + t);
        const bool measure = g.every != 0 && ((t + 1) % g.every) == 0;
        DevRecord *rec = nullptr;
        if (measure) {
            const unsigned long long r = m.state->rec_head + (t + 1) / g.every - 1;
            rec = &m.series[(long long)chain * m.cap + (long long)(r % (unsigned long long)m.cap)];
            if (rank == 0 && threadIdx.x == 0) { // zeroed before barrier 1, summed into after it
                rec->sweep = (long long)sweep;
                rec->a = rec->b = 0;
                rec->d0 = rec->d1 = rec->d2 = 0.0;
            }
        }
        uint32_t anti = 0, up = 0;
        if (LAYOUT == MC_LAYOUT_INT8) {
            int8_t *s = reinterpret_cast<int8_t *>(lat);
            for (uint32_t u = start; u < units; u += stride)
                int8_group<0, false, kLdBatch>(s, ch, ks, u, sweep, anti, up);
            group_barrier(G, cluster);
            if (measure)
                for (uint32_t u = start; u < units; u += stride)
                    int8_group<1, true, kLdBatch>(s, ch, ks, u, sweep, anti, up);
            else
                for (uint32_t u = start; u < units; u += stride)
                    int8_group<1, false, kLdBatch>(s, ch, ks, u, sweep, anti, up);
        } else {
            uint32_t *p0 = reinterpret_cast<uint32_t *>(lat), *p1 = p0 + nw;
            for (uint32_t u = start; u < units; u += stride) {
                const uint32_t yy = u / ch.W, w = u - yy * ch.W;
                msc_row_pair<0, false, kLdBatch>(p0, p1, yy, w, ch, ks, sweep, anti, up);
            }
            group_barrier(G, cluster);
            if (measure)
                for (uint32_t u = start; u < units; u += stride) {
                    const uint32_t yy = u / ch.W, w = u - yy * ch.W;
                    msc_row_pair<1, true, kLdBatch>(p1, p0, yy, w, ch, ks, sweep, anti, up);
                }
            else
                for (uint32_t u = start; u < units; u += stride) {
                    const uint32_t yy = u / ch.W, w = u - yy * ch.W;
                    msc_row_pair<1, false, kLdBatch>(p1, p0, yy, w, ch, ks, sweep, anti, up);
                }
        }
        if (measure) {
            block_sum2(anti, up);
            if (threadIdx.x == 0) {
                atomicAdd(&rec->a, (unsigned long long)anti);
                atomicAdd(&rec->b, (unsigned long long)up);
            }
        }
        group_barrier(G, cluster);
    }
}

// SU(2) measurement in the batch kernel: one x1 pair of sites per thread step
// (su2_pair_plaquettes, 29 link loads per pair) measured 0.451 against 0.459 ms
// per measured sweep of the batched workload for one site per step.
#ifndef MC_GROUP_PAIR_PLAQ
#define MC_GROUP_PAIR_PLAQ 1
#endif

__device__ void run_su2(const GroupMember &m, int chain, int item, int G, int rank, const GroupArgs &g,
                        cg::cluster_group &cluster)
{
    const Su2Chain ch = static_cast<const Su2Chain *>(m.chains)[chain];
    const PhiloxSchedule ks = philox_schedule(ch.key);
    float4 *U = reinterpret_cast<float4 *>(m.lattice + ch.link_off);
    const unsigned long long base = m.state->sweep_base;
    const uint32_t stride = (uint32_t)G * blockDim.x, start = (uint32_t)rank * blockDim.x + threadIdx.x;
    long long *part = g.partials + (size_t)item * kMaxCluster * 2;
    for (uint32_t t = 0; t < g.n_sweeps; ++t) {
        const uint32_t sweep = (uint32_t)(base + t);
        for (int phase = 0; phase < 8; ++phase) { // (odd, mu = 0..3), then (even, mu = 0..3)
            for (uint32_t e = start; e < ch.nh; e += stride)
                su2_update_link_rt<kLdBatch>(phase, U, ch, ks, e, sweep, m.state);
            group_barrier(G, cluster);
        }
        for (int r = 0; r < m.n_or; ++r) // overrelaxation sweeps, same phase order
            for (int phase = 0; phase < 8; ++phase) {
                for (uint32_t e = start; e < ch.nh; e += stride)
                    su2_overrelax_link_rt<kLdBatch>(phase, U, ch, e);
                group_barrier(G, cluster);
            }
        if (g.every != 0 && ((t + 1) % g.every) == 0) {
            long long ps = 0, pt = 0;
#if MC_GROUP_PAIR_PLAQ
            for (uint32_t j = start; j < ch.nh; j += stride) // one x1 pair of sites per step
                su2_pair_plaquettes<kLdBatch>(U, ch, j, ps, pt);
#else
            for (uint32_t s = start; s < 2 * ch.nh; s += stride)
                su2_site_plaquettes<kLdBatch>(U, ch, s, ps, pt);
#endif
            block_sum2ll(ps, pt);
            if (threadIdx.x == 0) {
                part[2 * rank] = ps;
                part[2 * rank + 1] = pt;
            }
            group_barrier(G, cluster);
            if (rank == 0 && threadIdx.x == 0) { // exact fixed-point sum: same value as the context kernels
                long long A = 0, B = 0;
                for (int r = 0; r < G; ++r) {
                    A += part[2 * r];
                    B += part[2 * r + 1];
                }
                const unsigned long long ri = m.state->rec_head + (t + 1) / g.every - 1;
                DevRecord *rec = &m.series[(long long)chain * m.cap + (long long)(ri % (unsigned long long)m.cap)];
                rec->sweep = (long long)sweep;
                rec->a = (unsigned long long)A; // the exact sums; P, P_s, P_t are formed on the host
                rec->b = (unsigned long long)B;
                rec->d0 = rec->d1 = rec->d2 = 0.0;
            }
        }
    }
}

// At least MC_GROUP_MIN_BLOCKS resident blocks of 256 threads per SM.  The
// default 2 (128 registers) measured best on the batched workload: 1.63e11
// updates/s, against 1.29e11 with 1 block, 1.33e11 with 3 (80 registers,
// spills) and 1.32e11 with 4 (64 registers, heavy spills).
#ifndef MC_GROUP_MIN_BLOCKS
#define MC_GROUP_MIN_BLOCKS 2
#endif
__global__ void __launch_bounds__(256, MC_GROUP_MIN_BLOCKS) k_group(GroupArgs g)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = g.C > 1 ? (int)cluster.block_rank() : 0;
    const int cid = (int)(blockIdx.x / (unsigned)g.C);
    for (uint32_t r = g.round_start[cid]; r < g.round_start[cid + 1]; ++r) {
        const int it = g.rounds[(size_t)r * g.C + rank];
        if (it < 0)
            continue; // idle lane (never inside a shared round)
        const int G = g.round_shared[r] ? g.C : 1;
        const int2 item = g.items[it];
        const GroupMember m = g.members[item.x];
        if (m.kind == MC_KIND_SU2)
            run_su2(m, item.y, it, G, G > 1 ? rank : 0, g, cluster);
        else if (m.layout == MC_LAYOUT_INT8)
            run_ising<MC_LAYOUT_INT8>(m, item.y, G, G > 1 ? rank : 0, g, cluster);
        else
            run_ising<MC_LAYOUT_MSC32>(m, item.y, G, G > 1 ? rank : 0, g, cluster);
    }
}

__global__ void k_group_advance(DevState *st, unsigned long long n, unsigned long long recs)
{
    st->sweep_base += n;
    st->rec_head += recs;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace mc

using namespace mc;

struct mc_group {
    std::vector<mc_ctx *> members;
    std::vector<int2> items;
    std::vector<double> cost;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    cudaEvent_t fence_in = nullptr, fence_out = nullptr;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    GroupMember *d_members = nullptr;
    int2 *d_items = nullptr;
    uint32_t *d_round_start = nullptr;
    int32_t *d_rounds = nullptr;
    uint8_t *d_round_shared = nullptr;
    long long *d_partials = nullptr;
    size_t max_rounds = 0, max_clusters = 0;
    // configuration and schedule
    int C = 4, threads = 256;
    double split_cost = -1.0; // items at least this costly are shared by a cluster (< 0: automatic)
    int n_clusters = 0;
    std::vector<uint32_t> round_start;
    std::vector<int32_t> rounds;
    std::vector<uint8_t> round_shared;
    bool planned = false;
    std::vector<GroupMember> hm; // host copy of d_members
    std::map<std::tuple<long long, int>, cudaGraphExec_t> graphs;
};

namespace {

mc_status gfail(mc_status s, const std::string &msg)
{
    mc::set_last_error(msg);
    return s;
}

// Relative cost of one sweep of a chain, in MSC spin-flip units.
double item_cost(const mc_ctx *c, int k)
{
    if (c->kind == MC_KIND_SU2) {
        const Su2Chain &ch = c->su2[k];
        return 60.0 * 8.0 * ch.nh * (1.0 + 0.6 * c->n_or); // 4 N heat-bath (+ cheaper overrelaxation) updates
    }
    const IsingChain &ch = c->ising[k];
    return (c->layout == MC_LAYOUT_INT8 ? 2.0 : 1.0) * ch.Lx * ch.Ly;
}

struct Layout {
    size_t members, items, round_start, rounds, round_shared, partials, total, max_rounds, max_clusters;
};

Layout group_layout(size_t n_members, size_t n_items)
{
    Layout L{};
    L.max_rounds = n_items + 1;
    L.max_clusters = 4096;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off = align256(off + std::max<size_t>(b, 1));
        return o;
    };
    L.members = take(n_members * sizeof(GroupMember));
    L.items = take(n_items * sizeof(int2));
    L.round_start = take((L.max_clusters + 1) * sizeof(uint32_t));
    L.rounds = take(L.max_rounds * kMaxCluster * sizeof(int32_t));
    L.round_shared = take(L.max_rounds);
    L.partials = take(n_items * kMaxCluster * 2 * sizeof(long long));
    L.total = off;
    return L;
}

void destroy_group_graphs(mc_group *g)
{
    for (auto &kv : g->graphs)
        cudaGraphExecDestroy(kv.second);
    g->graphs.clear();
}

// Longest-processing-time schedule of the items over n_clusters clusters of C CTAs.
mc_status plan(mc_group *g)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)g->C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(g->C * sms));
    cfg.blockDim = dim3((unsigned)g->threads);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int max_clusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&max_clusters, k_group, &cfg);
    if (e != cudaSuccess || max_clusters < 1)
        return gfail(MC_ECUDA, std::string("cluster occupancy query failed: ") + cudaGetErrorString(e));
    const size_t n = g->items.size();
    g->n_clusters = (int)std::min<size_t>({(size_t)max_clusters, g->max_clusters, std::max<size_t>(n, 1)});
    const int C = g->C, NC = g->n_clusters;
    double total = std::accumulate(g->cost.begin(), g->cost.end(), 0.0);
    double split = g->split_cost >= 0 ? g->split_cost : total / (double)(NC * C); // > one CTA's fair share
    if (C == 1)
        split = 1e300;
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return g->cost[a] > g->cost[b]; });
    std::vector<double> lane(NC * C, 0.0);
    std::vector<std::vector<int>> shared(NC);
    std::vector<std::vector<int>> lanes(NC * C);
    for (int it : order) {
        if (g->cost[it] >= split) { // cluster-wide: goes to the cluster whose busiest lane is least loaded
            int best = 0;
            double bl = 1e300;
            for (int c = 0; c < NC; ++c) {
                const double l = *std::max_element(lane.begin() + c * C, lane.begin() + (c + 1) * C);
                if (l < bl) {
                    bl = l;
                    best = c;
                }
            }
            shared[best].push_back(it);
            for (int r = 0; r < C; ++r)
                lane[best * C + r] = bl + g->cost[it] / C;
        } else {
            const int l = (int)(std::min_element(lane.begin(), lane.end()) - lane.begin());
            lanes[l].push_back(it);
            lane[l] += g->cost[it];
        }
    }
    g->round_start.assign(NC + 1, 0);
    g->rounds.clear();
    g->round_shared.clear();
    for (int c = 0; c < NC; ++c) {
        g->round_start[c] = (uint32_t)g->round_shared.size();
        for (int it : shared[c]) {
            for (int r = 0; r < C; ++r)
                g->rounds.push_back(it);
            g->round_shared.push_back(1);
        }
        size_t depth = 0;
        for (int r = 0; r < C; ++r)
            depth = std::max(depth, lanes[c * C + r].size());
        for (size_t d = 0; d < depth; ++d) {
            for (int r = 0; r < C; ++r)
                g->rounds.push_back(d < lanes[c * C + r].size() ? lanes[c * C + r][d] : -1);
            g->round_shared.push_back(0);
        }
    }
    g->round_start[NC] = (uint32_t)g->round_shared.size();
    if (g->round_shared.size() > g->max_rounds)
        return gfail(MC_ENOMEM, "group schedule exceeds its workspace");
    e = cudaMemcpyAsync(g->d_round_start, g->round_start.data(), g->round_start.size() * 4, cudaMemcpyHostToDevice,
                        g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->d_rounds, g->rounds.data(), g->rounds.size() * 4, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->d_round_shared, g->round_shared.data(), g->round_shared.size(), cudaMemcpyHostToDevice,
                            g->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess)
        return gfail(MC_ECUDA, std::string("upload group schedule: ") + cudaGetErrorString(e));
    g->planned = true;
    destroy_group_graphs(g);
    return MC_OK;
}

cudaError_t enqueue_group(mc_group *g, cudaStream_t s, long long n, int every)
{
    GroupArgs a{};
    a.members = g->d_members;
    a.items = g->d_items;
    a.round_start = g->d_round_start;
    a.rounds = g->d_rounds;
    a.round_shared = g->d_round_shared;
    a.partials = g->d_partials;
    a.C = g->C;
    a.n_sweeps = (uint32_t)n;
    a.every = (uint32_t)every;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)g->C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(g->n_clusters * g->C));
    cfg.blockDim = dim3((unsigned)g->threads);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_group, a);
    if (e != cudaSuccess)
        return e;
    const long long recs = every > 0 ? n / every : 0;
    for (mc_ctx *c : g->members)
        k_group_advance<<<1, 1, 0, s>>>(c->d_state, (unsigned long long)n, (unsigned long long)recs);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

size_t mc_group_workspace_bytes(int32_t n_ctx, mc_ctx *const *ctxs)
{
    if (n_ctx < 1 || n_ctx > kMaxMembers || !ctxs) {
        mc::set_last_error("n_ctx must be in [1, 16] and ctxs non-NULL");
        return 0;
    }
    size_t items = 0;
    for (int i = 0; i < n_ctx; ++i) {
        if (!ctxs[i]) {
            mc::set_last_error("NULL context");
            return 0;
        }
        items += (size_t)ctxs[i]->n_chains;
    }
    return group_layout((size_t)n_ctx, items).total;
}

mc_status mc_group_create(mc_group **out, int32_t n_ctx, mc_ctx *const *ctxs, void *workspace, size_t bytes,
                          void *cuda_stream)
{
    if (!out)
        return gfail(MC_EINVAL, "out is NULL");
    *out = nullptr;
    const size_t need = mc_group_workspace_bytes(n_ctx, ctxs);
    if (need == 0)
        return MC_EINVAL;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u))
        return gfail(MC_EINVAL, "workspace must be a device pointer aligned to 256 bytes");
    if (bytes < need)
        return gfail(MC_ENOMEM, "group workspace too small: need " + std::to_string(need) + " bytes");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    for (int i = 0; i < n_ctx; ++i)
        if (ctxs[i]->stream != st)
            return gfail(MC_EINVAL, "every member context must use the group's stream");
    mc_group *g = new (std::nothrow) mc_group();
    if (!g)
        return gfail(MC_ENOMEM, "host allocation of the group failed");
    g->members.assign(ctxs, ctxs + n_ctx);
    g->stream = st;
    g->ws = static_cast<char *>(workspace);
    g->ws_bytes = bytes;
    std::vector<GroupMember> hm;
    for (int i = 0; i < n_ctx; ++i) {
        const mc_ctx *c = ctxs[i];
        hm.push_back(GroupMember{c->d_chains, c->d_lattice, c->d_series, c->d_state, c->cap, c->kind, c->layout,
                                 c->n_or, 0});
        for (int k = 0; k < c->n_chains; ++k) {
            g->items.push_back(make_int2(i, k));
            g->cost.push_back(item_cost(c, k));
        }
    }
    const Layout L = group_layout(hm.size(), g->items.size());
    g->max_rounds = L.max_rounds;
    g->max_clusters = L.max_clusters;
    g->d_members = reinterpret_cast<GroupMember *>(g->ws + L.members);
    g->d_items = reinterpret_cast<int2 *>(g->ws + L.items);
    g->d_round_start = reinterpret_cast<uint32_t *>(g->ws + L.round_start);
    g->d_rounds = reinterpret_cast<int32_t *>(g->ws + L.rounds);
    g->d_round_shared = reinterpret_cast<uint8_t *>(g->ws + L.round_shared);
    g->d_partials = reinterpret_cast<long long *>(g->ws + L.partials);
    cudaError_t e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&g->fence_in, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&g->fence_out, cudaEventDisableTiming);
    if (e == cudaSuccess) // allow clusters of 16 CTAs
        e = cudaFuncSetAttribute(k_group, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    g->hm = hm;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->d_members, g->hm.data(), hm.size() * sizeof(GroupMember), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->d_items, g->items.data(), g->items.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        mc_group_destroy(g);
        return gfail(MC_ECUDA, std::string("create group: ") + cudaGetErrorString(e));
    }
    *out = g;
    return MC_OK;
}

mc_status mc_group_configure(mc_group *g, int32_t cluster_size, int32_t threads_per_block, double split_cost)
{
    if (!g)
        return gfail(MC_EINVAL, "group is NULL");
    if (cluster_size != 0 && cluster_size != 1 && cluster_size != 2 && cluster_size != 4 && cluster_size != 8 &&
        cluster_size != 16)
        return gfail(MC_EINVAL, "cluster_size must be 1, 2, 4, 8 or 16");
    if (threads_per_block != 0 && (threads_per_block < 64 || threads_per_block > 256 || threads_per_block % 32))
        return gfail(MC_EINVAL, "threads_per_block must be a multiple of 32 in [64, 256]");
    if (cluster_size)
        g->C = cluster_size;
    if (threads_per_block)
        g->threads = threads_per_block;
    g->split_cost = split_cost;
    g->planned = false;
    destroy_group_graphs(g);
    return MC_OK;
}

mc_status mc_group_sweep(mc_group *g, int64_t n_sweeps, int32_t measure_every)
{
    if (!g)
        return gfail(MC_EINVAL, "group is NULL");
    if (n_sweeps < 0 || measure_every < 0)
        return gfail(MC_EINVAL, "n_sweeps and measure_every must be >= 0");
    if (n_sweeps == 0)
        return MC_OK;
    const long long recs = measure_every > 0 ? n_sweeps / measure_every : 0;
    for (mc_ctx *c : g->members) {
        if ((c->rec_written - c->rec_read) + recs > c->cap)
            return gfail(MC_EINVAL, "a member's measurement ring buffer would overflow");
        if (c->sweeps_done + n_sweeps > 0xFFFFFFFFll)
            return gfail(MC_EINVAL, "sweep counter would exceed 2^32");
    }
    bool or_changed = false; // a member context changed its overrelaxation count since the last call
    for (size_t i = 0; i < g->members.size(); ++i)
        if (g->hm[i].n_or != g->members[i]->n_or) {
            g->hm[i].n_or = g->members[i]->n_or;
            or_changed = true;
        }
    if (or_changed) {
        cudaError_t e = cudaMemcpyAsync(g->d_members, g->hm.data(), g->hm.size() * sizeof(GroupMember),
                                        cudaMemcpyHostToDevice, g->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess)
            return gfail(MC_ECUDA, std::string("update group members: ") + cudaGetErrorString(e));
        g->planned = false;
        destroy_group_graphs(g);
    }
    if (!g->planned) {
        mc_status s = plan(g);
        if (s != MC_OK)
            return s;
    }
    const auto key = std::make_tuple((long long)n_sweeps, (int)measure_every);
    auto it = g->graphs.find(key);
    if (it == g->graphs.end()) {
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess)
            return gfail(MC_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
        cudaError_t ek = enqueue_group(g, g->cap_stream, n_sweeps, measure_every);
        e = cudaStreamEndCapture(g->cap_stream, &gr);
        if (ek != cudaSuccess || e != cudaSuccess) {
            if (gr)
                cudaGraphDestroy(gr);
            return gfail(MC_ECUDA, std::string("capture group sweep: ") + cudaGetErrorString(ek != cudaSuccess ? ek : e));
        }
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess)
            return gfail(MC_ECUDA, std::string("instantiate group graph: ") + cudaGetErrorString(e));
        it = g->graphs.emplace(key, ge).first;
    }
    cudaError_t e = cudaEventRecord(g->fence_in, g->stream);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(g->cap_stream, g->fence_in, 0);
    if (e == cudaSuccess)
        e = cudaGraphLaunch(it->second, g->cap_stream);
    if (e == cudaSuccess)
        e = cudaEventRecord(g->fence_out, g->cap_stream);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(g->stream, g->fence_out, 0);
    if (e != cudaSuccess)
        return gfail(MC_ECUDA, std::string("group graph launch: ") + cudaGetErrorString(e));
    for (mc_ctx *c : g->members) {
        c->sweeps_done += n_sweeps;
        c->rec_written += recs;
    }
    return MC_OK;
}

mc_status mc_group_schedule(const mc_group *g, int32_t *n_clusters, int32_t *n_rounds)
{
    if (!g || !n_clusters || !n_rounds)
        return gfail(MC_EINVAL, "NULL argument");
    *n_clusters = g->planned ? g->n_clusters : 0;
    *n_rounds = g->planned ? (int32_t)g->round_shared.size() : 0;
    return MC_OK;
}

mc_status mc_group_destroy(mc_group *g)
{
    if (!g)
        return MC_OK;
    cudaError_t e = cudaStreamSynchronize(g->stream);
    destroy_group_graphs(g);
    if (g->fence_in)
        cudaEventDestroy(g->fence_in);
    if (g->fence_out)
        cudaEventDestroy(g->fence_out);
    if (g->cap_stream)
        cudaStreamDestroy(g->cap_stream);
    delete g;
    if (e != cudaSuccess)
        return gfail(MC_ECUDA, std::string("stream synchronize: ") + cudaGetErrorString(e));
    return MC_OK;
}

}  // extern "C"
