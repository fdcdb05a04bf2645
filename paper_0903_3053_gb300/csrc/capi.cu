// capi.cu -- the extern "C" boundary of libmc.so (declared in include/mc.h).
//
// Host-side bookkeeping only: argument validation, carving the caller's device
// workspace, CUDA-graph capture and replay of sweep sequences, the measurement
// ring buffer and configuration I/O.  Every step of the sweep itself runs in
// the kernels of ising.cu and su2.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "mc_internal.cuh"

using namespace mc;

namespace {

thread_local std::string g_err;

mc_status fail(mc_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

mc_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(MC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Metropolis thresholds T = floor(e^{-beta dE} 2^32), clamped to 2^32 - 1, for
// dE = 4 and 8 (the only positive energy changes of a single flip in 2D).
void thresholds(double beta, uint32_t &t2, uint32_t &t4)
{
    const double d[2] = {4.0, 8.0};
    uint32_t out[2];
    for (int i = 0; i < 2; ++i) {
        const double t = std::exp(-beta * d[i]) * 4294967296.0;
        out[i] = t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)std::floor(t);
    }
    t2 = out[0];
    t4 = out[1];
}

bool validate(int32_t n, const mc_chain_desc *chains, int32_t layout, int64_t cap, std::string &why)
{
    if (n < 1 || n > kMaxChains) {
        why = "n_chains must be in [1, " + std::to_string(kMaxChains) + "]";
        return false;
    }
    if (!chains) {
        why = "chains is NULL";
        return false;
    }
    if (cap < 1 || cap > (1ll << 32)) {
        why = "series_capacity must be in [1, 2^32]";
        return false;
    }
    const int kind = chains[0].kind;
    if (kind != MC_KIND_ISING && kind != MC_KIND_SU2) {
        why = "unknown chain kind";
        return false;
    }
    if (kind == MC_KIND_ISING && layout != MC_LAYOUT_INT8 && layout != MC_LAYOUT_MSC32) {
        why = "unknown Ising layout";
        return false;
    }
    for (int k = 0; k < n; ++k) {
        const mc_chain_desc &d = chains[k];
        const std::string tag = "chain " + std::to_string(k) + ": ";
        if (d.kind != kind) {
            why = tag + "all chains of a batch must be of one kind";
            return false;
        }
        if (!(d.beta >= 0.0) || !std::isfinite(d.beta)) {
            why = tag + "beta must be finite and >= 0";
            return false;
        }
        if (d.start != MC_COLD && d.start != MC_HOT) {
            why = tag + "start must be MC_COLD or MC_HOT";
            return false;
        }
        const int nd = kind == MC_KIND_ISING ? 2 : 4;
        double sites = 1.0;
        for (int m = 0; m < nd; ++m) {
            if (d.L[m] < 2 || (d.L[m] & 1)) {
                why = tag + "every extent must be even and >= 2 (checkerboard)";
                return false;
            }
            sites *= d.L[m];
        }
        if (kind == MC_KIND_ISING) {
            if (sites > 2147483648.0) { // colour index and 4 * group must fit in 32 bits
                why = tag + "Lx*Ly must be <= 2^31";
                return false;
            }
            if (layout == MC_LAYOUT_MSC32 && (d.L[0] % 64) != 0) {
                why = tag + "MC_LAYOUT_MSC32 needs Lx % 64 == 0";
                return false;
            }
        } else {
            if (sites * 4.0 > 1073741824.0) { // link index 4 s + mu in 32 bits, with margin
                why = tag + "number of links must be <= 2^30";
                return false;
            }
            if (!(d.beta < 1e30)) {
                why = tag + "beta too large";
                return false;
            }
        }
    }
    return true;
}

struct Plan {
    size_t state, chains, block_start, meas_start, series, scratch_rec, partials, staging, tries, lattice, total;
    size_t partial_count, staging_bytes;
    std::vector<size_t> lat_off, tries_off;
};

size_t ising_storage(const mc_chain_desc &d, int layout)
{
    const size_t n = (size_t)d.L[0] * d.L[1];
    return layout == MC_LAYOUT_INT8 ? n : n / 8;
}

Plan make_plan(int32_t n, const mc_chain_desc *chains, int32_t layout, int64_t cap)
{
    Plan p{};
    const int kind = chains[0].kind;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + std::max<size_t>(bytes, 1));
        return o;
    };
    p.state = take(sizeof(DevState));
    p.chains = take((size_t)n * (kind == MC_KIND_ISING ? sizeof(IsingChain) : sizeof(Su2Chain)));
    p.block_start = take((size_t)(n + 1) * sizeof(uint32_t));
    p.meas_start = take((size_t)(n + 1) * sizeof(uint32_t));
    p.series = take((size_t)n * (size_t)cap * sizeof(DevRecord));
    p.scratch_rec = take((size_t)n * sizeof(DevRecord));
    size_t staging = 0, meas_blocks = 0;
    for (int k = 0; k < n; ++k) {
        const mc_chain_desc &d = chains[k];
        if (kind == MC_KIND_ISING) {
            staging = std::max(staging, (size_t)d.L[0] * d.L[1]);
        } else {
            const size_t sites = (size_t)d.L[0] * d.L[1] * d.L[2] * d.L[3];
            staging = std::max(staging, sites * 4 * 16);
            // >= kSu2ResidentMaxCluster blocks: the resident mode keeps one partial pair per CTA of a chain
            meas_blocks += std::max<size_t>((sites / 2 + kPlaqThreads - 1) / kPlaqThreads, kSu2ResidentMaxCluster);
        }
    }
    p.partial_count = 2 * meas_blocks;
    p.partials = take(p.partial_count * sizeof(long long));
    p.staging_bytes = staging;
    p.staging = take(staging);
    p.tries_off.assign(n, 0);
    size_t tries_total = 0;
    if (kind == MC_KIND_SU2)
        for (int k = 0; k < n; ++k) {
            p.tries_off[k] = tries_total;
            tries_total += align_up((size_t)4 * chains[k].L[0] * chains[k].L[1] * chains[k].L[2] * chains[k].L[3]);
        }
    p.tries = take(tries_total);
    p.lat_off.assign(n, 0);
    size_t lat = 0;
    for (int k = 0; k < n; ++k) {
        p.lat_off[k] = lat;
        const mc_chain_desc &d = chains[k];
        const size_t bytes = kind == MC_KIND_ISING ? ising_storage(d, layout)
                                                   : (size_t)d.L[0] * d.L[1] * d.L[2] * d.L[3] * 4 * 16;
        lat += align_up(bytes);
    }
    p.lattice = take(lat);
    p.total = off;
    return p;
}

mc_status check_device(mc_ctx *c)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "stream synchronize");
    DevState st;
    e = cudaMemcpy(&st, c->d_state, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(e, "read device state");
    if (st.err_code != 0) {
        char buf[160];
        snprintf(buf, sizeof buf, "device fault latched: code %d info %d", st.err_code, st.err_info);
        return fail(st.err_code == kErrTimeout ? MC_ETIMEOUT : MC_EDEVICE, buf);
    }
    return MC_OK;
}

void destroy_graphs(mc_ctx *c)
{
    for (auto &kv : c->graphs)
        cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
}

void free_ctx(mc_ctx *c)
{
    destroy_graphs(c);
    for (cudaEvent_t ev : c->events)
        cudaEventDestroy(ev);
    if (c->fence_in)
        cudaEventDestroy(c->fence_in);
    if (c->fence_out)
        cudaEventDestroy(c->fence_out);
    if (c->cap_stream)
        cudaStreamDestroy(c->cap_stream);
    delete c;
}

int resolve_mode(mc_ctx *c)
{
    if (c->kind == MC_KIND_SU2) {
        if (c->record_tries) // the per-link try record is kept by the grid kernels only
            return MC_MODE_GRID;
        if (c->mode != MC_MODE_AUTO)
            return c->mode;
        return su2_resident_auto(c) ? MC_MODE_RESIDENT : MC_MODE_GRID;
    }
    if (c->mode != MC_MODE_AUTO)
        return c->mode;
    int smem = 0;
    if (!ising_resident_fits(c, &smem))
        return MC_MODE_GRID;
    uint64_t max_sites = 0;
    for (const auto &ch : c->ising)
        max_sites = std::max<uint64_t>(max_sites, (uint64_t)ch.Lx * ch.Ly);
    // small lattices: launch latency dominates a grid-mode sweep
    return max_sites <= 65536 ? MC_MODE_RESIDENT : MC_MODE_GRID;
}

mc_status upload_tables(mc_ctx *c)
{
    if (c->kind == MC_KIND_ISING)
        ising_plan_grid(c);
    else
        su2_plan_grid(c);
    cudaError_t e = cudaMemcpyAsync(c->d_block_start, c->block_start.data(), c->block_start.size() * 4,
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !c->meas_start.empty())
        e = cudaMemcpyAsync(c->d_meas_start, c->meas_start.data(), c->meas_start.size() * 4, cudaMemcpyHostToDevice,
                            c->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "upload block tables");
    e = cudaStreamSynchronize(c->stream); // the host vectors may change on the next set_mode
    if (e != cudaSuccess)
        return cuda_fail(e, "upload block tables");
    return MC_OK;
}

cudaError_t sweep_enqueue(mc_ctx *c, long long n, int every, int mode)
{
    if (c->kind == MC_KIND_ISING)
        return ising_sweep_enqueue(c, n, every, mode);
    return mode == MC_MODE_RESIDENT ? su2_resident_enqueue(c, n, every) : su2_sweep_enqueue(c, n, every);
}

// Capture `n` sweeps (+ state advance) into a graph, or replay a cached one.
mc_status run_chunk(mc_ctx *c, long long n, int every, int mode)
{
    if (c->profiling) { // direct launches, each sweep kernel bracketed by events
        cudaError_t ek = sweep_enqueue(c, n, every, mode);
        if (ek == cudaSuccess)
            ek = advance_state_launch(c, n, every > 0 ? n / every : 0);
        if (ek != cudaSuccess)
            return cuda_fail(ek, "enqueue sweep kernels");
        return MC_OK;
    }
    // Graphs are recorded and replayed on a private stream (capture is not
    // permitted on the legacy default stream a caller may pass), fenced with
    // events against the caller's stream so stream order is preserved.
    const auto key = std::make_tuple(n, every, mode, c->threads, c->record_tries, c->n_or);
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess)
            return cuda_fail(e, "begin graph capture");
        c->ls = c->cap_stream;
        cudaError_t ek = sweep_enqueue(c, n, every, mode);
        const long long recs = every > 0 ? n / every : 0;
        if (ek == cudaSuccess)
            ek = advance_state_launch(c, n, recs);
        c->ls = c->stream;
        e = cudaStreamEndCapture(c->cap_stream, &g);
        if (ek != cudaSuccess) {
            if (g)
                cudaGraphDestroy(g);
            return cuda_fail(ek, "enqueue sweep kernels");
        }
        if (e != cudaSuccess)
            return cuda_fail(e, "end graph capture");
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess)
            return cuda_fail(e, "instantiate graph");
        it = c->graphs.emplace(key, ge).first;
    }
    cudaError_t e = cudaEventRecord(c->fence_in, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(c->cap_stream, c->fence_in, 0);
    if (e == cudaSuccess)
        e = cudaGraphLaunch(it->second, c->cap_stream);
    if (e == cudaSuccess)
        e = cudaEventRecord(c->fence_out, c->cap_stream);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(c->stream, c->fence_out, 0);
    if (e != cudaSuccess)
        return cuda_fail(e, "graph launch");
    return MC_OK;
}

const char *kVersion = "mc-gb300 1.0 (sm_103a)";

}  // namespace

namespace mc {
static cudaError_t prof_record(mc_ctx *c)
{
    if (c->events_used == c->events.size()) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess)
            return e;
        c->events.push_back(ev);
    }
    return cudaEventRecord(c->events[c->events_used++], c->stream);
}
void set_last_error(const std::string &msg) { g_err = msg; }
cudaError_t prof_begin(mc_ctx *c) { return c->profiling ? prof_record(c) : cudaSuccess; }
cudaError_t prof_end(mc_ctx *c) { return c->profiling ? prof_record(c) : cudaSuccess; }
}  // namespace mc

extern "C" {

const char *mc_last_error(void) { return g_err.c_str(); }
const char *mc_version(void) { return kVersion; }

size_t mc_workspace_bytes(int32_t n_chains, const mc_chain_desc *chains, int32_t layout, int64_t series_capacity)
{
    std::string why;
    if (!validate(n_chains, chains, layout, series_capacity, why)) {
        g_err = why;
        return 0;
    }
    return make_plan(n_chains, chains, layout, series_capacity).total;
}

mc_status mc_batch_init(mc_ctx **out, int32_t n_chains, const mc_chain_desc *chains, int32_t layout,
                        int64_t series_capacity, void *workspace, size_t workspace_bytes, void *cuda_stream)
{
    if (!out)
        return fail(MC_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why;
    if (!validate(n_chains, chains, layout, series_capacity, why))
        return fail(MC_EINVAL, why);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0)
        return fail(MC_EINVAL, "workspace must be a non-NULL device pointer aligned to 256 bytes");
    cudaPointerAttributes attr{};
    cudaError_t e = cudaPointerGetAttributes(&attr, workspace);
    if (e != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(MC_EINVAL, "workspace is not device memory");
    }
    const Plan p = make_plan(n_chains, chains, layout, series_capacity);
    if (workspace_bytes < p.total)
        return fail(MC_ENOMEM, "workspace too small: need " + std::to_string(p.total) + " bytes");
    mc_ctx *c = new (std::nothrow) mc_ctx();
    if (!c)
        return fail(MC_ENOMEM, "host allocation of the context failed");
    c->kind = chains[0].kind;
    if (c->kind == MC_KIND_SU2) // 128-thread blocks: same occupancy, smaller tail (0.672 vs 0.679 ms per sweep
        c->threads = kSu2DefaultThreads; // of 4 x 32^4)
    c->layout = c->kind == MC_KIND_ISING ? layout : 0;
    c->n_chains = n_chains;
    c->cap = series_capacity;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->ls = c->stream;
    e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&c->fence_in, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&c->fence_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_ctx(c);
        return cuda_fail(e, "create capture stream");
    }
    c->ws = static_cast<char *>(workspace);
    c->ws_bytes = workspace_bytes;
    c->d_state = reinterpret_cast<DevState *>(c->ws + p.state);
    c->d_chains = c->ws + p.chains;
    c->d_block_start = reinterpret_cast<uint32_t *>(c->ws + p.block_start);
    c->d_meas_start = reinterpret_cast<uint32_t *>(c->ws + p.meas_start);
    c->d_series = reinterpret_cast<DevRecord *>(c->ws + p.series);
    c->d_scratch_rec = reinterpret_cast<DevRecord *>(c->ws + p.scratch_rec);
    c->d_partials = reinterpret_cast<long long *>(c->ws + p.partials);
    c->partial_count = p.partial_count;
    c->d_staging = c->ws + p.staging;
    c->staging_bytes = p.staging_bytes;
    c->d_tries = reinterpret_cast<uint8_t *>(c->ws + p.tries);
    c->d_lattice = c->ws + p.lattice;
    c->desc.assign(chains, chains + n_chains);
    if (c->kind == MC_KIND_ISING) {
        c->ising.resize(n_chains);
        for (int k = 0; k < n_chains; ++k) {
            IsingChain &ch = c->ising[k];
            ch = IsingChain{};
            ch.Lx = (uint32_t)chains[k].L[0];
            ch.Ly = (uint32_t)chains[k].L[1];
            ch.W = ch.Lx / 64;
            thresholds(chains[k].beta, ch.T2, ch.T4);
            ch.beta = chains[k].beta;
            ch.key = PhiloxKey{(uint32_t)chains[k].seed, (uint32_t)(chains[k].seed >> 32)};
            ch.chain_id = chains[k].chain_id;
            ch.spin_off = p.lat_off[k];
        }
        e = cudaMemcpyAsync(c->d_chains, c->ising.data(), sizeof(IsingChain) * n_chains, cudaMemcpyHostToDevice,
                            c->stream);
    } else {
        c->su2.resize(n_chains);
        for (int k = 0; k < n_chains; ++k) {
            Su2Chain &ch = c->su2[k];
            ch = Su2Chain{};
            for (int m = 0; m < 4; ++m)
                ch.L[m] = chains[k].L[m];
            ch.nh = (uint32_t)((size_t)ch.L[0] * ch.L[1] * ch.L[2] * ch.L[3] / 2);
            ch.beta = (float)chains[k].beta;
            ch.key = PhiloxKey{(uint32_t)chains[k].seed, (uint32_t)(chains[k].seed >> 32)};
            ch.chain_id = chains[k].chain_id;
            ch.link_off = p.lat_off[k];
            ch.tries_off = p.tries_off[k];
            ch.div1h = make_fastdiv((uint32_t)ch.L[1] / 2);
            ch.div1 = make_fastdiv((uint32_t)ch.L[1]);
            ch.div2 = make_fastdiv((uint32_t)ch.L[2]);
            ch.div3 = make_fastdiv((uint32_t)ch.L[3]);
        }
        e = cudaMemcpyAsync(c->d_chains, c->su2.data(), sizeof(Su2Chain) * n_chains, cudaMemcpyHostToDevice,
                            c->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->d_state, 0, sizeof(DevState), c->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->d_series, 0, (size_t)n_chains * series_capacity * sizeof(DevRecord), c->stream);
    if (e != cudaSuccess) {
        free_ctx(c);
        return cuda_fail(e, "initialise workspace");
    }
    mc_status s = upload_tables(c); // synchronises: the chain tables above are host vectors
    if (s != MC_OK) {
        free_ctx(c);
        return s;
    }
    e = c->kind == MC_KIND_ISING ? ising_init_launch(c, chains) : su2_init_launch(c, chains);
    if (e != cudaSuccess) {
        free_ctx(c);
        return cuda_fail(e, "launch lattice initialisation");
    }
    *out = c;
    return MC_OK;
}

mc_status mc_ising_init(mc_ctx **out, const int32_t L[2], double beta, uint64_t seed, int32_t start, int32_t layout,
                        int64_t series_capacity, void *workspace, size_t workspace_bytes, void *cuda_stream)
{
    if (!L)
        return fail(MC_EINVAL, "L is NULL");
    mc_chain_desc d{};
    d.kind = MC_KIND_ISING;
    d.L[0] = L[0];
    d.L[1] = L[1];
    d.L[2] = d.L[3] = 1;
    d.beta = beta;
    d.seed = seed;
    d.chain_id = 0;
    d.start = start;
    return mc_batch_init(out, 1, &d, layout, series_capacity, workspace, workspace_bytes, cuda_stream);
}

mc_status mc_su2_init(mc_ctx **out, const int32_t L[4], double beta, uint64_t seed, int32_t start,
                      int64_t series_capacity, void *workspace, size_t workspace_bytes, void *cuda_stream)
{
    if (!L)
        return fail(MC_EINVAL, "L is NULL");
    mc_chain_desc d{};
    d.kind = MC_KIND_SU2;
    for (int m = 0; m < 4; ++m)
        d.L[m] = L[m];
    d.beta = beta;
    d.seed = seed;
    d.chain_id = 0;
    d.start = start;
    return mc_batch_init(out, 1, &d, MC_LAYOUT_INT8, series_capacity, workspace, workspace_bytes, cuda_stream);
}

mc_status mc_set_mode(mc_ctx *c, int32_t mode, int32_t threads_per_block)
{
    if (!c)
        return fail(MC_EINVAL, "ctx is NULL");
    if (mode < MC_MODE_AUTO || mode > MC_MODE_RESIDENT)
        return fail(MC_EINVAL, "unknown mode");
    if (mode == MC_MODE_RESIDENT && c->kind == MC_KIND_ISING && !ising_resident_fits(c, nullptr))
        return fail(MC_EINVAL, "resident mode needs Ising chains whose lattices fit in one CTA's shared memory");
    if (threads_per_block != 0) {
        const int maxt = c->kind == MC_KIND_SU2 ? 256 : 1024;
        if (threads_per_block < 32 || threads_per_block > maxt || threads_per_block % 32)
            return fail(MC_EINVAL, "threads_per_block must be a multiple of 32 in [32, " + std::to_string(maxt) + "]");
    }
    c->mode = mode;
    if (threads_per_block != 0)
        c->threads_set = true;
    if (threads_per_block != 0 && threads_per_block != c->threads) {
        c->threads = threads_per_block;
        mc_status s = upload_tables(c);
        if (s != MC_OK)
            return s;
    }
    destroy_graphs(c);
    return MC_OK;
}

mc_status mc_sweep(mc_ctx *c, int64_t n_sweeps, int32_t measure_every)
{
    if (!c)
        return fail(MC_EINVAL, "ctx is NULL");
    if (n_sweeps < 0 || measure_every < 0)
        return fail(MC_EINVAL, "n_sweeps and measure_every must be >= 0");
    if (n_sweeps == 0)
        return MC_OK;
    const long long recs = measure_every > 0 ? n_sweeps / measure_every : 0;
    if ((c->rec_written - c->rec_read) + recs > c->cap)
        return fail(MC_EINVAL, "measurement ring buffer would overflow: read the series first or raise capacity");
    if (c->sweeps_done + n_sweeps > 0xFFFFFFFFll)
        return fail(MC_EINVAL, "sweep counter would exceed 2^32 (the Philox sweep word)");
    const int mode = resolve_mode(c);
    if (mode == MC_MODE_RESIDENT) {
        cudaError_t e = c->kind == MC_KIND_ISING ? ising_prepare_resident(c) : su2_prepare_resident(c);
        if (e != cudaSuccess)
            return cuda_fail(e, "configure resident kernel");
    }
    // Split long calls into replayable chunks whose length is a multiple of
    // measure_every, so the record cadence repeats exactly.
    long long chunk = 256;
    if (mode == MC_MODE_RESIDENT)
        chunk = 4096;
    if (measure_every > 0)
        chunk = std::max<long long>(measure_every, chunk / measure_every * measure_every);
    long long left = n_sweeps;
    while (left > 0) {
        const long long m = std::min(left, chunk);
        mc_status s = run_chunk(c, m, measure_every, mode);
        if (s != MC_OK)
            return s;
        left -= m;
    }
    c->sweeps_done += n_sweeps;
    c->rec_written += recs;
    return MC_OK;
}

mc_status mc_sync(mc_ctx *c)
{
    if (!c)
        return fail(MC_EINVAL, "ctx is NULL");
    return check_device(c);
}

static void convert_record(const mc_ctx *c, int k, const DevRecord &r, mc_record &o)
{
    o.sweep = r.sweep;
    if (c->kind == MC_KIND_ISING) {
        const long long n = (long long)c->ising[k].Lx * c->ising[k].Ly;
        o.E = 2 * (long long)r.a - 2 * n;
        o.M = 2 * (long long)r.b - n;
        o.P = o.Ps = o.Pt = 0.0;
    } else { // exact fixed-point sums over the N = 2 nh sites, 3 planes each
        const double n = 2.0 * (double)c->su2[k].nh;
        const long long A = (long long)r.a, B = (long long)r.b;
        o.E = o.M = 0;
        o.P = (double)(A + B) * kPlaqUnfix / (6.0 * n);
        o.Ps = (double)A * kPlaqUnfix / (3.0 * n);
        o.Pt = (double)B * kPlaqUnfix / (3.0 * n);
    }
}

mc_status mc_measure(mc_ctx *c, int32_t chain, mc_record *out)
{
    if (!c || !out)
        return fail(MC_EINVAL, "NULL argument");
    if (chain < 0 || chain >= c->n_chains)
        return fail(MC_EINVAL, "chain index out of range");
    DevRecord *d = c->d_scratch_rec + chain;
    cudaError_t e = c->kind == MC_KIND_ISING ? ising_measure_launch(c, chain, d) : su2_measure_launch(c, chain, d);
    if (e != cudaSuccess)
        return cuda_fail(e, "launch measurement");
    DevRecord r;
    e = cudaMemcpyAsync(&r, d, sizeof r, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "copy measurement");
    mc_status s = check_device(c);
    if (s != MC_OK)
        return s;
    r.sweep = c->sweeps_done - 1;
    convert_record(c, chain, r, *out);
    return MC_OK;
}

mc_status mc_su2_polyakov(mc_ctx *c, int32_t chain, double *out)
{
    if (!c || !out)
        return fail(MC_EINVAL, "NULL argument");
    if (c->kind != MC_KIND_SU2)
        return fail(MC_EINVAL, "the Polyakov loop is an SU(2) observable");
    if (chain < 0 || chain >= c->n_chains)
        return fail(MC_EINVAL, "chain index out of range");
    DevRecord *d = c->d_scratch_rec + chain;
    cudaError_t e = su2_polyakov_launch(c, chain, d);
    if (e != cudaSuccess)
        return cuda_fail(e, "launch Polyakov loop");
    DevRecord r;
    e = cudaMemcpyAsync(&r, d, sizeof r, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "copy Polyakov loop");
    mc_status s = check_device(c);
    if (s != MC_OK)
        return s;
    *out = r.d0;
    return MC_OK;
}

mc_status mc_read_series(mc_ctx *c, mc_record *dst, int64_t max_per_chain, int64_t *n_per_chain)
{
    if (!c || !n_per_chain || (!dst && max_per_chain > 0) || max_per_chain < 0)
        return fail(MC_EINVAL, "bad argument");
    const long long unread = c->rec_written - c->rec_read;
    const long long m = std::min<long long>(unread, max_per_chain);
    *n_per_chain = 0;
    if (m <= 0)
        return check_device(c);
    std::vector<DevRecord> tmp((size_t)c->n_chains * m);
    const long long start = c->rec_read % c->cap;
    const long long first = std::min<long long>(m, c->cap - start);
    const size_t pitch = (size_t)c->cap * sizeof(DevRecord);
    cudaError_t e = cudaMemcpy2DAsync(tmp.data(), (size_t)m * sizeof(DevRecord), c->d_series + start, pitch,
                                      (size_t)first * sizeof(DevRecord), c->n_chains, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && first < m)
        e = cudaMemcpy2DAsync(tmp.data() + first, (size_t)m * sizeof(DevRecord), c->d_series, pitch,
                              (size_t)(m - first) * sizeof(DevRecord), c->n_chains, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "copy series");
    mc_status s = check_device(c);
    if (s != MC_OK)
        return s;
    for (int k = 0; k < c->n_chains; ++k)
        for (long long i = 0; i < m; ++i)
            convert_record(c, k, tmp[(size_t)k * m + i], dst[(size_t)k * max_per_chain + i]);
    c->rec_read += m;
    *n_per_chain = m;
    return MC_OK;
}

// Bytes and device address of a chain's storage (the MC_FMT_NATIVE format).
static size_t native_bytes(const mc_ctx *c, int32_t chain)
{
    if (c->kind == MC_KIND_SU2)
        return su2_config_bytes(c->su2[chain]);
    const IsingChain &ch = c->ising[chain];
    const size_t n = (size_t)ch.Lx * ch.Ly;
    return c->layout == MC_LAYOUT_INT8 ? n : n / 8;
}

static char *native_ptr(const mc_ctx *c, int32_t chain)
{
    return c->d_lattice + (c->kind == MC_KIND_SU2 ? c->su2[chain].link_off : c->ising[chain].spin_off);
}

size_t mc_config_bytes(const mc_ctx *c, int32_t chain, int32_t fmt)
{
    if (!c || chain < 0 || chain >= c->n_chains)
        return 0;
    if (fmt == MC_FMT_NATIVE)
        return native_bytes(c, chain);
    if (c->kind == MC_KIND_ISING)
        return ising_config_bytes(c->ising[chain], fmt);
    return fmt == MC_FMT_F32 ? su2_config_bytes(c->su2[chain]) : 0;
}

// Device address of a host buffer the GPU can read and write in place
// (page-locked memory, allocated or registered through CUDA), else nullptr.
static void *device_view_of_host(void *host)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError(); // clear the non-sticky error of an unknown pointer
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Host buffers: page-locked memory is read or written by the conversion kernel
// directly (one pass over the interconnect); other host memory goes through
// the staging region with a copy.
static mc_status config_io(mc_ctx *c, int32_t chain, int32_t fmt, void *buf, int32_t is_device, bool to_lattice)
{
    if (!c || !buf)
        return fail(MC_EINVAL, "NULL argument");
    if (chain < 0 || chain >= c->n_chains)
        return fail(MC_EINVAL, "chain index out of range");
    if (fmt == MC_FMT_NATIVE) { // the storage itself: one copy, no conversion
        char *lat = native_ptr(c, chain);
        const size_t bytes = native_bytes(c, chain);
        cudaError_t e = to_lattice ? cudaMemcpyAsync(lat, buf, bytes, cudaMemcpyDefault, c->stream)
                                   : cudaMemcpyAsync(buf, lat, bytes, cudaMemcpyDefault, c->stream);
        if (e != cudaSuccess)
            return cuda_fail(e, to_lattice ? "set native configuration" : "get native configuration");
        return to_lattice ? MC_OK : check_device(c);
    }
    const size_t bytes = mc_config_bytes(c, chain, fmt);
    if (bytes == 0)
        return fail(MC_EINVAL, "format not valid for this chain (Ising: MC_FMT_INT8, or MC_FMT_BITS with Lx % 32 == 0; "
                               "SU(2): MC_FMT_F32)");
    void *dev = buf;
    bool staged = false;
    if (!is_device) {
        dev = device_view_of_host(buf);
        if (!dev) {
            dev = c->d_staging;
            staged = true;
        }
    }
    cudaError_t e = cudaSuccess;
    if (to_lattice && staged)
        e = cudaMemcpyAsync(dev, buf, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = c->kind == MC_KIND_ISING ? ising_config_io(c, chain, fmt, dev, to_lattice)
                                     : su2_config_io(c, chain, dev, to_lattice);
    if (e == cudaSuccess && !to_lattice && staged)
        e = cudaMemcpyAsync(buf, dev, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "configuration copy");
    if (!to_lattice)
        return check_device(c);
    return MC_OK;
}

mc_status mc_get_config(mc_ctx *c, int32_t chain, int32_t fmt, void *dst, int32_t dst_is_device)
{
    return config_io(c, chain, fmt, dst, dst_is_device, false);
}

mc_status mc_set_config(mc_ctx *c, int32_t chain, int32_t fmt, const void *src, int32_t src_is_device)
{
    return config_io(c, chain, fmt, const_cast<void *>(src), src_is_device, true);
}

mc_status mc_get_sweep(const mc_ctx *c, int64_t *sweeps_done)
{
    if (!c || !sweeps_done)
        return fail(MC_EINVAL, "NULL argument");
    *sweeps_done = c->sweeps_done;
    return MC_OK;
}

mc_status mc_set_sweep(mc_ctx *c, int64_t sweeps_done)
{
    if (!c)
        return fail(MC_EINVAL, "ctx is NULL");
    if (sweeps_done < 0 || sweeps_done > 0xFFFFFFFFll)
        return fail(MC_EINVAL, "sweeps_done must be in [0, 2^32]");
    const unsigned long long v = (unsigned long long)sweeps_done;
    cudaError_t e = cudaMemcpyAsync(&c->d_state->sweep_base, &v, sizeof v, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "set sweep counter");
    c->sweeps_done = sweeps_done;
    return MC_OK;
}

mc_status mc_su2_record_tries(mc_ctx *c, int32_t enable)
{
    if (!c)
        return fail(MC_EINVAL, "ctx is NULL");
    if (c->kind != MC_KIND_SU2)
        return fail(MC_EINVAL, "not an SU(2) context");
    if ((bool)enable != c->record_tries) {
        c->record_tries = enable != 0;
        destroy_graphs(c);
    }
    return MC_OK;
}

mc_status mc_su2_set_overrelax(mc_ctx *c, int32_t n_or)
{
    if (!c)
        return fail(MC_EINVAL, "ctx is NULL");
    if (c->kind != MC_KIND_SU2)
        return fail(MC_EINVAL, "overrelaxation applies to SU(2) contexts");
    if (n_or < 0 || n_or > kMaxOverrelax)
        return fail(MC_EINVAL, "n_or must be in [0, " + std::to_string(kMaxOverrelax) + "]");
    if (n_or != c->n_or) {
        c->n_or = n_or;
        destroy_graphs(c);
    }
    return MC_OK;
}

mc_status mc_su2_get_overrelax(mc_ctx *c, int32_t *n_or)
{
    if (!c || !n_or)
        return fail(MC_EINVAL, "ctx or n_or is NULL");
    *n_or = c->n_or;
    return MC_OK;
}

mc_status mc_su2_get_tries(mc_ctx *c, int32_t chain, uint8_t *dst)
{
    if (!c || !dst)
        return fail(MC_EINVAL, "NULL argument");
    if (c->kind != MC_KIND_SU2 || chain < 0 || chain >= c->n_chains)
        return fail(MC_EINVAL, "not an SU(2) chain");
    const Su2Chain &ch = c->su2[chain];
    cudaError_t e = cudaMemcpyAsync(dst, c->d_tries + ch.tries_off, (size_t)8 * ch.nh, cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "copy tries");
    return check_device(c);
}

mc_status mc_su2_failed_updates(mc_ctx *c, int64_t *count)
{
    if (!c || !count)
        return fail(MC_EINVAL, "NULL argument");
    mc_status s = check_device(c);
    if (s != MC_OK)
        return s;
    DevState st;
    cudaError_t e = cudaMemcpy(&st, c->d_state, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(e, "read device state");
    *count = (int64_t)st.hb_failures;
    return MC_OK;
}

mc_status mc_profile_enable(mc_ctx *c, int32_t enable)
{
    if (!c)
        return fail(MC_EINVAL, "ctx is NULL");
    c->profiling = enable != 0;
    return MC_OK;
}

mc_status mc_profile_read(mc_ctx *c, int64_t *launches, double *total_ms)
{
    if (!c || !launches || !total_ms)
        return fail(MC_EINVAL, "NULL argument");
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "stream synchronize");
    double total = 0.0;
    for (size_t i = 0; i + 1 < c->events_used; i += 2) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, c->events[i], c->events[i + 1]);
        if (e != cudaSuccess)
            return cuda_fail(e, "event elapsed time");
        total += ms;
    }
    *launches = (int64_t)(c->events_used / 2);
    *total_ms = total;
    c->events_used = 0;
    return MC_OK;
}

mc_status mc_destroy(mc_ctx *c)
{
    if (!c)
        return MC_OK;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    destroy_graphs(c);
    free_ctx(c);
    if (e != cudaSuccess)
        return cuda_fail(e, "stream synchronize");
    return MC_OK;
}

}  // extern "C"
