// mc_internal.cuh -- structures shared by the kernels and the C ABI layer of
// libmc.so.  Nothing here is visible through include/mc.h.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/mc.h"
#include "fastdiv.cuh"
#include "philox.cuh"

namespace mc {

constexpr int kMaxChains = 4096;
constexpr int kDefaultThreads = 256;
constexpr int kSu2DefaultThreads = 128; // SU(2) phase kernels (launch bound 256 threads)
constexpr int kMaxOverrelax = 64;   // overrelaxation sweeps per heat-bath sweep
constexpr size_t kAlign = 256;

// Per-chain descriptor of a 2D Ising chain, resident in the workspace.
struct IsingChain {
    uint32_t Lx, Ly;    // extents (even)
    uint32_t W;         // MSC words per row per colour = Lx / 64
    uint32_t T2, T4;    // Metropolis thresholds for dE = 4 and dE = 8 (floor(e^{-beta dE} 2^32))
    PhiloxKey key;      // seed
    uint32_t chain_id;  // Philox counter word 3
    uint32_t pad0;
    uint64_t spin_off;  // byte offset of the chain's spins in the lattice region
    double beta;        // coupling (the Metropolis-Hastings step of the learned proposal needs it)
};

// Per-chain descriptor of a 4D SU(2) chain.
struct Su2Chain {
    int32_t L[4];       // extents, mu = 0 time (all even)
    uint32_t nh;        // sites per parity = N / 2
    float beta;
    PhiloxKey key;
    uint32_t chain_id;
    uint32_t pad0;
    uint64_t link_off;  // byte offset of the links: float4 [parity][mu][nh]
    uint64_t tries_off; // byte offset of the try record: uint8 [s][mu]
    FastDiv div1h, div1, div2, div3; // by L1 / 2, L1, L2, L3: site index -> coordinates
};

// Device-resident run state: lets one captured CUDA graph be replayed.
struct DevState {
    unsigned long long sweep_base;   // sweeps completed before the running call
    unsigned long long rec_head;     // records written before the running call
    unsigned long long hb_failures;  // SU(2) link updates with every try rejected
    int err_code;                    // first latched device fault (0 = none)
    int err_info;
    unsigned long long pad[4];
};

// Measurement record as kept on the device.  Ising: a = anti-aligned bonds,
// b = up spins (E = 2a - 2N, M = 2b - N are formed on the host).  SU(2): a, b =
// the exact int64 fixed-point sums of the spatial and temporal plaquettes (two's
// complement), from which the host forms P, P_s, P_t in FP64 (the device's FP64
// pipe is narrow, and the measuring thread would hold up the next phase).
constexpr double kPlaqUnfix = 1.0 / 536870912.0; // 2^-29, the unit of the plaquette sums
struct DevRecord {
    long long sweep;
    unsigned long long a, b;
    double d0, d1, d2;
};
static_assert(sizeof(DevRecord) == 48, "record size");

// Device fault codes latched in DevState::err_code.
enum DevErr : int { kErrNone = 0, kErrChainLookup = 1, kErrBounds = 2, kErrTimeout = 3 };

__device__ __forceinline__ void latch_error(DevState *st, int code, int info)
{
    if (atomicCAS(&st->err_code, 0, code) == 0)
        st->err_info = info;
}

// Lattice load policy.  Kernels that never read a location written during the
// same launch use the read-only path (kLdReadOnly).  Kernels whose later phases
// read what earlier phases wrote (possibly on other SMs of the cluster) either
// load through L2, the device's point of coherence (kLdCoherent: the SU(2)
// resident kernel, where L1-cacheable loads measured no faster), or use plain
// loads ordered by the barrier's acquire (kLdPlain: the batch kernel).
constexpr int kLdReadOnly = 0, kLdPlain = 1, kLdCoherent = 2;

// Threads per block of the SU(2) plaquette measurement; each thread measures
// one x1 pair of sites, so a chain of N sites has ceil(N / (2 kPlaqThreads))
// partial-sum blocks.
constexpr int kPlaqThreads = 128;
// Largest cluster of the SU(2) resident mode (CTAs per chain; 16 is non-portable).
constexpr int kSu2ResidentMaxCluster = 16;
template <int LD, typename T>
__device__ __forceinline__ T lat_load(const T *p)
{
    if (LD == kLdCoherent)
        return __ldcg(p);
    else if (LD == kLdReadOnly)
        return __ldg(p);
    else
        return *p;
}

// Largest k in [0, n) with block_start[k] <= b (block_start ascending, [0] = 0).
__device__ __forceinline__ int find_chain(const uint32_t *__restrict__ block_start, int n, uint32_t b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&block_start[mid]) <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Arguments common to the sweep kernels.
struct SweepArgs {
    const void *chains;          // IsingChain* or Su2Chain*
    const uint32_t *block_start; // grid-mode block offsets per chain (n_chains + 1 entries)
    int n_chains;
    char *lattice;               // lattice region base
    DevRecord *series;           // [chain][cap]
    DevState *state;
    long long cap;               // records per chain in the ring
    uint32_t k;                  // sweep offset within the running call
    int measure;                 // 1: this sweep is measured
    uint32_t rec_k;              // index of this record within the running call
    uint8_t *tries;              // SU(2) try record base, or nullptr
    uint32_t block_base;         // first block of this launch in the block table
};

}  // namespace mc

// Host-side context.  Lives in the global namespace because include/mc.h
// forward-declares `struct mc_ctx`.
struct mc_ctx {
    int kind = 0;
    int layout = 0;
    int n_chains = 0;
    long long cap = 0;
    cudaStream_t stream = nullptr;       // the caller's stream
    cudaStream_t ls = nullptr;           // stream kernels are launched on (== stream, or the
                                         // capture stream while a graph is being recorded)
    cudaStream_t cap_stream = nullptr;   // private non-blocking stream for graph capture/replay
    cudaEvent_t fence_in = nullptr, fence_out = nullptr;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    // carve-out of the workspace
    void *d_chains = nullptr;
    uint32_t *d_block_start = nullptr;   // grid-mode sweep launches
    uint32_t *d_meas_start = nullptr;    // measurement launches
    char *d_lattice = nullptr;
    mc::DevRecord *d_series = nullptr;
    mc::DevState *d_state = nullptr;
    char *d_staging = nullptr;
    size_t staging_bytes = 0;
    long long *d_partials = nullptr;     // SU(2) plaquette per-block partial sums (fixed point)
    size_t partial_count = 0;
    uint8_t *d_tries = nullptr;
    mc::DevRecord *d_scratch_rec = nullptr; // one record per chain for mc_measure
    // host copies
    std::vector<mc::IsingChain> ising;
    std::vector<mc::Su2Chain> su2;
    std::vector<mc_chain_desc> desc;
    std::vector<uint32_t> block_start, meas_start;
    std::vector<std::pair<int, int>> groups; // SU(2) launch groups of chains [first, last)
    uint32_t grid_blocks = 0, meas_blocks = 0;
    // run bookkeeping
    long long sweeps_done = 0;
    long long rec_written = 0, rec_read = 0;
    int mode = MC_MODE_AUTO;
    int threads = mc::kDefaultThreads;
    bool threads_set = false;            // threads chosen by the caller (mc_set_mode), not the default
    bool record_tries = false;
    int n_or = 0;                        // SU(2): overrelaxation sweeps after each heat-bath sweep
    int su2_res_cluster = 0;             // SU(2) resident mode: CTAs per chain (0 = not prepared)
    std::map<std::tuple<long long, int, int, int, bool, int>, cudaGraphExec_t> graphs;
    // kernel timing (mc_profile_enable)
    bool profiling = false;
    std::vector<cudaEvent_t> events; // pairs: [2i] before, [2i+1] after launch i
    size_t events_used = 0;
};

namespace mc {
// Launchers implemented in ising.cu / su2.cu; return a cudaError_t.
cudaError_t ising_init_launch(mc_ctx *c, const mc_chain_desc *desc);
cudaError_t ising_sweep_enqueue(mc_ctx *c, long long n, int every, int mode);
cudaError_t ising_measure_launch(mc_ctx *c, int chain, DevRecord *out);
cudaError_t ising_config_io(mc_ctx *c, int chain, int fmt, void *dev_buf, bool to_lattice);
size_t ising_config_bytes(const IsingChain &ch, int fmt);
bool ising_resident_fits(const mc_ctx *c, int *smem_bytes);
cudaError_t ising_prepare_resident(mc_ctx *c);
void ising_plan_grid(mc_ctx *c);

cudaError_t su2_init_launch(mc_ctx *c, const mc_chain_desc *desc);
cudaError_t su2_sweep_enqueue(mc_ctx *c, long long n, int every);
cudaError_t su2_measure_launch(mc_ctx *c, int chain, DevRecord *out);
cudaError_t su2_polyakov_launch(mc_ctx *c, int chain, DevRecord *out);
cudaError_t su2_config_io(mc_ctx *c, int chain, void *dev_buf, bool to_lattice);
size_t su2_config_bytes(const Su2Chain &ch);
void su2_plan_grid(mc_ctx *c);
bool su2_resident_auto(const mc_ctx *c);
cudaError_t su2_prepare_resident(mc_ctx *c);
cudaError_t su2_resident_enqueue(mc_ctx *c, long long n, int every);

cudaError_t advance_state_launch(mc_ctx *c, long long n, long long recs);

// Message returned by mc_last_error() on this thread.
void set_last_error(const std::string &msg);

// Bracket one sweep-kernel launch with events when the context is profiling.
cudaError_t prof_begin(mc_ctx *c);
cudaError_t prof_end(mc_ctx *c);
}  // namespace mc
