/*
 * mc.h -- C ABI of libmc.so: the checkerboard local-update sweep of
 * Demchik & Strelchenko, "Monte Carlo simulations on Graphics Processing Units"
 * (arXiv:0903.3053), for one NVIDIA GB300 (sm_103a).
 *
 * Models
 *   Ising : 2D Ising model of Eq. (1), H = -sum_<ij> s_i s_j, on an Lx x Ly
 *           periodic torus, Metropolis single-spin updates on the red/black
 *           checkerboard (Sec. 2.3); a sweep updates colour 0 ((x+y) even), then
 *           colour 1 (Sec. 2.1).
 *   SU(2) : 4D SU(2) Wilson gauge theory, Eqs. (2)-(3), on an L0 x L1 x L2 x L3
 *           periodic hypertorus (mu = 0 is time, Sec. 2.4); heat-bath
 *           replacement of each link by Eqs. (5)-(7) with the staple of Eq. (6);
 *           a sweep runs mu = 0..3 on the odd sites, then mu = 0..3 on the even
 *           sites (Sec. 2.4).  Links are the quaternions (U0, U1, U2, U3) of
 *           Eq. (4) in FP32.
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), keyed by the 64-bit
 *   seed and counted by (site, sweep, tag, chain id), so every result is
 *   reproducible and independent of the launch configuration.
 *
 * Conventions
 *   - Every function returns an mc_status; nothing throws across the ABI.  On a
 *     non-OK status mc_last_error() returns a message (thread-local).
 *   - Memory: the caller allocates ONE device workspace of
 *     mc_workspace_bytes(...) bytes (e.g. a torch uint8 tensor) and keeps it
 *     alive until mc_destroy; the library carves the lattice, series ring
 *     buffer, scratch and state out of it and allocates no device memory of its
 *     own.  The library owns the mc_ctx struct and its CUDA graphs.
 *   - Streams: all device work of a context is issued on the cudaStream_t given
 *     at init (passed as void*; NULL = legacy default stream).  Calls marked
 *     "async" return before the GPU has finished; device-side faults detected by
 *     the kernels (bad index, wait limit reached) are latched in the context and
 *     reported by the next synchronising call (mc_sync, mc_measure,
 *     mc_read_series, mc_get_config) as MC_EDEVICE.
 *   - Layout-free I/O: configurations cross the ABI in a canonical order that
 *     does not depend on the internal layout:
 *       Ising : MC_FMT_INT8 -- int8 s[y][x] = +-1;
 *               MC_FMT_BITS -- uint32 words, row-major, bit b of word w of row y
 *                              is site x = 32 w + b, 1 = spin +1 (Lx % 32 == 0).
 *       SU(2) : float q[s][mu][4], s = x1 + L1 (x2 + L2 (x3 + L3 x0)).
 *   - Threads: one context must not be used by two host threads at once.
 */
#ifndef MC_H
#define MC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MC_API __attribute__((visibility("default")))
#else
#define MC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mc_ctx mc_ctx; /* opaque, owned by the library */

typedef enum {
    MC_OK = 0,
    MC_EINVAL = -1,   /* bad argument (reported before any device work) */
    MC_ENOMEM = -2,   /* workspace too small */
    MC_ECUDA = -3,    /* a CUDA runtime call failed */
    MC_ETIMEOUT = -4, /* a device-side wait reached its iteration limit */
    MC_ESTATE = -5,   /* call not valid in the context's current state */
    MC_EDEVICE = -6   /* a kernel detected a fault and latched it */
} mc_status;

enum { MC_COLD = 0, MC_HOT = 1 };              /* initial configuration (Sec. 2.1, 2.4) */
enum { MC_KIND_ISING = 1, MC_KIND_SU2 = 2 };   /* model */
enum { MC_LAYOUT_INT8 = 0, MC_LAYOUT_MSC32 = 1 }; /* Ising storage: 1 byte / 1 bit per spin */
enum { MC_FMT_INT8 = 0, MC_FMT_BITS = 1, MC_FMT_F32 = 2, MC_FMT_NATIVE = 3 }; /* config formats */
enum { MC_MODE_AUTO = 0, MC_MODE_GRID = 1, MC_MODE_RESIDENT = 2 }; /* sweep execution */

/* One Markov chain of a batch. */
typedef struct {
    int32_t kind;      /* MC_KIND_ISING or MC_KIND_SU2 */
    int32_t L[4];      /* Ising: L[0] = Lx, L[1] = Ly (L[2], L[3] ignored); SU(2): L[mu] */
    double beta;       /* Ising: coupling beta of Eq. (1); SU(2): beta = 4/g^2 of Eq. (2); >= 0 */
    uint64_t seed;     /* Philox key */
    uint32_t chain_id; /* Philox counter word 3: distinguishes chains sharing a seed */
    int32_t start;     /* MC_COLD or MC_HOT */
} mc_chain_desc;

/* One measurement record (per chain, per measured sweep). */
typedef struct {
    int64_t sweep; /* global index of the sweep after which it was taken (0-based) */
    int64_t E;     /* Ising: H of Eq. (1), exact */
    int64_t M;     /* Ising: sum of spins, exact */
    double P;      /* SU(2): plaquette (1/6N) sum_x sum_{mu<nu} (1/2) Tr U_munu(x), Eq. (3); FP32 per-site
                      values, summed exactly in int64 fixed point (2^-29), averaged in FP64 */
    double Ps;     /* SU(2): spatial plaquettes only (mu, nu in 1..3) */
    double Pt;     /* SU(2): temporal plaquettes only (one index 0) */
} mc_record;

/* Sizes.  Each chain needs all extents even (checkerboard / parity split);
 * MC_LAYOUT_MSC32 additionally needs Lx % 64 == 0.  series_capacity = records
 * per chain the ring buffer holds between two mc_read_series calls (>= 1).
 * Returns 0 when the arguments are invalid (see mc_last_error). */
MC_API size_t mc_workspace_bytes(int32_t n_chains, const mc_chain_desc *chains, int32_t layout,
                          int64_t series_capacity);

/* Create a context over n_chains chains, all of the same kind, and launch their
 * initialisation (hot/cold, Sec. 2.1 and Sec. 2.4; async).  `workspace` is a
 * device pointer to at least mc_workspace_bytes(...) bytes, 256-byte aligned,
 * borrowed until mc_destroy.  `cuda_stream` is a cudaStream_t or NULL.  The
 * global sweep counter starts at 0. */
MC_API mc_status mc_batch_init(mc_ctx **out, int32_t n_chains, const mc_chain_desc *chains, int32_t layout,
                        int64_t series_capacity, void *workspace, size_t workspace_bytes, void *cuda_stream);

/* Single-chain conveniences (chain_id 0). */
MC_API mc_status mc_ising_init(mc_ctx **out, const int32_t L[2], double beta, uint64_t seed, int32_t start,
                        int32_t layout, int64_t series_capacity, void *workspace, size_t workspace_bytes,
                        void *cuda_stream);
MC_API mc_status mc_su2_init(mc_ctx **out, const int32_t L[4], double beta, uint64_t seed, int32_t start,
                      int64_t series_capacity, void *workspace, size_t workspace_bytes, void *cuda_stream);

/* Advance every chain by n_sweeps sweeps (async).  When measure_every > 0 a
 * record is appended after the k-th sweep of this call (k = 1..n_sweeps) for
 * every k divisible by measure_every (the measuring kernels of Sec. 2.3/2.4);
 * MC_EINVAL if that would overrun the unread part of the ring buffer.
 * Repeated calls with the same (n_sweeps, measure_every) replay one captured
 * CUDA graph. */
MC_API mc_status mc_sweep(mc_ctx *ctx, int64_t n_sweeps, int32_t measure_every);

/* Execution mode for later sweeps: MC_MODE_GRID (one launch per half-sweep /
 * phase over all chains), MC_MODE_RESIDENT (all sweeps of a call in one
 * launch -- Ising: one CTA per chain with its lattice in shared memory, for
 * lattices that fit there; SU(2): one thread-block cluster of up to 16 CTAs
 * per chain, the phases of Sec. 2.4 separated by the hardware cluster barrier,
 * any lattice size, fastest up to ~4096 links per phase) or MC_MODE_AUTO
 * (resident for small lattices).  An SU(2) context that records heat-bath
 * tries (mc_su2_record_tries) always sweeps in grid mode.  threads_per_block
 * = 0 keeps the default (256 for Ising, 128 for SU(2), at most 256 for SU(2)):
 * the block size of grid mode, and for Ising resident mode the largest block.
 * Without one, an Ising resident CTA has the largest chain's work units (int8:
 * groups of four same-colour sites; MSC32: pairs of rows) rounded up to a
 * warp, at most 1024 threads when no more chains than SMs share the GPU and at
 * most 256 otherwise.  The SU(2) resident kernel always runs 1024-thread CTAs.  Results are bit-identical in
 * every mode and for every block size. */
MC_API mc_status mc_set_mode(mc_ctx *ctx, int32_t mode, int32_t threads_per_block);

/* Wait for the context's stream; report latched device faults. */
MC_API mc_status mc_sync(mc_ctx *ctx);

/* Measure chain `chain` now (synchronous) and return the record (sweep field =
 * number of sweeps done - 1, or -1 before the first sweep). */
MC_API mc_status mc_measure(mc_ctx *ctx, int32_t chain, mc_record *out);

/* Copy the unread records (oldest first, chain-major: all of chain 0, then
 * chain 1, ...) into host_dst, which must hold n_chains * max_per_chain
 * records; *n_per_chain receives how many records each chain returned.  The
 * copied records are marked read.  Synchronous. */
MC_API mc_status mc_read_series(mc_ctx *ctx, mc_record *host_dst, int64_t max_per_chain, int64_t *n_per_chain);

/* Configuration of one chain, to/from host or device memory (dst_is_device /
 * src_is_device).  Canonical formats (above): Ising MC_FMT_INT8 or MC_FMT_BITS,
 * SU(2) MC_FMT_F32.  MC_FMT_NATIVE is the chain's storage in the context's own
 * layout, copied as it is (one copy, no conversion kernel), for checkpoints
 * restored into a context of the same kind and layout:
 *   Ising, int8 layout : int8 s[y][x], as MC_FMT_INT8;
 *   Ising, MSC32       : uint32 plane[c][y][w], c = (x + y) & 1 the colour;
 *                        bit b of word w is the site x = 2 (32 w + b) +
 *                        ((y + c) & 1) of row y, 1 = spin +1;
 *   SU(2)              : float4 U[p][mu][s >> 1], p = (x0 + x1 + x2 + x3) & 1
 *                        the parity of site s (canonical index above).
 * For the canonical formats, page-locked host memory (allocated or registered
 * through CUDA) is read or written in place by the layout-conversion kernel;
 * other host memory passes through the context's staging region with a copy.
 * mc_get_config is synchronous.  mc_set_config is asynchronous on the context's
 * stream: a device or page-locked source must stay unchanged until the next
 * synchronising call; other host memory may be reused when the call returns. */
MC_API mc_status mc_get_config(mc_ctx *ctx, int32_t chain, int32_t fmt, void *dst, int32_t dst_is_device);
MC_API mc_status mc_set_config(mc_ctx *ctx, int32_t chain, int32_t fmt, const void *src, int32_t src_is_device);
MC_API size_t mc_config_bytes(const mc_ctx *ctx, int32_t chain, int32_t fmt); /* 0 if invalid */

/* Checkpoint: the global sweep counter is the whole RNG state (counter-based
 * stream); together with the configurations it makes resume bit-exact. */
MC_API mc_status mc_get_sweep(const mc_ctx *ctx, int64_t *sweeps_done);
MC_API mc_status mc_set_sweep(mc_ctx *ctx, int64_t sweeps_done);

/* SU(2) debugging: when enabled, every sweep writes, per link, the index of
 * the heat-bath try whose draw was taken (0..7 Kennedy-Pendleton, 8..71 Creutz,
 * 255 = all rejected, link unchanged) into a per-chain byte array readable with
 * mc_su2_get_tries (canonical [s][mu] order, 4 N bytes, host memory). */
MC_API mc_status mc_su2_record_tries(mc_ctx *ctx, int32_t enable);
MC_API mc_status mc_su2_get_tries(mc_ctx *ctx, int32_t chain, uint8_t *host_dst);

/* Number of SU(2) link updates, summed over chains and sweeps so far, whose
 * every heat-bath try was rejected (link kept; still exact).  Synchronous. */
MC_API mc_status mc_su2_failed_updates(mc_ctx *ctx, int64_t *count);

/* Overrelaxation (Sec. 2.4: "heat-bath algorithm with overrelaxation"): from
 * the next mc_sweep on, every sweep of every chain of an SU(2) context is one
 * heat-bath sweep followed by n_or overrelaxation sweeps, 0 <= n_or <= 64
 * (default 0), each in the heat-bath's phase order (odd sites mu = 0..3, then
 * even sites).  An overrelaxation update replaces U_mu(x) by V U^dag V with
 * V = W / |W| (W the staple of Eq. (6)): it keeps the action, uses no random
 * numbers and leaves a link with W = 0 unchanged.  The sweep counter and the
 * measurement cadence count compound sweeps.  MC_EINVAL for an Ising context
 * or n_or out of range.  The paper does not fix n_or; it calls the run-time
 * choice the "number of link updates per one MC sweep". */
MC_API mc_status mc_su2_set_overrelax(mc_ctx *ctx, int32_t n_or);
MC_API mc_status mc_su2_get_overrelax(mc_ctx *ctx, int32_t *n_or);

/* Polyakov loop of one SU(2) chain's current configuration: the average over
 * the L1 L2 L3 spatial sites x of (1/2) Tr U_0(0, x) U_0(1, x) ... U_0(L0-1, x)
 * (mu = 0 is time).  The paper measures plaquettes only (Eq. (3)); this is the
 * order parameter of its finite-temperature lattices L_t x L_s^3 (Sec. 2.4).
 * FP32 products, exact fixed-point sum; written to *out (host).  Synchronous;
 * MC_EINVAL for an Ising context or a chain index out of range. */
MC_API mc_status mc_su2_polyakov(mc_ctx *ctx, int32_t chain, double *out);

/* Kernel timing.  While enabled, sweeps are enqueued without CUDA graphs and
 * every launch of a sweep kernel (Ising half-sweep, SU(2) (parity, mu) phase)
 * is bracketed by CUDA events recorded on the context stream. */
MC_API mc_status mc_profile_enable(mc_ctx *ctx, int32_t enable);
/* Number of bracketed launches and their summed duration in milliseconds since
 * the previous read (synchronous; resets the counters). */
MC_API mc_status mc_profile_read(mc_ctx *ctx, int64_t *launches, double *total_ms);

/* Multiply ceiling of the Ising sweep's roofline.  Every attempted flip uses
 * one word of a Philox4x32-10 block (Salmon et al., SC'11, the counter-based
 * generator in place of the paper's RANMAR, Sec. 2.2): 40 32-bit multiplies
 * (the high and low halves of 20 products) per block.  This launches
 * blocks x threads threads that each generate `iters` blocks, counter
 * (thread id, i, TAG_PROBE, 0) under key `seed`, and nothing else; thread id
 * writes the xor of all its words to dev_out[id] (caller-owned, blocks x
 * threads uint32).  Async on cuda_stream; the caller times it (40 x blocks x
 * threads x iters multiplies per launch).  MC_EINVAL unless blocks >= 1 and
 * threads is a multiple of 32 in [32, 256]. */
MC_API mc_status mc_philox_rate(int32_t blocks, int32_t threads, uint32_t iters, uint64_t seed, uint32_t *dev_out,
                                void *cuda_stream);

/* ---- Batched chains in one persistent launch ---------------------------------
 * A group advances every chain of up to 16 contexts (any mix of Ising layouts
 * and SU(2)) with ONE persistent kernel launch per call, replayed from a CUDA
 * graph -- the paper runs independent parameter points side by side (Sec. 3);
 * here they share one GPU.  The grid is a set of thread-block clusters; a
 * host-computed longest-first schedule gives each cluster a list of rounds,
 * each either one large chain split over the cluster's CTAs (phases separated
 * by the hardware cluster barrier) or up to cluster-size small chains, one per
 * CTA.  Results are bit-identical to the contexts' own mc_sweep (same Philox
 * counters), so any configuration may be chosen for speed alone.
 * Member contexts must have been created on the group's stream and stay alive
 * until mc_group_destroy; records go to each member's own ring buffer. */
typedef struct mc_group mc_group; /* opaque, owned by the library */

/* Device workspace the group needs for its schedule and scratch (0 = error). */
MC_API size_t mc_group_workspace_bytes(int32_t n_ctx, mc_ctx *const *ctxs);
MC_API mc_status mc_group_create(mc_group **out, int32_t n_ctx, mc_ctx *const *ctxs, void *workspace,
                                 size_t workspace_bytes, void *cuda_stream);
/* cluster_size in {1, 2, 4, 8, 16} (0 = keep; default 4; 16 is a non-portable
 * cluster size: a device that cannot co-schedule it fails the next
 * mc_group_sweep with MC_ECUDA); threads_per_block a
 * multiple of 32 in [64, 256] (0 = keep; default 256); a chain whose estimated
 * cost (MSC spin-flip units per sweep: Ising int8 2 per site, MSC 1 per site,
 * SU(2) 60 per link) is at least split_cost is shared by a whole cluster
 * (split_cost < 0: one CTA's fair share of the total).  Invalidates the
 * schedule; the next mc_group_sweep recomputes it. */
MC_API mc_status mc_group_configure(mc_group *g, int32_t cluster_size, int32_t threads_per_block, double split_cost);
/* Advance every member chain by n_sweeps (async), recording as mc_sweep does. */
MC_API mc_status mc_group_sweep(mc_group *g, int64_t n_sweeps, int32_t measure_every);
/* Clusters in the launch and rounds in the schedule (0 before the first sweep). */
MC_API mc_status mc_group_schedule(const mc_group *g, int32_t *n_clusters, int32_t *n_rounds);
MC_API mc_status mc_group_destroy(mc_group *g);

/* ---- Learned global proposal ------------------------------------------------
 * Not in the paper: a masked autoregressive convolutional network over Ising
 * spins (variational autoregressive network, Wu, Wang & Zhang, PRL 122 (2019)
 * 080602) -- layer 1 a 5x5 convolution 1 -> 32 channels with mask A, layers
 * 2..depth-1 5x5 convolutions 32 -> 32 with mask B, ReLU after each, the last a
 * 5x5 convolution 32 -> 1 with mask B giving p(s_k = +1 | s_<k) =
 * sigmoid(f_k) in raster order, zero padding -- used as an independence
 * proposal for the chains of an int8-layout Ising context and corrected by
 * Metropolis-Hastings with q_sym(s) = (q(s) + q(-s)) / 2, so the stationary
 * distribution stays that of Eq. (1).  BF16 weights and activations, FP32
 * accumulation (tensor cores for the 32 -> 32 layers), FP64 log q.
 * Parameters cross the ABI as FP32 in the order: for each layer l,
 * W[out][in][5][5] then b[out] (taps outside the mask are ignored). */
typedef struct mc_van mc_van;

MC_API size_t mc_van_param_count(int32_t depth);                          /* 0 if depth not in [3, 7] */
MC_API size_t mc_van_workspace_bytes(int32_t L, int32_t batch, int32_t depth); /* L even, <= 128 */
/* batch = most configurations one call handles (and chains one MH round serves). */
MC_API mc_status mc_van_create(mc_van **out, int32_t L, int32_t batch, int32_t depth, uint64_t seed, void *workspace,
                               size_t workspace_bytes, void *cuda_stream);
MC_API mc_status mc_van_set_params(mc_van *w, const float *host_params, size_t n); /* resets Adam */
/* Parameters (and, if host_grads != NULL, the gradient of the last training step). */
MC_API mc_status mc_van_get_params(mc_van *w, float *host_params, size_t n, float *host_grads);
/* Hidden activations of the last forward pass (log_prob, train_step; not the
 * sampler), for element-wise parity checks of the network: the BF16 output of
 * layer `layer` (0 = the first 1 -> 32 layer, ..., depth - 2 = the last hidden
 * layer), after its ReLU, for the first n configurations of that pass, as raw
 * BF16 bit patterns uint16 [n][L][L][32] into host memory (synchronous).
 * MC_EINVAL for a layer outside [0, depth - 2] or n outside [1, batch]. */
MC_API mc_status mc_van_get_activations(mc_van *w, int32_t layer, int32_t n, uint16_t *host_dst);
/* log q of n device configurations int8 [n][L][L] (or of their global flips if
 * negate) into device doubles (async). */
MC_API mc_status mc_van_log_prob(mc_van *w, const int8_t *dev_spins, int32_t n, int32_t negate, double *dev_logq);
/* Maximum likelihood: loss = -mean log q over n device configurations; forward,
 * backward and (if apply) one Adam step with learning rate lr.  *host_loss (if
 * non-NULL) receives the loss before the step (synchronous then). */
MC_API mc_status mc_van_train_step(mc_van *w, const int8_t *dev_spins, int32_t n, float lr, int32_t apply,
                                   double *host_loss);
/* n autoregressive samples into device int8 [n][L][L] and their log q into
 * device doubles; sample i uses Philox key `seed`, counter (k >> 2, round,
 * TAG_SAMPLE, id_i) word k & 3 for position k, id_i = dev_ids[i] or i.
 * Asynchronous; a device wait of the sampler that reached its limit is
 * reported by the next mc_van_sync (or synchronous train / MH call). */
MC_API mc_status mc_van_sample(mc_van *w, int32_t n, uint32_t round, const uint32_t *dev_ids, int8_t *dev_out,
                               double *dev_logq);
/* One Metropolis-Hastings round for every chain of an int8-layout Ising
 * context (all chains L x L, same stream): sample a proposal per chain, flip it
 * globally with probability 1/2, accept with min(1, e^{-beta dE} q_sym(s) /
 * q_sym(s')) using Philox (0, round, TAG_MH, chain id), write accepted
 * proposals into the chains.  *host_accepted (if non-NULL) receives the number
 * accepted (synchronous then).  The round counter advances by one. */
MC_API mc_status mc_van_mh_round(mc_van *w, mc_ctx *c, int32_t *host_accepted);
MC_API mc_status mc_van_set_round(mc_van *w, uint32_t round);
/* Wait for the network's stream; MC_ETIMEOUT (and the latch cleared) if a
 * bounded device wait of an earlier call on this network gave up. */
MC_API mc_status mc_van_sync(mc_van *w);
MC_API mc_status mc_van_destroy(mc_van *w);
/* Copy every chain of an int8-layout Ising context (all L x L) into / from
 * (back != 0) one contiguous device buffer int8 [n_chains][L][L] (async). */
MC_API mc_status mc_ising_gather(mc_ctx *c, int8_t *dev_buf, int32_t back);

/* Plaquette averages {P, P_s, P_t} (as in mc_record) of an SU(2) link field
 * held by the caller in device memory in the canonical order (float
 * q[s][mu][4], 16-byte aligned), written to three doubles of device memory at
 * `out` on `cuda_stream` (async; NULL = legacy default stream).  The paper has
 * no counterpart: this entry point is for callers that cannot allocate device
 * memory -- a process whose device memory is owned by another allocator (a
 * framework's pool, an arena fixed at start-up), or a monitoring loop that must
 * not enter the CUDA allocator -- so it needs no context or workspace and
 * allocates nothing.  Its partial sums live in a fixed 256 KiB array inside
 * libmc.so, held on every device that loads the library until the process
 * exits; lattices of more than 4,194,304 sites are rejected with MC_EINVAL.
 * The launch and the array are those of the CURRENT device, which must be the
 * device holding `links`, `out` and `cuda_stream`.  The first call on a
 * device, made with that device current, looks up the array's device address
 * and keeps it for the life of the process; make that first call before any
 * stream capture.  A cudaDeviceReset (or anything else that destroys the
 * device's primary context) invalidates the kept address: do not call this
 * entry point on that device afterwards.
 * Every call uses the same array: calls that overlap on the GPU (other
 * streams, other host threads) race and give wrong results. */
MC_API mc_status mc_su2_plaquette_noalloc(const float *links, const int32_t L[4], double *out, void *cuda_stream);

/* Destroy the context (synchronises its stream first; frees graphs). */
MC_API mc_status mc_destroy(mc_ctx *ctx);

/* Message for the last non-OK status returned on this thread. */
MC_API const char *mc_last_error(void);

/* Library version string. */
MC_API const char *mc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MC_H */
