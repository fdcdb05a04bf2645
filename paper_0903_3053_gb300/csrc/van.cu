// van.cu -- the learned global proposal: masked autoregressive conv net
// (forward, backward, Adam), autoregressive sampler, and the symmetrised
// Metropolis-Hastings round over the chains of an Ising context.  See
// van_dev.cuh for the network.  The paper has no learned component.
#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "tc_dev.cuh"
#include "van_dev.cuh"

using bf16 = __nv_bfloat16;

namespace mc {
namespace van {
namespace {

// Per-CTA partial gradient of a hidden layer (13 x 32 x 32 weights + 32 biases)
// and the most CTAs k_dw32_tc is launched with.
constexpr int kDwPart = kTapsB * kCh * kCh + kCh;
constexpr int kMaxDwBlocks = 512;

// ------------------------------------------------------------------ parameters
// Canonical FP32 parameter layout (the same as the FP64 oracle): for each layer
// l, W[o][i][5][5] then b[o]; cin = 1 for l = 0, cout = 1 for l = D - 1.
struct ParamLayout {
    int D;
    size_t w_off[kMaxDepth], b_off[kMaxDepth], total;
};

__host__ __device__ inline int layer_cin(int l) { return l == 0 ? 1 : kCh; }
__host__ __device__ inline int layer_cout(int l, int D) { return l == D - 1 ? 1 : kCh; }

ParamLayout param_layout(int D)
{
    ParamLayout p{};
    p.D = D;
    size_t off = 0;
    for (int l = 0; l < D; ++l) {
        p.w_off[l] = off;
        off += (size_t)layer_cout(l, D) * layer_cin(l) * 25;
        p.b_off[l] = off;
        off += (size_t)layer_cout(l, D);
    }
    p.total = off;
    return p;
}

struct DevParams {
    size_t w_off[kMaxDepth], b_off[kMaxDepth];
    int D;
};

__device__ __forceinline__ size_t canon_w(const DevParams &P, int l, int o, int i, int dy, int dx)
{
    return P.w_off[l] + (((size_t)o * layer_cin(l) + i) * 5 + (dy + 2)) * 5 + (dx + 2);
}

// Kernel-side copies of the weights, rounded to BF16: hidden layers as
// [l][tap][o][c] (BF16), layer 1 as [o][tap] and the last layer as [tap][c]
// (FP32 holding BF16-rounded values), biases FP32.
__global__ void k_prep_weights(const float *p, DevParams P, bf16 *wh, float *w1, float *wD, float *bias)
{
    const int D = P.D;
    const int nh = (D - 2) * kTapsB * kCh * kCh;
    const int total = nh + kCh * kTapsA + kTapsB * kCh + (D - 1) * kCh + 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < nh) {
            const int l = 1 + i / (kTapsB * kCh * kCh), r = i % (kTapsB * kCh * kCh);
            const int t = r / (kCh * kCh), o = (r / kCh) % kCh, c = r % kCh;
            wh[i] = __float2bfloat16(p[canon_w(P, l, o, c, tap_dy(t), tap_dx(t))]);
        } else if (i < nh + kCh * kTapsA) {
            const int r = i - nh, o = r / kTapsA, t = r % kTapsA;
            w1[r] = bf(__float2bfloat16(p[canon_w(P, 0, o, 0, tap_dy(t), tap_dx(t))]));
        } else if (i < nh + kCh * kTapsA + kTapsB * kCh) {
            const int r = i - nh - kCh * kTapsA, t = r / kCh, c = r % kCh;
            wD[r] = bf(__float2bfloat16(p[canon_w(P, D - 1, 0, c, tap_dy(t), tap_dx(t))]));
        } else {
            const int r = i - nh - kCh * kTapsA - kTapsB * kCh; // biases: layers 0..D-2 x 32, then the last
            const int l = r / kCh, o = r % kCh;
            bias[r] = l < D - 1 ? p[P.b_off[l] + o] : p[P.b_off[D - 1]];
        }
    }
}

// ------------------------------------------------------------------ forward
// 32 -> 32 masked convolutions on the fifth-generation tensor cores: implicit
// GEMMs D[q][o] = sum_{t,c} A_t[q][c] W[t][o][c] with tcgen05.mma (M = 128
// positions, N = 32 channels, K = 16, BF16 in, FP32 accumulator in tensor
// memory).  Positions are indexed on a padded grid, q = r P + xp with
// xp = x + 2 and a row pitch P >= L + 4, so that every tap (dy, dx) of output q
// reads input index q + (dy + 2) P + dx of the staged rows y0-2 .. y0+R-1 -- a
// shifted view of the same shared-memory chunk planes (see tc_dev.cuh), zero
// halo columns giving the zero padding.  Outputs on halo columns or past the
// last row are computed and discarded.  One CTA item = R rows of one sample,
// cut into 128-position tiles; tiles are issued 3 at a time by one thread into
// one of two tensor-memory buffers (26 MMAs per tile: 13 taps x 2 k-steps)
// while 4 warps drain the other (tcgen05.ld, bias, ReLU, BF16, stores).
//
// Geometry of the gradient kernel (k_conv32_bwd_tc: P = L + 4, rows staged with
// cp.async by the CTA's threads, `nplanes` chunk planes, two CTAs per SM).
struct TcConvGeom {
    int L, P, R, YB, Qpad, tiles, PL;
    uint32_t plane_bytes, smem_bytes;
};
constexpr uint32_t kTcB = kTapsB * 4 * kCh * 16; // B planes: [tap][chunk][out channel] x 16 bytes
constexpr int kTcGroup = 3;                       // tiles per commit
constexpr uint32_t kTcCols = 256;                 // 2 buffers x 3 tiles x 32 columns, rounded to a power of 2
constexpr int kTcMaxPolls = 1 << 22;              // bounded completion wait

// Rows per CTA item: the R <= 16 whose `nplanes` planes (plus the weights)
// fit two CTAs per SM and that needs the fewest 128-position tiles per sample.
TcConvGeom tc_conv_geom(int L, int nplanes)
{
    TcConvGeom best{};
    long best_tiles = -1;
    for (int R = 1; R <= 16 && R <= L; ++R) {
        TcConvGeom g{};
        g.L = L;
        g.P = L + 4;
        g.R = R;
        g.Qpad = (R * g.P + 127) / 128 * 128;
        g.PL = (g.Qpad + 2 * g.P + 4 + 7) / 8 * 8; // 2-entry guard each side of every tap's view
        g.plane_bytes = (uint32_t)g.PL * 16;
        g.smem_bytes = (uint32_t)nplanes * g.plane_bytes + kTcB + 32;
        g.YB = (L + R - 1) / R;
        g.tiles = g.Qpad / 128;
        if (g.smem_bytes > 110u * 1024)
            continue;
        const long t = (long)g.YB * g.tiles;
        if (best_tiles < 0 || t < best_tiles || (t == best_tiles && R > best.R)) {
            best = g;
            best_tiles = t;
        }
    }
    return best;
}

// Layer 1 (1 -> 32 channels, mask A, ReLU) on the fifth-generation tensor
// cores: one MMA per tile of 128 consecutive positions (M = 128, N = 32,
// K = 16: the 12 taps and 4 zeros).  Each thread builds its position's A row
// from the (negated) spins -- +-1 or 0 outside the lattice, exact in BF16 --
// into two K-major chunk planes; B holds the layer's weights (BF16 values, as
// k_prep_weights leaves them) as [chunk][out channel] rows.  After the MMA each
// thread reads its position's 32 accumulator columns from its tensor-memory
// lane, adds the bias, applies ReLU and stores the 64-byte BF16 row.  Several
// CTAs per SM overlap one another's MMA waits; every wait is bounded and a
// timeout latches *err.
constexpr int kL1Threads = 128;
constexpr uint32_t kL1Cols = 32;

__global__ void __launch_bounds__(kL1Threads, 8) k_layer1_tc(const int8_t *__restrict__ spins, int negate,
                                                             const float *__restrict__ w1, const float *__restrict__ b1,
                                                             bf16 *__restrict__ h1, int n, int L, int *err)
{
    __shared__ __align__(128) uint4 A[2][kL1Threads]; // chunk planes: taps 0-7, taps 8-15
    __shared__ __align__(128) uint4 B[2][kCh];        // chunk planes: [out channel] taps 0-7, 8-15
    __shared__ float Bias[kCh];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid < kCh)
        Bias[tid] = b1[tid];
    if (tid < 2 * kCh) { // w1 is [o][t]
        const int pl = tid / kCh, o = tid % kCh;
        bf16 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int t = 8 * pl + k;
            v[k] = __float2bfloat16(t < kTapsA ? w1[o * kTapsA + t] : 0.f);
        }
        B[pl][o] = *reinterpret_cast<uint4 *>(v);
    }
    const uint32_t bar_s = smem_u32(&bar);
    if (warp == 0)
        tc::tmem_alloc(smem_u32(&tslot), kL1Cols);
    if (tid == 0)
        tc::mbar_init(bar_s, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t *>(&tslot);
    const uint64_t adesc = tc::smem_desc(smem_u32(&A[0][0]), kL1Threads * 16, 128);
    const uint64_t bdesc = tc::smem_desc(smem_u32(&B[0][0]), kCh * 16, 128);
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kCh);
    const long long total = (long long)n * L * L, tiles = (total + kL1Threads - 1) / kL1Threads;
    int ok = 1;
    uint32_t uses = 0;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++uses) {
        const long long p = tile * kL1Threads + tid;
        const bool live = p < total;
        int b = 0, y = 0, x = 0;
        if (live) {
            b = (int)(p / ((long long)L * L));
            const int r = (int)(p - (long long)b * L * L);
            y = r / L;
            x = r - y * L;
        }
        bf16 a[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            float v = 0.f;
            if (t < kTapsA && live) {
                const int yy = y + tap_dy(t), xx = x + tap_dx(t);
                if (yy >= 0 && xx >= 0 && xx < L) {
                    const int s = spins[((size_t)b * L + yy) * L + xx];
                    v = (float)(negate ? -s : s);
                }
            }
            a[t] = __float2bfloat16(v);
        }
        A[0][tid] = *reinterpret_cast<uint4 *>(&a[0]);
        A[1][tid] = *reinterpret_cast<uint4 *>(&a[8]);
        tc::fence_smem_for_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            tc::mma_bf16(tbase, adesc, bdesc, idesc, 0u);
            tc::commit(bar_s);
        }
        if (!__syncthreads_and(tc::mbar_wait(bar_s, uses & 1u, kTcMaxPolls))) { // block-uniform
            ok = 0;
            break;
        }
        tc::fence_after_sync();
        float v[kCh];
        tc::ld_32x32b_x32(tbase + ((uint32_t)(32 * warp) << 16), v);
        if (live) {
            uint4 pk[4];
            uint32_t *pw = reinterpret_cast<uint32_t *>(pk);
#pragma unroll
            for (int c = 0; c < kCh; c += 2) {
                const __nv_bfloat162 h =
                    __floats2bfloat162_rn(fmaxf(v[c] + Bias[c], 0.f), fmaxf(v[c + 1] + Bias[c + 1], 0.f));
                pw[c / 2] = *reinterpret_cast<const uint32_t *>(&h);
            }
            uint4 *dst = reinterpret_cast<uint4 *>(h1 + (size_t)p * kCh);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                dst[k] = pk[k];
        }
        tc::fence_before_sync(); // this tile's tensor-memory reads precede the next MMA
    }
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0)
        atomicExch(err, 1);
    tc::fence_after_sync();
    if (warp == 0)
        tc::tmem_free(tbase, kL1Cols);
}

// ---------------------------------------------------------------- TMA-pipelined forward convolution
// out = ReLU(conv(in) + bias).  The staging is taken off the threads and the
// three stages of an item overlap across items: warp 4 streams the
// input rows of the next item by TMA (one box of all 32 channels: R + 2 rows of
// P positions from x = -2, everything outside the lattice arriving zero-filled,
// 64-byte rows in the 64-byte swizzle, which the MMA reads through swizzled
// descriptors -- a tap is still an offset of whole rows) into the second of two
// stage buffers, one thread of warp 5 issues the MMAs of the current item, and warps
// 0-3 drain tensor memory (bias, ReLU, BF16, stores).  They hand over through
// mbarriers: stage full (TMA bytes), stage free (MMA commit), accumulator full
// (MMA commit) and accumulator free (epilogue arrivals); every wait is bounded
// and a timeout latches MC_ETIMEOUT.  Every TMA destination starts on a
// 1024-byte boundary.  Two CTAs of 6 warps per SM (stages of at most 110 KB,
// so fewer rows per item) where that costs at most 15% more tiles than one CTA
// with 200 KB: the other CTA's MMAs fill one CTA's pipeline gaps (L = 64,
// batch 4096: 4.94 against 5.95 ms per forward pass); else one.
struct TmaConvGeom {
    int L, P, R, YB, Qpad, tiles, PL, ctas_per_sm;
    uint32_t plane_bytes, stage_bytes, smem_bytes;
};
constexpr int kTmaGuard = 16;                  // positions ahead of staged row 0 (>= 2; 16 x 64 bytes = one
                                               // 1024-byte boundary, so that the TMA box lands swizzle-aligned)
constexpr uint32_t kTmaMaxSmem1 = 200u * 1024; // two stages + weights + barriers, one CTA per SM
constexpr uint32_t kTmaMaxSmem2 = 110u * 1024; // the same, two CTAs per SM
constexpr uint32_t kTmaBarBytes = 128;         // 9 mbarriers, tensor-memory slot

// Rows per item: the R whose two stages fit `max_smem` and that needs the
// fewest 128-position tiles per sample.
TmaConvGeom tma_conv_geom_cap(int L, uint32_t max_smem)
{
    TmaConvGeom best{};
    long best_tiles = -1;
    for (int R = 1; R <= 32 && R <= L; ++R) {
        TmaConvGeom g{};
        g.L = L;
        g.P = (L + 4 + 7) / 8 * 8;
        g.R = R;
        g.Qpad = (R * g.P + 127) / 128 * 128;
        g.PL = (kTmaGuard + 2 * g.P + g.Qpad + 15) / 16 * 16; // whole 1024-byte swizzle spans
        g.plane_bytes = (uint32_t)g.PL * 64;                 // 64 bytes (32 channels) per position
        g.stage_bytes = g.plane_bytes;
        g.smem_bytes = 2 * g.stage_bytes + kTcB + kTmaBarBytes + 1024; // + alignment slack
        g.YB = (L + R - 1) / R;
        g.tiles = g.Qpad / 128;
        if (g.smem_bytes > max_smem)
            continue;
        const long t = (long)g.YB * g.tiles;
        if (best_tiles < 0 || t < best_tiles || (t == best_tiles && R > best.R)) {
            best = g;
            best_tiles = t;
        }
    }
    return best;
}

TmaConvGeom tma_conv_geom(int L)
{
    TmaConvGeom one = tma_conv_geom_cap(L, kTmaMaxSmem1), two = tma_conv_geom_cap(L, kTmaMaxSmem2);
    one.ctas_per_sm = 1;
    two.ctas_per_sm = 2;
    const long t1 = (long)one.YB * one.tiles, t2 = (long)two.YB * two.tiles;
    return two.R > 0 && 100 * t2 <= 115 * t1 ? two : one;
}

// The last layer (32 -> 1) on the same pipeline: B has N = 16 rows (the
// smallest tile of an M = 128 MMA), the layer's weights -- BF16 values, as
// k_prep_weights leaves them -- in row 0 and zeros elsewhere, so that the
// logit is f = D[p][0] + b; the epilogue forms f, log sigmoid(s f) and
// (training) dF = -(1/n) s sigmoid(-s f) per position.
struct LastLayerArgs {
    const float *wD; // [t][c], BF16-representable
    const float *bD; // the layer's bias (one value)
    const int8_t *spins;
    int negate;
    float *f, *ll, *dF; // dF may be null
    float inv_n;
};

template <int MINB, bool LAST>
__global__ void __launch_bounds__(192, MINB) k_conv32_tma(const __grid_constant__ CUtensorMap in_map,
                                                       bf16 *__restrict__ out, const bf16 *__restrict__ W,
                                                       const float *__restrict__ bias, LastLayerArgs la, int n,
                                                       TmaConvGeom g, int *err)
{
    constexpr int NB = LAST ? 16 : kCh; // output columns of the MMA
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the stages hold 64-byte-swizzled rows: round the base up to 1024 bytes
    // (the launch reserves 1024 extra bytes)
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sb = smem_u32(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t boff = 2 * g.stage_bytes, bars = boff + kTcB;
    const uint32_t full0 = sb + bars, empty0 = full0 + 16, tfull0 = full0 + 32, tempty0 = full0 + 48,
                   drain = full0 + 64, tslot_off = bars + 80;
    for (uint32_t i = tid; i < 2 * g.stage_bytes / 16; i += blockDim.x) // padding columns and guards stay zero
        reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (LAST) {
        for (int i = tid; i < kTapsB * 4 * NB; i += blockDim.x) { // [t][c8][row]: row 0 the weights
            const int t = i / (4 * NB), c8 = (i / NB) % 4, o = i % NB;
            bf16 v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                v[k] = __float2bfloat16(o == 0 ? la.wD[t * kCh + c8 * 8 + k] : 0.f);
            *reinterpret_cast<uint4 *>(smem + boff + ((t * 4 + c8) * NB + o) * 16) = *reinterpret_cast<uint4 *>(v);
        }
    } else {
        for (int i = tid; i < kTapsB * kCh * 4; i += blockDim.x) {
            const int t = i / (kCh * 4), o = (i / 4) % kCh, c8 = i % 4;
            *reinterpret_cast<uint4 *>(smem + boff + ((t * 4 + c8) * kCh + o) * 16) =
                *reinterpret_cast<const uint4 *>(W + ((size_t)(t * kCh + o) * kCh + c8 * 8));
        }
    }
    if (warp == 0)
        tc::tmem_alloc(sb + tslot_off, kTcCols);
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            tc::mbar_init(full0 + 8 * k, 1);
            tc::mbar_init(empty0 + 8 * k, 1);
            tc::mbar_init(tfull0 + 8 * k, 1);
            tc::mbar_init(tempty0 + 8 * k, 4);
        }
        tc::mbar_init(drain, 1);
    }
    tc::fence_smem_for_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t *>(smem + tslot_off);
    const int total = n * g.YB, rounds = (g.tiles + kTcGroup - 1) / kTcGroup;
    int ok = 1;
    if (warp == 4) {
        if (lane == 0) { // producer
            const uint32_t bytes = (uint32_t)(g.R + 2) * (uint32_t)g.P * 64u;
            int k = 0, armed[2] = {-1, -1};
            for (int it = blockIdx.x; it < total; it += gridDim.x, ++k) {
                const int s = k & 1;
                if (k >= 2 && !tc::mbar_wait(empty0 + 8 * s, ((k >> 1) - 1) & 1, kTcMaxPolls)) {
                    ok = 0;
                    break;
                }
                const int b = it / g.YB, y0 = (it - b * g.YB) * g.R;
                tc::mbar_arrive_expect_tx(full0 + 8 * s, bytes);
                const uint32_t st = sb + (uint32_t)s * g.stage_bytes;
                // rows y0-2 .. y0+R-1, columns -2 .. P-3, all 32 channels: one box
                tc::tma_load_5d(st + (uint32_t)kTmaGuard * 64u, &in_map, 0, 0, -2, y0 - 2, b, full0 + 8 * s);
                armed[s] = k;
            }
            for (int s = 0; s < 2; ++s) // the last loads of each stage have landed before the CTA ends
                if (armed[s] >= 0 && !tc::mbar_wait(full0 + 8 * s, (armed[s] >> 1) & 1, kTcMaxPolls))
                    ok = 0;
        }
    } else if (warp == 5) {
        if (lane == 0) { // MMA issuer
            const uint32_t idesc = tc::idesc_bf16_f32(128, NB);
            uint64_t adesc[kTapsB * 2], bdesc[kTapsB * 2];
            for (int t = 0; t < kTapsB; ++t)
                for (int kc = 0; kc < 2; ++kc) {
                    adesc[t * 2 + kc] = tc::smem_desc_sw64(
                        sb + (uint32_t)(kTmaGuard + (tap_dy(t) + 2) * g.P + tap_dx(t)) * 64u + (uint32_t)kc * 32u);
                    bdesc[t * 2 + kc] = tc::smem_desc(sb + boff + (uint32_t)(t * 4 + 2 * kc) * (NB * 16), NB * 16, 128);
                }
            uint32_t tcount = 0;
            int k = 0;
            for (int it = blockIdx.x; ok && it < total; it += gridDim.x, ++k) {
                const int s = k & 1;
                if (!tc::mbar_wait(full0 + 8 * s, (k >> 1) & 1, kTcMaxPolls)) {
                    ok = 0;
                    break;
                }
                tc::fence_after_sync();
                const uint64_t soff = (uint64_t)(((uint32_t)s * g.stage_bytes) >> 4);
                for (int rd = 0; rd < rounds; ++rd, ++tcount) {
                    const uint32_t bb = tcount & 1u;
                    if (tcount >= 2 && !tc::mbar_wait(tempty0 + 8 * bb, ((tcount >> 1) - 1) & 1u, kTcMaxPolls)) {
                        ok = 0;
                        break;
                    }
                    tc::fence_after_sync();
                    const int m0 = rd * kTcGroup, m1 = m0 + kTcGroup < g.tiles ? m0 + kTcGroup : g.tiles;
                    for (int m = m0; m < m1; ++m) {
                        const uint32_t d = tbase + (bb * kTcGroup + (uint32_t)(m - m0)) * NB;
                        const uint64_t off = soff + (uint64_t)((uint32_t)m * 128u * 4u); // 128 positions x 64 B
#pragma unroll
                        for (int j = 0; j < kTapsB * 2; ++j)
                            tc::mma_bf16(d, adesc[j] + off, bdesc[j], idesc, j != 0);
                    }
                    tc::commit(tfull0 + 8 * bb);
                }
                if (!ok)
                    break;
                tc::commit(empty0 + 8 * s); // stage s is free once this item's MMAs have read it
            }
            tc::commit(drain); // every MMA issued above has completed before the CTA ends
            if (!tc::mbar_wait(drain, 0u, kTcMaxPolls))
                ok = 0;
        }
    } else { // warps 0-3: epilogue, tensor-memory lanes 32 warp .. 32 warp + 31
        float bv[kCh];
#pragma unroll
        for (int c = 0; c < kCh; ++c)
            bv[c] = LAST ? 0.f : __ldg(&bias[c]);
        const float b0 = LAST ? __ldg(la.bD) : 0.f;
        uint32_t tcount = 0;
        for (int it = blockIdx.x; ok && it < total; it += gridDim.x) {
            const int b = it / g.YB, y0 = (it - b * g.YB) * g.R;
            for (int rd = 0; rd < rounds; ++rd, ++tcount) {
                const uint32_t bb = tcount & 1u;
                const bool got =
                    __any_sync(0xffffffffu, tc::mbar_wait(tfull0 + 8 * bb, (tcount >> 1) & 1u, kTcMaxPolls));
                tc::fence_after_sync();
                if (!got) {
                    ok = 0;
                    break;
                }
                const int m0 = rd * kTcGroup, m1 = m0 + kTcGroup < g.tiles ? m0 + kTcGroup : g.tiles;
                for (int m = m0; m < m1; ++m) {
                    const uint32_t col = tbase + ((uint32_t)(32 * warp) << 16) + (bb * kTcGroup + (uint32_t)(m - m0)) * NB;
                    const int q = m * 128 + 32 * warp + lane, r = q / g.P, xp = q - r * g.P;
                    if (LAST) {
                        const float acc = tc::ld_32x32b_x1(col);
                        if (r < g.R && y0 + r < g.L && xp >= 2 && xp < g.L + 2) {
                            const size_t p = ((size_t)b * g.L + y0 + r) * g.L + (xp - 2);
                            const float fv = b0 + acc;
                            const float sv = la.negate ? -(float)la.spins[p] : (float)la.spins[p];
                            la.f[p] = fv;
                            la.ll[p] = log_sigmoid(sv * fv);
                            if (la.dF)
                                la.dF[p] = -la.inv_n * sv * sigmoid(-sv * fv);
                        }
                        continue;
                    }
                    float v[kCh];
                    tc::ld_32x32b_x32(col, v);
                    if (r < g.R && y0 + r < g.L && xp >= 2 && xp < g.L + 2) {
                        uint4 pk[4];
                        uint32_t *pw = reinterpret_cast<uint32_t *>(pk);
#pragma unroll
                        for (int c = 0; c < kCh; c += 2) {
                            const __nv_bfloat162 h =
                                __floats2bfloat162_rn(fmaxf(v[c] + bv[c], 0.f), fmaxf(v[c + 1] + bv[c + 1], 0.f));
                            pw[c / 2] = *reinterpret_cast<const uint32_t *>(&h);
                        }
                        uint4 *dst = reinterpret_cast<uint4 *>(out + (((size_t)b * g.L + y0 + r) * g.L + (xp - 2)) * kCh);
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            dst[k] = pk[k];
                    }
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0)
                    tc::mbar_arrive(tempty0 + 8 * bb);
            }
        }
    }
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0)
        atomicExch(err, 1);
    tc::fence_after_sync();
    if (warp == 0)
        tc::tmem_free(tbase, kTcCols);
}

// Encoder of tensor maps, from the driver through the runtime (no link
// dependency on the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Activations [n][L][L][32] BF16 as a 5-D tensor (32 channels, 1, x, y,
// sample); one box is R + 2 rows of P positions from x = -2, all channels: it
// lands in shared memory as 64-byte rows in the 64-byte swizzle, the columns
// outside the lattice zero-filled.
cudaError_t activation_map(CUtensorMap *m, const bf16 *base, int n, int L, int P, int rows)
{
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc)
        return cudaErrorNotSupported;
    const cuuint64_t dims[5] = {32, 1, (cuuint64_t)L, (cuuint64_t)L, (cuuint64_t)n};
    const cuuint64_t strides[4] = {64, 64, (cuuint64_t)64 * L, (cuuint64_t)64 * L * L};
    const cuuint32_t box[5] = {32, 1, (cuuint32_t)P, (cuuint32_t)rows, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16 *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Gradients travel between the backward kernels as a BF16 hi + lo pair
// (hi = bf16(v), lo = bf16(v - hi), ~16 mantissa bits): two [n][L][L][32] BF16
// arrays in the space of one FP32 array, which the tensor cores read directly.
__device__ __forceinline__ void split8(const float *v, uint4 &hi, uint4 &lo)
{
    bf16 h[8], l[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        h[k] = __float2bfloat16(v[k]);
        l[k] = __float2bfloat16(v[k] - bf(h[k]));
    }
    hi = *reinterpret_cast<uint4 *>(h);
    lo = *reinterpret_cast<uint4 *>(l);
}

// Gradient with respect to a 32 -> 32 layer's input, masked by the previous
// layer's ReLU, on the fifth-generation tensor cores:
//   out(p)[c] = [mask(p)[c] > 0] sum_t sum_o W[t][o][c] dz(p - d_t)[o].
// Same padded-position implicit GEMM as the forward kernel with the taps negated
// (rows y0 .. y0+R+1 staged) and the weights transposed into the B planes;
// dz arrives as hi + lo (8 A planes) and each k step issues two MMAs into
// the same FP32 accumulator; the masked result leaves as hi + lo.
constexpr int kTcBwdGroup = 2;
constexpr uint32_t kTcBwdCols = 128;

__global__ void __launch_bounds__(128, 2) k_conv32_bwd_tc(const bf16 *__restrict__ dzh, const bf16 *__restrict__ dzl,
                                                          bf16 *__restrict__ outh, bf16 *__restrict__ outl,
                                                          const bf16 *__restrict__ W, const bf16 *__restrict__ mask,
                                                          int n, TcConvGeom g, int *err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t sb = smem_u32(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t abytes = 8 * g.plane_bytes; // planes 0-3: hi, 4-7: lo
    const uint32_t boff = abytes, bar0 = sb + boff + kTcB, tslot_off = boff + kTcB + 16;
    for (uint32_t i = tid; i < abytes / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid; i < kTapsB * 4 * kCh; i += blockDim.x) { // B planes [t][o8][c] = W[t][8 o8 .. +7][c]
        const int t = i / (4 * kCh), o8 = (i / kCh) % 4, c = i % kCh;
        bf16 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            v[k] = W[((size_t)t * kCh + o8 * 8 + k) * kCh + c];
        *reinterpret_cast<uint4 *>(smem + boff + ((t * 4 + o8) * kCh + c) * 16) = *reinterpret_cast<uint4 *>(v);
    }
    if (warp == 0)
        tc::tmem_alloc(sb + tslot_off, kTcBwdCols);
    if (tid == 0) {
        tc::mbar_init(bar0, 1);
        tc::mbar_init(bar0 + 8, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t *>(smem + tslot_off);
    const uint32_t idesc = tc::idesc_bf16_f32(128, kCh);
    uint64_t adesc[kTapsB * 2], bdesc[kTapsB * 2];
    if (tid == 0)
        for (int t = 0; t < kTapsB; ++t)
            for (int kc = 0; kc < 2; ++kc) {
                adesc[t * 2 + kc] = tc::smem_desc(sb + (uint32_t)(2 * kc) * g.plane_bytes +
                                                      (uint32_t)(2 - tap_dy(t) * g.P - tap_dx(t)) * 16u,
                                                  g.plane_bytes, 128);
                bdesc[t * 2 + kc] = tc::smem_desc(sb + boff + (uint32_t)(t * 4 + 2 * kc) * (kCh * 16), kCh * 16, 128);
            }
    const uint64_t lo_off = (uint64_t)((4u * g.plane_bytes) >> 4);
    const int rounds = (g.tiles + kTcBwdGroup - 1) / kTcBwdGroup;
    auto issue = [&](int rd) {
        const int m0 = rd * kTcBwdGroup, m1 = m0 + kTcBwdGroup < g.tiles ? m0 + kTcBwdGroup : g.tiles;
        for (int m = m0; m < m1; ++m) {
            const uint32_t d = tbase + (uint32_t)((rd & 1) * kTcBwdGroup + (m - m0)) * kCh;
            const uint64_t off = (uint64_t)((uint32_t)m * 128u);
#pragma unroll
            for (int j = 0; j < kTapsB * 2; ++j) {
                tc::mma_bf16(d, adesc[j] + off, bdesc[j], idesc, j != 0);
                tc::mma_bf16(d, adesc[j] + off + lo_off, bdesc[j], idesc, 1u);
            }
        }
        tc::commit(bar0 + 8u * (uint32_t)(rd & 1));
    };
    uint32_t uses[2] = {0u, 0u};
    int ok = 1;
    for (int it = blockIdx.x; ok && it < n * g.YB; it += gridDim.x) {
        const int b = it / g.YB, y0 = (it - b * g.YB) * g.R;
        for (int i = tid; i < (g.R + 2) * g.L * 8; i += blockDim.x) { // rows y0 .. y0+R+1, hi and lo
            const int rho = i / (g.L * 8), rem = i - rho * g.L * 8, x = rem >> 3, pl = rem & 7, yy = y0 + rho;
            const bool inside = yy < g.L;
            const bf16 *src = (pl < 4 ? dzh : dzl) + (((size_t)b * g.L + (inside ? yy : 0)) * g.L + x) * kCh + (pl & 3) * 8;
            const uint32_t dst = sb + (uint32_t)pl * g.plane_bytes + (uint32_t)(4 + rho * g.P + x) * 16u;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(inside ? 16 : 0)
                         : "memory");
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        tc::fence_smem_for_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0)
            issue(0);
        for (int rd = 0; rd < rounds; ++rd) {
            if (tid == 0 && rd + 1 < rounds)
                issue(rd + 1);
            const int s = rd & 1;
            const bool got = tc::mbar_wait(bar0 + 8u * s, uses[s] & 1u, kTcMaxPolls);
            ++uses[s];
            tc::fence_after_sync();
            const int m0 = rd * kTcBwdGroup, m1 = m0 + kTcBwdGroup < g.tiles ? m0 + kTcBwdGroup : g.tiles;
            for (int m = m0; m < m1; ++m) {
                float v[kCh];
                tc::ld_32x32b_x32(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(s * kTcBwdGroup + (m - m0)) * kCh,
                                  v);
                const int q = m * 128 + 32 * warp + lane, r = q / g.P, xp = q - r * g.P;
                if (got && r < g.R && y0 + r < g.L && xp >= 2 && xp < g.L + 2) {
                    const size_t p = ((size_t)b * g.L + y0 + r) * g.L + (xp - 2);
                    const uint4 *mk = reinterpret_cast<const uint4 *>(mask + p * kCh);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint4 mv = mk[k];
                        const bf16 *m8 = reinterpret_cast<const bf16 *>(&mv);
                        float o[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            o[j] = bf(m8[j]) > 0.f ? v[8 * k + j] : 0.f;
                        uint4 hi, lo;
                        split8(o, hi, lo);
                        reinterpret_cast<uint4 *>(outh + p * kCh)[k] = hi;
                        reinterpret_cast<uint4 *>(outl + p * kCh)[k] = lo;
                    }
                }
            }
            tc::fence_before_sync();
            ok = __syncthreads_and(ok && got);
            tc::fence_after_sync();
            if (!ok)
                break;
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (!ok && tid == 0)
        atomicExch(err, 1);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0)
        tc::tmem_free(tbase, kTcBwdCols);
}

// Stage rows y-2..y of a [n][L][L][32] BF16 activation into smem rows of L+4
// positions (x offset 2, zero padded), 16-byte chunks.
__device__ __forceinline__ void stage_rows3(bf16 (*H)[(kMaxL + 4) * kCh], const bf16 *src, int b, int y, int L)
{
    for (int i = threadIdx.x; i < 3 * (L + 4) * 4; i += blockDim.x) {
        const int r = i / ((L + 4) * 4), rem = i - r * (L + 4) * 4, xx = rem / 4 - 2, ch = rem & 3, yy = y - 2 + r;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (yy >= 0 && xx >= 0 && xx < L)
            v = *reinterpret_cast<const uint4 *>(src + (((size_t)b * L + yy) * L + xx) * kCh + ch * 8);
        *reinterpret_cast<uint4 *>(&H[r][(xx + 2) * kCh + ch * 8]) = v;
    }
}

// log q per sample: fixed-order FP64 sum of its L^2 log-probabilities.
__global__ void k_logq(const float *ll, double *logq, int L)
{
    __shared__ double part[32];
    const int b = blockIdx.x, n = L * L;
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        acc += (double)ll[(size_t)b * n + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0)
        part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            s += part[w];
        logq[b] = s;
    }
}

// ------------------------------------------------------------------ backward
// Last layer: dZ_{D-1}(p)[c] = (sum_t wD[t][c] dF(p - d_t)) * [h_{D-1}(p)[c] > 0]
// (the forward read h at q + d_t for output q).  One CTA item = one row: dF of
// rows y..y+2 staged in smem (zero padded); 4 threads per position.
__global__ void __launch_bounds__(256) k_layerD_bwd_data(const float *dF, const float *wD, const bf16 *hD,
                                                         bf16 *dzh, bf16 *dzl, int n, int L)
{
    __shared__ float W[kTapsB * kCh];
    __shared__ float G[3][kMaxL + 4];
    const int tid = threadIdx.x;
    for (int i = tid; i < kTapsB * kCh; i += blockDim.x)
        W[i] = wD[i];
    for (int item = blockIdx.x; item < n * L; item += gridDim.x) {
        const int b = item / L, y = item - b * L;
        __syncthreads();
        for (int i = tid; i < 3 * (L + 4); i += blockDim.x) {
            const int r = i / (L + 4), xx = i - r * (L + 4) - 2, yy = y + r;
            G[r][xx + 2] = (yy < L && xx >= 0 && xx < L) ? dF[((size_t)b * L + yy) * L + xx] : 0.f;
        }
        __syncthreads();
        for (int j = tid; j < L * 4; j += blockDim.x) {
            const int x = j >> 2, c0 = (j & 3) * 8;
            float acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                acc[q] = 0.f;
#pragma unroll
            for (int t = 0; t < kTapsB; ++t) {
                const float gv = G[-tap_dy(t)][x - tap_dx(t) + 2];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    acc[q] += W[t * kCh + c0 + q] * gv;
            }
            const size_t p = ((size_t)b * L + y) * L + x;
            const uint4 hv = *reinterpret_cast<const uint4 *>(hD + p * kCh + c0);
            const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&hv);
            float o[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                o[2 * q] = bf(h2[q].x) > 0.f ? acc[2 * q] : 0.f;
                o[2 * q + 1] = bf(h2[q].y) > 0.f ? acc[2 * q + 1] : 0.f;
            }
            uint4 hi, lo;
            split8(o, hi, lo);
            *reinterpret_cast<uint4 *>(dzh + p * kCh + c0) = hi;
            *reinterpret_cast<uint4 *>(dzl + p * kCh + c0) = lo;
        }
    }
}

// Last-layer weight and bias gradients: gW[t][c] = sum_p dF(p) h(p + d_t)[c],
// gb = sum_p dF(p).  One CTA item = one row, staged in smem.  Lane c of warp w
// accumulates the 13 tap outputs of channel c (and the bias) over its segment
// w of every row, the tap activations held in a window of registers that
// slides along x (3 shared-memory loads per position); at the end the 8
// segment warps are added in warp order and the CTA writes its partial sums to
// part[output][CTA] (summed in a fixed order by k_edge_grad_reduce: the
// gradient does not depend on the order the CTAs finish in).
constexpr int kEdgeOutD = kTapsB * kCh + 1;  // last layer: 13 x 32 weights + bias
constexpr int kEdgeOut1 = kCh * (kTapsA + 1); // first layer: 32 x (12 weights + bias)
__global__ void __launch_bounds__(256) k_layerD_bwd_w(const float *dF, const bf16 *hD, float *part, int n, int L)
{
    __shared__ float Gs[kMaxL];
    __shared__ __align__(16) bf16 H[3][(kMaxL + 4) * kCh];
    __shared__ float R[8][kEdgeOutD];
    const int tid = threadIdx.x, c = tid & 31, seg = tid >> 5;
    const int seg_len = (L + 7) / 8, x0 = seg * seg_len, x1 = min(x0 + seg_len, L);
    float acc[kTapsB + 1];
#pragma unroll
    for (int t = 0; t <= kTapsB; ++t)
        acc[t] = 0.f;
    for (int item = blockIdx.x; item < n * L; item += gridDim.x) {
        const int b = item / L, y = item - b * L;
        __syncthreads();
        stage_rows3(H, hD, b, y, L);
        for (int x = tid; x < L; x += blockDim.x)
            Gs[x] = dF[((size_t)b * L + y) * L + x];
        __syncthreads();
        if (x0 < x1) {
            // taps 0-4: row y-2 at x - 2 .. x + 2; 5-9: row y-1; 10-12: row y at x - 2 .. x (mask B)
            float w0[5], w1[5], w2[3];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                w0[k + 1] = bf(H[0][(x0 + k) * kCh + c]);
                w1[k + 1] = bf(H[1][(x0 + k) * kCh + c]);
            }
            w2[1] = bf(H[2][x0 * kCh + c]);
            w2[2] = bf(H[2][(x0 + 1) * kCh + c]);
            for (int x = x0; x < x1; ++x) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    w0[k] = w0[k + 1];
                    w1[k] = w1[k + 1];
                }
                w0[4] = bf(H[0][(x + 4) * kCh + c]);
                w1[4] = bf(H[1][(x + 4) * kCh + c]);
                w2[0] = w2[1];
                w2[1] = w2[2];
                w2[2] = bf(H[2][(x + 2) * kCh + c]);
                const float gf = Gs[x];
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    acc[k] += gf * w0[k];
                    acc[5 + k] += gf * w1[k];
                }
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    acc[10 + k] += gf * w2[k];
                acc[13] += gf;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kTapsB; ++t)
        R[seg][t * kCh + c] = acc[t];
    if (c == 0)
        R[seg][kTapsB * kCh] = acc[kTapsB];
    __syncthreads();
    for (int o = tid; o < kEdgeOutD; o += blockDim.x) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w)
            v += R[w][o];
        part[(size_t)o * gridDim.x + blockIdx.x] = v;
    }
}

// Gradient of the first (FIRST) or last layer: one CTA per output adds its
// nb per-CTA partial sums (part[output][CTA]) in a fixed order -- strided
// per-thread sums, then a fixed shuffle and shared-memory tree -- and writes
// the canonical parameter.
template <bool FIRST>
__global__ void __launch_bounds__(256) k_edge_grad_reduce(const float *part, int nb, float *g, DevParams P)
{
    __shared__ float ws[8];
    const int o = blockIdx.x, tid = threadIdx.x;
    float v = 0.f;
    for (int b = tid; b < nb; b += blockDim.x)
        v += part[(size_t)o * nb + b];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, d);
    if ((tid & 31) == 0)
        ws[tid >> 5] = v;
    __syncthreads();
    if (tid != 0)
        return;
    v = ((ws[0] + ws[1]) + (ws[2] + ws[3])) + ((ws[4] + ws[5]) + (ws[6] + ws[7]));
    if (FIRST) {
        const int oc = o / (kTapsA + 1), t = o - oc * (kTapsA + 1);
        g[t < kTapsA ? canon_w(P, 0, oc, 0, tap_dy(t), tap_dx(t)) : P.b_off[0] + oc] = v;
    } else {
        const int t = o / kCh, c = o - t * kCh;
        g[t < kTapsB ? canon_w(P, P.D - 1, 0, c, tap_dy(t), tap_dx(t)) : P.b_off[P.D - 1]] = v;
    }
}

// Weight gradient of a 32 -> 32 layer on the fifth-generation tensor cores:
//   dW[t][o][c] = sum_(b, y, x) dz(b, y, x)[o] X(b, y + dy_t, x + dx_t)[c],
//   db[o] = sum_(b, y, x) dz(b, y, x)[o],
// dz as its BF16 hi + lo pair.  One item is one row (b, y): its dz hi and lo
// rows and the input rows y-2 .. y (columns -2 .. PX-3, zero outside the
// lattice) arrive by TMA in the 64-byte swizzle, and the positions of the row
// are the reduction dimension K.  Both operands are read MN-major.  A = the
// input rows, whose M dimension takes four taps at once: the taps (dy, dx ..
// dx+3) of one kernel row are the same staged row shifted by one position,
// i.e. 32-channel atoms 64 bytes apart (the descriptor's leading offset), and
// taps (-2, 2), (-1, 2) are one staged row apart (M = 64).  B = dz (N = 64: 32
// columns of hi, then 32 of lo, the lo plane one descriptor stride away).  The
// 13 taps are four MMAs per 16 positions (M = 128, 128, 128 with one unused
// tap, 64), accumulated in 256 tensor-memory columns over all items of the
// CTA; tensor-memory lane (tap, c) then holds the hi and the lo sums of
// channel c, added in the drain.  Roles: warp 4 loads (ring of NS stages),
// warp 5 issues, warps 0-3 sum the bias gradient from the staged dz rows and
// drain the accumulator.  Per-CTA partial sums [t][o][c] then the 32 biases,
// reduced in CTA order by k_dw_reduce.  Two CTAs per SM, so that one's MMAs
// fill the other's gaps.  Every wait is bounded; a timeout latches *err.
struct DwTcGeom {
    int L, PZ, PX, KS, NS;
    uint32_t zbytes, xbytes, stage_bytes, smem_bytes;
};
constexpr uint32_t kDwTcAlloc = 256;       // tensor-memory columns: 4 tap groups x (32 hi + 32 lo)
constexpr uint32_t kDwTcMaxSmem = 110u * 1024;
constexpr int kDwTcMaxStages = 6;

DwTcGeom dw_tc_geom(int L)
{
    DwTcGeom g{};
    g.L = L;
    g.PZ = (L + 15) / 16 * 16;
    g.PX = (g.PZ + 4 + 7) / 8 * 8;
    g.KS = g.PZ / 16;
    g.zbytes = (uint32_t)g.PZ * 64u;
    g.xbytes = ((uint32_t)(3 * g.PX) * 64u + 1023u) / 1024u * 1024u;
    g.stage_bytes = 2 * g.zbytes + g.xbytes;
    const uint32_t extra = 256 + 512 + 1024; // barriers and tensor-memory slot, bias sums, alignment slack
    g.NS = (int)std::min<uint32_t>(kDwTcMaxStages, (kDwTcMaxSmem - extra) / g.stage_bytes);
    g.smem_bytes = (uint32_t)g.NS * g.stage_bytes + extra;
    return g;
}

__global__ void __launch_bounds__(192, 2) k_dw32_tc(const __grid_constant__ CUtensorMap zh_map,
                                                    const __grid_constant__ CUtensorMap zl_map,
                                                    const __grid_constant__ CUtensorMap x_map, float *__restrict__ part,
                                                    int n, DwTcGeom g, int *err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sb = smem_u32(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, NS = g.NS;
    const uint32_t ring = (uint32_t)NS * g.stage_bytes;
    const uint32_t full0 = sb + ring, empty0 = full0 + 8 * kDwTcMaxStages, done = empty0 + 8 * kDwTcMaxStages,
                   tslot_off = ring + 16 * kDwTcMaxStages + 8;
    float *bsum_s = reinterpret_cast<float *>(smem + ring + 256); // [4][32]
    if (warp == 0)
        tc::tmem_alloc(sb + tslot_off, kDwTcAlloc);
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(full0 + 8 * s, 1);
            tc::mbar_init(empty0 + 8 * s, 5); // the MMA commit and the four bias warps
        }
        tc::mbar_init(done, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t *>(smem + tslot_off);
    const int total = n * g.L;
    int ok = 1;
    if (warp == 4) {
        if (lane == 0) { // producer
            const uint32_t bytes = 2 * g.zbytes + (uint32_t)(3 * g.PX) * 64u;
            int k = 0, armed[kDwTcMaxStages];
            for (int s = 0; s < kDwTcMaxStages; ++s)
                armed[s] = -1;
            for (int it = blockIdx.x; it < total; it += gridDim.x, ++k) {
                const int s = k % NS, use = k / NS;
                if (use >= 1 && !tc::mbar_wait(empty0 + 8 * s, (use - 1) & 1, kTcMaxPolls)) {
                    ok = 0;
                    break;
                }
                const int b = it / g.L, y = it - b * g.L;
                const uint32_t st = sb + (uint32_t)s * g.stage_bytes;
                tc::mbar_arrive_expect_tx(full0 + 8 * s, bytes);
                tc::tma_load_5d(st, &zh_map, 0, 0, 0, y, b, full0 + 8 * s);
                tc::tma_load_5d(st + g.zbytes, &zl_map, 0, 0, 0, y, b, full0 + 8 * s);
                tc::tma_load_5d(st + 2 * g.zbytes, &x_map, 0, 0, -2, y - 2, b, full0 + 8 * s);
                armed[s] = use;
            }
            for (int s = 0; s < NS; ++s) // the last loads of each stage have landed before the CTA ends
                if (armed[s] >= 0 && !tc::mbar_wait(full0 + 8 * s, armed[s] & 1, kTcMaxPolls))
                    ok = 0;
        }
    } else if (warp == 5) {
        if (lane == 0) { // MMA issuer
            // tap group q: first tap (dy, dx), atom stride, M; descriptors of stage 0 at
            // position 0, advanced by 16-byte units (1024 bytes per 16 positions)
            const int cdy[4] = {-2, -1, 0, -2}, cdx[4] = {-2, -2, -2, 2};
            const uint32_t clbo[4] = {64u, 64u, 64u, (uint32_t)g.PX * 64u};
            uint64_t abase[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                abase[q] = tc::smem_desc_mn_sw64(sb + 2 * g.zbytes + (uint32_t)((cdy[q] + 2) * g.PX + cdx[q] + 2) * 64u,
                                                 clbo[q]);
            const uint64_t bbase = tc::smem_desc_mn_sw64(sb, g.zbytes);
            constexpr uint32_t id128 = tc::idesc_bf16_f32_mn(128, 64), id64 = tc::idesc_bf16_f32_mn(64, 64);
            int k = 0;
            for (int it = blockIdx.x; ok && it < total; it += gridDim.x, ++k) {
                const int s = k % NS, use = k / NS;
                if (!tc::mbar_wait(full0 + 8 * s, use & 1, kTcMaxPolls)) {
                    ok = 0;
                    break;
                }
                tc::fence_after_sync();
                const uint64_t soff = (uint64_t)(((uint32_t)s * g.stage_bytes) >> 4);
                for (int j = 0; j < g.KS; ++j) {
                    const uint64_t jo = soff + (uint64_t)(64 * j);
                    const uint32_t acc = (k > 0 || j > 0) ? 1u : 0u;
                    const uint64_t bd = bbase + jo;
                    tc::mma_bf16(tbase, abase[0] + jo, bd, id128, acc);
                    tc::mma_bf16(tbase + 64u, abase[1] + jo, bd, id128, acc);
                    tc::mma_bf16(tbase + 128u, abase[2] + jo, bd, id128, acc);
                    tc::mma_bf16(tbase + 192u, abase[3] + jo, bd, id64, acc);
                }
                tc::commit(empty0 + 8 * s); // stage s is free once this item's MMAs have read it
            }
            tc::commit(done); // every MMA issued above has completed before the drain
        }
    } else { // warps 0-3: bias gradient per item, then the drain
        float bsum = 0.f;
        int k = 0;
        for (int it = blockIdx.x; ok && it < total; it += gridDim.x, ++k) {
            const int s = k % NS, use = k / NS;
            const bool got = __any_sync(0xffffffffu, tc::mbar_wait(full0 + 8 * s, use & 1, kTcMaxPolls));
            if (!got) {
                ok = 0;
                break;
            }
            const unsigned char *zh = smem + (size_t)s * g.stage_bytes, *zl = zh + g.zbytes;
            for (int x = warp; x < g.L; x += 4) { // channel `lane` of position x, 64-byte swizzle
                const uint32_t off = (uint32_t)x * 64u + ((((uint32_t)lane >> 3) ^ (((uint32_t)x >> 1) & 3u)) << 4) +
                                     ((uint32_t)lane & 7u) * 2u;
                bsum += bf(*reinterpret_cast<const bf16 *>(zh + off)) + bf(*reinterpret_cast<const bf16 *>(zl + off));
            }
            __syncwarp();
            if (lane == 0)
                tc::mbar_arrive(empty0 + 8 * s);
        }
        bsum_s[warp * 32 + lane] = bsum;
        const bool got = __any_sync(0xffffffffu, tc::mbar_wait(done, 0u, kTcMaxPolls));
        tc::fence_after_sync();
        if (!got)
            ok = 0;
        float *mine = part + (size_t)blockIdx.x * kDwPart;
        const bool any = blockIdx.x < total;
        // tap groups 0-2 (M = 128): lane 32 w + c holds tap w of the group, channel c;
        // group 3 (M = 64): lanes 0-15 of warp w hold tap (w < 2 ? 4 : 9), channel 16 (w & 1) + lane
        for (int q = 0; q < 4; ++q) {
            float v[32], u[32];
            const uint32_t col = tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(64 * q);
            tc::ld_32x32b_x32(col, v);
            tc::ld_32x32b_x32(col + 32u, u);
            int t, c;
            if (q < 3) {
                t = 5 * q + warp; // (dy, dx) = (q - 2, warp - 2): raster index 5 (dy + 2) + dx + 2
                c = lane;
                if (q == 2 && warp == 3)
                    continue; // (0, 1) is not a tap of the mask
            } else {
                if (lane >= 16)
                    continue;
                t = warp < 2 ? 4 : 9;
                c = 16 * (warp & 1) + lane;
            }
#pragma unroll
            for (int o = 0; o < kCh; ++o)
                mine[(t * kCh + o) * kCh + c] = any ? v[o] + u[o] : 0.f;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (tid < kCh)
            mine[kTapsB * kCh * kCh + tid] = bsum_s[tid] + bsum_s[32 + tid] + bsum_s[64 + tid] + bsum_s[96 + tid];
    }
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0)
        atomicExch(err, 1);
    tc::fence_after_sync();
    if (warp == 0)
        tc::tmem_free(tbase, kDwTcAlloc);
}

// Sum the per-CTA partials of k_dw32_tc in CTA order (deterministic) into the
// canonical gradient of hidden layer `layer`.
__global__ void k_dw_reduce(const float *__restrict__ part, int nparts, float *g, DevParams P, int layer)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kDwPart)
        return;
    float v = 0.f;
    for (int k = 0; k < nparts; ++k)
        v += part[(size_t)k * kDwPart + i];
    if (i < kTapsB * kCh * kCh) {
        const int t = i / (kCh * kCh), o = (i / kCh) % kCh, c = i % kCh;
        g[canon_w(P, layer, o, c, tap_dy(t), tap_dx(t))] += v;
    } else {
        g[P.b_off[layer] + (i - kTapsB * kCh * kCh)] += v;
    }
}

// Layer-1 weight and bias gradients: gW1[o][t] = sum_p dZ1(p)[o] s(p + d_t),
// gb1[o] = sum_p dZ1(p)[o].  One CTA item = one row: spins of rows y-2..y and
// dZ1 of row y staged in smem.  Lane o of warp w accumulates the 13 outputs
// of channel o over its segment w of every row, the 12 tap spins held in a
// window of registers that slides along x (3 shared-memory loads per
// position instead of one per tap and channel); at the end the 8 segment
// warps are added in warp order and the CTA writes its partial sums to
// part[output][CTA] (summed in a fixed order by k_edge_grad_reduce).
__global__ void __launch_bounds__(256) k_layer1_bwd_w(const bf16 *dzh, const bf16 *dzl, const int8_t *spins,
                                                      float *part, int n, int L)
{
    __shared__ float S[3][kMaxL + 4];
    __shared__ __align__(16) float Z[kMaxL * kCh];
    __shared__ float R[8][kEdgeOut1];
    const int tid = threadIdx.x, o = tid & 31, seg = tid >> 5;
    const int seg_len = (L + 7) / 8, x0 = seg * seg_len, x1 = min(x0 + seg_len, L);
    float acc[kTapsA + 1];
#pragma unroll
    for (int t = 0; t <= kTapsA; ++t)
        acc[t] = 0.f;
    for (int item = blockIdx.x; item < n * L; item += gridDim.x) {
        const int b = item / L, y = item - b * L;
        __syncthreads();
        for (int i = tid; i < 3 * (L + 4); i += blockDim.x) {
            const int r = i / (L + 4), xx = i - r * (L + 4) - 2, yy = y - 2 + r;
            S[r][xx + 2] = (yy >= 0 && xx >= 0 && xx < L) ? (float)spins[((size_t)b * L + yy) * L + xx] : 0.f;
        }
        const uint4 *zh = reinterpret_cast<const uint4 *>(dzh + ((size_t)b * L + y) * L * kCh);
        const uint4 *zl = reinterpret_cast<const uint4 *>(dzl + ((size_t)b * L + y) * L * kCh);
        for (int i = tid; i < L * kCh / 8; i += blockDim.x) { // value = hi + lo
            const uint4 h = zh[i], l = zl[i];
            const bf16 *h8 = reinterpret_cast<const bf16 *>(&h), *l8 = reinterpret_cast<const bf16 *>(&l);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                Z[8 * i + k] = bf(h8[k]) + bf(l8[k]);
        }
        __syncthreads();
        if (x0 < x1) {
            // taps 0-4: S[0][x + t]; 5-9: S[1][x + t - 5]; 10, 11: S[2][x + t - 10] (mask A)
            float w0[5], w1[5], w2[2];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                w0[k + 1] = S[0][x0 + k];
                w1[k + 1] = S[1][x0 + k];
            }
            w2[1] = S[2][x0];
            for (int x = x0; x < x1; ++x) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    w0[k] = w0[k + 1];
                    w1[k] = w1[k + 1];
                }
                w0[4] = S[0][x + 4];
                w1[4] = S[1][x + 4];
                w2[0] = w2[1];
                w2[1] = S[2][x + 1];
                const float z = Z[x * kCh + o];
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    acc[k] += z * w0[k];
                    acc[5 + k] += z * w1[k];
                }
                acc[10] += z * w2[0];
                acc[11] += z * w2[1];
                acc[12] += z;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t <= kTapsA; ++t)
        R[seg][o * (kTapsA + 1) + t] = acc[t];
    __syncthreads();
    for (int idx = tid; idx < kEdgeOut1; idx += blockDim.x) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w)
            v += R[w][idx];
        part[(size_t)idx * gridDim.x + blockIdx.x] = v;
    }
}

__global__ void k_adam(float *p, float *m, float *v, const float *g, size_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace
}  // namespace van
}  // namespace mc

namespace mc {
namespace van {
namespace {

constexpr uint32_t kTagVanSample = 0x21000000u; // sampler uniforms
constexpr uint32_t kTagVanMH = 0x22000000u;     // accept uniform and global flip
constexpr int kSampleTile = 32;                 // samples per sampler CTA (two m16 tiles)
constexpr int kTapBytes = kSampleTile * kCh * 2; // one tap of the 32 samples of a CTA: 2 KB
constexpr int kTileBytes = kTapsA * kTapBytes;      // a gathered tile [12 taps][32 samples][32 ch]
constexpr int kSampleMaxBufs = 3;                   // gathered hidden-layer tiles in flight
constexpr size_t kSampleSmemLimit = 232448;         // 227 KB, the opt-in maximum per block
constexpr int kGroupThreads = 128;                  // main warps 0-3, side warps 4-7
constexpr int kSampleThreads = 2 * kGroupThreads + 32; // + the producer warp (gathers)

// Ring arrays of the sampler, per layer [32-sample block][row % 3][x][32 samples]
// [32 ch]: a block's five taps of one row are one contiguous run (one bulk
// copy), and the 16-byte channel chunks of sample s are stored in the order
// c ^ ((s >> 1) & 3), so that eight consecutive samples' rows of one chunk fall
// on distinct shared-memory banks when a tile is read by ldmatrix.  The same
// layout holds the layer values of the current position (Hc) and, per tap, the
// weights (row = output channel).
__device__ __forceinline__ int ring_elem(int s, int o) { return s * kCh + ((((o >> 3) ^ (s >> 1)) & 3) << 3) + (o & 7); }

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// BF16 pair <-> two floats as plain bit operations (BF16 -> FP32 is exact);
// the pack rounds to nearest even, lo in the low half.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    uint32_t u;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(u) : "f"(hi), "f"(lo));
    return u;
}
__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }

// Named barriers of the sampler's warp groups (0 is __syncthreads).
constexpr int kBarMain = 1, kBarSide = 2;
__device__ __forceinline__ void group_sync(int id, int threads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Wait for an mbarrier phase.  A wait that gives up latches *err and sets the
// CTA's abort flag; once the flag is set every wait returns at once, so that
// all threads run to the end (no barrier is left short of threads) and the
// sampled values are garbage, reported through *err.
__device__ __forceinline__ void wait_phase(uint32_t bar, uint32_t parity, volatile int *abort, int *err)
{
    for (int it = 0; it < kTcMaxPolls; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done || *abort)
            return;
    }
    *abort = 1;
    atomicExch(err, 1);
}

// The tap of position k = y L + x whose position is k - 1 (the one just sampled),
// or -1: tap 11 (dx = -1) for x > 0; for x = 0 the position k - 1 is (y - 1,
// L - 1), a tap only when L = 2 (tap 8).  In either case no later tap of 0..11
// is inside the lattice.
__device__ __forceinline__ int newest_tap(int L, int y, int x) { return x > 0 ? 11 : (L == 2 && y > 0 ? 8 : -1); }

// One 16 x 16 output tile of a 32 -> 32 layer for this warp (m-tile w >> 1,
// n-tiles 2 (w & 1) + 0, 1): accumulate one tap (K = 32) from the [32][32]
// operand at shared address `a` with the tap's weights at `wt`.
__device__ __forceinline__ void mma_tap(float (&c0)[4], float (&c1)[4], uint32_t a, uint32_t wt, uint32_t ao0,
                                        uint32_t ao1, uint32_t bo0, uint32_t bo1)
{
    uint32_t a0, a1, a2, a3, b0, b1, b2, b3;
    ldsm_x4(a + ao0, a0, a1, a2, a3);
    ldsm_x4(wt + bo0, b0, b1, b2, b3);
    mma_bf16(c0, a0, a1, a2, a3, b0, b1);
    mma_bf16(c1, a0, a1, a2, a3, b2, b3);
    ldsm_x4(a + ao1, a0, a1, a2, a3);
    ldsm_x4(wt + bo1, b0, b1, b2, b3);
    mma_bf16(c0, a0, a1, a2, a3, b0, b1);
    mma_bf16(c1, a0, a1, a2, a3, b2, b3);
}

// Autoregressive sampling, one position k = y L + x at a time in raster order,
// 32 samples per CTA.  Layer l at position k sums its taps over the 12 earlier
// positions (values of layer l - 1 from earlier steps, gathered from that
// layer's ring array) and tap 12, the value of layer l - 1 at k itself; s_k =
// +1 iff u < sigmoid(f_k), u from Philox (k >> 2, round, TAG_SAMPLE, id) word
// k & 3, and log q accumulates log sigmoid(s_k f_k) in FP64.  Warp roles:
//   * main warps 0-3 run the chain of dependent layers of step k: the first
//     layer (its partial plus w s_{k-1}), the hidden layers on the tensor cores
//     (a 16 x 16 output tile per warp, 26 MMA k-steps), the output layer (its
//     partial plus tap 12) and the draw; they write each hidden value to the
//     layer's ring array (followed by a proxy fence, for the bulk copies);
//   * side warps 4-7 compute, off that chain, the output layer's partial sum
//     over its 12 earlier taps for step k and the first layer's partial over
//     its taps other than s_{k-1} for step k + 1, and accumulate log q -- in
//     the order of one pass over all taps, so that the result is that of the
//     plain evaluation;
//   * a producer warp gathers, per (position, consuming layer g = 1..G, G = D -
//     1), the 12 earlier taps of the CTA's samples from the ring array by bulk
//     copies into one of `nbuf` tiles (taps outside the lattice copy a zero
//     page), in the sequence q = k G + g - 1.  Main releases a hidden layer's
//     tile after the layer; side releases the output layer's tile of step k
//     once main has finished step k, so that every release comes after the ring
//     stores that the gather nbuf later may read (nbuf <= G).
// Signals between main and side are mbarriers with one completion per step:
// E0 (first layer of step k done: its partial consumed), E1 (step k done:
// output partial consumed, s_k drawn), R0 (first-layer partial of step k
// written), R1 (output partial of step k written).  Every wait is bounded; one
// that gives up latches *err and sets an abort flag after which all waits return
// at once, so that every thread still reaches every barrier.
__global__ void __launch_bounds__(kSampleThreads, 1) k_sample(const bf16 *__restrict__ wh, const float *__restrict__ w1,
                                                   const float *__restrict__ wD, const float *__restrict__ bias, int D,
                                                   int L, int n, int nbuf, bf16 *hist, const bf16 *zero, int8_t *out,
                                                   double *logq, PhiloxKey key, uint32_t round, const uint32_t *ids,
                                                   int *err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int nh = D - 2, G = nh + 1;
    bf16 *Ws = reinterpret_cast<bf16 *>(smem);                      // [nh][13][32 o][32 c] (ring_elem)
    bf16 *Ts = Ws + (size_t)nh * kTapsB * kCh * kCh;                // nbuf + 1 x [12][32][32] gathered taps
    bf16 *Hc = Ts + (size_t)(nbuf + 1) * kTapsA * kSampleTile * kCh; // [2 (layer & 1)][32][32] values at k
    float *P0 = reinterpret_cast<float *>(Hc + (size_t)2 * kSampleTile * kCh); // [32 s][32 o] first-layer partial
    float *Po = P0 + kSampleTile * kCh;                             // [32 s][8 parts] output partial
    float *W1 = Po + kSampleTile * 8;                               // [12][32] (tap-major)
    float *WD = W1 + kCh * kTapsA;                                  // [13][32]
    float *Bs = WD + kTapsB * kCh;                                  // [(D-1) 32 + 1]
    float *LT = Bs + (D - 1) * kCh + 1;                             // [32] s_k f_k of the last draw
    int8_t *Sr = reinterpret_cast<int8_t *>(LT + kSampleTile);      // [32][3][L] spins of rows y-2..y
    const uint32_t bar0 = (smem_u32(Sr + kSampleTile * 3 * L) + 7u) & ~7u;
    const uint32_t full0 = bar0, empty0 = bar0 + 8u * (kSampleMaxBufs + 1), E0 = empty0 + 8u * (kSampleMaxBufs + 1),
                   E1 = E0 + 8u, R0 = E0 + 16u, R1 = E0 + 24u;
    __shared__ int abort_flag;
    volatile int *abort = &abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int s0 = blockIdx.x * kSampleTile;
    for (int i = tid; i < nh * kTapsB * kCh * kCh; i += blockDim.x) {
        const int row = i / kCh, c = i % kCh, o = row % kCh; // row = (l, t, o)
        Ws[(size_t)(row - o) * kCh + ring_elem(o, c)] = wh[i];
    }
    for (int i = tid; i < kCh * kTapsA; i += blockDim.x)
        W1[(i % kTapsA) * kCh + i / kTapsA] = w1[i]; // w1 is [o][t]
    for (int i = tid; i < kTapsB * kCh; i += blockDim.x)
        WD[i] = wD[i];
    for (int i = tid; i < (D - 1) * kCh + 1; i += blockDim.x)
        Bs[i] = bias[i];
    if (tid == 0) {
        abort_flag = 0;
        for (int b = 0; b <= nbuf; ++b) {
            tc::mbar_init(full0 + 8u * b, 1);
            tc::mbar_init(empty0 + 8u * b, 1);
        }
        for (int j = 0; j < 4; ++j)
            tc::mbar_init(E0 + 8u * j, 1);
    }
    const int nsb = (n + kSampleTile - 1) / kSampleTile;
    const size_t pblk = (size_t)kSampleTile * kCh;                  // ring elements per position of a block
    const size_t lstride = (size_t)nsb * 3 * L * pblk;             // ring elements per layer
    bf16 *ring = hist + (size_t)blockIdx.x * 3 * L * pblk;         // this CTA's block of layer 0
    const int P = L * L, Q = P * G;
    const uint32_t ts0 = smem_u32(Ts), ws0 = smem_u32(Ws);
    __syncthreads();

    if (warp == 8) { // ---------------------------------------------------------------- producer
        int issued = 0;
        for (int q = 0; q < Q; ++q) {
            const int kq = q / G, g = q - kq * G + 1, yq = kq / L, xq = kq - yq * L;
            // hidden-layer gathers cycle through slots 0..nbuf-1, output-layer gathers use slot nbuf
            const int hq = kq * nh + g - 1, slot = g < G ? hq % nbuf : nbuf, use = g < G ? hq / nbuf : kq;
            if (use > 0)
                wait_phase(empty0 + 8u * (uint32_t)slot, (uint32_t)(use - 1) & 1u, abort, err);
            if (*abort)
                break;
            const uint32_t bar = full0 + 8u * (uint32_t)slot;
            if (lane == 0)
                tc::mbar_arrive_expect_tx(bar, kTileBytes);
            __syncwarp();
            // lane 3 r + p copies part p (0 zeros left of the lattice, 1 the positions inside, 2 zeros right
            // of it) of tap row r: rows y-2 and y-1 (taps 5 r .. 5 r + 4, dx = -2..2), row y (taps 10, 11)
            const int r = lane / 3, part = lane - 3 * r;
            if (r < 3) {
                const int ntap = r < 2 ? 5 : 2, yy = yq - 2 + r, xlo = xq - 2;
                int zl = ntap, nd = 0;
                if (yy >= 0) {
                    zl = xlo < 0 ? -xlo : 0;
                    nd = ntap - zl - max(0, xlo + ntap - L);
                }
                const int first = part == 0 ? 0 : part == 1 ? zl : zl + nd;
                const int cnt = part == 0 ? zl : part == 1 ? nd : ntap - zl - nd;
                if (cnt > 0) {
                    const bf16 *src = part == 1 ? ring + (size_t)(g - 1) * lstride + ((size_t)(yy % 3) * L + xlo + zl) * pblk
                                                : zero;
                    bulk_g2s(ts0 + (uint32_t)(slot * kTileBytes + (5 * r + first) * kTapBytes), src,
                             (uint32_t)cnt * kTapBytes, bar);
                }
            }
            issued = q + 1;
        }
        // copies still in flight (the consumers stopped early): let them land before the CTA ends
        if (lane == 0 && *abort) {
            uint32_t seen = 0; // the last fill of each slot
            for (int q = issued - 1; q >= 0 && seen != (2u << nbuf) - 1u; --q) {
                const int kq = q / G, g = q - kq * G + 1, hq = kq * nh + g - 1;
                const int slot = g < G ? hq % nbuf : nbuf, use = g < G ? hq / nbuf : kq;
                if (!(seen >> slot & 1u)) {
                    seen |= 1u << slot;
                    tc::mbar_wait(full0 + 8u * (uint32_t)slot, (uint32_t)use & 1u, kTcMaxPolls);
                }
            }
        }
        return;
    }

    if (warp >= 4) { // ---------------------------------------------------------------------- side
        const int h = tid - 128, s = h >> 2, sub = h & 3;
        double lq = 0.0; // owned by side thread s < 32
        // the first-layer partial of position k: bias + taps 0..11 inside, except the one at k - 1
        auto first_partial = [&](int k) {
            const int y = k / L, x = k % L, tn = newest_tap(L, y, x), o0 = sub * 8;
            float acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                acc[j] = Bs[o0 + j];
#pragma unroll
            for (int t = 0; t < kTapsA; ++t) {
                const int yy = y + tap_dy(t), xx = x + tap_dx(t);
                if (t != tn && yy >= 0 && xx >= 0 && xx < L) {
                    const float v = (float)Sr[(s * 3 + yy % 3) * L + xx];
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        acc[j] = __fmaf_rn(W1[t * kCh + o0 + j], v, acc[j]);
                }
            }
            *reinterpret_cast<float4 *>(P0 + s * kCh + o0) = make_float4(acc[0], acc[1], acc[2], acc[3]);
            *reinterpret_cast<float4 *>(P0 + s * kCh + o0 + 4) = make_float4(acc[4], acc[5], acc[6], acc[7]);
        };
        first_partial(0);
        group_sync(kBarSide, kGroupThreads);
        if (h == 0)
            tc::mbar_arrive(R0);
        for (int k = 0; k < P; ++k) {
            const int y = k / L, x = k % L;
            if (k > 0) {
                wait_phase(E1, (uint32_t)(k - 1) & 1u, abort, err); // step k - 1 done
                if (h == 0) // its output tile: every ring store of step k - 1 is in
                    tc::mbar_arrive(empty0 + 8u * (uint32_t)nbuf);
                if (h < kSampleTile && s0 + h < n)
                    lq += (double)log_sigmoid(LT[h]);
            }
            // ---- output partial of step k: taps 0..11 inside, 8 parts of 4 channels per sample
            wait_phase(full0 + 8u * (uint32_t)nbuf, (uint32_t)k & 1u, abort, err);
            {
                const bf16 *tl = Ts + (size_t)nbuf * kTapsA * kSampleTile * kCh;
                float po0 = 0.f, po1 = 0.f;
                for (int t = 0; t < kTapsA; ++t) {
                    const int yy = y + tap_dy(t), xx = x + tap_dx(t);
                    if (yy < 0 || xx < 0 || xx >= L)
                        continue;
                    const bf16 *src = tl + t * kSampleTile * kCh;
                    const uint2 hv0 = *reinterpret_cast<const uint2 *>(src + ring_elem(s, sub * 8));
                    const uint2 hv1 = *reinterpret_cast<const uint2 *>(src + ring_elem(s, sub * 8 + 4));
                    const float4 w0 = *reinterpret_cast<const float4 *>(WD + t * kCh + sub * 8);
                    const float4 wv1 = *reinterpret_cast<const float4 *>(WD + t * kCh + sub * 8 + 4);
                    po0 = __fmaf_rn(w0.x, bf16_lo(hv0.x), po0);
                    po0 = __fmaf_rn(w0.y, bf16_hi(hv0.x), po0);
                    po0 = __fmaf_rn(w0.z, bf16_lo(hv0.y), po0);
                    po0 = __fmaf_rn(w0.w, bf16_hi(hv0.y), po0);
                    po1 = __fmaf_rn(wv1.x, bf16_lo(hv1.x), po1);
                    po1 = __fmaf_rn(wv1.y, bf16_hi(hv1.x), po1);
                    po1 = __fmaf_rn(wv1.z, bf16_lo(hv1.y), po1);
                    po1 = __fmaf_rn(wv1.w, bf16_hi(hv1.y), po1);
                }
                *reinterpret_cast<float2 *>(Po + s * 8 + sub * 2) = make_float2(po0, po1);
            }
            group_sync(kBarSide, kGroupThreads);
            if (h == 0)
                tc::mbar_arrive(R1);
            // ---- first-layer partial of step k + 1 (its spins at positions <= k - 1 are drawn)
            if (k + 1 < P) {
                wait_phase(E0, (uint32_t)k & 1u, abort, err); // the partial of step k consumed
                first_partial(k + 1);
                group_sync(kBarSide, kGroupThreads);
                if (h == 0)
                    tc::mbar_arrive(R0);
            }
        }
        wait_phase(E1, (uint32_t)(P - 1) & 1u, abort, err); // the last draw
        if (h < kSampleTile && s0 + h < n)
            logq[s0 + h] = lq + (double)log_sigmoid(LT[h]);
        return;
    }

    // ----------------------------------------------------------------------------------------- main
    const int c = tid, s = c >> 2, sub = c & 3, gs = s0 + s;
    const int mt = warp >> 1, np = warp & 1; // this warp's 16 x 16 output tile of a hidden layer
    const int ar = mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8, br = (2 * np + (lane >> 4)) * 8 + (lane & 7);
    const uint32_t ao0 = 2u * ring_elem(ar, (lane >> 4) * 8), ao1 = 2u * ring_elem(ar, 16 + (lane >> 4) * 8);
    const uint32_t bo0 = 2u * ring_elem(br, ((lane >> 3) & 1) * 8), bo1 = 2u * ring_elem(br, 16 + ((lane >> 3) & 1) * 8);
    const int fg = lane >> 2, ft = lane & 3; // accumulator fragment: rows fg, fg + 8; columns 2 ft, 2 ft + 1
    uint32_t my_id = 0;
    if (sub == 0 && gs < n)
        my_id = ids ? ids[gs] : (uint32_t)gs;
    for (int k = 0; k < P; ++k) {
        const int y = k / L, x = k % L, tn = newest_tap(L, y, x);
        bf16 *hpos = ring + ((size_t)(y % 3) * L + x) * pblk; // position k in the ring of layer 0
        // ---- first layer: partial + w s_{k-1}
        wait_phase(R0, (uint32_t)k & 1u, abort, err);
        {
            const int o0 = sub * 8;
            float v = 0.f;
            if (tn >= 0)
                v = (float)Sr[(s * 3 + (y + tap_dy(tn)) % 3) * L + x + tap_dx(tn)];
            float a[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                a[j] = P0[s * kCh + o0 + j];
                if (tn >= 0)
                    a[j] = __fmaf_rn(W1[tn * kCh + o0 + j], v, a[j]);
            }
            const uint4 pk =
                make_uint4(pack_bf16x2(fmaxf(a[0], 0.f), fmaxf(a[1], 0.f)), pack_bf16x2(fmaxf(a[2], 0.f), fmaxf(a[3], 0.f)),
                           pack_bf16x2(fmaxf(a[4], 0.f), fmaxf(a[5], 0.f)), pack_bf16x2(fmaxf(a[6], 0.f), fmaxf(a[7], 0.f)));
            *reinterpret_cast<uint4 *>(Hc + ring_elem(s, o0)) = pk;
            *reinterpret_cast<uint4 *>(hpos + ring_elem(s, o0)) = pk;
            asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        group_sync(kBarMain, kGroupThreads);
        if (c == 0)
            tc::mbar_arrive(E0);
        // ---- hidden layers (tensor cores): M = 32 samples, N = 32, K = 13 x 32
        for (int l = 1; l <= nh; ++l) {
            const int hq = k * nh + l - 1, slot = hq % nbuf;
            const uint32_t tile = ts0 + (uint32_t)(slot * kTileBytes);
            const uint32_t wl = ws0 + (uint32_t)((l - 1) * kTapsB * kCh * kCh * 2);
            wait_phase(full0 + 8u * (uint32_t)slot, (uint32_t)(hq / nbuf) & 1u, abort, err);
            float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
            for (int t = 0; t < kTapsA; ++t)
                mma_tap(c0, c1, tile + (uint32_t)t * kTapBytes, wl + (uint32_t)t * kCh * kCh * 2, ao0, ao1, bo0, bo1);
            mma_tap(c0, c1, smem_u32(Hc + (size_t)((l - 1) & 1) * kSampleTile * kCh), wl + (uint32_t)kTapsA * kCh * kCh * 2,
                    ao0, ao1, bo0, bo1);
            bf16 *hn = Hc + (size_t)(l & 1) * kSampleTile * kCh;
            bf16 *hr = hpos + (size_t)l * lstride;
            // bias, ReLU, BF16 of n-tile j's fragment (rows fg, fg + 8), to Hc and the ring
            auto store = [&](const float(&acc)[4], int j) {
                const int o = (2 * np + j) * 8 + 2 * ft;
                const float bo = Bs[l * kCh + o], b1v = Bs[l * kCh + o + 1];
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int sr = mt * 16 + fg + 8 * hh;
                    const uint32_t v = pack_bf16x2(fmaxf(acc[2 * hh] + bo, 0.f), fmaxf(acc[2 * hh + 1] + b1v, 0.f));
                    *reinterpret_cast<uint32_t *>(hn + ring_elem(sr, o)) = v;
                    *reinterpret_cast<uint32_t *>(hr + ring_elem(sr, o)) = v;
                }
            };
            store(c0, 0);
            store(c1, 1);
            asm volatile("fence.proxy.async.global;" ::: "memory");
            group_sync(kBarMain, kGroupThreads);
            if (c == 0)
                tc::mbar_arrive(empty0 + 8u * (uint32_t)slot);
        }
        // ---- output layer: partial + tap 12, then the draw
        wait_phase(R1, (uint32_t)k & 1u, abort, err);
        {
            const bf16 *hp = Hc + (size_t)(nh & 1) * kSampleTile * kCh;
            float a2[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int part = sub * 2 + j;
                float acc = Po[s * 8 + part];
                const uint2 hv = *reinterpret_cast<const uint2 *>(hp + ring_elem(s, part * 4));
                const float4 w = *reinterpret_cast<const float4 *>(WD + kTapsA * kCh + part * 4);
                acc = __fmaf_rn(w.x, bf16_lo(hv.x), acc);
                acc = __fmaf_rn(w.y, bf16_hi(hv.x), acc);
                acc = __fmaf_rn(w.z, bf16_lo(hv.y), acc);
                acc = __fmaf_rn(w.w, bf16_hi(hv.y), acc);
                a2[j] = acc;
            }
            float f = a2[0] + a2[1];
            f += __shfl_xor_sync(0xffffffffu, f, 1);
            f += __shfl_xor_sync(0xffffffffu, f, 2);
            f += Bs[(D - 1) * kCh];
            if (sub == 0 && gs < n) {
                const uint4 r = philox4x32_10(make_uint4((uint32_t)k >> 2, round, kTagVanSample, my_id), key);
                const uint32_t rk = (k & 2) ? ((k & 1) ? r.w : r.z) : ((k & 1) ? r.y : r.x);
                const float sp = uniform_open0(rk) < sigmoid(f) ? 1.f : -1.f;
                Sr[(s * 3 + y % 3) * L + x] = (int8_t)sp;
                out[((size_t)gs * L + y) * L + x] = (int8_t)sp;
                LT[s] = sp * f;
            }
        }
        group_sync(kBarMain, kGroupThreads);
        if (c == 0)
            tc::mbar_arrive(E1);
    }
}

// Copy the int8 lattices of every chain of an int8-layout Ising context into
// one contiguous [n][L][L] buffer (or back, when `back`).
__global__ void k_gather(const IsingChain *chains, char *lattice, int8_t *buf, int L, int n, int back)
{
    const size_t per = (size_t)L * L;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < per * n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t k = i / per, j = i % per;
        int8_t *lat = reinterpret_cast<int8_t *>(lattice + chains[k].spin_off);
        if (back)
            lat[j] = buf[i];
        else
            buf[i] = lat[j];
    }
}

// H of Eq. (1) per configuration (exact).
__global__ void k_energy(const int8_t *s, long long *E, int L)
{
    __shared__ long long part[32];
    const size_t base = (size_t)blockIdx.x * L * L;
    long long acc = 0;
    for (int i = threadIdx.x; i < L * L; i += blockDim.x) {
        const int y = i / L, x = i % L;
        const int v = s[base + i];
        acc -= v * (s[base + y * L + (x + 1) % L] + s[base + ((y + 1) % L) * L + x]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0)
        part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            t += part[w];
        E[blockIdx.x] = t;
    }
}

__device__ __forceinline__ double log_add_exp(double a, double b)
{
    const double m = fmax(a, b);
    return m + log1p(exp(-fabs(a - b)));
}

// Metropolis-Hastings for an independence proposal from q_sym(s) = (q(s) +
// q(-s)) / 2: accept s' with probability min(1, e^{-beta (E' - E)} q_sym(s) /
// q_sym(s')).  The proposal is the sample s'' or its global flip -s'' (one bit
// of the chain's MH Philox block), and q_sym, E are flip-invariant.  Accepted
// proposals are written into the chain's lattice.
__global__ void k_mh_accept(const IsingChain *chains, char *lattice, const int8_t *prop, const double *lq_p,
                            const double *lq_pn, const double *lq_s, const double *lq_sn, const long long *E_s,
                            const long long *E_p, int L, int n, PhiloxKey key, uint32_t round, int *accepted,
                            double *log_ratio)
{
    const int k = blockIdx.x;
    __shared__ int take, flip;
    if (threadIdx.x == 0) {
        const IsingChain &ch = chains[k];
        const uint4 r = philox4x32_10(make_uint4(0u, round, kTagVanMH, ch.chain_id), key);
        const double u = (double)((r.x >> 8) + 1u) * (1.0 / 16777216.0);
        flip = (int)(r.y >> 31);
        const double lr = -ch.beta * (double)(E_p[k] - E_s[k]) + log_add_exp(lq_s[k], lq_sn[k]) -
                          log_add_exp(lq_p[k], lq_pn[k]);
        take = log(u) < lr;
        if (log_ratio)
            log_ratio[k] = lr;
        if (take)
            atomicAdd(accepted, 1);
    }
    __syncthreads();
    if (!take)
        return;
    int8_t *lat = reinterpret_cast<int8_t *>(lattice + chains[k].spin_off);
    const int8_t *p = prop + (size_t)k * L * L;
    for (int i = threadIdx.x; i < L * L; i += blockDim.x)
        lat[i] = flip ? (int8_t)(-p[i]) : p[i];
}

size_t a256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace van
}  // namespace mc

using namespace mc;
using namespace mc::van;

struct mc_van {
    int L = 0, D = 0, nmax = 0;
    PhiloxKey key{};
    uint32_t round = 0;
    int adam_t = 0;
    cudaStream_t stream = nullptr;
    char *ws = nullptr;
    ParamLayout P{};
    DevParams dp{};
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    bf16 *wh = nullptr;
    float *w1 = nullptr, *wD = nullptr, *bias = nullptr;
    bf16 *H = nullptr;
    float *dZa = nullptr, *dZb = nullptr;
    float *f = nullptr, *ll = nullptr, *dF = nullptr;
    int8_t *spins = nullptr, *prop = nullptr;
    double *lq = nullptr, *lq2 = nullptr, *lq3 = nullptr, *lq4 = nullptr, *mh_lr = nullptr;
    long long *E1 = nullptr, *E2 = nullptr;
    int *acc = nullptr;
    bf16 *hist = nullptr;
    const bf16 *zero = nullptr; // 5 kTapBytes of zeros
    float *dwpart = nullptr; // per-CTA partial gradients of k_dw32_tc
    int *err = nullptr;      // device fault latch (a bounded completion wait gave up)
    int sms = 0;
    bool weights_ready = false;
};

namespace {

mc_status vfail(mc_status s, const std::string &m)
{
    mc::set_last_error(m);
    return s;
}

// Synchronise the stream, then report (and clear) a fault a kernel latched --
// a bounded wait for a tensor-core or bulk-copy completion that gave up.
mc_status check_err(mc_van *w, const char *where)
{
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, w->err, sizeof v, cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess)
        return vfail(MC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
    if (v != 0) {
        cudaMemsetAsync(w->err, 0, sizeof v, w->stream);
        return vfail(MC_ETIMEOUT, std::string(where) + ": a tensor-core or bulk-copy completion wait timed out");
    }
    return MC_OK;
}

struct VanLayout {
    size_t p, m, v, g, wh, w1, wD, bias, H, dZa, dZb, f, ll, dF, spins, prop, lq, lq2, lq3, lq4, lr, E1, E2, acc, zero,
        hist, dwpart, err, total;
};

VanLayout van_layout(int L, int nmax, int D)
{
    VanLayout o{};
    const ParamLayout P = param_layout(D);
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t r = off;
        off = a256(off + std::max<size_t>(b, 1));
        return r;
    };
    const size_t pos = (size_t)nmax * L * L;
    o.p = take(P.total * 4);
    o.m = take(P.total * 4);
    o.v = take(P.total * 4);
    o.g = take(P.total * 4);
    o.wh = take((size_t)(D - 2) * kTapsB * kCh * kCh * 2);
    o.dwpart = take((size_t)kMaxDwBlocks * kDwPart * 4);
    o.err = take(16);
    o.w1 = take((size_t)kCh * kTapsA * 4);
    o.wD = take((size_t)kTapsB * kCh * 4);
    o.bias = take((size_t)((D - 1) * kCh + 1) * 4);
    o.H = take((size_t)(D - 1) * pos * kCh * 2);
    o.dZa = take(pos * kCh * 4);
    o.dZb = take(pos * kCh * 4);
    o.f = take(pos * 4);
    o.ll = take(pos * 4);
    o.dF = take(pos * 4);
    o.spins = take(pos);
    o.prop = take(pos);
    o.lq = take((size_t)nmax * 8);
    o.lq2 = take((size_t)nmax * 8);
    o.lq3 = take((size_t)nmax * 8);
    o.lq4 = take((size_t)nmax * 8);
    o.lr = take((size_t)nmax * 8);
    o.E1 = take((size_t)nmax * 8);
    o.E2 = take((size_t)nmax * 8);
    o.acc = take(64);
    o.zero = take((size_t)5 * kTapBytes); // zeros: the sampler's taps outside the lattice
    o.hist = take((size_t)(D - 1) * ((nmax + kSampleTile - 1) / kSampleTile) * kSampleTile * 3 * L * kCh * 2);
    o.total = off;
    return o;
}

unsigned grid_for(size_t n, int threads, int sms) { return (unsigned)std::min<size_t>((n + threads - 1) / threads, (size_t)sms * 16); }

size_t sample_smem(int D, int L, int nbuf)
{
    const size_t nh = (size_t)D - 2, tt = (size_t)kSampleTile * kCh;
    return nh * kTapsB * tt * 2 + (size_t)(nbuf + 1) * kTileBytes + 2 * tt * 2 + tt * 4 + (size_t)kSampleTile * 8 * 4 +
           (size_t)(kCh * kTapsA + kTapsB * kCh + (D - 1) * kCh + 1 + kSampleTile) * 4 + (size_t)kSampleTile * 3 * L +
           8 * (2 * (kSampleMaxBufs + 1) + 4) + 8;
}

// Hidden-layer tiles the sampler keeps in flight (besides the output layer's
// one): as many as fit, at most 3 and at most the D - 2 hidden layers (the
// release of the tile nbuf gathers back must come after the ring stores that
// a gather reads).
int sample_bufs(int D, int L)
{
    for (int b = std::min(kSampleMaxBufs, D - 2); b > 1; --b)
        if (sample_smem(D, L, b) <= kSampleSmemLimit)
            return b;
    return 1;
}

// Dynamic shared memory a kernel may use: raised to what this network needs,
// never lowered, so that creating a smaller network leaves larger ones usable.
cudaError_t raise_smem_limit(const void *kernel, size_t bytes)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess || (int)bytes <= a.maxDynamicSharedSizeBytes)
        return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t prep(mc_van *w)
{
    k_prep_weights<<<64, 256, 0, w->stream>>>(w->p, w->dp, w->wh, w->w1, w->wD, w->bias);
    w->weights_ready = true;
    return cudaGetLastError();
}

// Forward over n configurations in w->spins (negated when `negate`); log q
// into `logq`; dF (training) when dF != nullptr.
cudaError_t forward(mc_van *w, int n, int negate, double *logq, float *dF)
{
    if (!w->weights_ready) {
        cudaError_t e = prep(w);
        if (e != cudaSuccess)
            return e;
    }
    const int L = w->L, D = w->D;
    const size_t layer = (size_t)w->nmax * L * L * kCh;
    const unsigned l1g =
        (unsigned)std::min<long long>(((long long)n * L * L + kL1Threads - 1) / kL1Threads, (long long)w->sms * 8);
    k_layer1_tc<<<l1g, kL1Threads, 0, w->stream>>>(w->spins, negate, w->w1, w->bias, w->H, n, L, w->err);
    const TmaConvGeom tg = tma_conv_geom(L);
    const unsigned tcg = (unsigned)std::min<size_t>((size_t)n * tg.YB, (size_t)w->sms * tg.ctas_per_sm);
    const LastLayerArgs none{};
    const LastLayerArgs last{w->wD, w->bias + (D - 1) * kCh, w->spins, negate, w->f, w->ll, dF, 1.0f / n};
    for (int l = 1; l <= D - 1; ++l) { // hidden layers 1 .. D-2, then the last layer
        CUtensorMap in_map;
        const cudaError_t e = activation_map(&in_map, w->H + (l - 1) * layer, n, L, tg.P, tg.R + 2);
        if (e != cudaSuccess)
            return e;
        const bool is_last = l == D - 1;
        bf16 *out = is_last ? nullptr : w->H + l * layer;
        const bf16 *wl = is_last ? nullptr : w->wh + (size_t)(l - 1) * kTapsB * kCh * kCh;
        const float *bl = is_last ? nullptr : w->bias + l * kCh;
        if (tg.ctas_per_sm == 2 && is_last)
            k_conv32_tma<2, true><<<tcg, 192, tg.smem_bytes, w->stream>>>(in_map, out, wl, bl, last, n, tg, w->err);
        else if (tg.ctas_per_sm == 2)
            k_conv32_tma<2, false><<<tcg, 192, tg.smem_bytes, w->stream>>>(in_map, out, wl, bl, none, n, tg, w->err);
        else if (is_last)
            k_conv32_tma<1, true><<<tcg, 192, tg.smem_bytes, w->stream>>>(in_map, out, wl, bl, last, n, tg, w->err);
        else
            k_conv32_tma<1, false><<<tcg, 192, tg.smem_bytes, w->stream>>>(in_map, out, wl, bl, none, n, tg, w->err);
    }
    k_logq<<<n, 256, 0, w->stream>>>(w->ll, logq, L);
    return cudaGetLastError();
}

cudaError_t backward(mc_van *w, int n)
{
    const int L = w->L, D = w->D;
    const size_t layer = (size_t)w->nmax * L * L * kCh;
    cudaError_t e = cudaMemsetAsync(w->g, 0, w->P.total * 4, w->stream);
    if (e != cudaSuccess)
        return e;
    const bf16 *hD = w->H + (D - 2) * layer;
    const unsigned rows = (unsigned)std::min<size_t>((size_t)n * L, (size_t)w->sms * 8);
    const unsigned rg = (unsigned)std::min<size_t>((size_t)n * L, (size_t)w->sms * 12);
    // gradients as BF16 hi + lo pairs, each pair in the space of one FP32 buffer
    const size_t cap = (size_t)w->nmax * L * L * kCh;
    bf16 *dzh = reinterpret_cast<bf16 *>(w->dZa), *dzl = dzh + cap;
    bf16 *nxh = reinterpret_cast<bf16 *>(w->dZb), *nxl = nxh + cap;
    k_layerD_bwd_data<<<rows, 256, 0, w->stream>>>(w->dF, w->wD, hD, dzh, dzl, n, L);
    // edge-layer partial sums go to the dW partial buffer (free at these points)
    const unsigned eg = (unsigned)std::min<size_t>(rg, (size_t)kMaxDwBlocks * kDwPart / kEdgeOutD);
    k_layerD_bwd_w<<<eg, 256, 0, w->stream>>>(w->dF, hD, w->dwpart, n, L);
    k_edge_grad_reduce<false><<<kEdgeOutD, 256, 0, w->stream>>>(w->dwpart, (int)eg, w->g, w->dp);
    const TcConvGeom tgb = tc_conv_geom(L, 8);
    const unsigned tcg = (unsigned)std::min<size_t>((size_t)n * tgb.YB, (size_t)w->sms * 2);
    // k_dw32_tc: two CTAs per SM (256 tensor-memory columns and at most 110 KB of stages each)
    const DwTcGeom dg = dw_tc_geom(L);
    const unsigned dwg = (unsigned)std::min<size_t>(std::min<size_t>((size_t)n * L, (size_t)w->sms * 2), kMaxDwBlocks);
    for (int l = D - 2; l >= 1; --l) { // hidden layer l: input H[l-1], output H[l], grad dz wrt its pre-activation
        CUtensorMap zh_map, zl_map, x_map;
        e = activation_map(&zh_map, dzh, n, L, dg.PZ, 1);
        if (e == cudaSuccess)
            e = activation_map(&zl_map, dzl, n, L, dg.PZ, 1);
        if (e == cudaSuccess)
            e = activation_map(&x_map, w->H + (l - 1) * layer, n, L, dg.PX, 3);
        if (e != cudaSuccess)
            return e;
        k_dw32_tc<<<dwg, 192, dg.smem_bytes, w->stream>>>(zh_map, zl_map, x_map, w->dwpart, n, dg, w->err);
        k_dw_reduce<<<(kDwPart + 255) / 256, 256, 0, w->stream>>>(w->dwpart, (int)dwg, w->g, w->dp, l);
        k_conv32_bwd_tc<<<tcg, 128, tgb.smem_bytes, w->stream>>>(dzh, dzl, nxh, nxl,
                                                                 w->wh + (size_t)(l - 1) * kTapsB * kCh * kCh,
                                                                 w->H + (l - 1) * layer, n, tgb, w->err);
        std::swap(dzh, nxh);
        std::swap(dzl, nxl);
    }
    k_layer1_bwd_w<<<eg, 256, 0, w->stream>>>(dzh, dzl, w->spins, w->dwpart, n, L);
    k_edge_grad_reduce<true><<<kEdgeOut1, 256, 0, w->stream>>>(w->dwpart, (int)eg, w->g, w->dp);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

size_t mc_van_param_count(int32_t depth)
{
    if (depth < 3 || depth > kMaxDepth)
        return 0;
    return param_layout(depth).total;
}

size_t mc_van_workspace_bytes(int32_t L, int32_t batch, int32_t depth)
{
    if (L < 2 || L > kMaxL || (L & 1) || batch < 1 || depth < 3 || depth > kMaxDepth) {
        mc::set_last_error("mc_van_workspace_bytes: need even L in [2, 128], batch >= 1, depth in [3, 7]");
        return 0;
    }
    return van_layout(L, batch, depth).total;
}

mc_status mc_van_create(mc_van **out, int32_t L, int32_t batch, int32_t depth, uint64_t seed, void *workspace,
                        size_t bytes, void *cuda_stream)
{
    if (!out)
        return vfail(MC_EINVAL, "out is NULL");
    *out = nullptr;
    const size_t need = mc_van_workspace_bytes(L, batch, depth);
    if (need == 0)
        return MC_EINVAL;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u))
        return vfail(MC_EINVAL, "workspace must be a device pointer aligned to 256 bytes");
    if (bytes < need)
        return vfail(MC_ENOMEM, "van workspace too small: need " + std::to_string(need) + " bytes");
    mc_van *w = new (std::nothrow) mc_van();
    if (!w)
        return vfail(MC_ENOMEM, "host allocation failed");
    w->L = L;
    w->D = depth;
    w->nmax = batch;
    w->key = PhiloxKey{(uint32_t)seed, (uint32_t)(seed >> 32)};
    w->stream = static_cast<cudaStream_t>(cuda_stream);
    w->ws = static_cast<char *>(workspace);
    w->P = param_layout(depth);
    w->dp.D = depth;
    for (int l = 0; l < depth; ++l) {
        w->dp.w_off[l] = w->P.w_off[l];
        w->dp.b_off[l] = w->P.b_off[l];
    }
    const VanLayout o = van_layout(L, batch, depth);
    char *b = w->ws;
    w->p = reinterpret_cast<float *>(b + o.p);
    w->m = reinterpret_cast<float *>(b + o.m);
    w->v = reinterpret_cast<float *>(b + o.v);
    w->g = reinterpret_cast<float *>(b + o.g);
    w->wh = reinterpret_cast<bf16 *>(b + o.wh);
    w->dwpart = reinterpret_cast<float *>(b + o.dwpart);
    w->err = reinterpret_cast<int *>(b + o.err);
    w->w1 = reinterpret_cast<float *>(b + o.w1);
    w->wD = reinterpret_cast<float *>(b + o.wD);
    w->bias = reinterpret_cast<float *>(b + o.bias);
    w->H = reinterpret_cast<bf16 *>(b + o.H);
    w->dZa = reinterpret_cast<float *>(b + o.dZa);
    w->dZb = reinterpret_cast<float *>(b + o.dZb);
    w->f = reinterpret_cast<float *>(b + o.f);
    w->ll = reinterpret_cast<float *>(b + o.ll);
    w->dF = reinterpret_cast<float *>(b + o.dF);
    w->spins = reinterpret_cast<int8_t *>(b + o.spins);
    w->prop = reinterpret_cast<int8_t *>(b + o.prop);
    w->lq = reinterpret_cast<double *>(b + o.lq);
    w->lq2 = reinterpret_cast<double *>(b + o.lq2);
    w->lq3 = reinterpret_cast<double *>(b + o.lq3);
    w->lq4 = reinterpret_cast<double *>(b + o.lq4);
    w->mh_lr = reinterpret_cast<double *>(b + o.lr);
    w->E1 = reinterpret_cast<long long *>(b + o.E1);
    w->E2 = reinterpret_cast<long long *>(b + o.E2);
    w->acc = reinterpret_cast<int *>(b + o.acc);
    w->hist = reinterpret_cast<bf16 *>(b + o.hist);
    w->zero = reinterpret_cast<const bf16 *>(b + o.zero);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&w->sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaMemsetAsync(w->ws, 0, o.hist, w->stream); // params, Adam state, buffers
    if (e == cudaSuccess)
        e = raise_smem_limit(tma_conv_geom(L).ctas_per_sm == 2 ? (const void *)k_conv32_tma<2, false>
                                                               : (const void *)k_conv32_tma<1, false>,
                             tma_conv_geom(L).smem_bytes);
    if (e == cudaSuccess)
        e = raise_smem_limit(tma_conv_geom(L).ctas_per_sm == 2 ? (const void *)k_conv32_tma<2, true>
                                                               : (const void *)k_conv32_tma<1, true>,
                             tma_conv_geom(L).smem_bytes);
    if (e == cudaSuccess)
        e = raise_smem_limit((const void *)k_conv32_bwd_tc, tc_conv_geom(L, 8).smem_bytes);
    if (e == cudaSuccess)
        e = raise_smem_limit((const void *)k_dw32_tc, dw_tc_geom(L).smem_bytes);
    if (e == cudaSuccess)
        e = raise_smem_limit((const void *)k_sample, sample_smem(depth, L, sample_bufs(depth, L)));
    if (e != cudaSuccess) {
        delete w;
        return vfail(MC_ECUDA, std::string("mc_van_create: ") + cudaGetErrorString(e));
    }
    *out = w;
    return MC_OK;
}

mc_status mc_van_set_params(mc_van *w, const float *host_params, size_t n)
{
    if (!w || !host_params || n != w->P.total)
        return vfail(MC_EINVAL, "mc_van_set_params: need mc_van_param_count(depth) floats");
    cudaError_t e = cudaMemcpyAsync(w->p, host_params, n * 4, cudaMemcpyHostToDevice, w->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(w->m, 0, n * 4, w->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(w->v, 0, n * 4, w->stream);
    if (e == cudaSuccess)
        e = prep(w);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(w->stream);
    w->adam_t = 0;
    if (e != cudaSuccess)
        return vfail(MC_ECUDA, std::string("mc_van_set_params: ") + cudaGetErrorString(e));
    return MC_OK;
}

mc_status mc_van_get_params(mc_van *w, float *host_params, size_t n, float *host_grads)
{
    if (!w || !host_params || n != w->P.total)
        return vfail(MC_EINVAL, "mc_van_get_params: need mc_van_param_count(depth) floats");
    cudaError_t e = cudaMemcpyAsync(host_params, w->p, n * 4, cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess && host_grads)
        e = cudaMemcpyAsync(host_grads, w->g, n * 4, cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess)
        return vfail(MC_ECUDA, std::string("mc_van_get_params: ") + cudaGetErrorString(e));
    return MC_OK;
}

mc_status mc_van_get_activations(mc_van *w, int32_t layer, int32_t n, uint16_t *host_dst)
{
    if (!w || !host_dst || layer < 0 || layer > w->D - 2 || n < 1 || n > w->nmax)
        return vfail(MC_EINVAL, "mc_van_get_activations: bad argument (0 <= layer <= depth - 2, 1 <= n <= batch)");
    const size_t layer_elems = (size_t)w->nmax * w->L * w->L * kCh;
    cudaError_t e = cudaMemcpyAsync(host_dst, w->H + (size_t)layer * layer_elems, (size_t)n * w->L * w->L * kCh * 2,
                                    cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess)
        return vfail(MC_ECUDA, std::string("mc_van_get_activations: ") + cudaGetErrorString(e));
    return MC_OK;
}

mc_status mc_van_log_prob(mc_van *w, const int8_t *dev_spins, int32_t n, int32_t negate, double *dev_logq)
{
    if (!w || !dev_spins || !dev_logq || n < 1 || n > w->nmax)
        return vfail(MC_EINVAL, "mc_van_log_prob: bad argument (1 <= n <= batch)");
    cudaError_t e = cudaMemcpyAsync(w->spins, dev_spins, (size_t)n * w->L * w->L, cudaMemcpyDeviceToDevice, w->stream);
    if (e == cudaSuccess)
        e = forward(w, n, negate, dev_logq, nullptr);
    if (e != cudaSuccess)
        return vfail(MC_ECUDA, std::string("mc_van_log_prob: ") + cudaGetErrorString(e));
    return MC_OK;
}

mc_status mc_van_train_step(mc_van *w, const int8_t *dev_spins, int32_t n, float lr, int32_t apply, double *host_loss)
{
    if (!w || !dev_spins || n < 1 || n > w->nmax)
        return vfail(MC_EINVAL, "mc_van_train_step: bad argument (1 <= n <= batch)");
    cudaError_t e = cudaMemcpyAsync(w->spins, dev_spins, (size_t)n * w->L * w->L, cudaMemcpyDeviceToDevice, w->stream);
    if (e == cudaSuccess)
        e = forward(w, n, 0, w->lq, w->dF);
    if (e == cudaSuccess)
        e = backward(w, n);
    if (e == cudaSuccess && apply) {
        ++w->adam_t;
        const float b1 = 0.9f, b2 = 0.999f;
        k_adam<<<grid_for(w->P.total, 256, w->sms), 256, 0, w->stream>>>(
            w->p, w->m, w->v, w->g, w->P.total, lr, b1, b2, 1e-8f, 1.f - powf(b1, (float)w->adam_t),
            1.f - powf(b2, (float)w->adam_t));
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = prep(w);
    }
    if (e == cudaSuccess && host_loss) {
        std::vector<double> lq(n);
        e = cudaMemcpyAsync(lq.data(), w->lq, (size_t)n * 8, cudaMemcpyDeviceToHost, w->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(w->stream);
        double s = 0.0;
        for (double v : lq)
            s += v;
        *host_loss = -s / n;
    }
    if (e != cudaSuccess)
        return vfail(MC_ECUDA, std::string("mc_van_train_step: ") + cudaGetErrorString(e));
    return host_loss ? check_err(w, "mc_van_train_step") : MC_OK;
}

mc_status mc_van_sample(mc_van *w, int32_t n, uint32_t round, const uint32_t *dev_ids, int8_t *dev_out,
                        double *dev_logq)
{
    if (!w || n < 1 || n > w->nmax)
        return vfail(MC_EINVAL, "mc_van_sample: 1 <= n <= batch");
    if (!w->weights_ready) {
        cudaError_t e = prep(w);
        if (e != cudaSuccess)
            return vfail(MC_ECUDA, cudaGetErrorString(e));
    }
    int8_t *out = dev_out ? dev_out : w->prop;
    double *lq = dev_logq ? dev_logq : w->lq;
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)n * w->L * w->L, w->stream);
    if (e == cudaSuccess) {
        const unsigned blocks = (unsigned)((n + kSampleTile - 1) / kSampleTile);
        const int nbuf = sample_bufs(w->D, w->L);
        k_sample<<<blocks, kSampleThreads, sample_smem(w->D, w->L, nbuf), w->stream>>>(w->wh, w->w1, w->wD, w->bias, w->D, w->L, n,
                                                                      nbuf, w->hist, w->zero, out, lq, w->key, round, dev_ids, w->err);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return vfail(MC_ECUDA, std::string("mc_van_sample: ") + cudaGetErrorString(e));
    return MC_OK;
}

mc_status mc_van_sync(mc_van *w)
{
    if (!w)
        return vfail(MC_EINVAL, "mc_van_sync: NULL network");
    return check_err(w, "mc_van_sync");
}

mc_status mc_ising_gather(mc_ctx *c, int8_t *dev_out, int32_t back)
{
    if (!c || !dev_out || c->kind != MC_KIND_ISING || c->layout != MC_LAYOUT_INT8)
        return vfail(MC_EINVAL, "mc_ising_gather: needs an int8-layout Ising context");
    const int L = (int)c->ising[0].Lx;
    for (const auto &ch : c->ising)
        if ((int)ch.Lx != L || (int)ch.Ly != L)
            return vfail(MC_EINVAL, "mc_ising_gather: every chain must be L x L with the same L");
    const size_t total = (size_t)c->n_chains * L * L;
    k_gather<<<(unsigned)std::min<size_t>((total + 255) / 256, 4096), 256, 0, c->stream>>>(
        static_cast<const IsingChain *>(c->d_chains), c->d_lattice, dev_out, L, c->n_chains, back);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return vfail(MC_ECUDA, std::string("mc_ising_gather: ") + cudaGetErrorString(e));
    return MC_OK;
}

mc_status mc_van_mh_round(mc_van *w, mc_ctx *c, int32_t *host_accepted)
{
    if (!w || !c || c->kind != MC_KIND_ISING || c->layout != MC_LAYOUT_INT8)
        return vfail(MC_EINVAL, "mc_van_mh_round: needs an int8-layout Ising context");
    const int n = c->n_chains, L = w->L;
    if (n > w->nmax)
        return vfail(MC_EINVAL, "mc_van_mh_round: more chains than the network's batch");
    for (const auto &ch : c->ising)
        if ((int)ch.Lx != L || (int)ch.Ly != L)
            return vfail(MC_EINVAL, "mc_van_mh_round: every chain must be L x L with the network's L");
    if (c->stream != w->stream)
        return vfail(MC_EINVAL, "mc_van_mh_round: context and network must share a stream");
    // ids for the sampler: the chains' own Philox chain ids
    static_assert(sizeof(IsingChain) % 4 == 0, "chain layout");
    const uint32_t round = w->round++;
    mc_status s = mc_van_sample(w, n, round, nullptr, w->prop, w->lq); // q(s'')
    if (s != MC_OK)
        return s;
    cudaError_t e = cudaMemcpyAsync(w->spins, w->prop, (size_t)n * L * L, cudaMemcpyDeviceToDevice, w->stream);
    if (e == cudaSuccess)
        e = forward(w, n, 1, w->lq2, nullptr); // q(-s'')
    if (e == cudaSuccess)
        k_energy<<<n, 256, 0, w->stream>>>(w->prop, w->E2, L);
    if (e == cudaSuccess && mc_ising_gather(c, w->spins, 0) != MC_OK)
        return MC_ECUDA;
    if (e == cudaSuccess)
        e = forward(w, n, 0, w->lq3, nullptr); // q(s)
    if (e == cudaSuccess)
        e = forward(w, n, 1, w->lq4, nullptr); // q(-s)
    if (e == cudaSuccess)
        k_energy<<<n, 256, 0, w->stream>>>(w->spins, w->E1, L);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(w->acc, 0, 4, w->stream);
    if (e == cudaSuccess)
        k_mh_accept<<<n, 256, 0, w->stream>>>(static_cast<const IsingChain *>(c->d_chains), c->d_lattice, w->prop,
                                              w->lq, w->lq2, w->lq3, w->lq4, w->E1, w->E2, L, n, w->key, round, w->acc,
                                              w->mh_lr);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e == cudaSuccess && host_accepted) {
        e = cudaMemcpyAsync(host_accepted, w->acc, 4, cudaMemcpyDeviceToHost, w->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(w->stream);
    }
    if (e != cudaSuccess)
        return vfail(MC_ECUDA, std::string("mc_van_mh_round: ") + cudaGetErrorString(e));
    return host_accepted ? check_err(w, "mc_van_mh_round") : MC_OK;
}

mc_status mc_van_set_round(mc_van *w, uint32_t round)
{
    if (!w)
        return vfail(MC_EINVAL, "NULL network");
    w->round = round;
    return MC_OK;
}

mc_status mc_van_destroy(mc_van *w)
{
    if (!w)
        return MC_OK;
    cudaError_t e = cudaStreamSynchronize(w->stream);
    delete w;
    if (e != cudaSuccess)
        return vfail(MC_ECUDA, std::string("mc_van_destroy: ") + cudaGetErrorString(e));
    return MC_OK;
}

}  // extern "C"
