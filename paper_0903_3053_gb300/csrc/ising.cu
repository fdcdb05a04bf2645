// ising.cu -- 2D Ising Metropolis sweep on the red/black checkerboard
// (Eq. (1), Sec. 2.3), two storage layouts:
//
//   int8  : s[y][x] = +-1, one byte per spin.
//   MSC32 : multi-spin coding, 32 spins per 32-bit word and one bit per spin
//           (the paper stores spins as 1-bit variables, Sec. 2.3).  Each
//           colour c has its own plane of Ly rows x W = Lx/64 words; bit b of
//           word w in row y of plane c is the site of colour c with in-row
//           index j = 32 w + b, i.e. x = 2 j + ((y + c) & 1).  With that packing
//           the four neighbours of a whole word are: the same word of the other
//           plane in rows y-1, y and y+1, and the row-y word of the other plane
//           shifted by one bit (towards w-1 or w+1 depending on the row parity).
//           Anti-aligned neighbours are counted bit-sliced for 32 spins at once.
//
// Random numbers: site i = y*(Lx/2) + j of colour c uses word (i & 3) of the
// Philox block with counter (i >> 2, sweep, TAG_METRO | c, chain_id), so the
// stream does not depend on layout, tiling or launch shape.  A spin flips when
// dE = 2 s h <= 0, or when its word is below T[dE] = floor(e^{-beta dE} 2^32)
// (integer thresholds, no floating point on the path).
//
// Execution modes:
//   grid     : one launch per colour over every chain of the batch; chain of a
//              block found by binary search over per-chain block offsets.
//   resident : one CTA per chain holding its whole lattice in shared memory and
//              running all sweeps of a call in one launch (small lattices).
// The energy/magnetisation measurement (the paper's sweep+measure kernels) is
// fused into the colour-1 half-sweep: each colour-1 site counts its
// anti-aligned bonds (every bond joins exactly one colour-1 site) and pairs
// itself with one colour-0 site for the magnetisation; exact integer sums via
// warp reductions and one 64-bit atomic per CTA.
#include "ising_dev.cuh"

namespace mc {
namespace {

// ------------------------------------------------------------------ grid mode
template <int C, int LAYOUT>
__device__ __forceinline__ void half_sweep(const SweepArgs &a)
{
    const int k = find_chain(a.block_start, a.n_chains, blockIdx.x);
    const IsingChain ch = static_cast<const IsingChain *>(a.chains)[k];
    const uint32_t t = (blockIdx.x - a.block_start[k]) * blockDim.x + threadIdx.x;
    const uint32_t sweep = (uint32_t)(a.state->sweep_base + a.k);
    const bool measure = (C == 1) && a.measure;
    uint32_t anti = 0, up = 0;
    if (LAYOUT == MC_LAYOUT_INT8) {
        int8_t *s = reinterpret_cast<int8_t *>(a.lattice + ch.spin_off);
        const uint32_t groups = (((ch.Lx * ch.Ly) >> 1) + 3) >> 2;
        if (t < groups) {
            const PhiloxSchedule ks = philox_schedule(ch.key);
            if (measure)
                int8_group<C, true>(s, ch, ks, t, sweep, anti, up);
            else
                int8_group<C, false>(s, ch, ks, t, sweep, anti, up);
        }
    } else {
        const uint32_t W = ch.W, nw = W * ch.Ly;
        uint32_t *base = reinterpret_cast<uint32_t *>(a.lattice + ch.spin_off);
        uint32_t *pc = base + (size_t)C * nw;
        const uint32_t *po = base + (size_t)(1 - C) * nw;
        if (t < W * (ch.Ly >> 1)) { // one thread per row pair and word column
            const PhiloxSchedule ks = philox_schedule(ch.key);
            const uint32_t yy = t / W, w = t - yy * W;
            if (measure)
                msc_row_pair<C, true>(pc, po, yy, w, ch, ks, sweep, anti, up);
            else
                msc_row_pair<C, false>(pc, po, yy, w, ch, ks, sweep, anti, up);
        }
    }
    if (!a.measure)
        return;
    const long long slot = (long long)((a.state->rec_head + a.rec_k) % (unsigned long long)a.cap);
    DevRecord *rec = &a.series[(long long)k * a.cap + slot];
    if (C == 0) {
        if (t == 0) { // zero the record before the colour-1 kernel accumulates into it
            rec->sweep = (long long)(a.state->sweep_base + a.k);
            rec->a = 0;
            rec->b = 0;
            rec->d0 = rec->d1 = rec->d2 = 0.0;
        }
        return;
    }
    block_sum2(anti, up);
    if (threadIdx.x == 0) {
        atomicAdd(&rec->a, (unsigned long long)anti);
        atomicAdd(&rec->b, (unsigned long long)up);
    }
}

// Two launch-bound flavours of the same half-sweep: blocks of at most 256
// threads with 8 resident per SM (32 registers: full occupancy also for the
// measuring colour-1 kernel, +1.7% on the MSC benchmark batch), and blocks of
// up to 1024 threads for callers that ask for them.
template <int C, int LAYOUT>
__global__ void __launch_bounds__(256, 8) k_half_sweep(SweepArgs a) { half_sweep<C, LAYOUT>(a); }
template <int C, int LAYOUT>
__global__ void __launch_bounds__(1024) k_half_sweep_big(SweepArgs a) { half_sweep<C, LAYOUT>(a); }

template <int C, int LAYOUT>
void launch_half_sweep(mc_ctx *c, const SweepArgs &a)
{
    if (c->threads <= 256)
        k_half_sweep<C, LAYOUT><<<c->grid_blocks, c->threads, 0, c->ls>>>(a);
    else
        k_half_sweep_big<C, LAYOUT><<<c->grid_blocks, c->threads, 0, c->ls>>>(a);
}

// ------------------------------------------------------------------ resident mode
template <int LAYOUT>
__global__ void __launch_bounds__(1024) k_resident(SweepArgs a, uint32_t n_sweeps, uint32_t every)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int k = blockIdx.x;
    const IsingChain ch = static_cast<const IsingChain *>(a.chains)[k];
    const uint32_t bytes = LAYOUT == MC_LAYOUT_INT8 ? ch.Lx * ch.Ly : 8u * ch.Ly * ch.W;
    uint32_t *gl = reinterpret_cast<uint32_t *>(a.lattice + ch.spin_off);
    uint32_t *sl = reinterpret_cast<uint32_t *>(smem);
    for (uint32_t u = threadIdx.x; u < bytes / 4; u += blockDim.x)
        sl[u] = gl[u];
    __syncthreads();
    const PhiloxSchedule ks = philox_schedule(ch.key);
    const unsigned long long base = a.state->sweep_base;
    for (uint32_t t = 0; t < n_sweeps; ++t) {
        const uint32_t sweep = (uint32_t)(base + t);
        const bool measure = every != 0 && ((t + 1) % every) == 0;
        uint32_t anti = 0, up = 0;
        if (LAYOUT == MC_LAYOUT_INT8) {
            int8_t *s = reinterpret_cast<int8_t *>(smem);
            const uint32_t groups = (((ch.Lx * ch.Ly) >> 1) + 3) >> 2;
            for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x)
                int8_group<0, false>(s, ch, ks, g, sweep, anti, up);
            __syncthreads();
            if (measure) {
                for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x)
                    int8_group<1, true>(s, ch, ks, g, sweep, anti, up);
            } else {
                for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x)
                    int8_group<1, false>(s, ch, ks, g, sweep, anti, up);
            }
        } else {
            const uint32_t W = ch.W, nw = W * ch.Ly, pairs = W * (ch.Ly >> 1);
            uint32_t *p0 = sl, *p1 = sl + nw;
            for (uint32_t u = threadIdx.x; u < pairs; u += blockDim.x) {
                const uint32_t yy = u / W, w = u - yy * W;
                msc_row_pair<0, false>(p0, p1, yy, w, ch, ks, sweep, anti, up);
            }
            __syncthreads();
            if (measure) {
                for (uint32_t u = threadIdx.x; u < pairs; u += blockDim.x) {
                    const uint32_t yy = u / W, w = u - yy * W;
                    msc_row_pair<1, true>(p1, p0, yy, w, ch, ks, sweep, anti, up);
                }
            } else {
                for (uint32_t u = threadIdx.x; u < pairs; u += blockDim.x) {
                    const uint32_t yy = u / W, w = u - yy * W;
                    msc_row_pair<1, false>(p1, p0, yy, w, ch, ks, sweep, anti, up);
                }
            }
        }
        if (measure) {
            block_sum2(anti, up);
            if (threadIdx.x == 0) {
                const unsigned long long r = a.state->rec_head + (t + 1) / every - 1;
                DevRecord *rec = &a.series[(long long)k * a.cap + (long long)(r % (unsigned long long)a.cap)];
                rec->sweep = (long long)(base + t);
                rec->a = anti;
                rec->b = up;
                rec->d0 = rec->d1 = rec->d2 = 0.0;
            }
        }
        __syncthreads();
    }
    for (uint32_t u = threadIdx.x; u < bytes / 4; u += blockDim.x)
        gl[u] = sl[u];
}

// ------------------------------------------------------------------ init
// Hot start: spin +1 iff the top bit of its random word (sweep field 0, tag
// INIT | colour) is set; cold start: all +1 (Sec. 2.1).
__global__ void k_init_int8(IsingChain ch, int8_t *s, int hot)
{
    const uint32_t n = ch.Lx * ch.Ly;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const uint32_t y = p / ch.Lx, x = p - y * ch.Lx;
        int8_t v = 1;
        if (hot) {
            const uint32_t c = (x + y) & 1u, i = y * (ch.Lx >> 1) + (x >> 1);
            const uint4 r = philox4x32_10(make_uint4(i >> 2, 0u, kTagIsingInit | c, ch.chain_id), ch.key);
            const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
            v = (rr[i & 3u] >> 31) ? 1 : -1;
        }
        s[p] = v;
    }
}

__global__ void k_init_msc(IsingChain ch, uint32_t *base, int hot)
{
    const uint32_t nw = ch.Ly * ch.W;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < 2 * nw; u += gridDim.x * blockDim.x) {
        const uint32_t c = u / nw, t = u - c * nw, y = t / ch.W, w = t - y * ch.W;
        uint32_t word = 0xFFFFFFFFu;
        if (hot) {
            word = 0;
            const uint32_t blk0 = y * (ch.Lx >> 3) + 8 * w;
            for (int kk = 0; kk < 8; ++kk) {
                const uint4 r = philox4x32_10(make_uint4(blk0 + kk, 0u, kTagIsingInit | c, ch.chain_id), ch.key);
                word |= ((r.x >> 31) << (4 * kk)) | ((r.y >> 31) << (4 * kk + 1)) | ((r.z >> 31) << (4 * kk + 2)) |
                        ((r.w >> 31) << (4 * kk + 3));
            }
        }
        base[u] = word;
    }
}

// ------------------------------------------------------------------ measure (standalone)
template <int LAYOUT>
__global__ void k_measure(IsingChain ch, const char *lat, DevRecord *out)
{
    uint32_t anti = 0, up = 0;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (LAYOUT == MC_LAYOUT_INT8) {
        const int8_t *s = reinterpret_cast<const int8_t *>(lat);
        const uint32_t Lx = ch.Lx, Ly = ch.Ly, half = Lx >> 1, nc = (Lx * Ly) >> 1;
        if (tid < nc) {
            const uint32_t y = tid / half, j = tid - y * half, x = 2 * j + ((y + 1) & 1u);
            const int sv = s[y * Lx + x];
            const int ne = s[y * Lx + inc_wrap(x, Lx)], nw = s[y * Lx + dec_wrap(x, Lx)];
            const int nn = s[dec_wrap(y, Ly) * Lx + x], ns = s[inc_wrap(y, Ly) * Lx + x];
            anti = (ne != sv) + (nw != sv) + (nn != sv) + (ns != sv);
            up = (sv > 0) + (((x & 1u) ? nw : ne) > 0);
        }
    } else {
        const uint32_t W = ch.W, Ly = ch.Ly, nw = W * Ly;
        const uint32_t *p0 = reinterpret_cast<const uint32_t *>(lat), *p1 = p0 + nw;
        if (tid < nw) {
            const uint32_t y = tid / W, w = tid - y * W;
            uint32_t nu, nd, ns, side;
            msc_neighbours<1>(p0, y, w, W, Ly, nu, nd, ns, side);
            const uint32_t s = p1[tid];
            anti = __popc(s ^ nu) + __popc(s ^ nd) + __popc(s ^ ns) + __popc(s ^ side);
            up = __popc(s) + __popc(ns);
        }
    }
    block_sum2(anti, up);
    if (threadIdx.x == 0) {
        atomicAdd(&out->a, (unsigned long long)anti);
        atomicAdd(&out->b, (unsigned long long)up);
    }
}

// ------------------------------------------------------------------ config I/O
// Canonical int8 s[y][x] <-> MSC planes; one thread per MSC word.
__global__ void k_msc_from_int8(IsingChain ch, const int8_t *src, uint32_t *dst)
{
    const uint32_t nw = ch.Ly * ch.W;
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= 2 * nw)
        return;
    const uint32_t c = u / nw, t = u - c * nw, y = t / ch.W, w = t - y * ch.W;
    uint32_t word = 0;
    for (int b = 0; b < 32; ++b) {
        const uint32_t x = 2 * (32 * w + b) + ((y + c) & 1u);
        word |= (uint32_t)(src[y * ch.Lx + x] > 0) << b;
    }
    dst[u] = word;
}

__global__ void k_msc_to_int8(IsingChain ch, const uint32_t *src, int8_t *dst)
{
    const uint32_t nw = ch.Ly * ch.W;
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= 2 * nw)
        return;
    const uint32_t c = u / nw, t = u - c * nw, y = t / ch.W, w = t - y * ch.W;
    const uint32_t word = src[u];
    for (int b = 0; b < 32; ++b) {
        const uint32_t x = 2 * (32 * w + b) + ((y + c) & 1u);
        dst[y * ch.Lx + x] = ((word >> b) & 1u) ? 1 : -1;
    }
}

// Canonical bit rows (bit b of word v of row y = site x = 32 v + b) <-> MSC.
// Even bits of x to its low half and odd bits to its high half (the outer
// perfect unshuffle written as four delta swaps; Warren, "Hacker's Delight",
// Sec. 7-2), and the inverse shuffle.
__device__ __forceinline__ uint32_t bit_unshuffle(uint32_t x)
{
    uint32_t t;
    t = (x ^ (x >> 1)) & 0x22222222u; x ^= t ^ (t << 1);
    t = (x ^ (x >> 2)) & 0x0C0C0C0Cu; x ^= t ^ (t << 2);
    t = (x ^ (x >> 4)) & 0x00F000F0u; x ^= t ^ (t << 4);
    t = (x ^ (x >> 8)) & 0x0000FF00u; x ^= t ^ (t << 8);
    return x;
}
__device__ __forceinline__ uint32_t bit_shuffle(uint32_t x)
{
    uint32_t t;
    t = (x ^ (x >> 8)) & 0x0000FF00u; x ^= t ^ (t << 8);
    t = (x ^ (x >> 4)) & 0x00F000F0u; x ^= t ^ (t << 4);
    t = (x ^ (x >> 2)) & 0x0C0C0C0Cu; x ^= t ^ (t << 2);
    t = (x ^ (x >> 1)) & 0x22222222u; x ^= t ^ (t << 1);
    return x;
}

// Canonical bit rows <-> the two colour planes.  One thread per 64-site chunk u
// = y W + w of a row (canonical words 2u, 2u + 1, read or written once, 8
// contiguous bytes per thread, so that a page-locked host buffer can be read
// or written by the kernel directly): its even-x sites are word u of plane
// y & 1, its odd-x sites word u of the other plane.
__global__ void k_msc_from_bits(IsingChain ch, const uint32_t *src, uint32_t *dst)
{
    const uint32_t nw = ch.Ly * ch.W;
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nw)
        return;
    const uint32_t y = u / ch.W;
    const uint32_t a = bit_unshuffle(src[2 * u]), b = bit_unshuffle(src[2 * u + 1]);
    dst[(y & 1u) * nw + u] = (a & 0xFFFFu) | (b << 16);          // x even
    dst[((y + 1u) & 1u) * nw + u] = (a >> 16) | (b & 0xFFFF0000u); // x odd
}

__global__ void k_msc_to_bits(IsingChain ch, const uint32_t *src, uint32_t *dst)
{
    const uint32_t nw = ch.Ly * ch.W;
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nw)
        return;
    const uint32_t y = u / ch.W;
    const uint32_t even = src[(y & 1u) * nw + u], odd = src[((y + 1u) & 1u) * nw + u];
    dst[2 * u] = bit_shuffle((even & 0xFFFFu) | (odd << 16));
    dst[2 * u + 1] = bit_shuffle((even >> 16) | (odd & 0xFFFF0000u));
}

__global__ void k_int8_from_bits(IsingChain ch, const uint32_t *src, int8_t *dst)
{
    const uint32_t n = ch.Lx * ch.Ly;
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n)
        dst[p] = ((src[p >> 5] >> (p & 31u)) & 1u) ? 1 : -1;
}

__global__ void k_int8_to_bits(IsingChain ch, const int8_t *src, uint32_t *dst)
{
    const uint32_t nwords = (ch.Lx * ch.Ly) >> 5;
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nwords)
        return;
    uint32_t word = 0;
    for (int b = 0; b < 32; ++b)
        word |= (uint32_t)(src[32 * v + b] > 0) << b;
    dst[v] = word;
}

__global__ void k_advance(DevState *st, unsigned long long n, unsigned long long recs)
{
    st->sweep_base += n;
    st->rec_head += recs;
}

inline unsigned blocks_for(size_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

// =========================================================================== host
size_t ising_config_bytes(const IsingChain &ch, int fmt)
{
    const size_t n = (size_t)ch.Lx * ch.Ly;
    if (fmt == MC_FMT_INT8)
        return n;
    if (fmt == MC_FMT_BITS)
        return (ch.Lx % 32 == 0) ? n / 8 : 0;
    return 0;
}

// Work units per chain for a grid-mode launch: Philox groups (int8) or row pairs (MSC).
static uint32_t grid_units(const mc_ctx *c, const IsingChain &ch)
{
    if (c->layout == MC_LAYOUT_INT8)
        return (((ch.Lx * ch.Ly) >> 1) + 3) >> 2;
    return (ch.Ly >> 1) * ch.W; // row pairs x words
}

void ising_plan_grid(mc_ctx *c)
{
    c->block_start.assign(c->n_chains + 1, 0);
    uint32_t acc = 0;
    for (int k = 0; k < c->n_chains; ++k) {
        c->block_start[k] = acc;
        acc += blocks_for(grid_units(c, c->ising[k]), c->threads);
    }
    c->block_start[c->n_chains] = acc;
    c->grid_blocks = acc;
}

static size_t resident_bytes(const mc_ctx *c, const IsingChain &ch)
{
    return c->layout == MC_LAYOUT_INT8 ? (size_t)ch.Lx * ch.Ly : (size_t)8 * ch.Ly * ch.W;
}

bool ising_resident_fits(const mc_ctx *c, int *smem_bytes)
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    size_t need = 0;
    for (const auto &ch : c->ising) {
        const size_t b = resident_bytes(c, ch);
        if (b % 4 != 0)
            return false;
        need = b > need ? b : need;
    }
    if (smem_bytes)
        *smem_bytes = (int)need;
    return need + 1024 <= (size_t)optin;
}

// Threads of a resident CTA: the work units of the largest chain (int8: groups
// of four same-colour sites; MSC32: row pairs) rounded up to a warp, at most
// the block size -- the caller's (mc_set_mode), else 1024 when every chain has
// an SM to itself and the default (256) when chains share SMs.  Threads past
// the last unit would idle through every half-sweep and hold the SM's warp
// slots: a 64^2 MSC32 lattice has 32 row pairs, and with one-warp CTAs a batch
// of 4096 such chains is resident on the 152 SMs in one wave (1.23e12 against
// 0.96e12 spin flips/s with 256-thread CTAs, four waves of one working warp
// each).  With a CTA per SM to spare, more threads shorten each half-sweep:
// one 64^2 int8 chain 2.44 against 2.99 us per sweep with 512 threads, one
// 256^2 MSC32 chain 7.8 against 9.2 us.
static int resident_threads(const mc_ctx *c)
{
    uint32_t units = 0;
    for (const auto &ch : c->ising) {
        const uint32_t u = c->layout == MC_LAYOUT_INT8 ? ((((ch.Lx * ch.Ly) >> 1) + 3) >> 2) : ch.W * (ch.Ly >> 1);
        units = u > units ? u : units;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int cap = c->threads_set || c->n_chains > sms ? c->threads : 1024;
    const int t = (int)((units + 31) / 32 * 32);
    return t < 32 ? 32 : (t < cap ? t : cap);
}

// Raise the dynamic shared-memory limit of the resident kernels (outside any
// graph capture).
cudaError_t ising_prepare_resident(mc_ctx *c)
{
    int smem = 0;
    if (!ising_resident_fits(c, &smem))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_resident<MC_LAYOUT_INT8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_resident<MC_LAYOUT_MSC32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

cudaError_t ising_init_launch(mc_ctx *c, const mc_chain_desc *desc)
{
    for (int k = 0; k < c->n_chains; ++k) {
        const IsingChain &ch = c->ising[k];
        char *p = c->d_lattice + ch.spin_off;
        if (c->layout == MC_LAYOUT_INT8) {
            k_init_int8<<<blocks_for((size_t)ch.Lx * ch.Ly, 256), 256, 0, c->ls>>>(
                ch, reinterpret_cast<int8_t *>(p), desc[k].start == MC_HOT);
        } else {
            k_init_msc<<<blocks_for((size_t)2 * ch.Ly * ch.W, 256), 256, 0, c->ls>>>(
                ch, reinterpret_cast<uint32_t *>(p), desc[k].start == MC_HOT);
        }
    }
    return cudaGetLastError();
}

cudaError_t advance_state_launch(mc_ctx *c, long long n, long long recs)
{
    k_advance<<<1, 1, 0, c->ls>>>(c->d_state, (unsigned long long)n, (unsigned long long)recs);
    return cudaGetLastError();
}

cudaError_t ising_sweep_enqueue(mc_ctx *c, long long n, int every, int mode)
{
    SweepArgs a{};
    a.chains = c->d_chains;
    a.block_start = c->d_block_start;
    a.n_chains = c->n_chains;
    a.lattice = c->d_lattice;
    a.series = c->d_series;
    a.state = c->d_state;
    a.cap = c->cap;
    a.tries = nullptr;
    if (mode == MC_MODE_RESIDENT) {
        int smem = 0;
        if (!ising_resident_fits(c, &smem))
            return cudaErrorInvalidValue;
        const int threads = resident_threads(c);
        cudaError_t e = prof_begin(c);
        if (e != cudaSuccess)
            return e;
        if (c->layout == MC_LAYOUT_INT8)
            k_resident<MC_LAYOUT_INT8><<<c->n_chains, threads, smem, c->ls>>>(a, (uint32_t)n, (uint32_t)every);
        else
            k_resident<MC_LAYOUT_MSC32><<<c->n_chains, threads, smem, c->ls>>>(a, (uint32_t)n, (uint32_t)every);
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
        return prof_end(c);
    }
    for (long long t = 0; t < n; ++t) {
        a.k = (uint32_t)t;
        a.measure = every > 0 && ((t + 1) % every) == 0;
        a.rec_k = a.measure ? (uint32_t)((t + 1) / every - 1) : 0u;
        for (int colour = 0; colour < 2; ++colour) {
            cudaError_t e = prof_begin(c);
            if (e != cudaSuccess)
                return e;
            if (c->layout == MC_LAYOUT_INT8) {
                if (colour == 0)
                    launch_half_sweep<0, MC_LAYOUT_INT8>(c, a);
                else
                    launch_half_sweep<1, MC_LAYOUT_INT8>(c, a);
            } else {
                if (colour == 0)
                    launch_half_sweep<0, MC_LAYOUT_MSC32>(c, a);
                else
                    launch_half_sweep<1, MC_LAYOUT_MSC32>(c, a);
            }
            e = prof_end(c);
            if (e != cudaSuccess)
                return e;
        }
    }
    return cudaGetLastError();
}

cudaError_t ising_measure_launch(mc_ctx *c, int chain, DevRecord *out)
{
    const IsingChain &ch = c->ising[chain];
    const char *lat = c->d_lattice + ch.spin_off;
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(DevRecord), c->ls);
    if (e != cudaSuccess)
        return e;
    if (c->layout == MC_LAYOUT_INT8)
        k_measure<MC_LAYOUT_INT8><<<blocks_for(((size_t)ch.Lx * ch.Ly) >> 1, 256), 256, 0, c->ls>>>(ch, lat, out);
    else
        k_measure<MC_LAYOUT_MSC32><<<blocks_for((size_t)ch.Ly * ch.W, 256), 256, 0, c->ls>>>(ch, lat, out);
    return cudaGetLastError();
}

cudaError_t ising_config_io(mc_ctx *c, int chain, int fmt, void *buf, bool to_lattice)
{
    const IsingChain &ch = c->ising[chain];
    char *lat = c->d_lattice + ch.spin_off;
    const size_t n = (size_t)ch.Lx * ch.Ly;
    if (c->layout == MC_LAYOUT_INT8) {
        if (fmt == MC_FMT_INT8) // buf: device memory or page-locked host memory
            return to_lattice ? cudaMemcpyAsync(lat, buf, n, cudaMemcpyDefault, c->ls)
                              : cudaMemcpyAsync(buf, lat, n, cudaMemcpyDefault, c->ls);
        if (to_lattice)
            k_int8_from_bits<<<blocks_for(n, 256), 256, 0, c->ls>>>(ch, static_cast<const uint32_t *>(buf),
                                                                        reinterpret_cast<int8_t *>(lat));
        else
            k_int8_to_bits<<<blocks_for(n / 32, 256), 256, 0, c->ls>>>(ch, reinterpret_cast<const int8_t *>(lat),
                                                                           static_cast<uint32_t *>(buf));
        return cudaGetLastError();
    }
    const size_t words = (size_t)2 * ch.Ly * ch.W;
    uint32_t *msc = reinterpret_cast<uint32_t *>(lat);
    if (fmt == MC_FMT_INT8) {
        if (to_lattice)
            k_msc_from_int8<<<blocks_for(words, 256), 256, 0, c->ls>>>(ch, static_cast<const int8_t *>(buf), msc);
        else
            k_msc_to_int8<<<blocks_for(words, 256), 256, 0, c->ls>>>(ch, msc, static_cast<int8_t *>(buf));
    } else {
        if (to_lattice)
            k_msc_from_bits<<<blocks_for(words / 2, 256), 256, 0, c->ls>>>(ch, static_cast<const uint32_t *>(buf), msc);
        else
            k_msc_to_bits<<<blocks_for(words / 2, 256), 256, 0, c->ls>>>(ch, msc, static_cast<uint32_t *>(buf));
    }
    return cudaGetLastError();
}

}  // namespace mc
