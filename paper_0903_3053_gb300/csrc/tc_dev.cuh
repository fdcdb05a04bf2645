// tc_dev.cuh -- Blackwell fifth-generation tensor core (tcgen05) building
// blocks in inline PTX: tensor-memory allocation, shared-memory matrix
// descriptors, the single-thread MMA issue, its completion on an mbarrier with
// a bounded wait, and the tensor-memory load for the epilogue.
//
// Operand layouts: K-major, no swizzle (below; the forward convolution's
// activations use the 64-byte swizzle instead, smem_desc_sw64, and the weight
// gradient reads its operands MN-major in that swizzle, smem_desc_mn_sw64).
// A matrix of R rows and K columns (16-bit elements) is stored as K/8 "chunk
// planes"; plane c
// holds elements 8c .. 8c+7 of every row, 16 bytes per row, rows contiguous.
// Eight consecutive rows of one plane form a core matrix (128 contiguous
// bytes), so the descriptor's leading-dimension offset (between core matrices
// adjacent in K) is the plane stride and its stride offset (between core
// matrices adjacent in M or N) is 128 bytes.  A row-shifted view of a plane is
// again a valid operand, which is what lets a convolution tap be an offset.
#pragma once
#include <cstdint>

namespace mc {
namespace tc {

// Shared-memory matrix descriptor (sm_100 format: start address, leading and
// stride byte offsets in 16-byte units, version 1, no swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo_bytes >> 4) << 16) |
           ((uint64_t)(sbo_bytes >> 4) << 32) | (1ull << 46);
}

// The same for a K-major operand of 64-byte rows (32 16-bit elements) in the
// 64-byte swizzle (16-byte chunk c of row r stored at chunk c ^ ((r >> 1) & 3),
// the pattern of a TMA box with CU_TENSOR_MAP_SWIZZLE_64B on a 1024-byte
// aligned buffer): stride offset 512 bytes (8 rows), base offset 0 -- the
// swizzle follows the absolute shared-memory address, so a view may start at any
// row and at the second 32-byte half of a row (K = 16..31).
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46) |
           (4ull << 61);
}

// The same swizzle for an MN-major operand (the M or N index runs along the
// 64-byte rows, K along the rows): a 512-byte atom holds 32 elements of M or N
// x 8 values of K; the stride offset (512 bytes) steps K by 8 and the leading
// offset `atom_stride` steps M or N by 32.  The atoms may overlap: a stride of
// 64 bytes makes atom a the view shifted by a rows, which is how a
// convolution's neighbouring taps share one staged row.
__device__ __forceinline__ uint64_t smem_desc_mn_sw64(uint32_t saddr, uint32_t atom_stride)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(atom_stride >> 4) << 16) |
           ((uint64_t)(512 >> 4) << 32) | (1ull << 46) | (4ull << 61);
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 accumulator,
// both operands K-major, tile M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The same with both operands MN-major (transpose bits 15 and 16).  With M = 64
// the accumulator's row m lies in tensor-memory lane 32 (m / 16) + m % 16:
// lanes 0-15 of each warp's quarter.
__host__ __device__ constexpr uint32_t idesc_bf16_f32_mn(int M, int N)
{
    return idesc_bf16_f32(M, N) | (1u << 15) | (1u << 16);
}

// Allocate / free `ncols` tensor-memory columns (one full warp, converged).
__device__ __forceinline__ void tmem_alloc(uint32_t dst_saddr, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_saddr), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Make this thread's generic-proxy shared-memory writes visible to the tensor core.
__device__ __forceinline__ void fence_smem_for_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (tensor memory) = A B^T (+ D when accumulate): one thread issues.
__device__ __forceinline__ void mma_bf16(uint32_t d_taddr, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_taddr),
                 "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
                 : "memory");
}

// Arrive on the mbarrier once every MMA this thread issued so far has completed.
__device__ __forceinline__ void commit(uint32_t bar_saddr)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_saddr)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar_saddr, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_saddr), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for the phase of the given parity to complete; gives up after
// `max_polls` polls and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar_saddr, uint32_t parity, int max_polls)
{
    uint32_t done = 0;
    for (int it = 0; it < max_polls; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar_saddr), "r"(parity)
                     : "memory");
        if (done)
            return true;
    }
    return false;
}

// Arrive on an mbarrier (count 1), optionally announcing `bytes` of
// asynchronous transfers that will complete on it.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar_saddr, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_saddr), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar_saddr)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar_saddr) : "memory");
}

// Tensor-map (TMA) load of one box at coordinates (c0 .. c4) into shared
// memory, completing `bytes` on the mbarrier.  `map` is the address of a
// __grid_constant__ CUtensorMap kernel parameter.  Coordinates outside the
// tensor read as zero.
__device__ __forceinline__ void tma_load_5d(uint32_t dst_saddr, const void *map, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t bar_saddr)
{
    asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst_saddr),
                 "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar_saddr)
                 : "memory");
}

// One FP32 column of this thread's tensor-memory lane.
__device__ __forceinline__ float ld_32x32b_x1(uint32_t taddr)
{
    uint32_t r0;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r0) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return __uint_as_float(r0);
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane (the warp
// reads lanes 32 (warp % 4) .. +31 starting at `taddr`).
__device__ __forceinline__ void ld_32x32b_x32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                 "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j)
        v[j] = __uint_as_float(r[j]);
}

}  // namespace tc
}  // namespace mc
