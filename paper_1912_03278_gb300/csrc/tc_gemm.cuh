// tc_gemm.cuh -- building blocks of a tcgen05 (5th-generation tensor core)
// BF16 GEMM for sm_103a, written against the PTX ISA: TMA tile loads into
// 128-byte-swizzled shared memory, mbarrier pipelines with bounded waits, MMA
// issued by one thread with the FP32 accumulator in tensor memory (TMEM), and
// tcgen05.ld for the epilogue.
//
// Tile: BM = 128 rows (M) x BN = 128 columns (N), BK = 64 BF16 (one 128-byte
// swizzle atom per row).  Both operands are K-major: A is M x K row-major,
// B is N x K row-major, D[m][n] = sum_k A[m][k] B[n][k].
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ihmc {
namespace tc {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int STAGES = 6;
constexpr int A_BYTES = BM * BK * 2;   // 16 KB
constexpr int B_BYTES = BN * BK * 2;   // 16 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 2 * BN;      // two FP32 accumulators of 128 lanes x 128 columns
constexpr int EPI_W = 16;              // columns per epilogue chunk
// The epilogue is memory-bound: EPI_GROUPS groups of four warps (one warp per
// TMEM lane quadrant) split a tile's column chunks, so that enough loads are
// in flight per SM to cover DRAM latency.
#ifndef IHMC_EPI_GROUPS
#define IHMC_EPI_GROUPS 3
#endif
constexpr int EPI_GROUPS = IHMC_EPI_GROUPS;
constexpr int EPI_WARPS = 4 * EPI_GROUPS;
constexpr int THREADS = 64 + 32 * EPI_WARPS;   // warp 0 TMA, warp 1 MMA, then the epilogue
// bounded waits: try_wait polls before the kernel gives up and flags an error
constexpr uint32_t WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 2D TMA tile load (x = inner coordinate in elements, y = row), completion
// signalled on the mbarrier as transaction bytes.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor for a K-major operand tile written by TMA
// with 128-byte swizzling: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::f16 with BF16 A and B, FP32 accumulate,
// both K-major, M = 128, N = BN.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4)                      // D format F32
           | (1u << 7)                    // A format BF16
           | (1u << 10)                   // B format BF16
           | ((uint32_t)(n >> 3) << 17)   // N / 8
           | ((uint32_t)(m >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory layout of one GEMM CTA (base aligned to 1024 bytes).
struct Smem {
    uint8_t stage[STAGES][STAGE_BYTES];
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint32_t tmem_base;
};
constexpr int SMEM_BYTES = (int)sizeof(Smem) + 1024;

// Persistent GEMM D = A B^T over an m_tiles x n_tiles grid of BM x BN tiles
// (K = nk * BK): CTA b takes tiles b, b + gridDim.x, ...  Warp 0 streams A and
// B tiles by TMA through the stage ring, warp 1 issues the MMAs into one of two TMEM
// accumulators, the epilogue warps run epi(row, col0, v[EPI_W]) on each
// 16-column chunk of each row of the other accumulator, so the epilogue of one
// tile overlaps the MMAs of the next.  Every wait is bounded; on a timeout
// the CTA flags *err and stops issuing work.
template <class Epi>
__device__ __forceinline__ void gemm_persistent(const CUtensorMap *ta, const CUtensorMap *tb,
                                                int m_tiles, int n_tiles, int nk, Epi &epi,
                                                int *err) {
    extern __shared__ uint8_t smem_raw[];
    Smem &s = *reinterpret_cast<Smem *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = m_tiles * n_tiles;
    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&s.full[i], 1);
            mbar_init(&s.empty[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&s.acc_full[b], 1);
            mbar_init(&s.acc_empty[b], EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tc_alloc(&s.tmem_base, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s.tmem_base;
    bool ok = true;

    if (warp == 0) {
        uint32_t it = 0;
        for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
            const int m0 = (t % m_tiles) * BM, n0 = (t / m_tiles) * BN;
            if (lane == 0) {
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const uint32_t st = it % STAGES;
                    if (it >= STAGES) ok = mbar_wait(&s.empty[st], ((it / STAGES) & 1) ^ 1);
                    if (!ok) break;
                    mbar_expect_tx(&s.full[st], STAGE_BYTES);
                    tma_load_2d(s.stage[st], ta, kb * BK, m0, &s.full[st]);
                    tma_load_2d(s.stage[st] + A_BYTES, tb, kb * BK, n0, &s.full[st]);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(BM, BN);
            uint32_t it = 0, lt = 0;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++lt) {
                const uint32_t buf = lt & 1;
                if (lt >= 2) ok = mbar_wait(&s.acc_empty[buf], ((lt >> 1) & 1) ^ 1);
                if (!ok) break;
                tc_fence_after();
                const uint32_t acc = tmem + buf * BN;
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const uint32_t st = it % STAGES;
                    ok = mbar_wait(&s.full[st], (it / STAGES) & 1);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t a_addr = smem_u32(s.stage[st]);
                    const uint32_t b_addr = a_addr + A_BYTES;
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k)
                        tc_mma(acc, smem_desc_sw128(a_addr + k * 32),
                               smem_desc_sw128(b_addr + k * 32), idesc,
                               (kb > 0 || k > 0) ? 1u : 0u);
                    tc_commit(&s.empty[st]);
                }
                if (!ok) break;
                tc_commit(&s.acc_full[buf]);
            }
        }
    } else {
        // epilogue warps: warp w reads TMEM lanes 32*(w%4) .. +31 and belongs
        // to group (w-2)/4, which takes chunks g, g + EPI_GROUPS, ...
        const int q = warp & 3;
        const int g = (warp - 2) >> 2;
        uint32_t lt = 0;
        for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++lt) {
            const uint32_t buf = lt & 1;
            ok = mbar_wait(&s.acc_full[buf], (lt >> 1) & 1);
            if (!ok) break;
            tc_fence_after();
            const int m0 = (t % m_tiles) * BM, n0 = (t / m_tiles) * BN;
            const int row = q * 32 + lane;
            const uint32_t base = tmem + buf * BN + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
            for (int c = g; c < BN / EPI_W; c += EPI_GROUPS) {
                float v[EPI_W];
                tc_ld16(base + (uint32_t)(c * EPI_W), v);
                epi(m0 + row, n0 + c * EPI_W, v);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&s.acc_empty[buf]);
        }
    }
    if (!ok) atomicOr(err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tc_dealloc(tmem, TMEM_COLS);
    }
}

}  // namespace tc
}  // namespace ihmc
