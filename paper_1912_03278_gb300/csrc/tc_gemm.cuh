// tc_gemm.cuh -- building blocks of a tcgen05 (5th-generation tensor core)
// BF16 GEMM for sm_103a, written against the PTX ISA: TMA tile loads into
// 128-byte-swizzled shared memory, mbarrier pipelines with bounded waits, MMA
// issued by one thread with the FP32 accumulator in tensor memory (TMEM), and
// tcgen05.ld for the epilogue.
//
// Two tile modes.  Single CTA: a 128 x 128 tile per CTA (M = 128, N = 128
// MMAs).  CTA pair (cta_group::2): a 256 x 256 tile per cluster of two CTAs;
// each CTA stages 128 rows of A and 128 of the 256 rows of B, the leader CTA
// issues M = 256, N = 256 MMAs that read both CTAs' shared memory, and each
// CTA's TMEM receives its 128 rows x 256 columns of the accumulator.  Per SM
// the pair mode moves half as many operand bytes through shared memory per
// MMA cycle, which is what bounds the single-CTA N = 128 mode.  BK = 64 BF16
// (one 128-byte swizzle atom per row).  Both operands are K-major: A is M x K
// row-major, B is N x K row-major, D[m][n] = sum_k A[m][k] B[n][k].
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mbarrier.cuh"

namespace ihmc {
namespace tc {

constexpr int BM = 128;                // rows of A per CTA (TMEM lanes)
constexpr int BR = 128;                // rows of B per CTA and stage
constexpr int BK = 64;
constexpr int STAGES = 6;
constexpr int A_BYTES = BM * BK * 2;   // 16 KB
constexpr int B_BYTES = BR * BK * 2;   // 16 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;

template <bool PAIR>
struct Mode {
    static constexpr int TILE_M = PAIR ? 256 : 128;   // rows of a (pair) tile
    static constexpr int TILE_N = PAIR ? 256 : 128;   // columns of a (pair) tile = MMA N
    static constexpr int TMEM_COLS = 2 * TILE_N;      // two FP32 accumulators
};
// Each epilogue functor states its chunk width Epi::W (16 or 32 columns).
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
constexpr uint32_t WAIT_LIMIT = mb::WAIT_LIMIT;
using mb::smem_u32;
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) { mb::init(bar, count); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    mb::expect_tx(bar, bytes);
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    return mb::try_wait(bar, parity);
}
// Wait for the phase with the given parity; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    return mb::wait(bar, parity);
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

// Instruction descriptor, FP32 accumulate, both operands K-major:
// kind::f16 with BF16 A and B, or kind::f8f6f4 with E4M3 A and B.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4)                      // D format F32
           | (1u << 7)                    // A format BF16
           | (1u << 10)                   // B format BF16
           | ((uint32_t)(n >> 3) << 17)   // N / 8
           | ((uint32_t)(m >> 4) << 24);  // M / 16
}
__host__ __device__ constexpr uint32_t idesc_e4m3(int m, int n) {
    return (1u << 4)                      // D format F32
           | (0u << 7)                    // A format E4M3
           | (0u << 10)                   // B format E4M3
           | ((uint32_t)(n >> 3) << 17)   // N / 8
           | ((uint32_t)(m >> 4) << 24);  // M / 16
}
// Elements of K in one 128-byte stage row, and per MMA (32 bytes).
template <bool FP8>
struct Elem {
    static constexpr int BK_ELEMS = FP8 ? 128 : 64;
};

template <bool PAIR, bool FP8 = false>
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
    if (PAIR && FP8)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    else if (FP8)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    else if (PAIR)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
}

// Arrive on bar once all prior MMAs of this thread have completed; in pair
// mode on the barrier at the same offset in both CTAs of the pair.
template <bool PAIR>
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    if (PAIR)
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster"
            ".b64 [%0], %1;" ::"r"(smem_u32(bar)),
            "h"((uint16_t)3)
            : "memory");
    else
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(bar))
            : "memory");
}

// TMEM allocation (one warp; in pair mode one warp of each CTA of the pair).
template <bool PAIR>
__device__ __forceinline__ void tc_alloc(uint32_t *dst_smem, uint32_t ncols) {
    if (PAIR) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(dst_smem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(dst_smem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
}

template <bool PAIR>
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    if (PAIR)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                     "r"(ncols)
                     : "memory");
    else
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                     "r"(ncols)
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

// ------------------------------------------------------------ clusters
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// All threads of all CTAs of the cluster.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Shared::cluster address of the object at this CTA's shared address a in CTA rank.
__device__ __forceinline__ uint32_t peer_addr(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

// 2D TMA tile load into this CTA's shared memory whose completion is signalled
// on an mbarrier of either CTA of the pair (shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, int x, int y,
                                                 uint32_t bar_cluster) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx"
        "::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar_cluster)
        : "memory");
}

// Arrive on an mbarrier of any CTA of the cluster (release at cluster scope).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster)
                 : "memory");
}

// Bounded wait with acquire at cluster scope (arrivals from the peer CTA).
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t *bar, uint32_t parity) {
    for (uint32_t i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], "
            "%2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

template <int NC>
__device__ __forceinline__ void tc_ld(uint32_t taddr, float (&v)[NC]) {
    static_assert(NC == 16 || NC == 32, "16 or 32 columns");
    if constexpr (NC == 16)
        tc_ld16(taddr, v);
    else
        tc_ld32(taddr, v);
}

// Programmatic dependent launch: wait until the grids this one depends on
// have completed and their memory is visible (no-op without the launch
// attribute), and allow the next grid on the stream to start launching.
__device__ __forceinline__ void grid_dependency_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void allow_dependent_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Shared-memory layout of one GEMM CTA (base aligned to 1024 bytes).
struct Smem {
    uint8_t stage[STAGES][STAGE_BYTES];
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t mma_done;
    uint32_t tmem_base;
};
constexpr int SMEM_BYTES = (int)sizeof(Smem) + 1024;

// Persistent GEMM D = A B^T over m_units x n_units tiles of the mode's
// TILE_M x TILE_N (K = nk * 128 bytes: 64 BF16 or, with FP8, 128 E4M3 elements per
// stage row), each computed reps times: repetition r reads
// A from row epi.a_off(r) on and B from row epi.b_off(r) on (stacked operand
// planes) and hands r to the epilogue.  Single mode: CTA b takes tiles b, b +
// gridDim.x, ..., each with all its repetitions in order.  Pair mode:
// clusters of two CTAs take tiles likewise; CTA r of a pair stages A rows
// TILE_M*um + 128 r .. +127 and B rows TILE_N*un + 128 r .. +127, signalling
// the leader's (rank 0) full barrier, whose MMA thread computes the whole
// 256 x 256 tile into both CTAs' TMEM.
//
// Warp 0 streams the stage ring by TMA, warp 1 (leader) issues the MMAs into
// one of two TMEM accumulators, and the epilogue warps of each CTA run
// epi(row, col0, v[Epi::W]) on each Epi::W-column chunk of each of its 128
// rows of the other accumulator, so the epilogue of one tile (or repetition)
// overlaps the MMAs of the next.  MMA completion releases a stage (and, per tile, an accumulator) on
// both CTAs of a pair; an accumulator is reused only after the epilogue warps
// of both CTAs have read it.  Every wait is bounded; on a timeout the CTA
// flags *err and stops issuing work.  Before teardown the producer waits for
// the release of every stage it filled and, after a timeout, the MMA thread
// for the MMAs it issued, so no copy, MMA or remote arrival is in flight when
// TMEM is freed or the CTA exits.  The set-up (barriers, TMEM, cluster) runs
// before the wait on the previous grid, so under programmatic dependent
// launch it overlaps that grid's tail.
template <bool PAIR, class Epi, bool FP8 = false>
__device__ __forceinline__ void gemm_persistent(const CUtensorMap *ta, const CUtensorMap *tb,
                                                int m_units, int n_units, int nk, int reps,
                                                Epi &epi, int *err) {
    using Md = Mode<PAIR>;
    constexpr int TN = Md::TILE_N;
    constexpr int KE = Elem<FP8>::BK_ELEMS;   // K elements per stage (128 bytes per row)
    extern __shared__ uint8_t smem_raw[];
    Smem &s = *reinterpret_cast<Smem *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = PAIR ? cluster_rank() : 0;
    const bool leader = rank == 0;
    const int c0 = PAIR ? (int)cluster_id() : (int)blockIdx.x;
    const int nclu = PAIR ? (int)cluster_count() : (int)gridDim.x;
    const int tiles = m_units * n_units;
    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&s.full[i], 1);
            mbar_init(&s.empty[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&s.acc_full[b], 1);
            mbar_init(&s.acc_empty[b], (PAIR ? 2 : 1) * EPI_WARPS);
        }
        mbar_init(&s.mma_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (PAIR) cluster_sync();   // both CTAs' barriers exist before any remote signal
    if (warp == 1) tc_alloc<PAIR>(&s.tmem_base, Md::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s.tmem_base;
    bool ok = true;
    grid_dependency_wait();
    allow_dependent_launch();

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int u = c0; u < tiles && ok; u += nclu)
            for (int r = 0; r < reps && ok; ++r) {
                const int a_row = (u % m_units) * Md::TILE_M + (int)rank * BM + epi.a_off(r);
                const int b_row = (u / m_units) * TN + (int)rank * BR + epi.b_off(r);
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const uint32_t st = it % STAGES;
                    if (it >= STAGES) ok = mbar_wait(&s.empty[st], ((it / STAGES) & 1) ^ 1);
                    if (!ok) break;
                    if (PAIR) {
                        if (leader) mbar_expect_tx(&s.full[st], 2 * STAGE_BYTES);
                        const uint32_t fb = peer_addr(smem_u32(&s.full[st]), 0);
                        tma_load_2d_pair(s.stage[st], ta, kb * KE, a_row, fb);
                        tma_load_2d_pair(s.stage[st] + A_BYTES, tb, kb * KE, b_row, fb);
                    } else {
                        mbar_expect_tx(&s.full[st], STAGE_BYTES);
                        tma_load_2d(s.stage[st], ta, kb * KE, a_row, &s.full[st]);
                        tma_load_2d(s.stage[st] + A_BYTES, tb, kb * KE, b_row, &s.full[st]);
                    }
                }
            }
            // tail: every stage filled must have been released by the MMAs
            const uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0;
            for (uint32_t i = first; i < it; ++i)
                if (!mbar_wait(&s.empty[i % STAGES], (i / STAGES) & 1)) ok = false;
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            constexpr uint32_t idesc = FP8 ? idesc_e4m3(Md::TILE_M, TN) : idesc_bf16(Md::TILE_M, TN);
            uint32_t it = 0, lt = 0;
            for (int u = c0; u < tiles && ok; u += nclu)
            for (int r = 0; r < reps && ok; ++r, ++lt) {
                const uint32_t buf = lt & 1;
                if (lt >= 2)
                    ok = PAIR ? mbar_wait_cluster(&s.acc_empty[buf], ((lt >> 1) & 1) ^ 1)
                              : mbar_wait(&s.acc_empty[buf], ((lt >> 1) & 1) ^ 1);
                if (!ok) break;
                tc_fence_after();
                const uint32_t acc = tmem + buf * TN;
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const uint32_t st = it % STAGES;
                    ok = mbar_wait(&s.full[st], (it / STAGES) & 1);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t a_addr = smem_u32(s.stage[st]);
                    const uint32_t b_addr = a_addr + A_BYTES;
#pragma unroll
                    for (int k = 0; k < 4; ++k)   // four MMAs of 32 bytes of K each
                        tc_mma<PAIR, FP8>(acc, smem_desc_sw128(a_addr + k * 32),
                                          smem_desc_sw128(b_addr + k * 32), idesc,
                                          (kb > 0 || k > 0) ? 1u : 0u);
                    tc_commit<PAIR>(&s.empty[st]);
                }
                if (!ok) break;
                tc_commit<PAIR>(&s.acc_full[buf]);
            }
            // On the normal path the epilogues have seen every accumulator
            // complete; after a timeout, wait for the MMAs already issued.
            if (!ok && it > 0) {
                tc_commit<PAIR>(&s.mma_done);
                mbar_wait(&s.mma_done, 0);
            }
        }
    } else {
        // epilogue warps: warp w reads TMEM lanes 32*(w%4) .. +31 and belongs
        // to group (w-2)/4, which takes chunks g, g + EPI_GROUPS, ...
        const int q = warp & 3;
        const int g = (warp - 2) >> 2;
        const uint32_t empty0 = PAIR ? peer_addr(smem_u32(&s.acc_empty[0]), 0) : 0;
        uint32_t lt = 0;
        for (int u = c0; u < tiles && ok; u += nclu)
        for (int r = 0; r < reps && ok; ++r, ++lt) {
            const uint32_t buf = lt & 1;
            ok = mbar_wait(&s.acc_full[buf], (lt >> 1) & 1);
            if (!ok) break;
            tc_fence_after();
            const int m0 = (u % m_units) * Md::TILE_M + (int)rank * BM;
            const int n0 = (u / m_units) * TN;
            const int row = q * 32 + lane;
            const uint32_t base = tmem + buf * TN + ((uint32_t)(q * 32) << 16);
            constexpr int EW = Epi::W;
#pragma unroll 1
            for (int c = g; c < TN / EW; c += EPI_GROUPS) {
                float v[EW];
                tc_ld<EW>(base + (uint32_t)(c * EW), v);
                epi(m0 + row, n0 + c * EW, v, r);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (PAIR)
                    mbar_arrive_cluster(empty0 + buf * (uint32_t)sizeof(uint64_t));
                else
                    mbar_arrive(&s.acc_empty[buf]);
            }
        }
    }
    if (!ok) atomicOr(err, 1);
    tc_fence_before();
    __syncthreads();
    if (PAIR) cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        tc_dealloc<PAIR>(tmem, Md::TMEM_COLS);
    }
}

}  // namespace tc
}  // namespace ihmc
