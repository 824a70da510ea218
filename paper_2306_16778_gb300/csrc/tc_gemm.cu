// tc_gemm.cu -- C -= A * B^T on the 5th-generation tensor cores (tcgen05: kind::tf32, or
// kind::f16 with bf16 operands).
//
// A is M x K and B is N x K, both K-major (row-major with the K index fastest): fp32 in
// memory read by the tensor cores as TF32, or bf16; C is M x N fp32 row-major, updated
// in place.  This is the trailing update of the mixed-precision LU: with the operands
// split into high and low parts and concatenated along K, one call computes
// C -= A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T (the 3xTF32 scheme), or with bf16 parts
// (h, m, l) the six products h h + h m + m h + h l + m m + l h (the bf16x3 scheme) --
// an update with binary32-level accuracy either way.
//
// One CTA computes one 128 x 256 tile of C: warp 0 issues TMA loads of tiles of A (128
// rows) and B (256 rows), one 128-byte row of K each (32 fp32 or 64 bf16; 128-byte
// swizzle), into a 4-stage shared-memory ring (48 KB a stage); one thread of warp 1
// issues tcgen05.mma (M = 128, N = 256, 32 bytes of K per instruction) into a 128 x 256
// fp32 accumulator in tensor memory and releases each stage with tcgen05.commit.  Then
// all four warps read the accumulator back with tcgen05.ld (warp w owns TMEM lanes
// 32w..32w+31, i.e. rows 32w..32w+31 of the tile), transpose 32-column chunks through
// shared memory (the ring is idle by then) and subtract them from C with coalesced row
// reads and writes.  The wide tile halves the operand bytes per MAC against 128 x 128
// (the operands of a K step come from L2, which does not feed every SM at the tensor
// pipe's rate).  The batch entry is the third coordinate of both tensor maps (grid z).
// Every mbarrier wait is bounded: on time-out the kernel records an error flag, stops
// issuing work, drains what it issued, frees its tensor memory and returns.
// That one-tile-per-CTA kernel runs its epilogue after the K loop, with the tensor pipe
// idle; the default launch is the persistent form further down (two accumulators, the
// epilogue of one tile under the MMAs of the next).
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "plan.cuh"
#include "tc_gemm.cuh"
#include "tcgen05_util.cuh"

namespace expm {

namespace {

constexpr int TC_BM = 128, TC_BN = 256;
constexpr int TC_ROW_BYTES = 128;                     // one 128-byte swizzled row per tile row and stage:
                                                      // 32 fp32 (TF32) or 64 bf16 elements of K
constexpr int TC_STAGES = 4;
constexpr int TC_A_BYTES = TC_BM * TC_ROW_BYTES;      // 16 KB of A per stage
constexpr int TC_B_BYTES = TC_BN * TC_ROW_BYTES;      // 32 KB of B per stage
constexpr int TC_SMEM = TC_STAGES * (TC_A_BYTES + TC_B_BYTES) + 1024 + 256;
using tcu::mbar_expect_tx;
using tcu::mbar_init;
using tcu::mbar_wait;
using tcu::smem_u32;
using tcu::tma_load_3d;

__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) { return tcu::smem_desc(saddr, 128); }

// Instruction descriptor: D fp32, A and B both TF32 (kind::tf32) or both bf16
// (kind::f16), K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tc(bool bf16, int M, int N) {
    return (1u << 4)                              // D format: F32
           | ((bf16 ? 1u : 2u) << 7)              // A format: BF16 / TF32
           | ((bf16 ? 1u : 2u) << 10)             // B format: BF16 / TF32
           | ((uint32_t)(N >> 3) << 17)           // N / 8
           | ((uint32_t)(M >> 4) << 24);          // M / 16
}

// BF16 = false: fp32 operands read as TF32, 32 of K per stage; true: bf16 operands, 64.
// Either way four MMAs of 32 bytes of K per stage.
template <bool BF16>
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                   int K, float *__restrict__ C, int ldc, int64_t cstride, int *__restrict__ err_flag) {
    constexpr int TC_BK = BF16 ? 64 : 32;
    const int bz = blockIdx.z;  // batch entry: the third coordinate of every tensor map
    C += (int64_t)bz * cstride;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned stage buffers (required by the 128-byte swizzle)
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;
    unsigned char *sB = base + TC_STAGES * TC_A_BYTES;
    uint64_t *full = (uint64_t *)(sB + TC_STAGES * TC_B_BYTES);
    uint64_t *empty = full + TC_STAGES;
    uint64_t *accum = empty + TC_STAGES;
    uint32_t *tmem_slot = (uint32_t *)(accum + 1);
    __shared__ int abort_flag;
    __shared__ int consumed;   // k-blocks whose stage the MMA issuer has taken
    __shared__ int produced;   // k-blocks whose TMA loads were issued

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int n0 = blockIdx.x * TC_BN, m0 = blockIdx.y * TC_BM;
    const int nk = (K + TC_BK - 1) / TC_BK;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        consumed = 0;
        produced = 0;
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {  // allocate 256 TMEM columns (the 128 x 256 fp32 accumulator)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer: the K ring
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % TC_STAGES;
            const uint32_t ph = (uint32_t)(kb / TC_STAGES) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            if (*(volatile int *)&abort_flag) break;
            mbar_expect_tx(&full[s], TC_A_BYTES + TC_B_BYTES);
            tma_load_3d(&mapA, &full[s], sA + s * TC_A_BYTES, kb * TC_BK, m0, bz);
            tma_load_3d(&mapB, &full[s], sB + s * TC_B_BYTES, kb * TC_BK, n0, bz);
            produced = kb + 1;
        }
    } else if (warp >= 2) {
        // idle during the K loop: pull this CTA's C tile (128 rows x 1 KB) into L2 for the
        // epilogue
        for (int e = threadIdx.x - 64; e < TC_BM * (TC_BN * 4 / 128); e += 64) {
            const int r = e / (TC_BN * 4 / 128), seg = e % (TC_BN * 4 / 128);
            const int row = m0 + r, col = n0 + seg * 32;
            if (row < M && col < N) asm volatile("prefetch.global.L2 [%0];" ::"l"(C + (int64_t)row * ldc + col));
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_tc(BF16, TC_BM, TC_BN);
        int issued = 0;
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % TC_STAGES;
            const uint32_t ph = (uint32_t)(kb / TC_STAGES) & 1u;
            if (!mbar_wait(&full[s], ph) || *(volatile int *)&abort_flag) {
                atomicExch(&abort_flag, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA + s * TC_A_BYTES), b0 = smem_u32(sB + s * TC_B_BYTES);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {  // 32 bytes of K per instruction (8 TF32 or 16 bf16)
                const uint64_t ad = smem_desc_sw128(a0 + kk * 32), bd = smem_desc_sw128(b0 + kk * 32);
                const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                if (BF16)
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.u32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                else
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.u32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
            }
            // release the stage once these MMAs have read it
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
            ++issued;
            consumed = kb + 1;
        }
        // accumulator complete (or, after an abort, everything issued has drained)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(accum))
                     : "memory");
        (void)issued;
    }
    __syncwarp();

    // epilogue: all four warps
    const bool ok = mbar_wait(accum, 0u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int aborted = *(volatile int *)&abort_flag;
    if (!ok || aborted) {
        if (threadIdx.x == 0) atomicExch(err_flag, 1);
    } else {
        // Each warp owns rows m0 + 32w .. +31.  Per 32-column chunk: tcgen05.ld gives each
        // lane one row of the accumulator; it is subtracted from the prefetched C tile in
        // shared memory, and the chunk is then written back one 128-byte row segment at a
        // time (lane = column).
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
        for (int c0 = 0; c0 < TC_BN; c0 += 32) {
            uint32_t v[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(tmem + lane_base + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            // transpose the chunk through a padded per-warp buffer (the K-ring stages are free now)
            float *stage = reinterpret_cast<float *>(base) + warp * 32 * 33;
#pragma unroll
            for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(v[j]);
            __syncwarp();
            const int col = n0 + c0 + lane;
            float cv[32];  // the chunk's 32 C values in flight together, then the stores
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int row = m0 + warp * 32 + r;
                cv[r] = (row < M && col < N) ? C[(int64_t)row * ldc + col] : 0.f;
            }
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int row = m0 + warp * 32 + r;
                if (row < M && col < N) C[(int64_t)row * ldc + col] = cv[r] - stage[r * 33 + lane];
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && (aborted || !ok)) {
        // after an abort, wait (bounded) for TMA copies that were issued but not consumed,
        // so that none lands in shared memory after this CTA has exited
        for (int kb = consumed; kb < produced; ++kb)
            mbar_wait(&full[kb % TC_STAGES], (uint32_t)(kb / TC_STAGES) & 1u);
    }
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
}

// ---------------------------------------------------------------------------------------
// Persistent form: one CTA per SM walks the tiles t = blockIdx.x, + gridDim.x, ... (N tile
// fastest, then M, then the batch entry) with two 128 x 256 accumulators in tensor memory
// (all 512 columns), so that the epilogue of one tile runs while the MMAs of the next one
// fill the other accumulator.  Warp roles (192 threads):
//   warp 0      TMA producer: the K ring, continuous across tiles (stage = global k-block
//               counter mod TC_STAGES)
//   warp 1      MMA issuer: waits until the epilogue has released the tile's accumulator
//               (acc_empty), issues the tile's MMAs, commits acc_full
//   warps 2-5   epilogue: warp w reads TMEM lanes 32 (w % 4) .. (rows of the tile), per
//               32-column chunk tcgen05.ld, a transpose through its own shared-memory
//               buffer and C -= chunk with coalesced row segments; then arrives on
//               acc_empty.  Before waiting for a tile they pull its C rows into L2.
// Every wait is bounded; on time-out the kernel raises the abort flag, every role leaves
// its loop, the MMA thread's last commit (drain) is awaited before the accumulators are
// freed, and copies issued but not consumed are awaited before the CTA exits.
constexpr int TCP_THREADS = 192;
constexpr int TCP_EPI_BYTES = 4 * 32 * 33 * 4;  // per epilogue warp a 32 x 33 fp32 transpose buffer
constexpr int TCP_SMEM = TC_STAGES * (TC_A_BYTES + TC_B_BYTES) + TCP_EPI_BYTES + 1024 + 256;

template <bool BF16>
__global__ void __launch_bounds__(TCP_THREADS, 1)
    tc_gemm_persistent(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                       int K, int batch, float *__restrict__ C, int ldc, int64_t cstride, int *__restrict__ err_flag) {
    constexpr int TC_BK = BF16 ? 64 : 32;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;
    unsigned char *sB = base + TC_STAGES * TC_A_BYTES;
    float *epi = reinterpret_cast<float *>(sB + TC_STAGES * TC_B_BYTES);
    uint64_t *full = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(epi) + TCP_EPI_BYTES);
    uint64_t *empty = full + TC_STAGES;
    uint64_t *acc_full = empty + TC_STAGES;   // [2]
    uint64_t *acc_empty = acc_full + 2;       // [2]
    uint64_t *drain = acc_empty + 2;
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    __shared__ int abort_flag;
    __shared__ long long consumed, produced;  // global k-blocks taken by the MMA issuer / issued by TMA

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nk = (K + TC_BK - 1) / TC_BK;
    const int tn = (N + TC_BN - 1) / TC_BN, tm = (M + TC_BM - 1) / TC_BM;
    const long long ntiles = (long long)tn * tm * batch;
    auto decode = [&](long long t, int &m0, int &n0, int &bz) {
        bz = (int)(t / ((long long)tn * tm));
        const int r = (int)(t % ((long long)tn * tm));
        m0 = (r / tn) * TC_BM;
        n0 = (r % tn) * TC_BN;
    };

    if (threadIdx.x == 0) {
        abort_flag = 0;
        consumed = 0;
        produced = 0;
        for (int st = 0; st < TC_STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], 4);  // the four epilogue warps
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {  // both accumulators: 512 TMEM columns (one CTA per SM)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            long long g = 0;
            for (long long t = blockIdx.x; t < ntiles && !*(volatile int *)&abort_flag; t += gridDim.x) {
                int m0, n0, bz;
                decode(t, m0, n0, bz);
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int st = (int)(g % TC_STAGES);
                    const uint32_t ph = (uint32_t)(g / TC_STAGES) & 1u;
                    if (!mbar_wait(&empty[st], ph ^ 1u) || *(volatile int *)&abort_flag) {
                        atomicExch(&abort_flag, 1);
                        break;
                    }
                    mbar_expect_tx(&full[st], TC_A_BYTES + TC_B_BYTES);
                    tma_load_3d(&mapA, &full[st], sA + st * TC_A_BYTES, kb * TC_BK, m0, bz);
                    tma_load_3d(&mapB, &full[st], sB + st * TC_B_BYTES, kb * TC_BK, n0, bz);
                    produced = g + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tc(BF16, TC_BM, TC_BN);
            long long g = 0;
            int i = 0;
            for (long long t = blockIdx.x; t < ntiles && !*(volatile int *)&abort_flag; t += gridDim.x, ++i) {
                const int a = i & 1;
                // the epilogue has read this accumulator's previous tile (first use: passes)
                if (!mbar_wait(&acc_empty[a], (uint32_t)((i >> 1) & 1) ^ 1u)) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dst = tmem + (uint32_t)(a * TC_BN);
                bool ok = true;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int st = (int)(g % TC_STAGES);
                    const uint32_t ph = (uint32_t)(g / TC_STAGES) & 1u;
                    if (!mbar_wait(&full[st], ph) || *(volatile int *)&abort_flag) {
                        atomicExch(&abort_flag, 1);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(sA + st * TC_A_BYTES), b0 = smem_u32(sB + st * TC_B_BYTES);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t ad = smem_desc_sw128(a0 + kk * 32), bd = smem_desc_sw128(b0 + kk * 32);
                        const uint32_t accu = (kb > 0 || kk > 0) ? 1u : 0u;
                        if (BF16)
                            asm volatile(
                                "{\n\t.reg .pred p;\n\t"
                                "setp.ne.u32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dst),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(accu)
                                : "memory");
                        else
                            asm volatile(
                                "{\n\t.reg .pred p;\n\t"
                                "setp.ne.u32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dst),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(accu)
                                : "memory");
                    }
                    tcu::mma_commit(&empty[st]);  // the stage is free once these MMAs have read it
                    consumed = g + 1;
                }
                if (!ok) break;
                tcu::mma_commit(&acc_full[a]);  // the tile's accumulator is complete
            }
            tcu::mma_commit(drain);  // everything issued has completed
        }
    } else {
        // epilogue warps 2..5: TMEM lane quadrant q = warp % 4 = tile rows 32 q .. 32 q + 31
        const int q = warp & 3;
        float *stage = epi + (warp - 2) * 32 * 33;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int i = 0;
        for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
            int m0, n0, bz;
            decode(t, m0, n0, bz);
            float *Cb = C + (int64_t)bz * cstride;
            // this warp's 32 rows of the C tile (1 KB each) into L2 while the MMAs run
            for (int e = lane; e < 32 * (TC_BN * 4 / 128); e += 32) {
                const int row = m0 + q * 32 + e / (TC_BN * 4 / 128), col = n0 + (e % (TC_BN * 4 / 128)) * 32;
                if (row < M && col < N) asm volatile("prefetch.global.L2 [%0];" ::"l"(Cb + (int64_t)row * ldc + col));
            }
            const int a = i & 1;
            if (!mbar_wait(&acc_full[a], (uint32_t)((i >> 1) & 1)) || *(volatile int *)&abort_flag) {
                atomicExch(&abort_flag, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int c0 = 0; c0 < TC_BN; c0 += 32) {
                uint32_t v[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                    "[%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                      "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(tmem + lane_base + (uint32_t)(a * TC_BN + c0)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (c0 + 32 >= TC_BN) {  // the accumulator is read: release it to the MMA issuer
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) tcu::mbar_arrive(&acc_empty[a]);
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(v[j]);
                __syncwarp();
                const int col = n0 + c0 + lane;
                float cv[32];
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    const int row = m0 + q * 32 + r;
                    cv[r] = (row < M && col < N) ? Cb[(int64_t)row * ldc + col] : 0.f;
                }
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    const int row = m0 + q * 32 + r;
                    if (row < M && col < N) Cb[(int64_t)row * ldc + col] = cv[r] - stage[r * 33 + lane];
                }
                __syncwarp();
            }
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    const int aborted = *(volatile int *)&abort_flag;
    if (threadIdx.x == 0) {
        // every MMA issued has completed before the accumulators are freed
        const bool drained = mbar_wait(drain, 0u);
        if (aborted || !drained) {
            atomicExch(err_flag, 1);
            // copies issued but not consumed must land before this CTA's shared memory goes
            for (long long g = consumed; g < produced; ++g)
                mbar_wait(&full[g % TC_STAGES], (uint32_t)(g / TC_STAGES) & 1u);
        }
    }
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

using tcu::EncodeFn;
using tcu::encode_fn;

// K-major operand tiles (one 128-byte swizzled row of K per tile row: 32 fp32 or 64
// bf16) or the plain fp32 C tile (TC_BN x TC_BM, no swizzle); out-of-range elements read
// as zero.
bool make_map(CUtensorMap *map, const void *ptr, int rows, int cols, int ld, int64_t bstride, int batch, int box_rows,
              bool bf16) {
    EncodeFn enc = encode_fn();
    if (!enc) return false;
    const size_t es = bf16 ? 2 : 4;
    const cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
    const cuuint64_t strides[2] = {(cuuint64_t)ld * es, (cuuint64_t)bstride * es};
    const cuuint32_t box[3] = {(cuuint32_t)(TC_ROW_BYTES / es), (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)ptr, dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The persistent two-accumulator kernel is the default; EXPM_TC_PERSISTENT=0 in the
// environment selects the one-tile-per-CTA kernel (kept for comparison).
static bool tc_persistent_enabled() {
    static const bool on = [] {
        const char *v = std::getenv("EXPM_TC_PERSISTENT");
        return !(v && v[0] == '0');
    }();
    return on;
}

template <bool BF16>
cudaError_t tc_gemm_sub(int M, int N, int K, const void *A, int lda, int64_t sA, const void *B, int ldb, int64_t sB,
                        float *C, int ldc, int64_t sC, int batch, int *err_flag, cudaStream_t st) {
    // a single matrix still gets a valid third stride (one matrix's extent)
    if (batch == 1) {
        sA = (int64_t)M * lda;
        sB = (int64_t)N * ldb;
        sC = (int64_t)M * ldc;
    }
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, M, K, lda, sA, batch, TC_BM, BF16) || !make_map(&mb, B, N, K, ldb, sB, batch, TC_BN, BF16))
        return cudaErrorInvalidValue;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(tc_gemm_kernel<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
        if (attr == cudaSuccess)
            attr = cudaFuncSetAttribute(tc_gemm_persistent<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, TCP_SMEM);
    });
    if (attr != cudaSuccess) return attr;
    const long long ntiles = (long long)((N + TC_BN - 1) / TC_BN) * ((M + TC_BM - 1) / TC_BM) * batch;
    if (tc_persistent_enabled()) {
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const unsigned grid = (unsigned)std::min<long long>(ntiles, sms);
        tc_gemm_persistent<BF16><<<grid, TCP_THREADS, TCP_SMEM, st>>>(ma, mb, M, N, K, batch, C, ldc, sC, err_flag);
        return cudaGetLastError();
    }
    dim3 grid((N + TC_BN - 1) / TC_BN, (M + TC_BM - 1) / TC_BM, batch);
    tc_gemm_kernel<BF16><<<grid, 128, TC_SMEM, st>>>(ma, mb, M, N, K, C, ldc, sC, err_flag);
    return cudaGetLastError();
}

int run_hook(bool bf16, int M, int N, int K, const void *A, int lda, const void *B, int ldb, float *C, int ldc) {
    if (!tc_gemm_supported(M, N, K, A, lda, B, ldb, C, ldc, bf16)) return 1;
    int *flag = nullptr;
    if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) return 1;
    cudaMemset(flag, 0, sizeof(int));
    cudaError_t e = bf16 ? tc_gemm_sub<true>(M, N, K, A, lda, 0, B, ldb, 0, C, ldc, 0, 1, flag, 0)
                         : tc_gemm_sub<false>(M, N, K, A, lda, 0, B, ldb, 0, C, ldc, 0, 1, flag, 0);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, flag, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(flag);
    if (e != cudaSuccess) return 1;
    return h ? 2 : 0;
}

// The time-out path of the bounded waits, with nothing in flight: one thread waits on an
// mbarrier that expects one arrival.  arrive = 0: nothing arrives, so mbar_wait gives up
// after `limit` polls; arrive = 1: the thread arrives first and the wait succeeds.
// status[0] = 1 if the wait gave up, status[1] = elapsed SM clocks / 1024.
__global__ void wait_probe_kernel(long long limit, int arrive, int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    tcu::mbar_init(&bar, 1);
    if (arrive) tcu::mbar_arrive(&bar);
    const long long t0 = clock64();
    const bool ok = mbar_wait(&bar, 0u, limit);
    const long long dt = (clock64() - t0) >> 10;
    status[0] = ok ? 0 : 1;
    status[1] = (int)(dt < 0x7fffffffLL ? dt : 0x7fffffffLL);
}

}  // namespace

bool tc_gemm_supported(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const void *C, int ldc,
                       bool bf16, int64_t sA, int64_t sB, int64_t sC) {
    if (M < 1 || N < 1 || K < 1) return false;
    const int q = bf16 ? 8 : 4;  // operand rows (and batch strides) a multiple of 16 bytes
    if ((lda % q) || (ldb % q) || (ldc % 4) || ((uintptr_t)A % 16) || ((uintptr_t)B % 16) || ((uintptr_t)C % 16))
        return false;
    if ((sA % q) || (sB % q) || (sC % 4)) return false;
    return encode_fn() != nullptr;
}

cudaError_t tc_gemm_tf32_sub(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
                             int *err_flag, cudaStream_t st) {
    return tc_gemm_sub<false>(M, N, K, A, lda, 0, B, ldb, 0, C, ldc, 0, 1, err_flag, st);
}

cudaError_t tc_gemm_bf16_sub(int M, int N, int K, const uint16_t *A, int lda, const uint16_t *B, int ldb, float *C,
                             int ldc, int *err_flag, cudaStream_t st) {
    return tc_gemm_sub<true>(M, N, K, A, lda, 0, B, ldb, 0, C, ldc, 0, 1, err_flag, st);
}

cudaError_t tc_gemm_batched(bool bf16, int M, int N, int K, const void *A, int lda, int64_t sA, const void *B, int ldb,
                            int64_t sB, float *C, int ldc, int64_t sC, int batch, int *err_flag, cudaStream_t st) {
    return bf16 ? tc_gemm_sub<true>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, batch, err_flag, st)
                : tc_gemm_sub<false>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, batch, err_flag, st);
}

}  // namespace expm

// Test hooks (not part of the documented interface): C -= A B^T with the tensor-core
// kernel on device buffers (fp32 operands read as TF32, or bf16 operands); return 0, or
// 1 for unsupported arguments / CUDA errors, or 2 when a bounded wait gave up.
extern "C" int expm_internal_tc_gemm_tf32(int M, int N, int K, const float *A, int lda, const float *B, int ldb,
                                          float *C, int ldc) {
    return expm::run_hook(false, M, N, K, A, lda, B, ldb, C, ldc);
}
extern "C" int expm_internal_tc_gemm_bf16(int M, int N, int K, const uint16_t *A, int lda, const uint16_t *B, int ldb,
                                          float *C, int ldc) {
    return expm::run_hook(true, M, N, K, A, lda, B, ldb, C, ldc);
}

// Test hook: runs the probe above on the current device; returns 0 (the wait completed),
// 2 (it gave up: the status the tensor-core kernels turn into EXPM_ETIMEOUT) or 1 (bad
// arguments, CUDA error).  elapsed_kclk (host, optional) receives the wait's SM clocks / 1024.
extern "C" int expm_internal_wait_probe(long long limit, int arrive, int *elapsed_kclk) {
    if (limit < 1 || limit > expm::tcu::SPIN_LIMIT) return 1;
    int *d = nullptr;
    if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) return 1;
    expm::wait_probe_kernel<<<1, 32>>>(limit, arrive ? 1 : 0, d);
    int h[2] = {0, 0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return 1;
    if (elapsed_kclk) *elapsed_kclk = h[1];
    return h[0] ? 2 : 0;
}
