// oz_gemm.cu -- the refinement residual R_s -= t A X_s with binary64-level accuracy on
// the bf16 tensor cores (tcgen05, kind::f16), by splitting both operands into integer
// slices (the error-free splitting of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Splitting.  Each row i of A (real view: K2 = n or 2n columns, re/im interleaved) gets
// a power-of-two scale 2^E_i > max_k |A_ik|; each complex column c of system s of X gets
// 2^F_sc > max_l max(|Re X_lc|, |Im X_lc|).  A value x with scale 2^E is rounded to the
// 55-bit fixed-point integer V = round(x 2^(55-E)) and written in balanced base-256
// digits, x = 2^(E-7) sum_{p=0..6} d_p 2^(-8p) (+ at most 2^(E-56)), with d_0 in
// [-128, 128] and d_1..d_6 in [-128, 127].  Slice p stores d_p 2^(-8p) in bf16 -- exact,
// eight significant bits at most.
//
// Products.  (A X)_ij = 2^(E_i + F_j - 14) sum_{p,q} sum_k a_p(ik) b_q(kj), where a_p, b_q
// are the slices.  The 28 slice products with p + q <= 6 are kept (the rest weigh about
// 2^-56 of max|A_i.| max|X_.j| K2 -- the scale is the row's largest entry, so a row whose
// other entries are much smaller, as in a dominant diagonal, needs these last bits) and
// summed on the tensor cores into five fp32 accumulators in tensor memory: p+q = 0, 1,
// 2, 3 (each an integer multiple of 2^(-8(p+q)) whose magnitude stays below 2^22 of
// those units over a K window of 64, hence exact whatever the accumulation's rounding),
// and p+q >= 4 together (it weighs 2^-32 of the first; the tensor core's fp32
// accumulation rounds it, measured to be toward zero, which is why p+q = 3 has an
// accumulator of its own).  After every window of 64 the accumulators are read back
// (tcgen05.ld); the four exact ones are turned into integers by adding a power-of-two
// "magic" constant (exact in the stated ranges) and added into one 64-bit integer per
// output in units of 2^-24 of the first accumulator's unit (|window| < 2^44.01, so the
// sum stays below 2^63 for any K2 <= 2^17), and the p+q >= 4 one is summed in fp32 --
// relative precision, which matters where the result is far below the scale product
// (entries much smaller than their row's largest).  The epilogue forms T 2^-24 + S in
// binary64, scales it by 2^(E_i + F_j - 14) and subtracts t times it from R.
//
// Layout of the real GEMM D = A' B'^T (M = n rows, N2 = 2 nsys kc output columns, K2):
// output column j = s (2 kc) + 2 c + part (part 0 = Re, 1 = Im), so row i of system s
// is 2 kc contiguous doubles of R.  For complex A, K index 2l + c' holds Re/Im of A_il and
// B' row j has (Re X_lc, -Im X_lc) (part 0) or (Im X_lc, Re X_lc) (part 1) at 2l, 2l+1;
// for real A, K index l and B' row j holds Re or Im of X_lc.
//
// Kernel: one CTA per 128 x 96 output tile, 320 threads.  Warp 8 issues TMA loads of
// 32-wide bf16 boxes of all seven slices of A (128 rows) and of B' (96 rows) -- 64-byte
// rows, 64-byte swizzle -- into a 2-stage ring (98 KB a stage); one thread of warp 9
// issues 56 tcgen05.mma (M = 128, N = 96, K = 16) per stage into the five accumulators
// (480 of the 512 TMEM columns); warps 0..7 drain the accumulators once per window (warp
// w: TMEM lanes 32 (w % 4) .., columns 48 (w / 4) ..) and hold the 64-bit sums in
// registers.  K beyond K2 and rows
// beyond n / N2 are zero-filled by TMA.  Every wait is bounded: on time-out the kernel
// sets an error flag, drains what it issued, frees tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "arith.cuh"
#include "oz_gemm.cuh"
#include "tcgen05_util.cuh"

namespace expm {

namespace {

using namespace tcu;

constexpr int OZ_S = 7;                       // slices of a binary64 operand
constexpr int OZ_BM = 128, OZ_BN = 96;        // output tile (5 accumulators x 96 <= 512 TMEM columns)
constexpr int OZ_BK = 32;                     // K per stage: 32 bf16 = 64-byte rows
constexpr int OZ_KW = 64;                     // K per accumulator window (two stages)
constexpr int OZ_ASLICE = OZ_BM * OZ_BK * 2;  // 8 KB: one slice of A per stage
constexpr int OZ_BSLICE = OZ_BN * OZ_BK * 2;  // 6 KB: one slice of B' per stage
constexpr int OZ_THREADS = 320;

// Kernel configurations.  Full: the residual V - M X, seven slices of A and of X, the 28
// products with p + q <= 6, accumulators p+q = 0, 1, 2, 3 exact and p+q >= 4 rounded.
// Light: the update -M D of a residual by a binary32 correction D (|D| ~ 1e-6 |X|, so
// its product is needed to about 2^-30 only): four slices of A and of D (32 bits below
// the row / column scale: three would hold a binary32 value exactly only near its
// column's largest entry), the 10 products with p + q <= 3, accumulators p+q = 0, 1, 2
// exact and 3 rounded.
#define OZ_TABLE(name, ...)                                              \
    static __host__ __device__ constexpr int name(int i) {               \
        constexpr unsigned char t[] = {__VA_ARGS__};                     \
        return t[i];                                                     \
    }
struct OzFull {
    static constexpr int SA = 7, SB = 7, NPAIR = 28, NACC = 5, STAGES = 2;
    static constexpr bool EXACT3 = true;
    OZ_TABLE(pp, 0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4, 0, 1, 2, 3, 4, 5, 0, 1, 2, 3, 4, 5, 6)
    OZ_TABLE(qq, 0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0, 5, 4, 3, 2, 1, 0, 6, 5, 4, 3, 2, 1, 0)
    OZ_TABLE(acc, 0, 1, 1, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4)
    OZ_TABLE(first, 1, 1, 0, 1, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0)
};
struct OzLight {
    static constexpr int SA = 4, SB = 4, NPAIR = 10, NACC = 4, STAGES = 4;
    static constexpr bool EXACT3 = false;
    OZ_TABLE(pp, 0, 0, 1, 0, 1, 2, 0, 1, 2, 3)
    OZ_TABLE(qq, 0, 1, 0, 2, 1, 0, 3, 2, 1, 0)
    OZ_TABLE(acc, 0, 1, 1, 2, 2, 2, 3, 3, 3, 3)
    OZ_TABLE(first, 1, 1, 0, 1, 0, 0, 1, 0, 0, 0)
};
#undef OZ_TABLE
template <class C> __host__ __device__ constexpr int oz_ahalf() { return C::SA * OZ_ASLICE; }
template <class C> __host__ __device__ constexpr int oz_stage() {  // a multiple of 1024
    return C::SA * OZ_ASLICE + C::SB * OZ_BSLICE;
}
template <class C> __host__ __device__ constexpr int oz_smem() { return C::STAGES * oz_stage<C>() + 1024 + 256; }

// kind::f16 instruction descriptor: D fp32, A and B bf16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ int biased_exp(double x) {
    const int e = (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff);
    return e > 0 ? e : 1;  // zero and subnormals: the subnormal exponent
}

// the seven slices of x (scale 2^(ebias - 1022)), as bf16 bit patterns of d_p 2^(-8p)
__device__ __forceinline__ void oz_digits(double x, int ebias, uint16_t out[OZ_S]) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    int ex = (int)((u >> 52) & 0x7ff);
    unsigned long long m = u & ((1ull << 52) - 1);
    long long V = 0;
    if (ex != 0x7ff) {  // non-finite values give zero slices; their row or column is flagged by its scale
        if (ex == 0) ex = 1;
        else m |= 1ull << 52;
        // |x| = m 2^(ex - 1075) < 2^(ebias - 1022), so V = round(m 2^(ex - ebias + 2)) < 2^55
        const int r = ebias - 2 - ex;  // >= -2
        if (r <= 0) V = (long long)(m << (-r));
        else V = r > 60 ? 0 : (long long)((m + (1ull << (r - 1))) >> r);
        if (u >> 63) V = -V;
    }
    int d[OZ_S];
#pragma unroll
    for (int p = OZ_S - 1; p >= 1; --p) {
        const int dig = (int)((V + 128) & 255) - 128;
        d[p] = dig;
        V = (V - dig) >> 8;
    }
    d[0] = (int)V;
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) {
        // d_p 2^(-8p): exact in binary32 and in bf16 (the low 16 bits of the float are zero).
        // |d_p| <= 2^8, so d_p becomes a float exactly by the 1.5 2^23 bias trick on the FP32
        // pipe (an integer-to-float conversion instruction would run on the FP64 unit)
        const float dp = __fsub_rn(__int_as_float(0x4b400000 + d[p]), 12582912.0f);
        const float f = dp * __int_as_float((127 - 8 * p) << 23);
        out[p] = (uint16_t)(__float_as_uint(f) >> 16);
    }
}

// max biased exponent of each row of the real view (n rows, K2 values, row stride ld)
__global__ void oz_row_exp(int K2, const double *__restrict__ A, int64_t ld, int *__restrict__ E) {
    const double *a = A + (int64_t)blockIdx.x * ld;
    int m = 1;
    for (int k = threadIdx.x; k < K2; k += blockDim.x) m = max(m, biased_exp(a[k]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ int wm[32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? wm[threadIdx.x] : 1;
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) E[blockIdx.x] = m;
    }
}

// slices of A: As[p][i][k] (ld K2p), two values of a row per thread
__global__ void oz_split_rows(int rows, int K2, int K2p, const double *__restrict__ A, int64_t ld,
                              const int *__restrict__ E, uint16_t *__restrict__ As) {
    const int hp = (K2 + 1) / 2;
    const int64_t total = (int64_t)rows * hp;
    const int64_t plane = (int64_t)rows * K2p;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / hp), k = 2 * (int)(idx % hp);
        const int eb = E[i];
        uint16_t d0[OZ_S], d1[OZ_S];
        oz_digits(A[(int64_t)i * ld + k], eb, d0);
        const bool two = k + 1 < K2;
        oz_digits(two ? A[(int64_t)i * ld + k + 1] : 0.0, eb, d1);
        uint16_t *o = As + (int64_t)i * K2p + k;
#pragma unroll
        for (int p = 0; p < OZ_S; ++p) {
            if (two) *reinterpret_cast<uint32_t *>(o + p * plane) = (uint32_t)d0[p] | ((uint32_t)d1[p] << 16);
            else o[p * plane] = d0[p];
        }
    }
}

// max biased exponent (binary64 terms) of each complex column (s, c) of X, binary64 or
// binary32 (F preset to zero)
template <class XT>
__global__ void oz_col_exp(int n, int kc, const cx<XT> *__restrict__ X, int64_t nk, int *__restrict__ F) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, s = blockIdx.z;
    if (c >= kc) return;
    const int l0 = blockIdx.y * 64, l1 = min(n, l0 + 64);
    int m = 1;
    for (int l = l0; l < l1; ++l) {
        const cx<XT> x = X[(int64_t)s * nk + (int64_t)l * kc + c];
        m = max(m, max(biased_exp((double)x.re), biased_exp((double)x.im)));
    }
    atomicMax(&F[s * kc + c], m);
}

// slices of B': Bs[q][j][k] (ld K2p), q < NS (the leading NS of the seven digits),
// one complex X value per thread (l fastest)
template <class XT, int NS>
__global__ void oz_split_cols(int n, int kc, int nsys, int complex_a, int K2p, int64_t N2,
                              const cx<XT> *__restrict__ X, int64_t nk, const int *__restrict__ F,
                              uint16_t *__restrict__ Bs) {
    const int64_t total = (int64_t)nsys * kc * n;
    const int64_t plane = N2 * K2p;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(idx % n);
        const int64_t sc = idx / n;
        const int c = (int)(sc % kc), s = (int)(sc / kc);
        const cx<XT> x = X[(int64_t)s * nk + (int64_t)l * kc + c];
        const int fb = F[s * kc + c];
        uint16_t dr[OZ_S], di[OZ_S];
        oz_digits((double)x.re, fb, dr);
        oz_digits((double)x.im, fb, di);
        const int64_t jre = (int64_t)s * 2 * kc + 2 * c;
        if (complex_a) {
            uint16_t *o0 = Bs + jre * K2p + 2 * l, *o1 = o0 + K2p;
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                const uint32_t ndi = (uint32_t)(di[q] ^ (di[q] ? 0x8000u : 0u));  // -Im (exact: a sign flip)
                *reinterpret_cast<uint32_t *>(o0 + q * plane) = (uint32_t)dr[q] | (ndi << 16);
                *reinterpret_cast<uint32_t *>(o1 + q * plane) = (uint32_t)di[q] | ((uint32_t)dr[q] << 16);
            }
        } else {
            uint16_t *o0 = Bs + jre * K2p + l, *o1 = o0 + K2p;
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                o0[q * plane] = dr[q];
                o1[q * plane] = di[q];
            }
        }
    }
}

// magic-constant conversion: bits(v + M) - bits(M) = v / ulp(M) for v a multiple of
// ulp(M) with |v| < M / 3 (exact), else v / ulp(M) rounded to nearest
__device__ __forceinline__ int magic_int(float v, float M) { return (int)(__float_as_uint(__fadd_rn(v, M)) - __float_as_uint(M)); }

__device__ __forceinline__ void tmem_ld4(uint32_t addr, uint32_t (&v)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(addr));
}

template <class Cfg>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M,
                   int64_t N2, int K2, int kc, int64_t nk, double t, const int *__restrict__ E,
                   const int *__restrict__ F, double *__restrict__ R, int *__restrict__ err_flag) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int STAGES = Cfg::STAGES, STAGE = oz_stage<Cfg>(), AHALF = oz_ahalf<Cfg>();
    // stage s: A slices at base + s * STAGE, B' slices AHALF after them
    uint64_t *full = (uint64_t *)(base + STAGES * STAGE);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;     // MMA -> drain: a window's accumulators are complete
    uint64_t *tempty = tfull + 1;         // drain -> MMA: the accumulators have been read
    uint64_t *done = tempty + 1;          // every MMA issued has completed
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    __shared__ int abort_flag;
    __shared__ int consumed, produced;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int m0 = blockIdx.x * OZ_BM;
    const int64_t n0 = (int64_t)blockIdx.y * OZ_BN;
    const int nst = (K2 + OZ_KW - 1) / OZ_KW * 2;  // stages (whole windows)
    const int nwin = nst / 2;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        consumed = produced = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tfull, 1);
        mbar_init(tempty, 8);
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 9) {  // 512 TMEM columns: five 128 x 96 fp32 accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 8) {
        if (lane == 0) {  // TMA producer
            for (int kb = 0; kb < nst; ++kb) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u)) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
                if (*(volatile int *)&abort_flag) break;
                unsigned char *st = base + s * STAGE;
                mbar_expect_tx(&full[s], STAGE);
                tma_load_3d(&mapA, &full[s], st, kb * OZ_BK, m0, 0);
                tma_load_3d(&mapB, &full[s], st + AHALF, kb * OZ_BK, (int)n0, 0);
                produced = kb + 1;
            }
        }
    } else if (warp == 9) {
        if (lane == 0) {  // MMA issuer
            constexpr uint32_t idesc = idesc_bf16(OZ_BM, OZ_BN);
            for (int kb = 0; kb < nst; ++kb) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                const bool wstart = (kb & 1) == 0;
                if ((wstart && kb > 0 && !mbar_wait(tempty, (uint32_t)((kb / 2 - 1) & 1))) ||
                    !mbar_wait(&full[s], ph) || *(volatile int *)&abort_flag) {
                    atomicExch(&abort_flag, 1);
                    mma_commit(tfull);  // wakes the drain warps, which then see the flag
                    break;
                }
                fence_after_sync();
                const uint32_t a0 = smem_u32(base + s * STAGE), b0 = a0 + AHALF;
#pragma unroll
                for (int kk = 0; kk < OZ_BK / 16; ++kk) {  // K = 16 bf16 = 32 bytes per instruction
#pragma unroll
                    for (int pr = 0; pr < Cfg::NPAIR; ++pr) {
                        const uint64_t ad = smem_desc(a0 + Cfg::pp(pr) * OZ_ASLICE + kk * 32, 64);
                        const uint64_t bd = smem_desc(b0 + Cfg::qq(pr) * OZ_BSLICE + kk * 32, 64);
                        const uint32_t acc = (wstart && kk == 0 && Cfg::first(pr)) ? 0u : 1u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\t"
                            "setp.ne.u32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                tmem + (uint32_t)Cfg::acc(pr) * OZ_BN),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                }
                mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
                if (!wstart) mma_commit(tfull);
                consumed = kb + 1;
            }
            mma_commit(done);
        }
    } else {
        // drain warps: rows m0 + 32 (warp % 4) + lane, columns n0 + 48 (warp / 4) + [0, 48)
        const int q4 = warp & 3, half = warp >> 2;
        const uint32_t tbase = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(half * 48);
        long long T[48];  // p+q <= 3, exact, in units of 2^-24 of the first accumulator's unit
        float S[48];      // p+q >= 4, in fp32 (relative precision)
#pragma unroll
        for (int c = 0; c < 48; ++c) {
            T[c] = 0;
            S[c] = 0.f;
        }
        const float M0 = 12582912.0f;  // 1.5 * 2^23: ulp 1
        const float M1 = 49152.0f;     // 1.5 * 2^15: ulp 2^-8
        const float M2 = 192.0f;       // 1.5 * 2^7:  ulp 2^-16
        const float M3 = 1.5f;         // ulp 2^-23
        const float M4 = 0.75f;        // 1.5 * 2^-1: ulp 2^-24
        bool ok = true;
        for (int w = 0; w < nwin; ++w) {
            if (!mbar_wait(tfull, (uint32_t)(w & 1)) || *(volatile int *)&abort_flag) {
                ok = false;
                break;
            }
            fence_after_sync();
#pragma unroll
            for (int g = 0; g < 12; ++g) {
                uint32_t v0[4], v1[4], v2[4], v3[4], v4[4];
                tmem_ld4(tbase + 0 * OZ_BN + 4 * g, v0);
                tmem_ld4(tbase + 1 * OZ_BN + 4 * g, v1);
                tmem_ld4(tbase + 2 * OZ_BN + 4 * g, v2);
                tmem_ld4(tbase + 3 * OZ_BN + 4 * g, v3);
                if (Cfg::EXACT3) tmem_ld4(tbase + 4 * OZ_BN + 4 * g, v4);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i0 = magic_int(__uint_as_float(v0[e]), M0);  // |.| <= 2^20
                    const int i1 = magic_int(__uint_as_float(v1[e]), M1);  // |.| <= 2^21
                    const int i2 = magic_int(__uint_as_float(v2[e]), M2);  // |.| <= 3 * 2^20
                    int i3 = 0;
                    float xr;  // the rounded accumulator: p+q >= 4 (full) or p+q = 3 (light)
                    if (Cfg::EXACT3) {
                        // p+q = 3: a multiple of 2^-24 with |.| <= 2^-2, in two exact steps
                        // (to 2^-23, then the remainder 0 or +-2^-24)
                        const float x3 = __uint_as_float(v3[e]);
                        const float h3 = __fsub_rn(__fadd_rn(x3, M3), M3);
                        i3 = 2 * magic_int(x3, M3) + magic_int(__fsub_rn(x3, h3), M4);  // x3 * 2^24
                        xr = __uint_as_float(v4[e]);
                    } else {
                        xr = __uint_as_float(v3[e]);
                    }
                    const int a = i0 * 256 + i1;  // |a| < 2^28.1
                    const int c = i2 * 256 + i3;  // |c| < 2^29.7
                    T[4 * g + e] += (long long)a * 65536 + (long long)c;
                    S[4 * g + e] = __fadd_rn(S[4 * g + e], xr);
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty);
        }
        if (!ok) {
            if (lane == 0) atomicExch(&abort_flag, 1);
        } else {
            // The operand ring is idle now (every stage was consumed before the last window
            // completed): each warp stages its 32 x 48 sums there ([row][column], padded),
            // then writes its rows with the lanes across columns (contiguous in R).
            long long *sT = reinterpret_cast<long long *>(base) + warp * 32 * 49;
            float *sS = reinterpret_cast<float *>(base + 8 * 32 * 49 * 8) + warp * 32 * 49;
#pragma unroll
            for (int c = 0; c < 48; ++c) {
                sT[lane * 49 + c] = T[c];
                sS[lane * 49 + c] = S[c];
            }
            __syncwarp();
            const int64_t skc = 2 * (int64_t)kc;
            for (int r = 0; r < 32; ++r) {
                const int i = m0 + q4 * 32 + r;
                if (i >= M) break;
                const int eb = E[i];
                for (int c = lane; c < 48; c += 32) {
                    const int64_t j = n0 + half * 48 + c;
                    if (j >= N2) continue;
                    const int64_t s = j / skc, rem = j - s * skc;
                    const int fb = F[s * kc + rem / 2];
                    double *rp = R + (s * nk + (int64_t)i * kc) * 2 + rem;
                    // (T 2^-24 + S) in units of 2^(E_i + F_j - 14)
                    const double v = (eb == 0x7ff || fb == 0x7ff)
                                         ? __longlong_as_double(0x7ff8000000000000ll)
                                         : ldexp(fma((double)sS[r * 49 + c], 16777216.0, (double)sT[r * 49 + c]),
                                                 eb + fb - 2082);
                    *rp = fma(-t, v, *rp);
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool aborted = *(volatile int *)&abort_flag != 0;
        // every issued MMA has completed before the tensor memory is freed; after an abort,
        // wait (bounded) for TMA copies that were issued but not consumed
        if (!mbar_wait(done, 0u)) atomicExch(err_flag, 1);
        if (aborted) {
            atomicExch(err_flag, 1);
            for (int kb = consumed; kb < produced; ++kb)
                mbar_wait(&full[kb % STAGES], (uint32_t)(kb / STAGES) & 1u);
        }
    }
    __syncthreads();
    if (warp == 9) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// 3-D map over the slices: dims (K2, rows, nslices), row stride K2p bf16, box 32 x box_rows x
// box_slices (the leading slices),
// 64-byte swizzle; out-of-range elements read as zero
bool make_slice_map(CUtensorMap *map, const uint16_t *ptr, int64_t rows, int K2, int K2p, int box_rows, int nslices,
                    int box_slices) {
    EncodeFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)K2, (cuuint64_t)rows, (cuuint64_t)nslices};
    const cuuint64_t strides[2] = {(cuuint64_t)K2p * 2, (cuuint64_t)rows * K2p * 2};
    const cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows, (cuuint32_t)box_slices};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)ptr, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct OzLayout {
    int K2, K2p;
    int64_t N2;
    size_t As, Bs, E, F, flag, total;
};

OzLayout oz_layout(int n, int kc, int nsys, int complex_a) {
    OzLayout L{};
    L.K2 = complex_a ? 2 * n : n;
    L.K2p = (L.K2 + OZ_KW - 1) / OZ_KW * OZ_KW;
    L.N2 = (int64_t)nsys * 2 * kc;
    size_t off = 0;
    L.As = off; off += al256((size_t)OZ_S * n * L.K2p * 2);  // A part first: independent of kc, nsys
    L.E = off; off += al256((size_t)n * 4);
    L.Bs = off; off += al256((size_t)OZ_S * L.N2 * L.K2p * 2);
    L.F = off; off += al256((size_t)nsys * kc * 4);
    L.flag = off; off += al256(4);
    L.total = off;
    return L;
}

}  // namespace

size_t oz_resid_bytes(int n, int kc, int nsys, int complex_a) { return oz_layout(n, kc, nsys, complex_a).total; }

bool oz_resid_supported(int n, int kc, int nsys) {
    if (n < 1 || kc < 1 || nsys < 1) return false;
    if ((int64_t)nsys * 2 * kc > (1ll << 30) || n > (1 << 16)) return false;  // K2 <= 2^17
    return encode_fn() != nullptr;
}

cudaError_t oz_split_a(int n, const double *A, int64_t lda, int complex_a, void *ws, cudaStream_t st) {
    const OzLayout L = oz_layout(n, 1, 1, complex_a);
    unsigned char *b = (unsigned char *)ws;
    int *E = (int *)(b + L.E);
    const int64_t ld = complex_a ? 2 * lda : lda;  // real view
    oz_row_exp<<<n, 256, 0, st>>>(L.K2, A, ld, E);
    const int64_t work = (int64_t)n * ((L.K2 + 1) / 2);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 16));
    oz_split_rows<<<grid, 256, 0, st>>>(n, L.K2, L.K2p, A, ld, E, (uint16_t *)(b + L.As));
    return cudaGetLastError();
}

cudaError_t oz_split_x(int n, int kc, int nsys, int complex_a, const cx<double> *X, int64_t nk, void *ws,
                       cudaStream_t st) {
    // the A part of the layout (slices, row scales) does not depend on kc or nsys
    const OzLayout L = oz_layout(n, kc, nsys, complex_a);
    unsigned char *b = (unsigned char *)ws;
    int *F = (int *)(b + L.F);
    cudaError_t e = cudaMemsetAsync(F, 0, sizeof(int) * (size_t)nsys * kc, st);
    if (e != cudaSuccess) return e;
    oz_col_exp<double><<<dim3((kc + 127) / 128, (n + 63) / 64, nsys), 128, 0, st>>>(n, kc, X, nk, F);
    const int64_t work = (int64_t)nsys * kc * n;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 16));
    oz_split_cols<double, OZ_S><<<grid, 256, 0, st>>>(n, kc, nsys, complex_a, L.K2p, L.N2, X, nk, F,
                                                      (uint16_t *)(b + L.Bs));
    return cudaGetLastError();
}

cudaError_t oz_split_d(int n, int kc, int nsys, int complex_a, const cx<float> *D, int64_t nk, void *ws,
                       cudaStream_t st) {
    const OzLayout L = oz_layout(n, kc, nsys, complex_a);
    unsigned char *b = (unsigned char *)ws;
    int *F = (int *)(b + L.F);
    cudaError_t e = cudaMemsetAsync(F, 0, sizeof(int) * (size_t)nsys * kc, st);
    if (e != cudaSuccess) return e;
    oz_col_exp<float><<<dim3((kc + 127) / 128, (n + 63) / 64, nsys), 128, 0, st>>>(n, kc, D, nk, F);
    const int64_t work = (int64_t)nsys * kc * n;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 16));
    oz_split_cols<float, OzLight::SB><<<grid, 256, 0, st>>>(n, kc, nsys, complex_a, L.K2p, L.N2, D, nk, F,
                                                            (uint16_t *)(b + L.Bs));
    return cudaGetLastError();
}

// every product within the slice counts and accumulators, ordered by p + q, and the
// last accumulator used
template <class Cfg> constexpr bool oz_tables_ok() {
    for (int i = 0; i < Cfg::NPAIR; ++i) {
        if (Cfg::pp(i) >= Cfg::SA || Cfg::qq(i) >= Cfg::SB || Cfg::acc(i) >= Cfg::NACC) return false;
        if (i > 0 && Cfg::pp(i) + Cfg::qq(i) < Cfg::pp(i - 1) + Cfg::qq(i - 1)) return false;
    }
    return Cfg::acc(Cfg::NPAIR - 1) == Cfg::NACC - 1;
}

template <class Cfg>
static cudaError_t oz_launch(int n, int kc, int nsys, int complex_a, double t, int64_t nk, cx<double> *R, void *ws,
                             cudaStream_t st, int *timeout) {
    static_assert(oz_tables_ok<Cfg>(), "slice-product tables");
    const OzLayout L = oz_layout(n, kc, nsys, complex_a);
    unsigned char *b = (unsigned char *)ws;
    int *F = (int *)(b + L.F), *flag = (int *)(b + L.flag);
    cudaError_t e;
    CUtensorMap ma, mb;
    // A's stored seven slices (the leading Cfg::SA read); B' holds Cfg::SB planes
    if (!make_slice_map(&ma, (const uint16_t *)(b + L.As), n, L.K2, L.K2p, OZ_BM, OZ_S, Cfg::SA) ||
        !make_slice_map(&mb, (const uint16_t *)(b + L.Bs), L.N2, L.K2, L.K2p, OZ_BN, Cfg::SB, Cfg::SB))
        return cudaErrorInvalidValue;
    static cudaError_t attr =
        cudaFuncSetAttribute(oz_gemm_kernel<Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize, oz_smem<Cfg>());
    if (attr != cudaSuccess) return attr;
    if ((e = cudaMemsetAsync(flag, 0, sizeof(int), st)) != cudaSuccess) return e;
    const dim3 gg((unsigned)((n + OZ_BM - 1) / OZ_BM), (unsigned)((L.N2 + OZ_BN - 1) / OZ_BN), 1);
    oz_gemm_kernel<Cfg><<<gg, OZ_THREADS, oz_smem<Cfg>(), st>>>(ma, mb, n, L.N2, L.K2, kc, nk, t,
                                                                (const int *)(b + L.E), F, (double *)R, flag);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (timeout) {
        e = cudaMemcpyAsync(timeout, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return e;
}

cudaError_t oz_product(int n, int kc, int nsys, int complex_a, double t, int64_t nk, cx<double> *R, void *ws,
                       cudaStream_t st, int *timeout) {
    return oz_launch<OzFull>(n, kc, nsys, complex_a, t, nk, R, ws, st, timeout);
}

cudaError_t oz_product_light(int n, int kc, int nsys, int complex_a, double t, int64_t nk, cx<double> *R, void *ws,
                             cudaStream_t st, int *timeout) {
    return oz_launch<OzLight>(n, kc, nsys, complex_a, t, nk, R, ws, st, timeout);
}

cudaError_t oz_read_timeout(int n, int kc, int nsys, int complex_a, void *ws, cudaStream_t st, int *timeout) {
    const OzLayout L = oz_layout(n, kc, nsys, complex_a);
    cudaError_t e = cudaMemcpyAsync(timeout, (unsigned char *)ws + L.flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    return e == cudaSuccess ? cudaStreamSynchronize(st) : e;
}

}  // namespace expm

// Test hook (not part of the documented interface): R_s -= t A X_s for s < nsys on
// device buffers (A n x n binary64, real or interleaved complex, row stride lda in
// elements; X_s and R_s n x kc interleaved complex, system stride n kc).  Returns 0,
// 1 for unsupported arguments or CUDA errors, 2 when a bounded wait gave up.
extern "C" int expm_internal_oz_resid(int n, int kc, int nsys, int complex_a, double t, const double *A, int64_t lda,
                                      const double *X, double *R) {
    using namespace expm;
    if (!oz_resid_supported(n, kc, nsys) || lda < n) return 1;
    void *ws = nullptr;
    if (cudaMalloc(&ws, oz_resid_bytes(n, kc, nsys, complex_a)) != cudaSuccess) return 1;
    int to = 0;
    cudaError_t e = oz_split_a(n, A, lda, complex_a, ws, 0);
    if (e == cudaSuccess) e = oz_split_x(n, kc, nsys, complex_a, (const cx<double> *)X, (int64_t)n * kc, ws, 0);
    if (e == cudaSuccess) e = oz_product(n, kc, nsys, complex_a, t, (int64_t)n * kc, (cx<double> *)R, ws, 0, &to);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(ws);
    if (e != cudaSuccess) return 1;
    return to ? 2 : 0;
}

// Test hook (not part of the documented interface): R_s -= t A D_s with the light product
// (D_s binary32 complex n x kc, system stride n kc).  Returns as the hook above.
extern "C" int expm_internal_oz_resid_light(int n, int kc, int nsys, int complex_a, double t, const double *A,
                                            int64_t lda, const float *D, double *R) {
    using namespace expm;
    if (!oz_resid_supported(n, kc, nsys) || lda < n) return 1;
    void *ws = nullptr;
    if (cudaMalloc(&ws, oz_resid_bytes(n, kc, nsys, complex_a)) != cudaSuccess) return 1;
    int to = 0;
    cudaError_t e = oz_split_a(n, A, lda, complex_a, ws, 0);
    if (e == cudaSuccess) e = oz_split_d(n, kc, nsys, complex_a, (const cx<float> *)D, (int64_t)n * kc, ws, 0);
    if (e == cudaSuccess)
        e = oz_product_light(n, kc, nsys, complex_a, t, (int64_t)n * kc, (cx<double> *)R, ws, 0, &to);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(ws);
    if (e != cudaSuccess) return 1;
    return to ? 2 : 0;
}
