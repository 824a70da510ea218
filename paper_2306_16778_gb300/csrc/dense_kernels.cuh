// dense_kernels.cuh -- building blocks of the pole-batched dense path (SIMT).
//
// All matrices are row-major complex (cx<T>, interleaved re/im) unless noted.
// Every kernel is batched over blockIdx.z ("batch" = pole pair); a batch stride
// of 0 shares one operand between batches.
//
//   form_shifted     M_s = t A - c I + theta_s I           (the shift of Sec. 3)
//   lu_diag          unpivoted LU of one nb x nb diagonal block in shared memory
//   trsm_left        op(T)^{-1} B for a triangular nb x nb block T (4 variants)
//   trsm_right_upper B U^{-1} (the L21 panel of the blocked LU)
//   cgemm            C = beta C + alpha op(A) op(B)  (op = N or conjugate transpose)
//   max_abs          max |x| over a (triangle of a) matrix, for the growth check
//
// No pivoting anywhere: (-i sign(Im theta)) (A + theta I) has the positive-definite
// Hermitian part |Im theta| I for Hermitian A, so unpivoted LU exists; its growth
// is monitored (max|U| / max|M|) and reported.
#pragma once
#include "arith.cuh"
#include "dense.cuh"

namespace expm {

constexpr int DN_NB = 64;  // diagonal block / panel width

template <class T> EXPM_D cx<T> cmake(T re, T im) { return {re, im}; }
template <class T> EXPM_D cx<T> cfma(cx<T> acc, cx<T> a, cx<T> b) {  // acc + a*b
    acc.re = acc.re + a.re * b.re - a.im * b.im;
    acc.im = acc.im + a.re * b.im + a.im * b.re;
    return acc;
}
template <class T> EXPM_D cx<T> cfms(cx<T> acc, cx<T> a, cx<T> b) {  // acc - a*b
    acc.re = acc.re - a.re * b.re + a.im * b.im;
    acc.im = acc.im - a.re * b.im - a.im * b.re;
    return acc;
}
template <class T> EXPM_D cx<T> cdiv(cx<T> a, cx<T> b) { return a * cinv(b); }
template <class T> EXPM_D T cabs2(cx<T> a) { return a.re * a.re + a.im * a.im; }

// ------------------------------------------------------------------ form_shifted
// Out[s] (n x n, ld n, precision T) = t A - c I + theta_s I.  A is real (a_cplx = 0)
// or complex, binary64, leading dimension lda.  amax[s] receives max |Out[s]_ij|
// (as the bit pattern of a non-negative float, atomicMax-ed).
// Batch z = instance * npairs + pair; instance i reads A + i * astride elements.
template <class T>
__global__ void form_shifted(int n, const double *__restrict__ A, int lda, int64_t astride, int a_cplx, int npairs,
                             double t, DenseSystems ps, cx<T> *__restrict__ Out, unsigned *amax) {
    const int z = blockIdx.z;
    const int s = z % npairs;
    A += (int64_t)(z / npairs) * astride * (a_cplx ? 2 : 1);
    const int64_t total = (int64_t)n * n;
    float local = 0.f;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / n), j = (int)(idx % n);
        double re, im;
        if (a_cplx) {
            re = t * A[2 * ((int64_t)i * lda + j)];
            im = t * A[2 * ((int64_t)i * lda + j) + 1];
        } else {
            re = t * A[(int64_t)i * lda + j];
            im = 0.0;
        }
        if (i == j) {
            re += ps.th_re[s] - ps.cshift;
            im += ps.th_im[s];
        }
        Out[(int64_t)z * total + idx] = {(T)re, (T)im};
        local = fmaxf(local, (float)sqrt(re * re + im * im));
    }
    for (int o = 16; o > 0; o >>= 1) local = fmaxf(local, __shfl_xor_sync(0xffffffffu, local, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax + z, __float_as_uint(local));
}

// ------------------------------------------------------------------ lu_diag
// In-place unpivoted LU of the nb x nb block at M + p*(ld+1) of every batch
// (unit lower L below the diagonal, U on and above).
// Dynamic shared memory of the block kernels: nb x (nb + 1) complex entries.
template <class T> constexpr size_t tri_smem_bytes() { return sizeof(cx<T>) * DN_NB * (DN_NB + 1); }
#define EXPM_SMEM_TRI(T, S) cx<T>(*S)[DN_NB + 1] = reinterpret_cast<cx<T>(*)[DN_NB + 1]>(dyn_smem)
extern __shared__ __align__(16) unsigned char dyn_smem[];

template <class T>
__global__ void __launch_bounds__(256) lu_diag(int nb, cx<T> *M, int ld, int64_t bstride) {
    EXPM_SMEM_TRI(T, S);
    cx<T> *blk = M + (int64_t)blockIdx.z * bstride;
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) S[idx / nb][idx % nb] = blk[(int64_t)(idx / nb) * ld + idx % nb];
    __syncthreads();
    for (int k = 0; k < nb; ++k) {
        const cx<T> inv = cinv(S[k][k]);
        for (int i = k + 1 + threadIdx.x; i < nb; i += blockDim.x) S[i][k] = S[i][k] * inv;
        __syncthreads();
        const int m = nb - k - 1;
        for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
            const int i = k + 1 + idx / m, j = k + 1 + idx % m;
            S[i][j] = cfms(S[i][j], S[i][k], S[k][j]);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) blk[(int64_t)(idx / nb) * ld + idx % nb] = S[idx / nb][idx % nb];
}

// ------------------------------------------------------------------ trsm_left
// B (nb x ncols, ld ldb) <- op(T)^{-1} B, T the nb x nb triangle at Tp (ld ldt).
// LOWER: solve with the lower triangle of op(T); UNIT: unit diagonal;
// CONJT: op(T) = T^H (so LOWER refers to the triangle of T^H).
// One thread per column; the triangle is staged in shared memory.
// Shared memory: the triangle (nb x (nb+1)) followed by the 64 columns (nb x 65).
template <class T, bool LOWER, bool UNIT, bool CONJT>
__global__ void __launch_bounds__(64) trsm_left(int nb, int ncols, const cx<T> *Tp, int ldt, int64_t tstride,
                                                cx<T> *B, int ldb, int64_t bstride) {
    EXPM_SMEM_TRI(T, S);
    cx<T>(*X)[DN_NB + 1] = S + DN_NB;
    const cx<T> *tri = Tp + (int64_t)blockIdx.z * tstride;
    cx<T> *b = B + (int64_t)blockIdx.z * bstride;
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const int i = idx / nb, j = idx % nb;
        cx<T> v = tri[(int64_t)i * ldt + j];
        if (CONJT) S[j][i] = conj(v); else S[i][j] = v;
    }
    __syncthreads();
    const int c = threadIdx.x;
    const int col = blockIdx.x * blockDim.x + c;
    if (col >= ncols) return;
    for (int i = 0; i < nb; ++i) X[i][c] = b[(int64_t)i * ldb + col];
    if (LOWER) {
        for (int i = 0; i < nb; ++i) {
            cx<T> acc = X[i][c];
            for (int l = 0; l < i; ++l) acc = cfms(acc, S[i][l], X[l][c]);
            X[i][c] = UNIT ? acc : cdiv(acc, S[i][i]);
        }
    } else {
        for (int i = nb - 1; i >= 0; --i) {
            cx<T> acc = X[i][c];
            for (int l = i + 1; l < nb; ++l) acc = cfms(acc, S[i][l], X[l][c]);
            X[i][c] = UNIT ? acc : cdiv(acc, S[i][i]);
        }
    }
    for (int i = 0; i < nb; ++i) b[(int64_t)i * ldb + col] = X[i][c];
}

// ------------------------------------------------------------------ trsm_right_upper
// B (nrows x nb, ld ldb) <- B U^{-1}, U the upper triangle (non-unit) of the nb x nb
// block at Up.  One thread per row.
// Shared memory: U (nb x (nb+1)) followed by the 64 rows (64 x (nb+1)).
template <class T>
__global__ void __launch_bounds__(64) trsm_right_upper(int nb, int nrows, const cx<T> *Up, int ldu, int64_t ustride,
                                                       cx<T> *B, int ldb, int64_t bstride) {
    EXPM_SMEM_TRI(T, S);
    cx<T>(*X)[DN_NB + 1] = S + DN_NB;
    const cx<T> *u = Up + (int64_t)blockIdx.z * ustride;
    cx<T> *b = B + (int64_t)blockIdx.z * bstride;
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) S[idx / nb][idx % nb] = u[(int64_t)(idx / nb) * ldu + idx % nb];
    __syncthreads();
    const int r = threadIdx.x;
    const int row = blockIdx.x * blockDim.x + r;
    if (row >= nrows) return;
    cx<T> *br = b + (int64_t)row * ldb;
    for (int j = 0; j < nb; ++j) {
        cx<T> acc = br[j];
        for (int l = 0; l < j; ++l) acc = cfms(acc, X[r][l], S[l][j]);
        X[r][j] = cdiv(acc, S[j][j]);
    }
    for (int j = 0; j < nb; ++j) br[j] = X[r][j];
}

// ------------------------------------------------------------------ cgemm
// C (m x n) = beta*C + alpha * op(A) op(B), op(X) = X or X^H (CONJ_A / CONJ_B).
// op(A) is m x K, op(B) is K x n.  AE is the element type of A: cx<T> or T (real A).
// 64x64 tiles, BK = 16, 256 threads, 4x4 complex outputs per thread.
template <class T> EXPM_D cx<T> as_cx(cx<T> v) { return v; }
template <class T> EXPM_D cx<T> as_cx(T v) { return {v, T(0)}; }

// Batch z uses A[z / adiv] (adiv > 1 shares one A among consecutive batches).
// Tile BM x BN, BK = 16, 256 threads, each computing TM x TN outputs.  The default
// 64 x 64 tile serves wide right-hand sides; the 128 x 8 tile serves narrow ones.
template <class T, class AE, bool CONJ_A, bool CONJ_B, int BM = 64, int BN = 64, int TM = 4, int TN = 4>
__global__ void __launch_bounds__(256) cgemm(int m, int n, int K, cx<T> alpha, T beta, const AE *__restrict__ A,
                                             int lda, int64_t sA, const cx<T> *__restrict__ B, int ldb, int64_t sB,
                                             cx<T> *__restrict__ C, int ldc, int64_t sC, int adiv) {
    constexpr int BK = 16;
    constexpr int NTX = BN / TN, NTY = BM / TM;
    static_assert(NTX * NTY == 256, "256 threads per tile");
    __shared__ cx<T> As[BK][BM + 1];
    __shared__ cx<T> Bs[BK][BN + 1];
    const AE *a = A + (int64_t)(blockIdx.z / adiv) * sA;
    const cx<T> *b = B + (int64_t)blockIdx.z * sB;
    cx<T> *c = C + (int64_t)blockIdx.z * sC;
    const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
    cx<T> acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int q = 0; q < TN; ++q) acc[r][q] = {T(0), T(0)};
    for (int l0 = 0; l0 < K; l0 += BK) {
        for (int idx = threadIdx.x; idx < BM * BK; idx += 256) {
            int ii, ll;
            if (CONJ_A) { ii = idx % BM; ll = idx / BM; } else { ii = idx / BK; ll = idx % BK; }
            const int gi = i0 + ii, gl = l0 + ll;
            cx<T> v = {T(0), T(0)};
            if (gi < m && gl < K) {
                if (CONJ_A) v = conj(as_cx<T>(a[(int64_t)gl * lda + gi]));
                else v = as_cx<T>(a[(int64_t)gi * lda + gl]);
            }
            As[ll][ii] = v;
        }
        for (int idx = threadIdx.x; idx < BK * BN; idx += 256) {
            int ll, jj;
            if (CONJ_B) { ll = idx % BK; jj = idx / BK; } else { ll = idx / BN; jj = idx % BN; }
            const int gl = l0 + ll, gj = j0 + jj;
            cx<T> v = {T(0), T(0)};
            if (gl < K && gj < n) {
                if (CONJ_B) v = conj(b[(int64_t)gj * ldb + gl]);
                else v = b[(int64_t)gl * ldb + gj];
            }
            Bs[ll][jj] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int l = 0; l < BK; ++l) {
            cx<T> av[TM], bv[TN];
#pragma unroll
            for (int r = 0; r < TM; ++r) av[r] = As[l][ty + NTY * r];
#pragma unroll
            for (int q = 0; q < TN; ++q) bv[q] = Bs[l][tx + NTX * q];
#pragma unroll
            for (int r = 0; r < TM; ++r)
#pragma unroll
                for (int q = 0; q < TN; ++q) acc[r][q] = cfma(acc[r][q], av[r], bv[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int q = 0; q < TN; ++q) {
            const int gi = i0 + ty + NTY * r, gj = j0 + tx + NTX * q;
            if (gi < m && gj < n) {
                cx<T> *cp = c + (int64_t)gi * ldc + gj;
                cx<T> out = alpha * acc[r][q];
                if (beta != T(0)) out = out + scale(beta, *cp);
                *cp = out;
            }
        }
}

// Launch helper: wide or narrow tile by the number of columns n.
template <class T, class AE, bool CONJ_A, bool CONJ_B>
inline void cgemm_launch(int m, int n, int K, cx<T> alpha, T beta, const AE *A, int lda, int64_t sA,
                         const cx<T> *B, int ldb, int64_t sB, cx<T> *C, int ldc, int64_t sC, int adiv, int batch,
                         cudaStream_t st) {
    if (n <= 8) {
        dim3 g(1, (m + 127) / 128, batch);
        cgemm<T, AE, CONJ_A, CONJ_B, 128, 8, 4, 1><<<g, 256, 0, st>>>(m, n, K, alpha, beta, A, lda, sA, B, ldb, sB,
                                                                      C, ldc, sC, adiv);
    } else {
        dim3 g((n + 63) / 64, (m + 63) / 64, batch);
        cgemm<T, AE, CONJ_A, CONJ_B><<<g, 256, 0, st>>>(m, n, K, alpha, beta, A, lda, sA, B, ldb, sB, C, ldc, sC,
                                                        adiv);
    }
}

// ------------------------------------------------------------------ resid_gemv
// R[z] -= t * A[z / adiv] * X[z] for at most 8 columns, binary64: one warp per row,
// lanes stride over K, shuffle reduction.  Narrow residuals are memory-bound, so the
// binary64 pipe suffices here.
template <class AE>
__global__ void __launch_bounds__(256) resid_gemv(int m, int n, int K, double t, const AE *__restrict__ A, int lda,
                                                  int64_t sA, const cx<double> *__restrict__ X, int ldx, int64_t sX,
                                                  cx<double> *__restrict__ Rm, int ldr, int64_t sR, int adiv) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int row = blockIdx.x * 8 + warp;
    if (row >= m) return;
    const AE *a = A + (int64_t)(blockIdx.z / adiv) * sA + (int64_t)row * lda;
    const cx<double> *x = X + (int64_t)blockIdx.z * sX;
    cx<double> acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = {0.0, 0.0};
    for (int l = lane; l < K; l += 32) {
        const cx<double> av = as_cx<double>(a[l]);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < n) acc[j] = cfma(acc[j], av, x[(int64_t)l * ldx + j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j < n) {
            double re = acc[j].re, im = acc[j].im;
            for (int o = 16; o > 0; o >>= 1) {
                re += __shfl_xor_sync(0xffffffffu, re, o);
                im += __shfl_xor_sync(0xffffffffu, im, o);
            }
            if (lane == 0) {
                cx<double> *rp = Rm + (int64_t)blockIdx.z * sR + (int64_t)row * ldr + j;
                rp->re -= t * re;
                rp->im -= t * im;
            }
        }
    }
}

// ------------------------------------------------------------------ resid_gemm_f32x2
// R[z] = R[z] - t * A[z / adiv] * X[z]  (A: m x K, X: K x n, all binary64 in memory)
// with binary64-level accuracy on the FP32 pipe.  Inside each K-block of 16 the
// products are accumulated in float-float (dd_fma); the block sums are added in
// binary64.  The rounding error of a block is ~16 * 2^-47 of its sum of |products|,
// and the blocks' errors are independent, so the total stays within a few 1e-15 of
// sum |a_il x_lj| -- far below what the refinement needs.
template <class AE> EXPM_D cx<f32x2> split_cx(AE v);
template <> EXPM_D cx<f32x2> split_cx<double>(double v) { return {split_bits(v), {0.f, 0.f}}; }
template <> EXPM_D cx<f32x2> split_cx<cx<double>>(cx<double> v) { return {split_bits(v.re), split_bits(v.im)}; }

template <class AE>
__global__ void __launch_bounds__(256) resid_gemm_f32x2(int m, int n, int K, double t, const AE *__restrict__ A,
                                                        int lda, int64_t sA, const cx<double> *__restrict__ X, int ldx,
                                                        int64_t sX, cx<double> *__restrict__ Rm, int ldr, int64_t sR,
                                                        int adiv) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ cx<f32x2> As[BK][BM + 1];
    __shared__ cx<f32x2> Bs[BK][BN + 1];
    const AE *a = A + (int64_t)(blockIdx.z / adiv) * sA;
    const cx<double> *x = X + (int64_t)blockIdx.z * sX;
    cx<double> *r = Rm + (int64_t)blockIdx.z * sR;
    const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const f32x2 z2 = {0.f, 0.f};
    cx<double> acc[4][4];
    cx<f32x2> blk[4][4];
#pragma unroll
    for (int rr = 0; rr < 4; ++rr)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[rr][q] = {0.0, 0.0};
    for (int l0 = 0; l0 < K; l0 += BK) {
        for (int idx = threadIdx.x; idx < BM * BK; idx += 256) {
            const int ii = idx / BK, ll = idx % BK;
            const int gi = i0 + ii, gl = l0 + ll;
            As[ll][ii] = (gi < m && gl < K) ? split_cx<AE>(a[(int64_t)gi * lda + gl]) : cx<f32x2>{z2, z2};
        }
        for (int idx = threadIdx.x; idx < BK * BN; idx += 256) {
            const int ll = idx / BN, jj = idx % BN;
            const int gl = l0 + ll, gj = j0 + jj;
            Bs[ll][jj] = (gl < K && gj < n) ? split_cx<cx<double>>(x[(int64_t)gl * ldx + gj]) : cx<f32x2>{z2, z2};
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int q = 0; q < 4; ++q) blk[rr][q] = {z2, z2};
#pragma unroll 2
        for (int l = 0; l < BK; ++l) {
            cx<f32x2> av[4], bv[4];
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) av[rr] = As[l][ty + 16 * rr];
#pragma unroll
            for (int q = 0; q < 4; ++q) bv[q] = Bs[l][tx + 16 * q];
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    cx<f32x2> &c = blk[rr][q];
                    c.re = dd_fma(av[rr].re, bv[q].re, c.re);
                    c.re = dd_fma(-av[rr].im, bv[q].im, c.re);
                    c.im = dd_fma(av[rr].re, bv[q].im, c.im);
                    c.im = dd_fma(av[rr].im, bv[q].re, c.im);
                }
        }
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                acc[rr][q].re += widen_bits(blk[rr][q].re.hi) + widen_bits(blk[rr][q].re.lo);
                acc[rr][q].im += widen_bits(blk[rr][q].im.hi) + widen_bits(blk[rr][q].im.lo);
            }
        __syncthreads();
    }
#pragma unroll
    for (int rr = 0; rr < 4; ++rr)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gi = i0 + ty + 16 * rr, gj = j0 + tx + 16 * q;
            if (gi < m && gj < n) {
                cx<double> *rp = r + (int64_t)gi * ldr + gj;
                rp->re -= t * acc[rr][q].re;
                rp->im -= t * acc[rr][q].im;
            }
        }
}

// ------------------------------------------------------------------ max_abs
// out[batch] = max |M_ij| over the upper triangle (j >= i) of an n x n matrix
// (as float bits, atomicMax) -- max |U| of an LU stored in place.
template <class T>
__global__ void max_abs_upper(int n, const cx<T> *M, int ld, int64_t bstride, unsigned *out) {
    const cx<T> *m = M + (int64_t)blockIdx.z * bstride;
    float local = 0.f;
    const int64_t total = (int64_t)n * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / n), j = (int)(idx % n);
        if (j >= i) {
            const cx<T> v = m[(int64_t)i * ld + j];
            local = fmaxf(local, (float)sqrt((double)(v.re * v.re + v.im * v.im)));
        }
    }
    for (int o = 16; o > 0; o >>= 1) local = fmaxf(local, __shfl_xor_sync(0xffffffffu, local, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + blockIdx.z, __float_as_uint(local));
}

}  // namespace expm
