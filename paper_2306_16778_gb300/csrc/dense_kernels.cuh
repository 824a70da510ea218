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
template <class T, class AE, bool CONJ_A, bool CONJ_B>
__global__ void __launch_bounds__(256) cgemm(int m, int n, int K, cx<T> alpha, T beta, const AE *__restrict__ A,
                                             int lda, int64_t sA, const cx<T> *__restrict__ B, int ldb, int64_t sB,
                                             cx<T> *__restrict__ C, int ldc, int64_t sC, int adiv) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ cx<T> As[BK][BM + 1];
    __shared__ cx<T> Bs[BK][BN + 1];
    const AE *a = A + (int64_t)(blockIdx.z / adiv) * sA;
    const cx<T> *b = B + (int64_t)blockIdx.z * sB;
    cx<T> *c = C + (int64_t)blockIdx.z * sC;
    const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    cx<T> acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = {T(0), T(0)};
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
            cx<T> av[4], bv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) av[r] = As[l][ty + 16 * r];
#pragma unroll
            for (int q = 0; q < 4; ++q) bv[q] = Bs[l][tx + 16 * q];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = cfma(acc[r][q], av[r], bv[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gi = i0 + ty + 16 * r, gj = j0 + tx + 16 * q;
            if (gi < m && gj < n) {
                cx<T> *cp = c + (int64_t)gi * ldc + gj;
                cx<T> out = alpha * acc[r][q];
                if (beta != T(0)) out = out + scale(beta, *cp);
                *cp = out;
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
