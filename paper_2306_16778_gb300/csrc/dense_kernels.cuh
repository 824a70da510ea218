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
//   cgemm_f32w       the same for wide binary32 operands (double-buffered 128 x 64 tile)
//   resid_gemv_f32x2 / resid_gemm_f32x2  binary64-accurate refinement residuals on the
//                    FP32 pipe (float pairs), at most 8 / more right-hand-side columns
//   max_abs          max |x| over a (triangle of a) matrix, for the growth check
//
// No pivoting anywhere: (-i sign(Im theta)) (A + theta I) has the positive-definite
// Hermitian part |Im theta| I for Hermitian A, so unpivoted LU exists; its growth
// is monitored (max|U| / max|M|) and reported.
#pragma once
#include <type_traits>
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
// Out[z] (n x n, ld n, precision T) = t A - c I + theta_s I for every pair s of every
// instance, z = instance * npairs + s.  A is real (a_cplx = 0) or complex, binary64,
// leading dimension lda; instance i reads A + i * astride elements.  One warp per row
// (grid.x = ceil(n / 8) blocks of 8 warps, grid.z = instances): A is read once and
// every pair's row written from it.  amax[z] receives max |Out[z]_ij| (as the bit
// pattern of a non-negative float, atomicMax-ed): the off-diagonal part is common to
// all pairs, only the diagonal entry differs.
template <class T>
__global__ void __launch_bounds__(256) form_shifted(int n, const double *__restrict__ A, int lda, int64_t astride,
                                                    int a_cplx, int npairs, double t, DenseSystems ps,
                                                    cx<T> *__restrict__ Out, unsigned *amax) {
    const int inst = blockIdx.z;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    const int64_t esz = a_cplx ? 2 : 1;
    const double *arow = A + (int64_t)inst * astride * esz + (int64_t)i * lda * esz;
    const int64_t nn = (int64_t)n * n;
    cx<T> *out0 = Out + (int64_t)inst * npairs * nn + (int64_t)i * n;
    float offmax = 0.f;
    for (int j = lane; j < n; j += 32) {
        const double re = t * arow[esz * j], im = a_cplx ? t * arow[2 * j + 1] : 0.0;
        if (j != i) {
            const cx<T> v = {(T)re, (T)im};
            for (int s = 0; s < npairs; ++s) out0[s * nn + j] = v;
            offmax = fmaxf(offmax, sqrtf((float)(re * re + im * im)));
        } else {
            for (int s = 0; s < npairs; ++s)
                out0[s * nn + j] = {(T)(re + ps.th_re[s] - ps.cshift), (T)(im + ps.th_im[s])};
        }
    }
    for (int o = 16; o > 0; o >>= 1) offmax = fmaxf(offmax, __shfl_xor_sync(0xffffffffu, offmax, o));
    if (lane == 0) {
        const double re = t * arow[esz * i], im = a_cplx ? t * arow[2 * i + 1] : 0.0;
        for (int s = 0; s < npairs; ++s) {
            const double dr = re + ps.th_re[s] - ps.cshift, di = im + ps.th_im[s];
            const float m = fmaxf(offmax, sqrtf((float)(dr * dr + di * di)));
            atomicMax(amax + (int64_t)inst * npairs + s, __float_as_uint(m));
        }
    }
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

// Binary32 complex GEMM for wide operands: C = beta C + alpha op(A) B, op(A) = A or A^H.
// 128 x 64 complex tile, BK = 8, 256 threads with 8 x 4 complex outputs each (rows
// ty + 16 r, columns tx + 16 q), two shared-memory stages: the next K tile is fetched
// into registers while the current one is consumed, then stored into the other stage,
// one barrier per K tile.  Two CTAs per SM.
template <bool CONJ_A>
__global__ void __launch_bounds__(256, 2) cgemm_f32w(int m, int n, int K, cx<float> alpha, float beta,
                                                     const cx<float> *__restrict__ A, int lda, int64_t sA,
                                                     const cx<float> *__restrict__ B, int ldb, int64_t sB,
                                                     cx<float> *__restrict__ C, int ldc, int64_t sC, int adiv) {
    constexpr int BM = 128, BN = 64, BK = 8;
    __shared__ cx<float> As[2][BK][BM + 4];
    __shared__ cx<float> Bs[2][BK][BN + 4];
    const cx<float> *a = A + (int64_t)(blockIdx.z / adiv) * sA;
    const cx<float> *b = B + (int64_t)blockIdx.z * sB;
    cx<float> *c = C + (int64_t)blockIdx.z * sC;
    const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    // this thread's share of a K tile: 4 elements of A, 2 of B
    cx<float> pa[4], pb[2];
    auto fetch = [&](int l0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = t + 256 * e;
            int ii, ll;
            if (CONJ_A) { ii = idx % BM; ll = idx / BM; } else { ii = idx / BK; ll = idx % BK; }
            const int gi = i0 + ii, gl = l0 + ll;
            cx<float> v = {0.f, 0.f};
            if (gi < m && gl < K) v = CONJ_A ? conj(a[(int64_t)gl * lda + gi]) : a[(int64_t)gi * lda + gl];
            pa[e] = v;
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int idx = t + 256 * e;
            const int ll = idx / BN, jj = idx % BN;
            const int gl = l0 + ll, gj = j0 + jj;
            pb[e] = (gl < K && gj < n) ? b[(int64_t)gl * ldb + gj] : cx<float>{0.f, 0.f};
        }
    };
    auto stash = [&](int st) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = t + 256 * e;
            int ii, ll;
            if (CONJ_A) { ii = idx % BM; ll = idx / BM; } else { ii = idx / BK; ll = idx % BK; }
            As[st][ll][ii] = pa[e];
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int idx = t + 256 * e;
            Bs[st][idx / BN][idx % BN] = pb[e];
        }
    };
    cx<float> acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = {0.f, 0.f};
    const int nt = (K + BK - 1) / BK;
    fetch(0);
    stash(0);
    __syncthreads();
    for (int kt = 0; kt < nt; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nt) fetch((kt + 1) * BK);
#pragma unroll
        for (int l = 0; l < BK; ++l) {
            cx<float> av[8], bv[4];
#pragma unroll
            for (int r = 0; r < 8; ++r) av[r] = As[cur][l][ty + 16 * r];
#pragma unroll
            for (int q = 0; q < 4; ++q) bv[q] = Bs[cur][l][tx + 16 * q];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = cfma(acc[r][q], av[r], bv[q]);
        }
        if (kt + 1 < nt) stash(cur ^ 1);  // the other stage was last read before the previous barrier
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gi = i0 + ty + 16 * r, gj = j0 + tx + 16 * q;
            if (gi < m && gj < n) {
                cx<float> *cp = c + (int64_t)gi * ldc + gj;
                cx<float> out = alpha * acc[r][q];
                if (beta != 0.f) out = out + scale(beta, *cp);
                *cp = out;
            }
        }
}

// Launch helper: wide or narrow tile by the number of columns n.
template <class T, class AE, bool CONJ_A, bool CONJ_B>
inline void cgemm_launch(int m, int n, int K, cx<T> alpha, T beta, const AE *A, int lda, int64_t sA,
                         const cx<T> *B, int ldb, int64_t sB, cx<T> *C, int ldc, int64_t sC, int adiv, int batch,
                         cudaStream_t st, int tile = 0) {
    // tile 0: 128 x 64 output tiles for binary32 (wider than 32 columns), tile 1: 64 x 64
    if constexpr (std::is_same<T, float>::value && std::is_same<AE, cx<float>>::value && !CONJ_B) {
        if (n > 32 && tile == 0) {
            dim3 g((n + 63) / 64, (m + 127) / 128, batch);
            cgemm_f32w<CONJ_A><<<g, 256, 0, st>>>(m, n, K, alpha, beta, A, lda, sA, B, ldb, sB, C, ldc, sC, adiv);
            return;
        }
    }
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

// ------------------------------------------------------------------ diagonal-panel inverses
// The wide triangular solves multiply by explicit inverses of the LU's diagonal panels
// (block triangular substitution with inverted diagonal blocks).  Panel q of batch entry z
// covers rows and columns q B .. q B + nb - 1, nb = min(B, n - q B).  This kernel copies
// it into the B x B block P[z][q] (packed unit-lower L and upper U, as in F), padded with
// the identity past nb so that every block is a full B x B LU, and sets both inverse slots
// Inv[z][q][0] (for L) and Inv[z][q][1] (for U) to the identity; the blocked solves on
// those identities then leave L_q^{-1} and U_q^{-1} there.
template <class T>
__global__ void __launch_bounds__(256) gather_diag_panels(int n, int B, int npan, const cx<T> *__restrict__ F,
                                                          int64_t fstride, cx<T> *__restrict__ P,
                                                          cx<T> *__restrict__ Inv) {
    const int q = blockIdx.y;
    const int64_t z = blockIdx.z;
    const int p0 = q * B, nb = min(B, n - p0);
    const int64_t zq = z * npan + q, bb = (int64_t)B * B;
    cx<T> *Pq = P + zq * bb;
    cx<T> *Iq = Inv + zq * 2 * bb;
    const cx<T> *Fq = F + z * fstride + (int64_t)p0 * n + p0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < bb; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / B), j = (int)(e % B);
        const cx<T> id = {i == j ? T(1) : T(0), T(0)};
        Pq[e] = (i < nb && j < nb) ? Fq[(int64_t)i * n + j] : id;
        Iq[e] = id;
        Iq[bb + e] = id;
    }
}

// ------------------------------------------------------------------ lu_solve_narrow
// X <- (L U)^{-1} X (CONJ = false) or (L U)^{-H} X = U^{-H} L^{-H} X (CONJ = true) for an
// LU stored in place (unit L below the diagonal, U on and above), at most 8 columns.
// One CTA per batch entry b: X_b (n x kc, row-major) lives in shared memory for the
// whole solve.  Per 64-row block: the update from the rows already solved (a GEMV on
// the factor, read once; row-wise when the needed triangle is stored by rows, column-
// wise -- lanes over the block's rows -- when it is the conjugate transpose), then the
// 64 x 64 diagonal block staged in shared memory and solved right-looking by one warp.
// Dynamic shared memory: n * kc complex entries, then DN_NB x (DN_NB + 1), then the
// cross-group partial sums 4 x DN_NB x 8.
template <class T, bool CONJ>
__global__ void __launch_bounds__(256) lu_solve_narrow(int n, int kc, const cx<T> *__restrict__ F, int64_t fstride,
                                                       cx<T> *X, int64_t xstride, const int *skip) {
    if (skip != nullptr && *skip) return;  // device-side refinement already converged
    constexpr int NB = DN_NB;
    cx<T> *xs = reinterpret_cast<cx<T> *>(dyn_smem);                       // [n][kc]
    cx<T>(*D)[NB + 1] = reinterpret_cast<cx<T>(*)[NB + 1]>(xs + (size_t)n * kc);  // diagonal block
    cx<T> *red = reinterpret_cast<cx<T> *>(D + NB);                        // [4][NB][8]
    const int64_t b = blockIdx.x;
    const cx<T> *Fb = F + b * fstride;
    cx<T> *Xb = X + b * xstride;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < n * kc; e += blockDim.x) xs[e] = Xb[e];
    __syncthreads();
    // element (i, j) of the triangle used: row-stored for !CONJ, conjugate of (j, i) for CONJ
    auto elem = [&](int i, int j) -> cx<T> { return CONJ ? conj(Fb[(int64_t)j * n + i]) : Fb[(int64_t)i * n + j]; };
    // xs[p + r] -= sum_{j in [j0, j1)} M(p + r, j) xs[j]  for r < nb
    auto offdiag = [&](int p, int nb, int j0, int j1) {
        if (j1 <= j0) return;
        if (!CONJ) {  // rows of F: one warp per row, lanes over j
            for (int r = warp; r < nb; r += 8) {
                cx<T> acc[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[c] = {T(0), T(0)};
                const cx<T> *frow = Fb + (int64_t)(p + r) * n;
                for (int j = j0 + lane; j < j1; j += 32) {
                    const cx<T> f = frow[j];
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (c < kc) acc[c] = cfma(acc[c], f, xs[(int64_t)j * kc + c]);
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    if (c < kc) {
                        T re = acc[c].re, im = acc[c].im;
                        for (int o = 16; o > 0; o >>= 1) {
                            re += __shfl_xor_sync(0xffffffffu, re, o);
                            im += __shfl_xor_sync(0xffffffffu, im, o);
                        }
                        if (lane == 0) {
                            xs[(int64_t)(p + r) * kc + c].re -= re;
                            xs[(int64_t)(p + r) * kc + c].im -= im;
                        }
                    }
                }
            }
        } else {  // columns of F: 64 lanes over the block's rows, 4 groups over j
            const int r = tid & (NB - 1), grp = tid / NB;
            cx<T> acc[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = {T(0), T(0)};
            if (r < nb) {
                for (int j = j0 + grp; j < j1; j += 4) {
                    const cx<T> f = conj(Fb[(int64_t)j * n + p + r]);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (c < kc) acc[c] = cfma(acc[c], f, xs[(int64_t)j * kc + c]);
                }
            }
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c < kc) red[(grp * NB + r) * 8 + c] = acc[c];
            __syncthreads();
            if (grp == 0 && r < nb) {
                for (int c = 0; c < kc; ++c) {
                    cx<T> sum = red[r * 8 + c];
                    for (int q = 1; q < 4; ++q) sum = sum + red[(q * NB + r) * 8 + c];
                    xs[(int64_t)(p + r) * kc + c] = xs[(int64_t)(p + r) * kc + c] - sum;
                }
            }
        }
    };
    // stage the diagonal block M(p .. p+nb, p .. p+nb) into D
    auto stage = [&](int p, int nb) {
        for (int e = tid; e < nb * nb; e += blockDim.x) {
            const int a = e / nb, c = e % nb;  // reads run along rows of F
            if (CONJ) D[c][a] = conj(Fb[(int64_t)(p + a) * n + p + c]);
            else D[a][c] = Fb[(int64_t)(p + a) * n + p + c];
        }
    };
    // right-looking solve of the staged block by warp 0: lower (forward) or upper (backward)
    auto diag_solve = [&](int p, int nb, bool lower, bool unit) {
        if (warp != 0) return;
        for (int step = 0; step < nb; ++step) {
            const int i = lower ? step : nb - 1 - step;
            if (!unit) {
                if (lane < kc) xs[(int64_t)(p + i) * kc + lane] = cdiv(xs[(int64_t)(p + i) * kc + lane], D[i][i]);
                __syncwarp();
            }
            const int cnt = lower ? nb - 1 - i : i;  // rows still to update
            for (int e = lane; e < cnt * kc; e += 32) {
                const int jj = e / kc, c = e % kc;
                const int j = lower ? i + 1 + jj : jj;
                xs[(int64_t)(p + j) * kc + c] = cfms(xs[(int64_t)(p + j) * kc + c], D[j][i], xs[(int64_t)(p + i) * kc + c]);
            }
            __syncwarp();
        }
    };
    // forward: lower triangle (L unit, or U^H with diagonal conj(U_ii))
    for (int p = 0; p < n; p += NB) {
        const int nb = min(NB, n - p);
        offdiag(p, nb, 0, p);
        stage(p, nb);
        __syncthreads();
        diag_solve(p, nb, true, !CONJ);
        __syncthreads();
    }
    // backward: upper triangle (U, or L^H with unit diagonal)
    for (int p = ((n - 1) / NB) * NB; p >= 0; p -= NB) {
        const int nb = min(NB, n - p);
        offdiag(p, nb, p + nb, n);
        stage(p, nb);
        __syncthreads();
        diag_solve(p, nb, false, CONJ);
        __syncthreads();
    }
    for (int e = tid; e < n * kc; e += blockDim.x) Xb[e] = xs[e];
}

template <class T> constexpr size_t narrow_smem_bytes(int n, int kc) {
    return sizeof(cx<T>) * ((size_t)n * kc + (size_t)DN_NB * (DN_NB + 1) + 4 * (size_t)DN_NB * 8);
}

// ------------------------------------------------------------------ resid_gemm_f32x2
// R[z] = R[z] - t * A[z / adiv] * X[z]  (A: m x K, X: K x n, all binary64 in memory)
// with binary64-level accuracy on the FP32 pipe.  Inside each K-block of 16 the
// products are accumulated as float pairs (pair_mac); the block sums are added in
// binary64.  The rounding error of a block is ~16 * 2^-47 of its sum of |products|,
// and the blocks' errors are independent, so the total stays within a few 1e-15 of
// sum |a_il x_lj| -- far below what the refinement needs.
template <class AE> EXPM_D cx<f32x2> split_cx(AE v);
template <> EXPM_D cx<f32x2> split_cx<double>(double v) { return {split_bits(v), {0.f, 0.f}}; }
template <> EXPM_D cx<f32x2> split_cx<cx<double>>(cx<double> v) { return {split_bits(v.re), split_bits(v.im)}; }

// a * b accumulated into the unnormalised pair (hi, lo): the product of the high parts
// split exactly by an FMA, the cross terms added to its error, the sum's rounding error
// from one TwoSum; lo collects all errors and is folded in once per K-block.
EXPM_D void pair_mac(float &hi, float &lo, f32x2 a, f32x2 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const f32x2 s = two_sum(hi, p);
    hi = s.hi;
    lo = __fadd_rn(lo, __fadd_rn(s.lo, e));
}

constexpr size_t RESID_GEMM_SMEM = 16 * 256 * sizeof(cx<double>);  // dynamic: the binary64 block sums

// ------------------------------------------------------------------ resid_gemv_f32x2
// R[inst, sys] -= t * A[inst] * X[inst, sys] for every system of an instance and at most
// 8 columns ((system, column) pairs taken CB at a time, so A is read once per CB pairs;
// a block holds 8 rows of A, one warp per row, lanes over K; X and R of (inst, sys)
// start at (inst * nsys + sys) * sX, row-major n x kc), with binary64-level accuracy on
// the FP32 pipe: A and X are split into float pairs (X once, when staged in
// shared memory), each product is error-free up to the dropped lo*lo term (pair_mac),
// a lane accumulates its terms of a 256-wide K chunk as an unnormalised pair and folds
// it into a normalised double-word sum once per chunk, and the warp's lanes are
// combined by double-word additions.  Relative error a few 2^-48 of sum |a_il x_l|.
template <class AE, int CB, int LPR>
__global__ void __launch_bounds__(256) resid_gemv_f32x2(int n, int kc, int nsys, double t, const AE *__restrict__ A,
                                                        int lda, int64_t sA, const cx<double> *__restrict__ X,
                                                        int64_t sX, cx<double> *__restrict__ Rm, const int *skip) {
    if (skip != nullptr && *skip) return;
    constexpr int KCH = 256;
    __shared__ cx<f32x2> xs[CB][KCH];
    const int inst = blockIdx.z;
    const int cb0 = blockIdx.y * CB, ncomb = nsys * kc;
    // LPR lanes per row (32, or 8 for short rows: fewer butterfly levels), 256 / LPR rows
    // per block
    const int lane = threadIdx.x % LPR;
    const int row = blockIdx.x * (256 / LPR) + threadIdx.x / LPR;
    const AE *arow = A + (int64_t)inst * sA + (int64_t)row * lda;
    const cx<double> *Xi = X + (int64_t)inst * nsys * sX;
    const f32x2 z2 = {0.f, 0.f};
    cx<f32x2> acc[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) acc[c] = {z2, z2};
    for (int k0 = 0; k0 < n; k0 += KCH) {
        const int lim = min(KCH, n - k0);
        __syncthreads();
        for (int e = threadIdx.x; e < CB * lim; e += blockDim.x) {  // only the live columns
            const int c = e / lim, l = e % lim, comb = cb0 + c;
            cx<f32x2> v = {z2, z2};
            if (comb < ncomb) v = split_cx<cx<double>>(Xi[(int64_t)(comb / kc) * sX + (int64_t)(k0 + l) * kc + comb % kc]);
            xs[c][l] = v;
        }
        __syncthreads();
        if (row < n) {
            float hr[CB], lr[CB], hi[CB], li[CB];
#pragma unroll
            for (int c = 0; c < CB; ++c) hr[c] = lr[c] = hi[c] = li[c] = 0.f;
            for (int l = lane; l < lim; l += LPR) {
                const cx<f32x2> av = split_cx<AE>(arow[k0 + l]);
                const f32x2 nai = {-av.im.hi, -av.im.lo};
#pragma unroll
                for (int c = 0; c < CB; ++c) {
                    const cx<f32x2> xv = xs[c][l];
                    pair_mac(hr[c], lr[c], av.re, xv.re);
                    pair_mac(hr[c], lr[c], nai, xv.im);
                    pair_mac(hi[c], li[c], av.re, xv.im);
                    pair_mac(hi[c], li[c], av.im, xv.re);
                }
            }
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                acc[c].re = acc[c].re + two_sum(hr[c], lr[c]);
                acc[c].im = acc[c].im + two_sum(hi[c], li[c]);
            }
        }
    }
    // the lanes' double-word sums combined by a butterfly of double-word additions (the
    // FP32 pipe; all lanes take part, rows past n with zero sums); binary64 only for the
    // final value
#pragma unroll
    for (int c = 0; c < CB; ++c) {
        f32x2 re = acc[c].re, im = acc[c].im;
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) {
            const f32x2 ro = {__shfl_xor_sync(0xffffffffu, re.hi, o), __shfl_xor_sync(0xffffffffu, re.lo, o)};
            const f32x2 io = {__shfl_xor_sync(0xffffffffu, im.hi, o), __shfl_xor_sync(0xffffffffu, im.lo, o)};
            re = re + ro;
            im = im + io;
        }
        const int comb = cb0 + c;
        if (lane == 0 && comb < ncomb && row < n) {
            cx<double> *rp = Rm + (int64_t)(inst * nsys + comb / kc) * sX + (int64_t)row * kc + comb % kc;
            rp->re -= t * (widen_bits(re.hi) + widen_bits(re.lo));
            rp->im -= t * (widen_bits(im.hi) + widen_bits(im.lo));
        }
    }
}

// pairs per block of resid_gemv_f32x2: 6 when that divides the pair count and 8 does not
inline int gemv_f32x2_cb(int ncomb) { return (ncomb % 8 != 0 && ncomb % 6 == 0) ? 6 : 8; }

template <class AE>
inline void resid_gemv_f32x2_launch(int n, int kc, int nsys, int ninst, double t, const AE *A, int lda, int64_t sA,
                                    const cx<double> *X, int64_t sX, cx<double> *R, const int *skip,
                                    cudaStream_t st) {
    const int ncomb = nsys * kc, cbw = gemv_f32x2_cb(ncomb);
    const bool shortrow = n <= 256;
    const int rpb = shortrow ? 32 : 8;  // rows per block
    const dim3 gg((n + rpb - 1) / rpb, (ncomb + cbw - 1) / cbw, ninst);
    if (shortrow) {
        if (cbw == 6) resid_gemv_f32x2<AE, 6, 8><<<gg, 256, 0, st>>>(n, kc, nsys, t, A, lda, sA, X, sX, R, skip);
        else resid_gemv_f32x2<AE, 8, 8><<<gg, 256, 0, st>>>(n, kc, nsys, t, A, lda, sA, X, sX, R, skip);
    } else {
        if (cbw == 6) resid_gemv_f32x2<AE, 6, 32><<<gg, 256, 0, st>>>(n, kc, nsys, t, A, lda, sA, X, sX, R, skip);
        else resid_gemv_f32x2<AE, 8, 32><<<gg, 256, 0, st>>>(n, kc, nsys, t, A, lda, sA, X, sX, R, skip);
    }
}

template <class AE>
__global__ void __launch_bounds__(256, 2) resid_gemm_f32x2(int m, int n, int K, double t, const AE *__restrict__ A,
                                                           int lda, int64_t sA, const cx<double> *__restrict__ X,
                                                           int ldx, int64_t sX, cx<double> *__restrict__ Rm, int ldr,
                                                           int64_t sR, int adiv) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ cx<f32x2> As[BK][BM + 1];
    __shared__ cx<f32x2> Bs[BK][BN + 1];
    // the binary64 block sums live in shared memory ([output][thread]: conflict-free), so
    // the registers hold only the float-pair accumulators of the current K-block
    extern __shared__ cx<double> accS[];  // 16 x 256
    const AE *a = A + (int64_t)(blockIdx.z / adiv) * sA;
    const cx<double> *x = X + (int64_t)blockIdx.z * sX;
    cx<double> *r = Rm + (int64_t)blockIdx.z * sR;
    const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const f32x2 z2 = {0.f, 0.f};
#pragma unroll
    for (int o = 0; o < 16; ++o) accS[o * 256 + threadIdx.x] = {0.0, 0.0};
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
        float hr[4][4], lr[4][4], hi_[4][4], li[4][4];  // (hi, lo) of the real and imaginary parts
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int q = 0; q < 4; ++q) hr[rr][q] = lr[rr][q] = hi_[rr][q] = li[rr][q] = 0.f;
#pragma unroll 1
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
                    pair_mac(hr[rr][q], lr[rr][q], av[rr].re, bv[q].re);
                    pair_mac(hr[rr][q], lr[rr][q], -av[rr].im, bv[q].im);
                    pair_mac(hi_[rr][q], li[rr][q], av[rr].re, bv[q].im);
                    pair_mac(hi_[rr][q], li[rr][q], av[rr].im, bv[q].re);
                }
        }
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                cx<double> &acc = accS[(rr * 4 + q) * 256 + threadIdx.x];
                acc.re += widen_bits(hr[rr][q]) + widen_bits(lr[rr][q]);
                acc.im += widen_bits(hi_[rr][q]) + widen_bits(li[rr][q]);
            }
        __syncthreads();
    }
#pragma unroll
    for (int rr = 0; rr < 4; ++rr)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gi = i0 + ty + 16 * rr, gj = j0 + tx + 16 * q;
            if (gi < m && gj < n) {
                const cx<double> acc = accS[(rr * 4 + q) * 256 + threadIdx.x];
                cx<double> *rp = r + (int64_t)gi * ldr + gj;
                rp->re -= t * acc.re;
                rp->im -= t * acc.im;
            }
        }
}

// ------------------------------------------------------------------ max_abs
// out[batch] = max |M_ij| over the upper triangle (j >= i) of an n x n matrix
// (as float bits, atomicMax) -- max |U| of an LU stored in place.  One warp per row.
template <class T>
__global__ void __launch_bounds__(256) max_abs_upper(int n, const cx<T> *M, int ld, int64_t bstride, unsigned *out) {
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    const cx<T> *m = M + (int64_t)blockIdx.z * bstride + (int64_t)i * ld;
    float local = 0.f;
    for (int j = i + lane; j < n; j += 32) {
        const cx<T> v = m[j];
        local = fmaxf(local, sqrtf((float)(v.re * v.re + v.im * v.im)));
    }
    for (int o = 16; o > 0; o >>= 1) local = fmaxf(local, __shfl_xor_sync(0xffffffffu, local, o));
    if (lane == 0) atomicMax(out + blockIdx.z, __float_as_uint(local));
}

}  // namespace expm
