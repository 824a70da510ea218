// dense_reduce.cu -- expm_apply_dense_reduced: Y = e^c R_n(tA - cI) V for a dense Hermitian
// A through a unitary reduction to real symmetric tridiagonal form.
//
// A = Q T Q^H with T real symmetric tridiagonal (Householder reflectors H_i = I - tau_i v_i
// v_i^H acting on rows i+1 .. n-1, each chosen so that it maps the column below the
// diagonal to a real multiple of the first unit vector), and R_n(tA - cI) = Q R_n(tT - cI)
// Q^H (Remark 3.1: R_n(P A P^{-1}) = P R_n(A) P^{-1}).  So
//     W = Q^H V,   Z = e^c R_n(tT - cI) W  (the pole-batched tridiagonal path),   Y = Q Z.
// The reduction costs about (8/3) n^3 complex multiply-adds once, independently of the
// number of poles, where the per-pole LU path needs (n/2) LUs of (1/3) n^3 each; the
// tridiagonal solves for all poles are then a small fraction of the time.
//
// The reduction is the classical unblocked one (Householder 1958; Golub and Van Loan,
// "Matrix Computations", Sec. 8.3.1): for each column i, the reflector from the column
// below the diagonal, p = tau A22 v, w = p - (tau/2)(p^H v) v, A22 <- A22 - v w^H - w v^H.
// All in binary64 on the working copy of A (the full Hermitian matrix is kept, so every
// kernel reads rows contiguously).  On GB300 every step is bound by the FP64 pipe or by
// HBM, not by the block structure, so the unblocked form is used as is.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/expm.h"
#include "arith.cuh"
#include "plan.cuh"

namespace expm {
namespace {

using cxd = cx<double>;

EXPM_D cxd cconj(cxd a) { return {a.re, -a.im}; }

// Ac (n x n complex, ld n) = A (real or complex, ld lda)
__global__ void to_complex(int n, const double *__restrict__ A, int64_t lda, int a_cplx, cxd *__restrict__ Ac) {
    const int i = blockIdx.x;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        cxd v;
        if (a_cplx) v = {A[2 * ((int64_t)i * lda + j)], A[2 * ((int64_t)i * lda + j) + 1]};
        else v = {A[(int64_t)i * lda + j], 0.0};
        Ac[(int64_t)i * n + j] = v;
    }
}

// Block-wide sum of a double (blockDim.x = 1024)
__device__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    if (threadIdx.x < 32)
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sh[32] = t;
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

constexpr int U_COLS = 256, U_ROWS = 16;  // her2 tile: columns per block, rows per block

// ---- fused step kernels: two launches per column instead of four
// Step i, kernel 1: every block forms the reflector of the column x = Ac[i+1.., i] itself
// (a block reduction for ||x_tail||; the column is only read in this step), keeps v in
// shared memory, and computes p_r = tau (A22 v)_r for its H_ROWS rows (one warp per row)
// with the partial sum of conj(p_r) v_r over them.  Block 0 also stores v (packed, Vp
// row i), tau_i, d_i and e_i = beta.
constexpr int H_ROWS = 16;
__global__ void __launch_bounds__(256) step_hemv(int n, int i, const cxd *__restrict__ Ac, cxd *__restrict__ Vp,
                                                 cxd *__restrict__ tau, double *__restrict__ d, double *__restrict__ e,
                                                 cxd *__restrict__ p, cxd *__restrict__ part) {
    extern __shared__ cxd vs[];  // m entries
    __shared__ double sh[33];
    __shared__ double pr[8][2];
    const int m = n - 1 - i;
    const cxd *col = Ac + (int64_t)(i + 1) * n + i;  // x_r at col[r * n]
    double s2 = 0.0;
    for (int r = 1 + threadIdx.x; r < m; r += blockDim.x) {
        const cxd x = col[(int64_t)r * n];
        s2 += x.re * x.re + x.im * x.im;
    }
    s2 = block_sum(s2, sh);
    const cxd alpha = col[0];
    const bool reflect = s2 > 0.0 || alpha.im != 0.0;
    cxd t = {0.0, 0.0}, scale = {0.0, 0.0};
    double beta = alpha.re;
    if (reflect) {
        const double nrm = sqrt(alpha.re * alpha.re + alpha.im * alpha.im + s2);
        beta = alpha.re >= 0.0 ? -nrm : nrm;
        t = {(beta - alpha.re) / beta, -alpha.im / beta};
        scale = cinv(cxd{alpha.re - beta, alpha.im});
    }
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        const cxd v = r == 0 ? cxd{1.0, 0.0} : (reflect ? col[(int64_t)r * n] * scale : cxd{0.0, 0.0});
        vs[r] = v;
        if (blockIdx.x == 0) Vp[(int64_t)i * n + r] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        tau[i] = t;
        d[i] = Ac[(int64_t)i * n + i].re;
        e[i] = beta;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double dre = 0.0, dim = 0.0;  // sum over this warp's rows of conj(p_r) v_r
    for (int rr = warp; rr < H_ROWS; rr += 8) {
        const int r = blockIdx.x * H_ROWS + rr;
        if (r >= m) break;
        const cxd *row = Ac + (int64_t)(i + 1 + r) * n + (i + 1);
        double re = 0.0, im = 0.0;
        for (int c = lane; c < m; c += 32) {
            const cxd a = row[c], x = vs[c];
            re = fma(a.re, x.re, fma(-a.im, x.im, re));
            im = fma(a.re, x.im, fma(a.im, x.re, im));
        }
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        const cxd pv = t * cxd{re, im};
        if (lane == 0) p[r] = pv;
        const cxd vr = vs[r];
        dre += pv.re * vr.re + pv.im * vr.im;
        dim += pv.re * vr.im - pv.im * vr.re;
    }
    if (lane == 0) {
        pr[warp][0] = dre;
        pr[warp][1] = dim;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cxd acc = {0.0, 0.0};
        for (int w = 0; w < 8; ++w) acc = acc + cxd{pr[w][0], pr[w][1]};
        part[blockIdx.x] = acc;
    }
}

// Step i, kernel 2: A22 -= v w^H + w v^H with w = p - (tau/2)(p^H v) v, the dot summed by
// every block from the per-block partials in a fixed order.  A block owns 256 columns x 16
// rows: each thread keeps its column's v_c, w_c in registers and walks the rows (row values
// from shared memory), so every entry costs one load, one store and eight FP64 operations.
__global__ void __launch_bounds__(256) step_her2(int n, int i, cxd *__restrict__ Ac, const cxd *__restrict__ Vp,
                                                 const cxd *__restrict__ tau, const cxd *__restrict__ p,
                                                 const cxd *__restrict__ part, int nparts) {
    __shared__ cxd sv[U_ROWS], sw[U_ROWS];
    __shared__ cxd salpha;
    const int m = n - 1 - i;
    const cxd *v = Vp + (int64_t)i * n;
    if (threadIdx.x < 32) {
        double re = 0.0, im = 0.0;
        for (int q = threadIdx.x; q < nparts; q += 32) {
            re += part[q].re;
            im += part[q].im;
        }
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (threadIdx.x == 0) salpha = cxd{-0.5, 0.0} * tau[i] * cxd{re, im};
    }
    __syncthreads();
    const cxd alpha = salpha;
    const int c = blockIdx.x * U_COLS + threadIdx.x, r0 = blockIdx.y * U_ROWS;
    if (threadIdx.x < U_ROWS && r0 + (int)threadIdx.x < m) {
        const cxd vr = v[r0 + threadIdx.x];
        sv[threadIdx.x] = vr;
        sw[threadIdx.x] = p[r0 + threadIdx.x] + alpha * vr;
    }
    __syncthreads();
    if (c >= m) return;
    const cxd vc = v[c], wc = p[c] + alpha * vc;
    cxd *base = Ac + (int64_t)(i + 1 + r0) * n + (i + 1) + c;
    const int rows = min(U_ROWS, m - r0);
#pragma unroll 4
    for (int rr = 0; rr < rows; ++rr) {
        const cxd vr = sv[rr], wr = sw[rr];
        cxd a = base[(int64_t)rr * n];
        a.re = fma(-vr.re, wc.re, fma(-vr.im, wc.im, fma(-wr.re, vc.re, fma(-wr.im, vc.im, a.re))));
        a.im = fma(-vr.im, wc.re, fma(vr.re, wc.im, fma(-wr.im, vc.re, fma(wr.re, vc.im, a.im))));
        base[(int64_t)rr * n] = a;
    }
}

__global__ void last_diag(int n, const cxd *Ac, double *d) { d[n - 1] = Ac[(int64_t)(n - 1) * n + (n - 1)].re; }

// The reflectors are kept packed by rows: Vp[i * n + r] = v_i[r], r < n-1-i.

// X <- Q^H X (adjoint: H_0^H first, t_i = conj(tau_i)) or X <- Q X (H_{n-2} first, t_i =
// tau_i), H_i = I - t_i v_i v_i^H on rows i+1.., with X held transposed (XT, k x n: row c
// is column c of X, so a column is contiguous).  The columns of X are independent under a
// left product, so one block owns AC of them and walks all n-1 reflectors itself: per
// reflector y = v^H X (block reduction), X -= t v y.
constexpr int AC = 2;  // columns per block
__global__ void __launch_bounds__(256) apply_q(int n, int k, const cxd *__restrict__ Vp, const cxd *__restrict__ tau,
                                               cxd *__restrict__ X, int adjoint) {
    __shared__ double red[8][AC][2];
    __shared__ cxd ty[AC];
    const int c0 = blockIdx.x * AC;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int s = 0; s < n - 1; ++s) {
        const int i = adjoint ? s : n - 2 - s;
        const int m = n - 1 - i;
        const cxd *v = Vp + (int64_t)i * n;
        cxd *Xi = X + (i + 1);  // column c0 + c, row i+1+r at Xi[(c0 + c) * n + r]
        double re[AC], im[AC];
#pragma unroll
        for (int c = 0; c < AC; ++c) re[c] = im[c] = 0.0;
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
            const cxd vr = v[r];
#pragma unroll
            for (int c = 0; c < AC; ++c) {
                if (c0 + c < k) {
                    const cxd x = Xi[(int64_t)(c0 + c) * n + r];
                    re[c] += vr.re * x.re + vr.im * x.im;  // conj(v_r) x
                    im[c] += vr.re * x.im - vr.im * x.re;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < AC; ++c) {
            for (int o = 16; o > 0; o >>= 1) {
                re[c] += __shfl_xor_sync(0xffffffffu, re[c], o);
                im[c] += __shfl_xor_sync(0xffffffffu, im[c], o);
            }
            if (lane == 0) {
                red[warp][c][0] = re[c];
                red[warp][c][1] = im[c];
            }
        }
        __syncthreads();
        if (threadIdx.x < AC) {
            cxd y = {0.0, 0.0};
            for (int w = 0; w < 8; ++w) y = y + cxd{red[w][threadIdx.x][0], red[w][threadIdx.x][1]};
            const cxd t = adjoint ? cconj(tau[i]) : tau[i];
            ty[threadIdx.x] = t * y;
        }
        __syncthreads();
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
            const cxd vr = v[r];
#pragma unroll
            for (int c = 0; c < AC; ++c)
                if (c0 + c < k) Xi[(int64_t)(c0 + c) * n + r] = Xi[(int64_t)(c0 + c) * n + r] - vr * ty[c];
        }
        __syncthreads();  // ty and red are rewritten by the next reflector
    }
}

// XT (k x n complex) = V^T (V real or complex, ld ldv), through 32 x 32 shared tiles
__global__ void load_t(int n, int k, const double *__restrict__ V, int64_t ldv, int v_cplx, cxd *__restrict__ XT) {
    __shared__ cxd tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int q = ty; q < 32; q += 8) {
        const int r = r0 + q, c = c0 + tx;
        if (r < n && c < k)
            tile[q][tx] = v_cplx ? cxd{V[2 * (r * ldv + c)], V[2 * (r * ldv + c) + 1]} : cxd{V[r * ldv + c], 0.0};
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
        const int c = c0 + q, r = r0 + tx;
        if (r < n && c < k) XT[(int64_t)c * n + r] = tile[tx][q];
    }
}
// out (cols x rows) = in^T (in: rows x cols), complex
__global__ void transpose_cx(int rows, int cols, const cxd *__restrict__ in, cxd *__restrict__ out) {
    __shared__ cxd tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y;
    for (int q = ty; q < 32; q += 8) {
        const int r = r0 + q, c = c0 + tx;
        if (r < rows && c < cols) tile[q][tx] = in[(int64_t)r * cols + c];
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
        const int c = c0 + q, r = r0 + tx;
        if (r < rows && c < cols) out[(int64_t)c * rows + r] = tile[tx][q];
    }
}
// Y (n x k, complex or its real part, ld ldy) = XT^T
__global__ void store_t(int n, int k, const cxd *__restrict__ XT, double *__restrict__ Y, int64_t ldy, int y_real) {
    __shared__ cxd tile[32][33];
    const int c0 = blockIdx.y * 32, r0 = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y;  // tile of XT: rows c, cols r
    for (int q = ty; q < 32; q += 8) {
        const int c = c0 + q, r = r0 + tx;
        if (c < k && r < n) tile[q][tx] = XT[(int64_t)c * n + r];
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
        const int r = r0 + q, c = c0 + tx;
        if (r < n && c < k) {
            const cxd x = tile[tx][q];
            if (y_real) Y[r * ldy + c] = x.re;
            else {
                Y[2 * (r * ldy + c)] = x.re;
                Y[2 * (r * ldy + c) + 1] = x.im;
            }
        }
    }
}

cudaError_t apply_reflectors(int n, int k, const cxd *Vp, const cxd *tau, cxd *X, bool adjoint, cudaStream_t st,
                             Profiler &prof) {
    return prof.timed(adjoint ? "reduce_apply_QH" : "reduce_apply_Q", st, [&]() -> cudaError_t {
        apply_q<<<(k + AC - 1) / AC, 256, 0, st>>>(n, k, Vp, tau, X, adjoint ? 1 : 0);
        return cudaGetLastError();
    });
}

}  // namespace
}  // namespace expm

using namespace expm;

extern "C" expm_status expm_apply_dense_reduced(expm_plan p, int n, const void *A, int lda, int a_is_complex,
                                                const void *V, int ldv, int k, int v_is_complex, void *Y, int ldy,
                                                const expm_opts *opts_in, expm_info *info) {
    if (!p) return set_error(EXPM_EINVAL, "apply_dense_reduced: NULL plan");
    expm_opts opts;
    if (opts_in) opts = *opts_in; else expm_opts_default(&opts);
    if (n < 1 || n > 12000 || k < 1 || k > 1024)
        return set_error(EXPM_EINVAL, "apply_dense_reduced: need 1 <= n <= 12000 and 1 <= k <= 1024");
    if (lda < n || ldv < k || ldy < k) return set_error(EXPM_EINVAL, "apply_dense_reduced: leading dimension too small");
    if (!A || !V || !Y) return set_error(EXPM_EINVAL, "apply_dense_reduced: NULL data pointer");
    if (!is_device_ptr(A) || !is_device_ptr(V) || !is_device_ptr(Y))
        return set_error(EXPM_EINVAL, "apply_dense_reduced: A, V and Y must be device memory");
    if (opts.flags != 0 && !(opts.prec == EXPM_MIXED_FP32 && opts.flags == EXPM_FLAG_SKIP_FINAL_RESIDUAL))
        return set_error(EXPM_EINVAL, "apply_dense_reduced: bad opts.flags");
    if (!std::isfinite(opts.t) || !std::isfinite(opts.shift_c))
        return set_error(EXPM_EINVAL, "apply_dense_reduced: t and shift_c must be finite");
    if (opts.prec != EXPM_FP64 && opts.prec != EXPM_MIXED_F32X2 && opts.prec != EXPM_MIXED_FP32)
        return set_error(EXPM_EINVAL, "apply_dense_reduced: precision (of the tridiagonal solves) must be "
                                      "EXPM_FP64, EXPM_MIXED_F32X2 or EXPM_MIXED_FP32");
    if (info) *info = expm_info{0, 0.0, 0.0, EXPM_OK};
    DeviceGuard guard(p->device);
    cudaStream_t st = (cudaStream_t)opts.stream;
    // stage: Ac | tau | d | e | X (n x k complex) | Z | packed reflectors | step vectors
    const size_t nn = (size_t)n * n, nk = (size_t)n * k;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t oAc = 0, oTau = oAc + al(nn * 16), oD = oTau + al((size_t)n * 16), oE = oD + al((size_t)n * 8),
                 oX = oE + al((size_t)n * 8), oZ = oX + al(nk * 16), oP = oZ + al(nk * 16),
                 oV = oP + al(nn * 16), oW = oV + al((size_t)n * 16), oQ = oW + al((size_t)n * 16),
                 total = oQ + al((size_t)n * 16);
    expm_status s = plan_reserve(p, &p->stage, &p->stage_bytes, total);
    if (s != EXPM_OK) return s;
    unsigned char *b = (unsigned char *)p->stage;
    cxd *Ac = (cxd *)(b + oAc), *tau = (cxd *)(b + oTau), *X = (cxd *)(b + oX), *Z = (cxd *)(b + oZ),
        *Vp = (cxd *)(b + oP), *part = (cxd *)(b + oW), *pbuf = (cxd *)(b + oQ);
    double *d = (double *)(b + oD), *e = (double *)(b + oE);
    Profiler &prof = p->prof;
    cudaError_t err = prof.timed("reduce_copy", st, [&] {
        to_complex<<<n, 256, 0, st>>>(n, (const double *)A, lda, a_is_complex, Ac);
        load_t<<<dim3((k + 31) / 32, (n + 31) / 32), dim3(32, 8), 0, st>>>(n, k, (const double *)V, ldv, v_is_complex,
                                                                          Z);  // Z holds X^T until the solve
        return cudaGetLastError();
    });
    if (err != cudaSuccess) return cuda_error(err, "apply_dense_reduced: copy");
    // reduction to tridiagonal form
    err = prof.timed("reduce_tridiag", st, [&]() -> cudaError_t {
        const size_t vsm = sizeof(cxd) * (size_t)std::max(n - 1, 1);
        cudaError_t e1 = cudaFuncSetAttribute(step_hemv, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10);
        if (e1 != cudaSuccess) return e1;
        for (int i = 0; i + 1 < n; ++i) {
            const int m = n - 1 - i;
            const int nb = (m + H_ROWS - 1) / H_ROWS;
            step_hemv<<<nb, 256, vsm, st>>>(n, i, Ac, Vp, tau, d, e, pbuf, part);
            step_her2<<<dim3((m + U_COLS - 1) / U_COLS, (m + U_ROWS - 1) / U_ROWS), 256, 0, st>>>(n, i, Ac, Vp, tau,
                                                                                                 pbuf, part, nb);
        }
        last_diag<<<1, 1, 0, st>>>(n, Ac, d);
        return cudaGetLastError();
    });
    if (err != cudaSuccess) return cuda_error(err, "apply_dense_reduced: reduction");
    if (n > 1) {
        err = apply_reflectors(n, k, Vp, tau, Z, true, st, prof);  // X^T = (Q^H V)^T
        if (err != cudaSuccess) return cuda_error(err, "apply_dense_reduced: Q^H V");
    }
    transpose_cx<<<dim3((n + 31) / 32, (k + 31) / 32), dim3(32, 8), 0, st>>>(k, n, Z, X);  // X = Q^H V, n x k
    // Z = e^c R_n(tT - cI) X on the real symmetric tridiagonal T (complex columns)
    expm_opts o2 = opts;
    expm_info i2{};
    s = expm_apply_tridiag(p, n, d, e, 0, X, k, 1, Z, &o2, info ? &i2 : nullptr);
    if (s != EXPM_OK && s != EXPM_ENOCONV) return s;
    transpose_cx<<<dim3((k + 31) / 32, (n + 31) / 32), dim3(32, 8), 0, st>>>(n, k, Z, X);  // X = Z^T, k x n
    if (n > 1) {
        err = apply_reflectors(n, k, Vp, tau, X, false, st, prof);  // (Q Z)^T
        if (err != cudaSuccess) return cuda_error(err, "apply_dense_reduced: Q Z");
    }
    store_t<<<dim3((n + 31) / 32, (k + 31) / 32), dim3(32, 8), 0, st>>>(n, k, X, (double *)Y, ldy,
                                                                      (a_is_complex || v_is_complex) ? 0 : 1);
    if ((err = cudaGetLastError()) != cudaSuccess) return cuda_error(err, "apply_dense_reduced: store");
    if (info) {
        *info = i2;
        if (s == EXPM_ENOCONV) return set_error(s, "apply_dense_reduced: refinement of the tridiagonal solves did not reach tol");
    }
    return EXPM_OK;
}
