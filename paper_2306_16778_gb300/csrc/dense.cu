// dense.cu -- pole-batched dense path: exp(tA)V ~ e^c sum_k a_k (tA - cI + theta_k I)^{-1} V.
//
// Eqs. ExpoMatRat / expAx of the paper with one unpivoted LU per conjugate pole
// pair.  Real A and real V: only the Im(theta) > 0 member of each pair is solved and
// the sum is 2 Re(a X) (Remark 5.1).  Complex Hermitian A: the conjugate pole's
// matrix is the conjugate transpose, tA - cI + conj(theta) I = (tA - cI + theta I)^H
// = U^H L^H, so one factorization serves both poles of a pair.
//
// Precision (opts.prec):
//   binary64      factor, solve and sum in binary64;
//   mixed         factor and solve in binary32; the solution is kept in binary64 and
//                 refined with binary64 residuals R = V - (tA - cI + theta I) X until
//                 ||R||_F <= tol (||tA||_F + |theta - c|) ||X||_F or max_refine sweeps;
//                 the residue sum is binary64.
//
// Blocked right-looking LU, panel width DN_NB, per step: diagonal-block LU,
// the two panel triangular solves, and the trailing update as a batched complex
// GEMM (all pole pairs in one launch).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "arith.cuh"
#include "dense.cuh"
#include "dense_kernels.cuh"
#include "plan.cuh"

namespace expm {

// ------------------------------------------------------------------ small kernels

// X[b] (n x kc, cx<T>) = V as complex; V real (v_cplx = 0, ldv in doubles) or complex
// (ldv in complex entries).  Shared by every batch b.
template <class T>
__global__ void load_rhs(int n, int kc, const double *__restrict__ V, int64_t ldv, int v_cplx, cx<T> *X,
                         int64_t xstride) {
    const int64_t total = (int64_t)n * kc;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / kc), j = (int)(idx % kc);
        cx<T> v;
        if (v_cplx) v = {(T)V[2 * (i * ldv + j)], (T)V[2 * (i * ldv + j) + 1]};
        else v = {(T)V[i * ldv + j], (T)0};
        X[(int64_t)blockIdx.z * xstride + idx] = v;
    }
}

// R[b] = V - (theta_b - c) X[b]   (the diagonal part of the residual; the tA X part
// is subtracted by a GEMM afterwards)
__global__ void residual_diag(int n, int kc, const double *__restrict__ V, int64_t ldv, int v_cplx,
                              const cx<double> *X, cx<double> *R, int64_t stride, DenseSystems sys) {
    const int b = blockIdx.z;
    const cx<double> sh = {sys.th_re[b] - sys.cshift, sys.th_im[b]};
    const int64_t total = (int64_t)n * kc;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / kc), j = (int)(idx % kc);
        cx<double> v;
        if (v_cplx) v = {V[2 * (i * ldv + j)], V[2 * (i * ldv + j) + 1]};
        else v = {V[i * ldv + j], 0.0};
        R[(int64_t)b * stride + idx] = v - sh * X[(int64_t)b * stride + idx];
    }
}

// Xc (binary32) = R (binary64) and sums of |R|^2, |X|^2 per batch
__global__ void demote_and_norms(int64_t total, const cx<double> *R, const cx<double> *X, cx<float> *Xc,
                                 int64_t stride, double *rn2, double *xn2) {
    const int b = blockIdx.z;
    double r2 = 0.0, x2 = 0.0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const cx<double> r = R[(int64_t)b * stride + idx];
        const cx<double> x = X[(int64_t)b * stride + idx];
        Xc[(int64_t)b * stride + idx] = {(float)r.re, (float)r.im};
        r2 += r.re * r.re + r.im * r.im;
        x2 += x.re * x.re + x.im * x.im;
    }
    for (int o = 16; o > 0; o >>= 1) {
        r2 += __shfl_xor_sync(0xffffffffu, r2, o);
        x2 += __shfl_xor_sync(0xffffffffu, x2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(rn2 + b, r2);
        atomicAdd(xn2 + b, x2);
    }
}

// X (binary64) += D (binary32 correction)
__global__ void add_correction(int64_t total, const cx<float> *D, cx<double> *X, int64_t stride) {
    const int b = blockIdx.z;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const cx<float> d = D[(int64_t)b * stride + idx];
        cx<double> &x = X[(int64_t)b * stride + idx];
        x.re += (double)d.re;
        x.im += (double)d.im;
    }
}

// Residue-weighted sum (a8): Y = sum_b W_b X_b, real part only when real_out.
// The sum over systems is taken in a fixed order per element (no atomics).
__global__ void accumulate(int n, int kc, int nsys, const cx<double> *__restrict__ X, int64_t stride,
                           DenseSystems sys, int real_out, double *__restrict__ Y, int64_t ldy) {
    const int64_t total = (int64_t)n * kc;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / kc), j = (int)(idx % kc);
        cx<double> acc = {0.0, 0.0};
        for (int b = 0; b < nsys; ++b) {
            const cx<double> w = {sys.w_re[b], sys.w_im[b]};
            acc = acc + w * X[(int64_t)b * stride + idx];
        }
        if (real_out) Y[i * ldy + j] = acc.re;
        else {
            Y[2 * (i * ldy + j)] = acc.re;
            Y[2 * (i * ldy + j) + 1] = acc.im;
        }
    }
}

// sum of |A_ij|^2 (binary64) into *out
__global__ void frob2(int n, const double *__restrict__ A, int64_t lda, int cplx, double *out) {
    double acc = 0.0;
    const int64_t total = (int64_t)n * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx % n;
        if (cplx) {
            const double re = A[2 * (i * lda + j)], im = A[2 * (i * lda + j) + 1];
            acc += re * re + im * im;
        } else {
            const double v = A[i * lda + j];
            acc += v * v;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// ------------------------------------------------------------------ host helpers

static unsigned grid1d(int64_t total, int threads = 256) {
    int64_t g = (total + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

template <class K> static cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define EXPM_TRY(x)                               \
    do {                                          \
        cudaError_t _e = (x);                     \
        if (_e != cudaSuccess) return _e;         \
    } while (0)

// Unpivoted blocked LU of `batch` n x n matrices F (ld n, batch stride n*n).
template <class T>
static cudaError_t lu_blocked(int n, int batch, cx<T> *F, cudaStream_t st, Profiler &prof) {
    const int64_t bs = (int64_t)n * n;
    const size_t sm1 = tri_smem_bytes<T>(), sm2 = 2 * tri_smem_bytes<T>();
    EXPM_TRY(set_smem(lu_diag<T>, sm1));
    EXPM_TRY(set_smem(trsm_left<T, true, true, false>, sm2));
    EXPM_TRY(set_smem(trsm_right_upper<T>, sm2));
    const char *tag = sizeof(T) == 8 ? "f64" : "f32";
    (void)tag;
    for (int p = 0; p < n; p += DN_NB) {
        const int nb = std::min(DN_NB, n - p);
        const int rest = n - p - nb;
        cx<T> *diag = F + (int64_t)p * n + p;
        EXPM_TRY(prof.timed(sizeof(T) == 8 ? "lu_diag<f64>" : "lu_diag<f32>", st, [&] {
            lu_diag<T><<<dim3(1, 1, batch), 256, sm1, st>>>(nb, diag, n, bs);
            return cudaGetLastError();
        }));
        if (rest <= 0) break;
        EXPM_TRY(prof.timed(sizeof(T) == 8 ? "trsm_panels<f64>" : "trsm_panels<f32>", st, [&] {
            // U12 = L11^{-1} A12 and L21 = A21 U11^{-1}
            trsm_left<T, true, true, false><<<dim3((rest + 63) / 64, 1, batch), 64, sm2, st>>>(
                nb, rest, diag, n, bs, diag + nb, n, bs);
            trsm_right_upper<T><<<dim3((rest + 63) / 64, 1, batch), 64, sm2, st>>>(nb, rest, diag, n, bs,
                                                                                 diag + (int64_t)nb * n, n, bs);
            return cudaGetLastError();
        }));
        EXPM_TRY(prof.timed(sizeof(T) == 8 ? "cgemm_update<f64>" : "cgemm_update<f32>", st, [&] {
            // A22 -= L21 U12
            dim3 g((rest + 63) / 64, (rest + 63) / 64, batch);
            cgemm<T, cx<T>, false, false><<<g, 256, 0, st>>>(
                rest, rest, nb, cx<T>{T(-1), T(0)}, T(1), diag + (int64_t)nb * n, n, bs, diag + nb, n, bs,
                diag + (int64_t)nb * n + nb, n, bs);
            return cudaGetLastError();
        }));
    }
    return cudaSuccess;
}

// In-place solve of the kc columns of X[b] (n x kc) with the factors in F.
// conj = false: L U x = b (forward unit-lower, back upper).
// conj = true : U^H L^H x = b (forward with U^H, back with unit L^H).
// Factor of system b is F[fidx[b]] -- systems of one pair share a factor.
template <class T>
static cudaError_t lu_solve(int n, int kc, int batch, const cx<T> *F, int64_t fstride, bool conj, cx<T> *X,
                            int64_t xstride, cudaStream_t st, Profiler &prof) {
    const size_t sm2 = 2 * tri_smem_bytes<T>();
    const int cb = (kc + 63) / 64;
    EXPM_TRY(set_smem(trsm_left<T, true, true, false>, sm2));
    EXPM_TRY(set_smem(trsm_left<T, false, false, false>, sm2));
    EXPM_TRY(set_smem(trsm_left<T, true, false, true>, sm2));
    EXPM_TRY(set_smem(trsm_left<T, false, true, true>, sm2));
    return prof.timed(sizeof(T) == 8 ? "lu_solve<f64>" : "lu_solve<f32>", st, [&]() -> cudaError_t {
        // forward sweep
        for (int p = 0; p < n; p += DN_NB) {
            const int nb = std::min(DN_NB, n - p), rest = n - p - nb;
            const cx<T> *dg = F + (int64_t)p * n + p;
            cx<T> *xp = X + (int64_t)p * kc;
            if (!conj) trsm_left<T, true, true, false><<<dim3(cb, 1, batch), 64, sm2, st>>>(nb, kc, dg, n, fstride, xp, kc, xstride);
            else trsm_left<T, true, false, true><<<dim3(cb, 1, batch), 64, sm2, st>>>(nb, kc, dg, n, fstride, xp, kc, xstride);
            if (rest > 0) {
                dim3 g(cb, (rest + 63) / 64, batch);
                if (!conj)  // X[p+nb:] -= L[p+nb:, p:p+nb] X[p:p+nb]
                    cgemm<T, cx<T>, false, false><<<g, 256, 0, st>>>(rest, kc, nb, cx<T>{T(-1), T(0)}, T(1),
                                                                     dg + (int64_t)nb * n, n, fstride, xp, kc, xstride,
                                                                     xp + (int64_t)nb * kc, kc, xstride);
                else  // X[p+nb:] -= (U[p:p+nb, p+nb:])^H X[p:p+nb]
                    cgemm<T, cx<T>, true, false><<<g, 256, 0, st>>>(rest, kc, nb, cx<T>{T(-1), T(0)}, T(1), dg + nb, n,
                                                                    fstride, xp, kc, xstride, xp + (int64_t)nb * kc, kc,
                                                                    xstride);
            }
        }
        // backward sweep
        const int nblk = (n + DN_NB - 1) / DN_NB;
        for (int bi = nblk - 1; bi >= 0; --bi) {
            const int p = bi * DN_NB, nb = std::min(DN_NB, n - p);
            const cx<T> *dg = F + (int64_t)p * n + p;
            cx<T> *xp = X + (int64_t)p * kc;
            if (!conj) trsm_left<T, false, false, false><<<dim3(cb, 1, batch), 64, sm2, st>>>(nb, kc, dg, n, fstride, xp, kc, xstride);
            else trsm_left<T, false, true, true><<<dim3(cb, 1, batch), 64, sm2, st>>>(nb, kc, dg, n, fstride, xp, kc, xstride);
            if (p > 0) {
                dim3 g(cb, (p + 63) / 64, batch);
                if (!conj)  // X[:p] -= U[:p, p:p+nb] X[p:p+nb]
                    cgemm<T, cx<T>, false, false><<<g, 256, 0, st>>>(p, kc, nb, cx<T>{T(-1), T(0)}, T(1), F + p, n,
                                                                     fstride, xp, kc, xstride, X, kc, xstride);
                else  // X[:p] -= (L[p:p+nb, :p])^H X[p:p+nb]
                    cgemm<T, cx<T>, true, false><<<g, 256, 0, st>>>(p, kc, nb, cx<T>{T(-1), T(0)}, T(1),
                                                                    F + (int64_t)p * n, n, fstride, xp, kc, xstride, X,
                                                                    kc, xstride);
            }
        }
        return cudaGetLastError();
    });
}

// ------------------------------------------------------------------ driver

size_t dense_workspace_bytes(const DenseGeom &g) {
    const size_t nn = (size_t)g.n * g.n, nk = (size_t)g.n * g.kc;
    const size_t fb = g.mixed ? sizeof(cx<float>) : sizeof(cx<double>);
    size_t bytes = g.npairs * nn * fb;                                  // factors
    bytes += (size_t)g.nsys * nk * sizeof(cx<double>);                  // X (binary64)
    if (g.mixed) bytes += (size_t)g.nsys * nk * (sizeof(cx<double>) + sizeof(cx<float>));  // R, correction
    bytes += 4096 + 64 * sizeof(double) * 4;
    return bytes + 8 * 256;
}

static inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

template <class T>
static cudaError_t factor_pairs(const DenseGeom &g, const double *A, int64_t lda, const DenseSystems &sys,
                                cx<T> *F, unsigned *amax, unsigned *umax, cudaStream_t st, Profiler &prof) {
    // pair s uses system 2s (complex A) or s (real data); both carry the Im(theta) > 0 member
    DenseSystems pairs = sys;
    for (int s = 0; s < g.npairs; ++s) {
        const int b = g.complex_a ? 2 * s : s;
        pairs.th_re[s] = sys.th_re[b];
        pairs.th_im[s] = sys.th_im[b];
    }
    EXPM_TRY(cudaMemsetAsync(amax, 0, sizeof(unsigned) * 2 * DENSE_MAXSYS, st));
    EXPM_TRY(prof.timed(sizeof(T) == 8 ? "form_shifted<f64>" : "form_shifted<f32>", st, [&] {
        form_shifted<T><<<dim3(grid1d((int64_t)g.n * g.n), 1, g.npairs), 256, 0, st>>>(
            g.n, A, (int)lda, g.complex_a, g.t, pairs, F, amax);
        return cudaGetLastError();
    }));
    EXPM_TRY(lu_blocked<T>(g.n, g.npairs, F, st, prof));
    max_abs_upper<T><<<dim3(grid1d((int64_t)g.n * g.n), 1, g.npairs), 256, 0, st>>>(g.n, F, g.n,
                                                                                     (int64_t)g.n * g.n, umax);
    return cudaGetLastError();
}

template <class T>
static cudaError_t solve_systems(const DenseGeom &g, const cx<T> *F, cx<T> *X, int64_t xstride, cudaStream_t st,
                                 Profiler &prof) {
    const int64_t fs = (int64_t)g.n * g.n;
    if (!g.complex_a) return lu_solve<T>(g.n, g.kc, g.npairs, F, fs, false, X, xstride, st, prof);
    // systems 2s (theta) and 2s+1 (conj theta) share factor s: run the two sweeps with
    // batch stride 2*xstride over the even and the odd systems
    EXPM_TRY(lu_solve<T>(g.n, g.kc, g.npairs, F, fs, false, X, 2 * xstride, st, prof));
    return lu_solve<T>(g.n, g.kc, g.npairs, F, fs, true, X + xstride, 2 * xstride, st, prof);
}

cudaError_t dense_run(const DenseGeom &g, const double *A, int64_t lda, const double *V, int64_t ldv, int v_cplx,
                      double *Y, int64_t ldy, const DenseSystems &sys, void *work, cudaStream_t st, Profiler &prof,
                      DenseResult *res) {
    const int64_t nk = (int64_t)g.n * g.kc;
    unsigned char *p = (unsigned char *)work;
    unsigned *amax = (unsigned *)p;
    unsigned *umax = amax + DENSE_MAXSYS;
    double *rn2 = (double *)(p + 1024);
    double *xn2 = rn2 + DENSE_MAXSYS;
    p += align_up(4096);
    const size_t fb = g.mixed ? sizeof(cx<float>) : sizeof(cx<double>);
    void *F = p;
    p += align_up((size_t)g.npairs * g.n * g.n * fb);
    cx<double> *X = (cx<double> *)p;
    p += align_up((size_t)g.nsys * nk * sizeof(cx<double>));
    const unsigned gx = grid1d(nk);
    res->iters = 0;
    res->resid_rel_max = 0.0;
    if (!g.mixed) {
        EXPM_TRY(factor_pairs<double>(g, A, lda, sys, (cx<double> *)F, amax, umax, st, prof));
        load_rhs<double><<<dim3(gx, 1, g.nsys), 256, 0, st>>>(g.n, g.kc, V, ldv, v_cplx, X, nk);
        EXPM_TRY(cudaGetLastError());
        EXPM_TRY(solve_systems<double>(g, (cx<double> *)F, X, nk, st, prof));
    } else {
        cx<double> *R = (cx<double> *)p;
        p += align_up((size_t)g.nsys * nk * sizeof(cx<double>));
        cx<float> *D = (cx<float> *)p;
        EXPM_TRY(factor_pairs<float>(g, A, lda, sys, (cx<float> *)F, amax, umax, st, prof));
        EXPM_TRY(cudaMemsetAsync(X, 0, (size_t)g.nsys * nk * sizeof(cx<double>), st));
        std::vector<double> h(2 * DENSE_MAXSYS);
        // ||tA||_F for the relative residual of the stopping test
        EXPM_TRY(cudaMemsetAsync(rn2, 0, sizeof(double), st));
        frob2<<<grid1d((int64_t)g.n * g.n), 256, 0, st>>>(g.n, A, lda, g.complex_a, rn2);
        EXPM_TRY(cudaGetLastError());
        EXPM_TRY(cudaMemcpyAsync(h.data(), rn2, sizeof(double), cudaMemcpyDeviceToHost, st));
        EXPM_TRY(cudaStreamSynchronize(st));
        const double anorm = std::sqrt(h[0]) * std::fabs(g.t);
        // it = 0: initial solve; it = 1 .. max_refine: refinement sweeps; the residual
        // of the current X is checked before every sweep and once after the last one
        for (int it = 0;; ++it) {
            // R = V - (tA - cI + theta I) X, binary64
            residual_diag<<<dim3(gx, 1, g.nsys), 256, 0, st>>>(g.n, g.kc, V, ldv, v_cplx, X, R, nk, sys);
            EXPM_TRY(cudaGetLastError());
            if (it > 0) {
                EXPM_TRY(prof.timed("residual_gemm<f64>", st, [&] {
                    dim3 gg((g.kc + 63) / 64, (g.n + 63) / 64, g.nsys);
                    if (g.complex_a)
                        cgemm<double, cx<double>, false, false><<<gg, 256, 0, st>>>(
                            g.n, g.kc, g.n, cx<double>{-g.t, 0.0}, 1.0, (const cx<double> *)A, (int)lda, 0, X, g.kc, nk,
                            R, g.kc, nk);
                    else
                        cgemm<double, double, false, false><<<gg, 256, 0, st>>>(g.n, g.kc, g.n, cx<double>{-g.t, 0.0}, 1.0,
                                                                                A, (int)lda, 0, X, g.kc, nk, R, g.kc, nk);
                    return cudaGetLastError();
                }));
            }
            EXPM_TRY(cudaMemsetAsync(rn2, 0, sizeof(double) * 2 * DENSE_MAXSYS, st));
            demote_and_norms<<<dim3(gx, 1, g.nsys), 256, 0, st>>>(nk, R, X, D, nk, rn2, xn2);
            EXPM_TRY(cudaGetLastError());
            if (it > 0) {
                EXPM_TRY(cudaMemcpyAsync(h.data(), rn2, sizeof(double) * 2 * DENSE_MAXSYS, cudaMemcpyDeviceToHost, st));
                EXPM_TRY(cudaStreamSynchronize(st));
                bool done = true;
                double worst = 0.0;
                for (int b = 0; b < g.nsys; ++b) {
                    const double shift = std::hypot(sys.th_re[b] - sys.cshift, sys.th_im[b]);
                    const double den = (anorm + shift) * std::sqrt(h[DENSE_MAXSYS + b]);
                    const double rel = den > 0 ? std::sqrt(h[b]) / den : 0.0;
                    worst = std::max(worst, rel);
                    if (!(rel <= g.tol)) done = false;
                }
                res->resid_rel_max = worst;
                res->iters = it - 1;
                if (done || it > g.max_refine) break;
            }
            EXPM_TRY(solve_systems<float>(g, (const cx<float> *)F, D, nk, st, prof));
            add_correction<<<dim3(gx, 1, g.nsys), 256, 0, st>>>(nk, D, X, nk);
            EXPM_TRY(cudaGetLastError());
        }
    }
    EXPM_TRY(prof.timed("accumulate", st, [&] {
        accumulate<<<grid1d(nk), 256, 0, st>>>(g.n, g.kc, g.nsys, X, nk, sys, g.complex_a ? 0 : 1, Y, ldy);
        return cudaGetLastError();
    }));
    // growth factors
    std::vector<unsigned> hm(2 * DENSE_MAXSYS);
    EXPM_TRY(cudaMemcpyAsync(hm.data(), amax, sizeof(unsigned) * 2 * DENSE_MAXSYS, cudaMemcpyDeviceToHost, st));
    EXPM_TRY(cudaStreamSynchronize(st));
    res->growth_max = 0.0;
    for (int s = 0; s < g.npairs; ++s) {
        float a, u;
        std::memcpy(&a, &hm[s], 4);
        std::memcpy(&u, &hm[DENSE_MAXSYS + s], 4);
        if (a > 0) res->growth_max = std::max(res->growth_max, (double)u / (double)a);
    }
    return cudaSuccess;
}

}  // namespace expm
