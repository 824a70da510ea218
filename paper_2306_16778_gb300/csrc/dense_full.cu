// dense_full.cu -- expm_apply_dense_full: the full matrix e^c R_n(tA - cI).
//
// Eq. ExpoMatRat itself: R_n(A) = sum_k a_k (A + theta_k I)^{-1}, i.e. the dense path
// with V = I.  The per-pair LUs are formed once (dense_factor) and the identity is fed
// through the solve part (triangular solves, refinement, residue sum) in column blocks,
// so the factorization is not repeated per block.
#include <algorithm>
#include <cmath>

#include "../../include/expm.h"
#include "dense.cuh"
#include "plan.cuh"

namespace expm {
namespace {

// V = columns c0 .. c0+kc-1 of the n x n identity, row-major n x kc (real or interleaved complex)
__global__ void identity_block(int n, int kc, int c0, int cplx, double *V) {
    const int64_t total = (int64_t)n * kc;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / kc;
        const int j = (int)(idx % kc);
        const double one = (i == (int64_t)c0 + j) ? 1.0 : 0.0;
        if (cplx) {
            V[2 * idx] = one;
            V[2 * idx + 1] = 0.0;
        } else {
            V[idx] = one;
        }
    }
}

constexpr int FULL_KC = 512;  // identity columns per solve block

}  // namespace
}  // namespace expm

using namespace expm;

extern "C" expm_status expm_apply_dense_full(expm_plan p, int n, const void *A, int lda, int a_is_complex, void *Y,
                                             int ldy, const expm_opts *opts_in, expm_info *info) {
    if (!p) return set_error(EXPM_EINVAL, "apply_dense_full: NULL plan");
    expm_opts opts;
    if (opts_in) opts = *opts_in; else expm_opts_default(&opts);
    if (n < 1) return set_error(EXPM_EINVAL, "apply_dense_full: need n >= 1");
    if (lda < n || ldy < n) return set_error(EXPM_EINVAL, "apply_dense_full: leading dimension too small");
    if (!A || !Y) return set_error(EXPM_EINVAL, "apply_dense_full: NULL data pointer");
    if (opts.prec < EXPM_FP64 || opts.prec > EXPM_MIXED_BF16X3)
        return set_error(EXPM_EINVAL, "apply_dense_full: unknown precision");
    if (opts.flags != 0) return set_error(EXPM_EINVAL, "apply_dense_full: opts.flags must be 0");
    if (!std::isfinite(opts.t) || !std::isfinite(opts.shift_c) || !(opts.tol > 0) || opts.max_refine < 0)
        return set_error(EXPM_EINVAL, "apply_dense_full: bad t, shift_c, tol or max_refine");
    if (info) *info = expm_info{0, 0.0, 0.0, EXPM_OK};
    DeviceGuard guard(p->device);
    cudaStream_t st = (cudaStream_t)opts.stream;
    const int S = p->degree / 2;
    const bool complex_a = a_is_complex != 0;
    const int kcw = std::min(n, FULL_KC);
    DenseGeom g{};
    g.n = n;
    g.ninst = 1;
    g.complex_a = complex_a;
    g.npairs = S;
    g.nsys = complex_a ? 2 * S : S;
    g.kc = kcw;
    g.mixed = opts.prec != EXPM_FP64;
    g.tc = opts.prec == EXPM_MIXED_TF32X3 ? 1 : opts.prec == EXPM_MIXED_BF16X3 ? 2 : 0;
    g.t = opts.t;
    g.tol = opts.tol;
    g.max_refine = opts.max_refine;
    DenseSystems sys{};
    sys.cshift = opts.shift_c;
    const double ec = std::exp(opts.shift_c);
    for (int s = 0; s < S; ++s) {
        const double tr = -p->lam[4 * s], ti = -p->lam[4 * s + 1];  // theta = -lambda (Im > 0 member first)
        const double ar = p->w[4 * s], ai = p->w[4 * s + 1];
        if (complex_a) {
            sys.th_re[2 * s] = tr; sys.th_im[2 * s] = ti; sys.w_re[2 * s] = ec * ar; sys.w_im[2 * s] = ec * ai;
            sys.th_re[2 * s + 1] = tr; sys.th_im[2 * s + 1] = -ti;
            sys.w_re[2 * s + 1] = ec * ar; sys.w_im[2 * s + 1] = -ec * ai;
        } else {
            sys.th_re[s] = tr; sys.th_im[s] = ti; sys.w_re[s] = 2 * ec * ar; sys.w_im[s] = 2 * ec * ai;
        }
    }
    const size_t ea = complex_a ? 2 : 1;
    const size_t nA = (size_t)n * lda * ea, nY = (size_t)n * ldy * ea, nV = (size_t)n * kcw * ea;
    const bool da = is_device_ptr(A), dy = is_device_ptr(Y);
    // stage: [identity block | A copy (host A) | Y copy (host Y)]
    expm_status s = plan_reserve(p, &p->stage, &p->stage_bytes,
                                 sizeof(double) * (nV + (da ? 0 : nA) + (dy ? 0 : nY)) + 1024);
    if (s != EXPM_OK) return s;
    double *Vb = (double *)p->stage;
    const double *dA = (const double *)A;
    double *dY = (double *)Y;
    cudaError_t err = cudaSuccess;
    if (!da) {
        err = cudaMemcpyAsync(Vb + nV, A, sizeof(double) * nA, cudaMemcpyHostToDevice, st);
        dA = Vb + nV;
    }
    if (!dy) dY = Vb + nV + (da ? 0 : nA);
    if (err != cudaSuccess) return cuda_error(err, "apply_dense_full: staging copy");
    const size_t fbytes = dense_factor_bytes(g);
    s = plan_reserve(p, &p->work, &p->work_bytes, fbytes + dense_solve_bytes(g));
    if (s != EXPM_OK) return s;
    void *fwork = p->work;
    void *swork = (unsigned char *)p->work + fbytes;
    DenseIO io{};
    io.A = dA;
    io.lda = lda;
    io.v_cplx = complex_a ? 1 : 0;
    io.y_real = complex_a ? 0 : 1;
    io.V = Vb;
    io.ldv = kcw;
    io.ldy = ldy;
    err = dense_factor(g, io, sys, fwork, st, p->prof);
    if (err != cudaSuccess) return cuda_error(err, "apply_dense_full: factor");
    DenseResult res{}, gr{};
    err = dense_growth(g, fwork, st, &gr);
    if (err != cudaSuccess) return cuda_error(err, "apply_dense_full: growth");
    if (gr.tc_timeout) return set_error(EXPM_ETIMEOUT, "apply_dense_full: a bounded wait in the tensor-core kernel gave up");
    int iters = 0;
    double resid = 0.0;
    for (int c0 = 0; c0 < n; c0 += kcw) {
        DenseGeom gb = g;
        gb.kc = std::min(kcw, n - c0);
        identity_block<<<(unsigned)std::min<int64_t>(((int64_t)n * gb.kc + 255) / 256, 1024), 256, 0, st>>>(
            n, gb.kc, c0, complex_a ? 1 : 0, Vb);
        if ((err = cudaGetLastError()) != cudaSuccess) return cuda_error(err, "apply_dense_full: identity");
        DenseIO iob = io;
        iob.ldv = gb.kc;
        iob.Y = dY + (size_t)c0 * ea;
        err = dense_solve(gb, iob, sys, fwork, swork, st, p->prof, &res);
        if (err != cudaSuccess) return cuda_error(err, "apply_dense_full: solve");
        if (res.tc_timeout)
            return set_error(EXPM_ETIMEOUT, "apply_dense_full: a bounded wait in the tensor-core kernel gave up");
        iters = std::max(iters, res.iters);
        resid = std::max(resid, res.resid_rel_max);
    }
    if (!dy) {
        err = cudaMemcpyAsync(Y, dY, sizeof(double) * nY, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        if (err != cudaSuccess) return cuda_error(err, "apply_dense_full: result copy");
    }
    expm_status out = EXPM_OK;
    if (gr.growth_max > opts.growth_max) out = EXPM_EGROWTH;
    else if (g.mixed && !(resid <= opts.tol)) out = EXPM_ENOCONV;
    if (info) {
        info->refine_iters_max = iters;
        info->growth_max_seen = gr.growth_max;
        info->resid_rel_max = resid;
        info->status_worst = out;
    }
    if (out == EXPM_EGROWTH) return set_error(out, "apply_dense_full: LU growth exceeds opts.growth_max");
    if (out == EXPM_ENOCONV) return set_error(out, "apply_dense_full: refinement did not reach opts.tol");
    return EXPM_OK;
}
