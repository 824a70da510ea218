// batched.cu -- expm_apply_batched: many independent dense problems of uneven size.
//
// Each instance i asks for e^c R_n(tA_i - cI) V_i (eq. expAx per instance).  The
// instances are grouped into size buckets; inside a bucket every matrix is padded
// to the bucket's order n_b with zero rows and columns.  Padding is exact: the padded
// part of tA - cI + theta I is the diagonal (theta - c) I, so its LU is diagonal, the
// padded rows of V are zero and so are the padded rows of the solution.  A bucket is
// then one uniform batch of (instance, pole pair) units for the dense kernels -- all
// its LUs, triangular solves, refinement sweeps and residue sums run as batched
// launches over (instance, pair).  Buckets are processed largest first.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <numeric>
#include <vector>

#include "../../include/expm.h"
#include "dense.cuh"
#include "plan.cuh"

namespace expm {

struct InstPtr {
    const double *A;
    const double *V;
    double *Y;
    int n, k;
};

// Apad[z] (nb x nb) = A of instance z, zero padded; Vpad[z] (nb x kb) likewise.
__global__ void gather_pad(const InstPtr *__restrict__ ip, int nb, int kb, int a_words, int v_words,
                           double *__restrict__ Apad, double *__restrict__ Vpad) {
    const InstPtr in = ip[blockIdx.z];
    const int64_t na = (int64_t)nb * nb * a_words;
    double *Ad = Apad + (int64_t)blockIdx.z * na;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < na; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = idx / a_words, w = idx % a_words;
        const int64_t i = e / nb, j = e % nb;
        Ad[idx] = (i < in.n && j < in.n) ? in.A[(i * in.n + j) * a_words + w] : 0.0;
    }
    const int64_t nv = (int64_t)nb * kb * v_words;
    double *Vd = Vpad + (int64_t)blockIdx.z * nv;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nv; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = idx / v_words, w = idx % v_words;
        const int64_t i = e / kb, j = e % kb;
        Vd[idx] = (i < in.n && j < in.k) ? in.V[(i * in.k + j) * v_words + w] : 0.0;
    }
}

// Y of instance z (n x k) = the leading block of Ypad[z] (nb x kb)
__global__ void scatter_unpad(const InstPtr *__restrict__ ip, int nb, int kb, int y_words, const double *__restrict__ Ypad) {
    const InstPtr in = ip[blockIdx.z];
    const int64_t ny = (int64_t)in.n * in.k * y_words;
    const double *Ys = Ypad + (int64_t)blockIdx.z * nb * kb * y_words;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < ny; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = idx / y_words, w = idx % y_words;
        const int64_t i = e / in.k, j = e % in.k;
        in.Y[idx] = Ys[(i * kb + j) * y_words + w];
    }
}

// Padded order of a bucket: multiples of 32 up to 128, then steps of about 1/4.
int bucket_order(int n) {
    static const int edges[] = {32, 64, 96, 128, 160, 192, 256, 320, 384, 448, 512, 640, 768, 896, 1024,
                                1280, 1536, 1792, 2048};
    for (int e : edges)
        if (n <= e) return e;
    return (n + 255) / 256 * 256;
}

}  // namespace expm

using namespace expm;

extern "C" expm_status expm_apply_batched(expm_plan p, int count, const int *n, const void *const *A, int a_is_complex,
                                          const void *const *V, const int *k, int v_is_complex, void *const *Y,
                                          const expm_opts *opts_in, expm_info *per_instance) {
    if (!p) return set_error(EXPM_EINVAL, "apply_batched: NULL plan");
    if (count < 0 || (count > 0 && (!n || !A || !V || !k || !Y)))
        return set_error(EXPM_EINVAL, "apply_batched: NULL array argument");
    if (count == 0) return EXPM_OK;
    expm_opts opts;
    if (opts_in) opts = *opts_in; else expm_opts_default(&opts);
    if (opts.prec != EXPM_FP64 && opts.prec != EXPM_MIXED_FP32 && opts.prec != EXPM_MIXED_F32X2)
        return set_error(EXPM_EINVAL, "apply_batched: precision must be EXPM_FP64, EXPM_MIXED_FP32 or EXPM_MIXED_F32X2");
    if (opts.flags != 0) return set_error(EXPM_EINVAL, "apply_batched: opts.flags must be 0");
    if (!std::isfinite(opts.t) || !std::isfinite(opts.shift_c) || !(opts.tol > 0) || opts.max_refine < 0)
        return set_error(EXPM_EINVAL, "apply_batched: bad t, shift_c, tol or max_refine");
    const bool complex_a = a_is_complex != 0;
    if (!complex_a && v_is_complex)
        return set_error(EXPM_ENOTSUP, "apply_batched: complex V with real A (use complex A or split V)");
    DeviceGuard guard(p->device);
    for (int i = 0; i < count; ++i) {
        if (n[i] < 1 || k[i] < 1 || k[i] > 4096) return set_error(EXPM_EINVAL, "apply_batched: bad n[i] or k[i]");
        if (!A[i] || !V[i] || !Y[i]) return set_error(EXPM_EINVAL, "apply_batched: NULL instance pointer");
        if (!is_device_ptr(A[i]) || !is_device_ptr(V[i]) || !is_device_ptr(Y[i]))
            return set_error(EXPM_EINVAL, "apply_batched: instance data must be device memory");
    }
    if (per_instance)
        for (int i = 0; i < count; ++i) per_instance[i] = expm_info{0, 0.0, 0.0, EXPM_OK};
    cudaStream_t st = (cudaStream_t)opts.stream;
    const int S = p->degree / 2;
    DenseSystems sys{};
    sys.cshift = opts.shift_c;
    const double ec = std::exp(opts.shift_c);
    for (int s = 0; s < S; ++s) {
        const double tr = -p->lam[4 * s], ti = -p->lam[4 * s + 1];
        const double ar = p->w[4 * s], ai = p->w[4 * s + 1];
        if (complex_a) {
            sys.th_re[2 * s] = tr; sys.th_im[2 * s] = ti; sys.w_re[2 * s] = ec * ar; sys.w_im[2 * s] = ec * ai;
            sys.th_re[2 * s + 1] = tr; sys.th_im[2 * s + 1] = -ti;
            sys.w_re[2 * s + 1] = ec * ar; sys.w_im[2 * s + 1] = -ec * ai;
        } else {
            sys.th_re[s] = tr; sys.th_im[s] = ti; sys.w_re[s] = 2 * ec * ar; sys.w_im[s] = 2 * ec * ai;
        }
    }
    const int nsys = complex_a ? 2 * S : S;
    const int aw = complex_a ? 2 : 1, vw = v_is_complex ? 2 : 1, yw = (complex_a || v_is_complex) ? 2 : 1;

    // buckets, largest first; instances of a bucket in input order
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return bucket_order(n[a]) > bucket_order(n[b]); });
    expm_status worst = EXPM_OK;
    size_t pos = 0;
    while (pos < order.size()) {
        const int nb = bucket_order(n[order[pos]]);
        size_t end = pos;
        int kb = 1;
        while (end < order.size() && bucket_order(n[order[end]]) == nb) kb = std::max(kb, k[order[end++]]);
        // chunk so that the batch fits a launch grid and a workspace of a few GB
        DenseGeom g{};
        g.n = nb;
        g.kc = kb;
        g.npairs = S;
        g.nsys = nsys;
        g.complex_a = complex_a;
        g.mixed = opts.prec != EXPM_FP64;
        g.t = opts.t;
        g.tol = opts.tol;
        g.max_refine = opts.max_refine;
        g.ninst = 1;
        const size_t per_inst = dense_workspace_bytes(g) + sizeof(double) * ((size_t)nb * nb * aw + 2 * (size_t)nb * kb * 2);
        size_t chunk = std::max<size_t>(1, ((size_t)8 << 30) / per_inst);
        chunk = std::min<size_t>(chunk, 65535 / nsys);
        for (size_t c0 = pos; c0 < end; c0 += chunk) {
            const size_t c1 = std::min(end, c0 + chunk);
            g.ninst = (int)(c1 - c0);
            const size_t bytesA = sizeof(double) * (size_t)g.ninst * nb * nb * aw;
            const size_t bytesV = sizeof(double) * (size_t)g.ninst * nb * kb * vw;
            const size_t bytesY = sizeof(double) * (size_t)g.ninst * nb * kb * yw;
            const size_t bytesP = sizeof(InstPtr) * g.ninst;
            const size_t need = dense_workspace_bytes(g);
            expm_status s = plan_reserve(p, &p->work, &p->work_bytes, need);
            if (s != EXPM_OK) return s;
            s = plan_reserve(p, &p->stage, &p->stage_bytes, bytesA + bytesV + bytesY + bytesP + 1024);
            if (s != EXPM_OK) return s;
            unsigned char *sp = (unsigned char *)p->stage;
            double *Apad = (double *)sp;
            double *Vpad = (double *)(sp + bytesA);
            double *Ypad = (double *)(sp + bytesA + bytesV);
            InstPtr *dptr = (InstPtr *)(sp + ((bytesA + bytesV + bytesY + 255) & ~size_t(255)));
            std::vector<InstPtr> hp(g.ninst);
            for (int z = 0; z < g.ninst; ++z) {
                const int i = order[c0 + z];
                hp[z] = InstPtr{(const double *)A[i], (const double *)V[i], (double *)Y[i], n[i], k[i]};
            }
            cudaError_t err = cudaMemcpyAsync(dptr, hp.data(), bytesP, cudaMemcpyHostToDevice, st);
            if (err != cudaSuccess) return cuda_error(err, "apply_batched: pointer upload");
            const unsigned gx = (unsigned)std::min<int64_t>(((int64_t)nb * nb * aw + 255) / 256, 1024);
            gather_pad<<<dim3(gx, 1, g.ninst), 256, 0, st>>>(dptr, nb, kb, aw, vw, Apad, Vpad);
            if ((err = cudaGetLastError()) != cudaSuccess) return cuda_error(err, "apply_batched: gather");
            DenseIO io{};
            io.A = Apad;
            io.lda = nb;
            io.astride = (int64_t)nb * nb;
            io.V = Vpad;
            io.ldv = kb;
            io.vstride = (int64_t)nb * kb;
            io.v_cplx = v_is_complex ? 1 : 0;
            io.Y = Ypad;
            io.ldy = kb;
            io.ystride = (int64_t)nb * kb;
            io.y_real = yw == 1 ? 1 : 0;
            DenseResult res;
            err = dense_run(g, io, sys, p->work, st, p->prof, &res);
            if (err != cudaSuccess) return cuda_error(err, "apply_batched: kernels");
            scatter_unpad<<<dim3((unsigned)std::min<int64_t>(((int64_t)nb * kb * yw + 255) / 256, 1024), 1, g.ninst),
                            256, 0, st>>>(dptr, nb, kb, yw, Ypad);
            if ((err = cudaGetLastError()) != cudaSuccess) return cuda_error(err, "apply_batched: scatter");
            // the pointer table and staging buffers are reused by the next chunk
            if ((err = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_error(err, "apply_batched: sync");
            for (int z = 0; z < g.ninst; ++z) {
                const int i = order[c0 + z];
                expm_status si = EXPM_OK;
                if (res.inst_growth[z] > opts.growth_max) si = EXPM_EGROWTH;
                else if (g.mixed && !(res.inst_resid[z] <= opts.tol)) si = EXPM_ENOCONV;
                if (si != EXPM_OK && worst == EXPM_OK) worst = si;
                if (per_instance)
                    per_instance[i] = expm_info{res.inst_iters[z], res.inst_growth[z], res.inst_resid[z], si};
            }
        }
        pos = end;
    }
    if (worst == EXPM_EGROWTH) return set_error(worst, "apply_batched: LU growth exceeds opts.growth_max");
    if (worst == EXPM_ENOCONV) return set_error(worst, "apply_batched: refinement did not reach opts.tol");
    return EXPM_OK;
}
