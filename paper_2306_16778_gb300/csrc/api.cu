// api.cu -- the C interface declared in include/expm.h: plans, validation,
// host/device staging and dispatch to the kernels.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/expm.h"
#include "plan.cuh"
#include "tridiag.cuh"
#include "dense.cuh"

using namespace expm;

namespace {
thread_local std::string g_last_error;
}

namespace expm {

expm_status set_error(expm_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

expm_status cuda_error(cudaError_t e, const char *where) {
    if (e == cudaSuccess) return EXPM_OK;
    return set_error(e == cudaErrorMemoryAllocation ? EXPM_ENOMEM : EXPM_ECUDA,
                     std::string(where) + ": " + cudaGetErrorString(e));
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

expm_status plan_reserve(expm_plan p, void **buf, size_t *have, size_t need) {
    if (need <= *have) return EXPM_OK;
    if (*buf) {
        cudaError_t e = cudaFree(*buf);
        *buf = nullptr;
        *have = 0;
        if (e != cudaSuccess) return cuda_error(e, "cudaFree");
    }
    cudaError_t e = cudaMalloc(buf, need);
    if (e != cudaSuccess) {
        *buf = nullptr;
        cudaGetLastError();
        return cuda_error(e, "cudaMalloc(workspace)");
    }
    *have = need;
    (void)p;
    return EXPM_OK;
}

// the plan's second stream and its two events, created on first use (false if unavailable)
bool plan_copy_stream(expm_plan p) {
    if (p->copy && p->ev_fork && p->ev_copied) return true;
    if (!p->copy && cudaStreamCreateWithFlags(&p->copy, cudaStreamNonBlocking) != cudaSuccess) p->copy = nullptr;
    if (!p->ev_fork && cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess) p->ev_fork = nullptr;
    if (!p->ev_copied && cudaEventCreateWithFlags(&p->ev_copied, cudaEventDisableTiming) != cudaSuccess)
        p->ev_copied = nullptr;
    return p->copy && p->ev_fork && p->ev_copied;
}

int Profiler::kernel_index(const char *name) {
    for (size_t i = 0; i < names.size(); ++i)
        if (names[i] == name || std::strcmp(names[i], name) == 0) return (int)i;
    names.push_back(name);
    launches.push_back(0);
    total_ms.push_back(0.0);
    return (int)names.size() - 1;
}

cudaEvent_t Profiler::take() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void Profiler::flush() {
    for (auto &p : pending) {
        cudaEventSynchronize(p.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            total_ms[p.kernel] += ms;
            launches[p.kernel] += 1;
        }
        pool.push_back(p.a);
        pool.push_back(p.b);
    }
    pending.clear();
}

void Profiler::reset() {
    flush();
    names.clear();
    launches.clear();
    total_ms.clear();
}

void Profiler::release() {
    flush();
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
}

DeviceGuard::DeviceGuard(int dev) {
    cudaGetDevice(&prev_);
    if (prev_ != dev) cudaSetDevice(dev);
}
DeviceGuard::~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != prev_) cudaSetDevice(prev_);
}

}  // namespace expm

extern "C" {

void expm_opts_default(expm_opts *o) {
    if (!o) return;
    o->prec = EXPM_FP64;
    o->tol = 1e-14;
    o->max_refine = 6;
    o->t = 1.0;
    o->shift_c = 0.0;
    o->growth_max = 1e6;
    o->stream = nullptr;
    o->flags = 0;
}

const char *expm_status_string(expm_status s) {
    switch (s) {
        case EXPM_OK: return "EXPM_OK";
        case EXPM_EINVAL: return "EXPM_EINVAL";
        case EXPM_ENOMEM: return "EXPM_ENOMEM";
        case EXPM_EGROWTH: return "EXPM_EGROWTH";
        case EXPM_ENOCONV: return "EXPM_ENOCONV";
        case EXPM_ETIMEOUT: return "EXPM_ETIMEOUT";
        case EXPM_EAGAIN: return "EXPM_EAGAIN";
        case EXPM_ECUDA: return "EXPM_ECUDA";
        case EXPM_ENOTFOUND: return "EXPM_ENOTFOUND";
        case EXPM_ENOTSUP: return "EXPM_ENOTSUP";
    }
    return "EXPM_UNKNOWN";
}

const char *expm_last_error(void) { return g_last_error.c_str(); }

expm_status expm_plan_create(const double *poles_ri, const double *residues_ri, int degree, expm_plan *out) {
    if (!out) return set_error(EXPM_EINVAL, "plan_create: out is NULL");
    *out = nullptr;
    if (!poles_ri || !residues_ri) return set_error(EXPM_EINVAL, "plan_create: NULL pole data");
    if (degree < 2 || degree > 64 || (degree & 1))
        return set_error(EXPM_EINVAL, "plan_create: degree must be even, 2..64");
    for (int k = 0; k < 2 * degree; ++k)
        if (!std::isfinite(poles_ri[k]) || !std::isfinite(residues_ri[k]))
            return set_error(EXPM_EINVAL, "plan_create: non-finite pole data");
    double r0_re = 0.0, r0_im = 0.0;
    for (int k = 0; k < degree; ++k) {
        const double lr = poles_ri[2 * k], li = poles_ri[2 * k + 1];
        const double wr = residues_ri[2 * k], wi = residues_ri[2 * k + 1];
        const double den = lr * lr + li * li;
        if (!(den > 0)) return set_error(EXPM_EINVAL, "plan_create: zero pole");
        // -w/lambda
        r0_re += -(wr * lr + wi * li) / den;
        r0_im += -(wi * lr - wr * li) / den;
        if (k & 1) {
            const double pr = poles_ri[2 * k - 2], pi = poles_ri[2 * k - 1];
            const double qr = residues_ri[2 * k - 2], qi = residues_ri[2 * k - 1];
            const double sc = std::sqrt(pr * pr + pi * pi), sw = std::sqrt(qr * qr + qi * qi);
            if (std::fabs(lr - pr) > 1e-12 * sc || std::fabs(li + pi) > 1e-12 * sc ||
                std::fabs(wr - qr) > 1e-12 * sw || std::fabs(wi + qi) > 1e-12 * sw)
                return set_error(EXPM_EINVAL, "plan_create: poles/weights not in adjacent conjugate pairs");
            if (pi == 0.0) return set_error(EXPM_EINVAL, "plan_create: real pole");
        }
    }
    if (std::fabs(r0_re - 1.0) > 1e-8 || std::fabs(r0_im) > 1e-8)
        return set_error(EXPM_EINVAL, "plan_create: pole data does not satisfy R_n(0) = 1");
    expm_plan p = new (std::nothrow) expm_plan_s();
    if (!p) return set_error(EXPM_ENOMEM, "plan_create: host allocation");
    static std::atomic<uint64_t> next_id{1};
    p->id = next_id.fetch_add(1);
    p->degree = degree;
    p->lam.assign(poles_ri, poles_ri + 2 * degree);
    p->w.assign(residues_ri, residues_ri + 2 * degree);
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        delete p;
        cudaGetLastError();
        return cuda_error(e, "plan_create");
    }
    *out = p;
    return EXPM_OK;
}

expm_status expm_plan_destroy(expm_plan p) {
    if (!p) return EXPM_OK;
    DeviceGuard guard(p->device);
    cudaDeviceSynchronize();
    p->prof.release();
    if (p->work) cudaFree(p->work);
    if (p->stage) cudaFree(p->stage);
    if (p->copy) cudaStreamDestroy(p->copy);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_copied) cudaEventDestroy(p->ev_copied);
    delete p;
    return EXPM_OK;
}

expm_status expm_apply_tridiag(expm_plan p, int64_t N, const double *d, const void *e, int e_is_complex,
                               const void *V, int r, int v_is_complex, void *Y, const expm_opts *opts_in,
                               expm_info *info) {
    if (!p) return set_error(EXPM_EINVAL, "apply_tridiag: NULL plan");
    expm_opts opts;
    if (opts_in) opts = *opts_in; else expm_opts_default(&opts);
    if (N < 1) return set_error(EXPM_EINVAL, "apply_tridiag: N must be >= 1");
    if (r < 1 || r > 1024) return set_error(EXPM_EINVAL, "apply_tridiag: r must be in 1..1024");
    if (!d || !V || !Y || (N > 1 && !e)) return set_error(EXPM_EINVAL, "apply_tridiag: NULL data pointer");
    if (opts.prec != EXPM_FP64 && opts.prec != EXPM_MIXED_F32X2 && opts.prec != EXPM_MIXED_FP32)
        return set_error(EXPM_EINVAL, "apply_tridiag: precision must be EXPM_FP64, EXPM_MIXED_F32X2 or EXPM_MIXED_FP32");
    const bool mixed = opts.prec == EXPM_MIXED_FP32;
    if (opts.flags != 0 && !(mixed && opts.flags == EXPM_FLAG_SKIP_FINAL_RESIDUAL))
        return set_error(EXPM_EINVAL, "apply_tridiag: opts.flags must be 0 (or EXPM_FLAG_SKIP_FINAL_RESIDUAL with EXPM_MIXED_FP32)");
    if (mixed && (opts.max_refine < 0 || opts.max_refine > 64 || !(opts.tol >= 0.0)))
        return set_error(EXPM_EINVAL, "apply_tridiag: need 0 <= max_refine <= 64 and tol >= 0");
    if (!std::isfinite(opts.t) || !std::isfinite(opts.shift_c))
        return set_error(EXPM_EINVAL, "apply_tridiag: t and shift_c must be finite");
    if (info) *info = expm_info{0, 0.0, 0.0, EXPM_OK};

    DeviceGuard guard(p->device);
    const bool ff = opts.prec == EXPM_MIXED_F32X2;
    const bool herm = e_is_complex != 0;  // complex T: solved as D^H T D (real) on D^H V
    const int Rin = r * (v_is_complex ? 2 : 1);  // real doubles per row of V
    // the kernels' real columns: complex V with real T has its real and imaginary parts as
    // columns; complex T always gives a complex V' = D^H V and a complex Y
    const int Rc = herm ? 2 * r : Rin;
    const int S = p->degree / 2;
    TriPoles ps{};
    const double ec = std::exp(opts.shift_c);
    for (int s = 0; s < S; ++s) {  // one member of each conjugate pair: theta = -lambda, W = 2 e^c a
        ps.th_re[s] = -p->lam[4 * s];
        ps.th_im[s] = -p->lam[4 * s + 1];
        ps.w_re[s] = 2.0 * ec * p->w[4 * s];
        ps.w_im[s] = 2.0 * ec * p->w[4 * s + 1];
    }
    TriGeom g = mixed ? tri_mixed_geometry(N, S, Rc, p->sm_count) : tri_geometry(N, S, Rc, ff, p->sm_count);
    g.t = opts.t;
    g.cshift = opts.shift_c;
    cudaStream_t st = (cudaStream_t)opts.stream;
    const MixOpts mo{opts.max_refine, (opts.flags & EXPM_FLAG_SKIP_FINAL_RESIDUAL) ? 0 : 1, opts.tol};
    const size_t mix_factor = mixed ? tri_mixed_factor_bytes(g) : 0;

    const size_t base_need =
        mixed ? mix_factor + tri_mixed_solve_bytes(g, mo.max_refine) : tri_workspace_bytes(g, ff);
    const size_t herm_off = (base_need + 255) & ~(size_t)255;
    const size_t need = herm ? herm_off + herm_scratch_bytes(N, r) : base_need;
    expm_status s = plan_reserve(p, &p->work, &p->work_bytes, need);
    if (s != EXPM_OK) return s;

    const bool dd = is_device_ptr(d), de = (N == 1) || is_device_ptr(e), dv = is_device_ptr(V),
               dy = is_device_ptr(Y);
    const double *dD = d, *dE = (const double *)e, *dV = (const double *)V;
    double *dY = (double *)Y;
    const size_t nV = (size_t)N * Rin, nY = (size_t)N * Rc;
    const size_t ew = e_is_complex ? 2 : 1;  // doubles per off-diagonal entry
    const bool staged = !(dd && de && dv && dy);
    cudaEvent_t v_ready = nullptr;  // set when V is copied on the second stream
    if (staged) {
        const size_t bytes = sizeof(double) * ((size_t)N + ew * (size_t)N + nV + nY) + 1024;
        s = plan_reserve(p, &p->stage, &p->stage_bytes, bytes);
        if (s != EXPM_OK) return s;
        double *base = (double *)p->stage;
        double *sD = base, *sE = base + N, *sV = sE + ew * N, *sY = sV + nV;
        cudaError_t err = cudaSuccess;
        if (!dd) { err = cudaMemcpyAsync(sD, d, sizeof(double) * N, cudaMemcpyHostToDevice, st); dD = sD; }
        if (err == cudaSuccess && !de && N > 1) {
            err = cudaMemcpyAsync(sE, e, sizeof(double) * ew * (N - 1), cudaMemcpyHostToDevice, st);
            dE = sE;
        }
        if (err == cudaSuccess && !dv) {
            // V is first read after the factorization (which needs d and e only): its copy
            // runs on the plan's second stream, overlapping the factor kernels, and st
            // waits for it just before the solve
            if (plan_copy_stream(p)) {
                err = cudaEventRecord(p->ev_fork, st);
                if (err == cudaSuccess) err = cudaStreamWaitEvent(p->copy, p->ev_fork, 0);
                if (err == cudaSuccess) err = cudaMemcpyAsync(sV, V, sizeof(double) * nV, cudaMemcpyHostToDevice, p->copy);
                if (err == cudaSuccess) err = cudaEventRecord(p->ev_copied, p->copy);
                v_ready = p->ev_copied;
            } else {
                err = cudaMemcpyAsync(sV, V, sizeof(double) * nV, cudaMemcpyHostToDevice, st);
            }
            dV = sV;
        }
        if (!dy) dY = sY;
        if (err != cudaSuccess) return cuda_error(err, "apply_tridiag: staging copy");
    }
    cudaError_t err;
    HermWork hw{};
    if (herm) {  // |e|, phi and D^H V; the kernels below then see a real symmetric T
        hw = herm_carve((unsigned char *)p->work + herm_off, N, r);
        if (v_ready) err = cudaStreamWaitEvent(st, v_ready, 0);
        else err = cudaSuccess;
        v_ready = nullptr;
        if (err == cudaSuccess) err = herm_prepare(N, dE, dV, r, v_is_complex, hw, p->sm_count, st);
        if (err != cudaSuccess) return cuda_error(err, "apply_tridiag: Hermitian phases");
        dE = hw.eabs;
        dV = hw.Vp;
    }
    if (mixed) {
        void *swork = (unsigned char *)p->work + mix_factor;
        err = tri_mixed_factor(g, dD, dE, ps, p->work, st, p->prof);
        if (err == cudaSuccess && v_ready) err = cudaStreamWaitEvent(st, v_ready, 0);
        if (err == cudaSuccess) err = tri_mixed_solve(g, dV, dY, ps, p->work, swork, mo, st, p->prof);
        if (err != cudaSuccess) return cuda_error(err, "apply_tridiag: kernel launch");
        if (info) {
            MixResult mr{};
            err = tri_mixed_read_state(g, swork, mo.max_refine, &mr, st);
            if (err != cudaSuccess) return cuda_error(err, "apply_tridiag: refinement state");
            info->refine_iters_max = mr.iters;
            info->resid_rel_max = mr.resid;
            if (mo.verify && !mr.converged) info->status_worst = EXPM_ENOCONV;
        }
    } else {
        err = tri_run(g, ff, dD, dE, dV, dY, ps, p->work, st, p->prof, v_ready);
        if (err != cudaSuccess) return cuda_error(err, "apply_tridiag: kernel launch");
    }
    if (herm) {  // Y = D Y'
        err = herm_finish(N, r, hw, dY, p->sm_count, st);
        if (err != cudaSuccess) return cuda_error(err, "apply_tridiag: Hermitian phases");
    }
    if (staged) {
        if (!dy) err = cudaMemcpyAsync(Y, dY, sizeof(double) * nY, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        if (err != cudaSuccess) return cuda_error(err, "apply_tridiag: result copy");
    }
    if (info && info->status_worst == EXPM_ENOCONV)
        return set_error(EXPM_ENOCONV, "apply_tridiag: refinement did not reach tol");
    return EXPM_OK;
}

expm_status expm_apply_dense(expm_plan p, int n, const void *A, int lda, int a_is_complex, const void *V, int ldv,
                             int k, int v_is_complex, void *Y, int ldy, const expm_opts *opts_in, expm_info *info) {
    if (!p) return set_error(EXPM_EINVAL, "apply_dense: NULL plan");
    expm_opts opts;
    if (opts_in) opts = *opts_in; else expm_opts_default(&opts);
    if (n < 1 || k < 1 || k > 4096) return set_error(EXPM_EINVAL, "apply_dense: need n >= 1 and 1 <= k <= 4096");
    if (lda < n || ldv < k || ldy < k) return set_error(EXPM_EINVAL, "apply_dense: leading dimension too small");
    if (!A || !V || !Y) return set_error(EXPM_EINVAL, "apply_dense: NULL data pointer");
    if (opts.prec < EXPM_FP64 || opts.prec > EXPM_MIXED_BF16X3)
        return set_error(EXPM_EINVAL, "apply_dense: unknown precision");
    if (opts.flags != 0) return set_error(EXPM_EINVAL, "apply_dense: opts.flags must be 0");
    if (!std::isfinite(opts.t) || !std::isfinite(opts.shift_c) || !(opts.tol > 0) || opts.max_refine < 0)
        return set_error(EXPM_EINVAL, "apply_dense: bad t, shift_c, tol or max_refine");
    if (info) *info = expm_info{0, 0.0, 0.0, EXPM_OK};
    DeviceGuard guard(p->device);
    cudaStream_t st = (cudaStream_t)opts.stream;
    const int S = p->degree / 2;
    const bool complex_a = a_is_complex != 0;
    DenseGeom g{};
    g.n = n;
    g.ninst = 1;
    g.complex_a = complex_a;
    g.npairs = S;
    g.nsys = complex_a ? 2 * S : S;
    // real A with complex V: real and imaginary parts are separate real columns
    const bool split_v = !complex_a && v_is_complex;
    g.kc = split_v ? 2 * k : k;
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
    const bool da = is_device_ptr(A), dv = is_device_ptr(V), dy = is_device_ptr(Y);
    const size_t ea = complex_a ? 2 : 1, ev = v_is_complex ? 2 : 1, ey = (complex_a || v_is_complex) ? 2 : 1;
    const size_t nA = (size_t)n * lda * ea, nV = (size_t)n * ldv * ev, nY = (size_t)n * ldy * ey;
    const double *dA = (const double *)A, *dV = (const double *)V;
    double *dY = (double *)Y;
    const bool staged = !(da && dv && dy);
    if (staged) {
        expm_status s = plan_reserve(p, &p->stage, &p->stage_bytes, sizeof(double) * (nA + nV + nY) + 1024);
        if (s != EXPM_OK) return s;
        double *base = (double *)p->stage;
        cudaError_t err = cudaSuccess;
        if (!da) { err = cudaMemcpyAsync(base, A, sizeof(double) * nA, cudaMemcpyHostToDevice, st); dA = base; }
        if (err == cudaSuccess && !dv) {
            err = cudaMemcpyAsync(base + nA, V, sizeof(double) * nV, cudaMemcpyHostToDevice, st);
            dV = base + nA;
        }
        if (!dy) dY = base + nA + nV;
        if (err != cudaSuccess) return cuda_error(err, "apply_dense: staging copy");
    }
    const bool small = dense_small_fits(g);  // one cluster launch (dense_small.cu)
    expm_status s = plan_reserve(p, &p->work, &p->work_bytes,
                                 small ? dense_small_workspace_bytes() : dense_workspace_bytes(g));
    if (s != EXPM_OK) return s;
    DenseResult res{};
    DenseIO io{};
    io.A = dA;
    io.lda = lda;
    io.astride = 0;
    io.V = dV;
    io.ldv = split_v ? 2 * (int64_t)ldv : ldv;  // in units of the loaded element
    io.vstride = 0;
    io.v_cplx = (complex_a && v_is_complex) ? 1 : 0;
    io.Y = dY;
    io.ldy = split_v ? 2 * (int64_t)ldy : ldy;
    io.ystride = 0;
    io.y_real = complex_a ? 0 : 1;
    cudaError_t err = small ? dense_small_run(g, io, sys, p->work, st, p->prof, &res)
                            : dense_run(g, io, sys, p->work, st, p->prof, &res);
    if (err != cudaSuccess) return cuda_error(err, "apply_dense: kernels");
    if (staged && !dy) {
        err = cudaMemcpyAsync(Y, dY, sizeof(double) * nY, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        if (err != cudaSuccess) return cuda_error(err, "apply_dense: result copy");
    }
    expm_status out = EXPM_OK;
    if (res.tc_timeout) return set_error(EXPM_ETIMEOUT, "apply_dense: a bounded wait in the tensor-core kernel gave up");
    if (res.growth_max > opts.growth_max) out = EXPM_EGROWTH;
    else if (g.mixed && !(res.resid_rel_max <= opts.tol)) out = EXPM_ENOCONV;
    if (info) {
        info->refine_iters_max = res.iters;
        info->growth_max_seen = res.growth_max;
        info->resid_rel_max = res.resid_rel_max;
        info->status_worst = out;
    }
    if (out == EXPM_EGROWTH) return set_error(out, "apply_dense: LU growth exceeds opts.growth_max");
    if (out == EXPM_ENOCONV) return set_error(out, "apply_dense: refinement did not reach opts.tol");
    return EXPM_OK;
}

expm_status expm_profile_enable(expm_plan p, int on) {
    if (!p) return set_error(EXPM_EINVAL, "profile_enable: NULL plan");
    DeviceGuard guard(p->device);
    p->prof.reset();
    p->prof.on = on != 0;
    return EXPM_OK;
}

expm_status expm_profile_read(expm_plan p, int idx, const char **name, int64_t *launches, double *total_ms) {
    if (!p || !name || !launches || !total_ms) return set_error(EXPM_EINVAL, "profile_read: NULL argument");
    DeviceGuard guard(p->device);
    p->prof.flush();
    if (idx < 0 || idx >= (int)p->prof.names.size()) return EXPM_ENOTFOUND;
    *name = p->prof.names[idx];
    *launches = p->prof.launches[idx];
    *total_ms = p->prof.total_ms[idx];
    return EXPM_OK;
}

}  // extern "C"
