// server.cu -- continuous-batching request server for exp(tA)V evaluations.
//
// Requests name a registered operator (a Hermitian tridiagonal T or a dense Hermitian
// A, copied into server-owned device memory at registration) and bring their own
// right-hand sides.  A pool of `max_inflight` worker threads, each with its own CUDA
// stream and scratch, takes requests as soon as they fit the HBM budget: a request
// that arrives while others run is admitted when a worker and enough memory are free,
// and its kernels overlap on the device with the others'.  Factorizations (the
// per-pole block LUs and spikes of the tridiagonal path, the per-pair LUs of the dense
// path) are kept resident in an LRU cache keyed by (operator, plan id, precision, t, c)
// and counted in the budget; a request finding its factor part cached runs only the
// solve part.  The plan id is unique over the process, so a plan destroyed and another
// created at the same address never meets the first one's factors; an entry whose build
// failed or whose tensor-core waits gave up is dropped as soon as no request uses it,
// so the next request for that operator rebuilds it.  Workers are supervised: a worker
// thread found stopped (between requests) is joined and started again by the next
// submit or poll, and the queued requests go on.  A factor part is built once, by the worker that first needs it, on
// its own stream; other workers order their use after it with a CUDA event, without
// blocking the host.  Each request's result depends only on its own inputs -- the
// kernels are deterministic and nothing is reduced across requests -- so it is the
// same alone and in the mix.
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/expm.h"
#include "dense.cuh"
#include "plan.cuh"
#include "tridiag.cuh"

namespace expm {
namespace {

using Clock = std::chrono::steady_clock;

struct Op {
    int kind = 0;
    int64_t n = 0;
    int a_cplx = 0;
    int herm = 0;          // tridiag with complex e: data holds d, |e| and the phases phi
    void *data = nullptr;  // tridiag: d (n) then e (n-1) [then phi (n complex)]; dense: A (n x n, ld n)
    size_t bytes = 0;
};

using FactorKey = std::tuple<uint64_t, uint64_t, int, double, double>;  // op, plan id, prec, t, c

struct FactorEntry {
    void *buf = nullptr;
    size_t bytes = 0;
    int degree = 0;              // the plan degree it was built for (a hit must match it and `bytes`)
    cudaEvent_t done = nullptr;  // recorded after the factor kernels
    bool ready = false;          // kernels enqueued and `done` recorded
    bool failed = false;
    int users = 0;
    uint64_t last_use = 0;
    DenseResult growth;          // dense: growth factors of the factorization
};

struct Request {
    uint64_t ticket = 0;
    uint64_t op = 0;
    Op opv;  // copy of the operator record (the map may change while the request runs)
    expm_plan plan = nullptr;
    const void *V = nullptr;
    void *Y = nullptr;
    int k = 0;
    int v_cplx = 0;
    expm_opts opts{};
    size_t solve_bytes = 0;
    size_t factor_bytes = 0;
    bool done = false;
    expm_status status = EXPM_OK;
    expm_info info{};
    double ts[4] = {0, 0, 0, 0};  // submit, admit, start, done (seconds since creation)
};

struct Worker {
    std::thread th;
    cudaStream_t stream = nullptr;
    void *work = nullptr;
    size_t work_bytes = 0;
    bool alive = false;          // its thread runs worker_loop (server lock)
    bool stop_after = false;     // test hook: leave the loop after the current request
};

}  // namespace
}  // namespace expm

using namespace expm;

struct expm_server_s {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0;
    size_t in_use = 0;  // admitted solve scratch + cached factor parts
    int max_inflight = 1;
    int max_queue = 1 << 16;
    bool fail_next_factor = false;  // test hook: the next factor build reports a failure
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    uint64_t next_ticket = 1, next_op = 1, use_clock = 0;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> requests;
    std::map<uint64_t, Op> ops;
    std::map<FactorKey, FactorEntry> cache;
    std::vector<std::unique_ptr<Worker>> workers;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

TriPoles tri_poles(expm_plan p, double shift_c) {
    TriPoles ps{};
    const double ec = std::exp(shift_c);
    for (int s = 0; s < p->degree / 2; ++s) {
        ps.th_re[s] = -p->lam[4 * s];
        ps.th_im[s] = -p->lam[4 * s + 1];
        ps.w_re[s] = 2.0 * ec * p->w[4 * s];
        ps.w_im[s] = 2.0 * ec * p->w[4 * s + 1];
    }
    return ps;
}

DenseSystems dense_systems(expm_plan p, bool complex_a, double shift_c) {
    DenseSystems sys{};
    sys.cshift = shift_c;
    const double ec = std::exp(shift_c);
    for (int s = 0; s < p->degree / 2; ++s) {
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
    return sys;
}

DenseGeom dense_geom(const Op &op, expm_plan p, const expm_opts &o, int k, int v_cplx) {
    DenseGeom g{};
    g.n = (int)op.n;
    g.ninst = 1;
    g.complex_a = op.a_cplx;
    g.npairs = p->degree / 2;
    g.nsys = op.a_cplx ? p->degree : p->degree / 2;
    g.kc = (!op.a_cplx && v_cplx) ? 2 * k : k;
    g.mixed = o.prec != EXPM_FP64;
    g.t = o.t;
    g.tol = o.tol;
    g.max_refine = o.max_refine;
    return g;
}

DenseIO dense_io(const Op &op, const Request &r) {
    DenseIO io{};
    const bool split_v = !op.a_cplx && r.v_cplx;
    io.A = (const double *)op.data;
    io.lda = op.n;
    io.V = (const double *)r.V;
    io.ldv = split_v ? 2 * (int64_t)r.k : r.k;
    io.v_cplx = (op.a_cplx && r.v_cplx) ? 1 : 0;
    io.Y = (double *)r.Y;
    io.ldy = io.ldv;
    io.y_real = op.a_cplx ? 0 : 1;
    return io;
}

// The test hook of expm_internal_server_fail_next_factor: true once, for the first
// factor build after it was set (the build is then reported as failed).
bool take_fail_hook(expm_server_s *sv) {
    std::lock_guard<std::mutex> lk(sv->mu);
    const bool f = sv->fail_next_factor;
    sv->fail_next_factor = false;
    return f;
}

// Marks a factor part as usable by other workers (its kernels are enqueued and its
// event recorded, or its build failed).
void publish(expm_server_s *sv, FactorEntry &fe, bool failed) {
    std::lock_guard<std::mutex> lk(sv->mu);
    fe.ready = true;
    fe.failed = failed;
    sv->cv.notify_all();
}

// Runs one admitted request on worker w.  Called without the server lock.
void run_request(expm_server_s *sv, Worker &w, Request &r, FactorEntry &fe, bool build) {
    Profiler off;
    const Op &op = r.opv;
    expm_status st = EXPM_OK;
    cudaError_t err = cudaSuccess;
    r.ts[2] = sv->now();
    const bool ff = r.opts.prec != EXPM_FP64;
    // complex Hermitian T: the kernels solve with D^H V (in the worker's scratch past the
    // solve part) for the real symmetric D^H T D, and Y's rows are then multiplied by phi
    const double *Vin = (const double *)r.V;
    const double *phi = op.herm ? (const double *)op.data + 2 * op.n : nullptr;
    auto herm_in = [&](size_t solve_part) {
        double *Vp = (double *)((unsigned char *)w.work + ((solve_part + 255) & ~(size_t)255));
        Vin = Vp;
        return herm_scale(op.n, r.k, phi, (const double *)r.V, r.v_cplx, Vp, 1, sv->sm_count, w.stream);
    };
    if (op.kind == EXPM_OP_TRIDIAG && r.opts.prec == EXPM_MIXED_FP32) {
        // binary32 factors + refinement: the factor part is cached like the others
        const int Rc = op.herm ? 2 * r.k : r.k * (r.v_cplx ? 2 : 1);
        TriGeom g = tri_mixed_geometry(op.n, r.plan->degree / 2, Rc, sv->sm_count);
        g.t = r.opts.t;
        g.cshift = r.opts.shift_c;
        const TriPoles ps = tri_poles(r.plan, r.opts.shift_c);
        const MixOpts mo{r.opts.max_refine, (r.opts.flags & EXPM_FLAG_SKIP_FINAL_RESIDUAL) ? 0 : 1, r.opts.tol};
        const double *d = (const double *)op.data;
        if (build) {
            err = tri_mixed_factor(g, d, d + op.n, ps, fe.buf, w.stream, off);
            if (err == cudaSuccess) err = cudaEventRecord(fe.done, w.stream);
            if (err == cudaSuccess && take_fail_hook(sv)) err = cudaErrorUnknown;
            publish(sv, fe, err != cudaSuccess);
        } else {
            err = fe.failed ? cudaErrorUnknown : cudaStreamWaitEvent(w.stream, fe.done, 0);
        }
        if (err == cudaSuccess && op.herm) err = herm_in(tri_mixed_solve_bytes(g, mo.max_refine));
        if (err == cudaSuccess) err = tri_mixed_solve(g, Vin, (double *)r.Y, ps, fe.buf, w.work, mo, w.stream, off);
        if (err == cudaSuccess && op.herm)
            err = herm_scale(op.n, r.k, phi, (const double *)r.Y, 1, (double *)r.Y, 0, sv->sm_count, w.stream);
        MixResult mr{};
        if (err == cudaSuccess) err = tri_mixed_read_state(g, w.work, mo.max_refine, &mr, w.stream);  // synchronises
        if (err == cudaSuccess) {
            r.info.refine_iters_max = mr.iters;
            r.info.resid_rel_max = mr.resid;
            if (mo.verify && !mr.converged) st = EXPM_ENOCONV;
        }
    } else if (op.kind == EXPM_OP_TRIDIAG) {
        const int Rc = op.herm ? 2 * r.k : r.k * (r.v_cplx ? 2 : 1);
        TriGeom g = tri_geometry(op.n, r.plan->degree / 2, Rc, ff, sv->sm_count);
        g.t = r.opts.t;
        g.cshift = r.opts.shift_c;
        const TriPoles ps = tri_poles(r.plan, r.opts.shift_c);
        const double *d = (const double *)op.data;
        if (build) {
            err = tri_factor(g, ff, d, d + op.n, ps, fe.buf, w.stream, off);
            if (err == cudaSuccess) err = cudaEventRecord(fe.done, w.stream);
            if (err == cudaSuccess && take_fail_hook(sv)) err = cudaErrorUnknown;
            publish(sv, fe, err != cudaSuccess);
        } else {
            err = fe.failed ? cudaErrorUnknown : cudaStreamWaitEvent(w.stream, fe.done, 0);
        }
        if (err == cudaSuccess && op.herm) err = herm_in(tri_solve_bytes(g, ff));
        if (err == cudaSuccess) err = tri_solve(g, ff, Vin, (double *)r.Y, ps, fe.buf, w.work, w.stream, off);
        if (err == cudaSuccess && op.herm)
            err = herm_scale(op.n, r.k, phi, (const double *)r.Y, 1, (double *)r.Y, 0, sv->sm_count, w.stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(w.stream);
    } else {
        const DenseGeom g = dense_geom(op, r.plan, r.opts, r.k, r.v_cplx);
        const DenseSystems sys = dense_systems(r.plan, op.a_cplx, r.opts.shift_c);
        const DenseIO io = dense_io(op, r);
        DenseResult res;
        if (build) {
            err = dense_factor(g, io, sys, fe.buf, w.stream, off);
            if (err == cudaSuccess) err = dense_growth(g, fe.buf, w.stream, &fe.growth);
            if (err == cudaSuccess) err = cudaEventRecord(fe.done, w.stream);
            if (err == cudaSuccess && take_fail_hook(sv)) err = cudaErrorUnknown;
            publish(sv, fe, err != cudaSuccess);
        } else {
            err = fe.failed ? cudaErrorUnknown : cudaStreamWaitEvent(w.stream, fe.done, 0);
        }
        if (err == cudaSuccess) err = dense_solve(g, io, sys, fe.buf, w.work, w.stream, off, &res);
        if (err == cudaSuccess) err = cudaStreamSynchronize(w.stream);
        if (err == cudaSuccess) {
            r.info.refine_iters_max = res.iters;
            r.info.resid_rel_max = res.resid_rel_max;
            r.info.growth_max_seen = fe.growth.growth_max;
            if (fe.growth.tc_timeout || res.tc_timeout) st = EXPM_ETIMEOUT;
            else if (fe.growth.growth_max > r.opts.growth_max) st = EXPM_EGROWTH;
            else if (g.mixed && !(res.resid_rel_max <= r.opts.tol)) st = EXPM_ENOCONV;
        }
    }
    if (err != cudaSuccess) {
        cudaGetLastError();
        st = err == cudaErrorMemoryAllocation ? EXPM_ENOMEM : EXPM_ECUDA;
    }
    r.status = st;
    r.info.status_worst = st;
    r.ts[3] = sv->now();
}

// Frees a cache entry that no request uses (its kernels are finished or never ran).
// Lock held.
void drop_entry(expm_server_s *sv, std::map<FactorKey, FactorEntry>::iterator it) {
    if (it->second.done) {
        cudaEventSynchronize(it->second.done);
        cudaEventDestroy(it->second.done);
    }
    if (it->second.buf) cudaFree(it->second.buf);
    sv->in_use -= it->second.bytes;
    sv->cache.erase(it);
}

// Picks the first queued request that fits; reserves its memory.  Lock held.
Request *admit(expm_server_s *sv, Worker &w, FactorEntry **fe_out, bool *build_out) {
    for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
        Request *r = *it;
        // factor parts differ by precision: binary64; float-float; binary32 (the dense mixed
        // precisions share one binary32 LU; the tridiagonal binary32 factors are their own)
        int fprec = r->opts.prec == EXPM_FP64 ? 0
                    : (r->opv.kind == EXPM_OP_TRIDIAG && r->opts.prec == EXPM_MIXED_FP32) ? 2 : 1;
        // a dense factor part that carries the diagonal-panel inverses of the wide solves
        // (more than 8 columns) is an entry of its own
        if (r->opv.kind != EXPM_OP_TRIDIAG && dense_uses_inv(dense_geom(r->opv, r->plan, r->opts, r->k, r->v_cplx)))
            fprec += 8;
        const FactorKey key{r->op, r->plan->id, fprec, r->opts.t, r->opts.shift_c};
        auto ce = sv->cache.find(key);
        if (ce != sv->cache.end() && ce->second.ready &&
            (ce->second.degree != r->plan->degree || ce->second.bytes != r->factor_bytes)) {
            // not this request's factorization: drop it once unused, build a fresh one
            if (ce->second.users > 0) continue;
            drop_entry(sv, ce);
            ce = sv->cache.end();
        }
        const bool cached = ce != sv->cache.end();
        if (cached && !ce->second.ready) continue;  // its factor is being built: wait for it
        const size_t grow = r->solve_bytes > w.work_bytes ? r->solve_bytes - w.work_bytes : 0;
        size_t need = grow + (cached ? 0 : r->factor_bytes);
        // make room by dropping unused cached factor parts, least recently used first
        while (sv->in_use + need > sv->budget) {
            auto victim = sv->cache.end();
            for (auto c = sv->cache.begin(); c != sv->cache.end(); ++c)
                if (c->second.ready && c->second.users == 0 && c != ce &&
                    (victim == sv->cache.end() || c->second.last_use < victim->second.last_use))
                    victim = c;
            if (victim == sv->cache.end()) break;
            drop_entry(sv, victim);
        }
        if (sv->in_use + need > sv->budget) continue;
        // admitted: grow the worker's scratch, create the cache entry if needed
        if (grow > 0) {
            if (w.work) cudaFree(w.work);
            sv->in_use -= w.work_bytes;
            w.work = nullptr;
            w.work_bytes = 0;
            if (cudaMalloc(&w.work, r->solve_bytes) != cudaSuccess) {
                cudaGetLastError();
                w.work = nullptr;
                continue;
            }
            w.work_bytes = r->solve_bytes;
            sv->in_use += w.work_bytes;
        }
        bool build = false;
        if (!cached) {
            FactorEntry fe;
            fe.bytes = r->factor_bytes;
            fe.degree = r->plan->degree;
            if (cudaMalloc(&fe.buf, fe.bytes) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            cudaEventCreateWithFlags(&fe.done, cudaEventDisableTiming);
            ce = sv->cache.emplace(key, fe).first;
            sv->in_use += fe.bytes;
            build = true;
        }
        ce->second.users += 1;
        ce->second.last_use = ++sv->use_clock;
        sv->queue.erase(it);
        r->ts[1] = sv->now();
        *fe_out = &ce->second;
        *build_out = build;
        return r;
    }
    return nullptr;
}

void worker_loop(expm_server_s *sv, Worker *w) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        FactorEntry *fe = nullptr;
        bool build = false;
        Request *r = nullptr;
        sv->cv.wait(lk, [&] { return sv->stop || w->stop_after || (r = admit(sv, *w, &fe, &build)) != nullptr; });
        if (!r) break;  // stop requested (server shutdown, or the test hook)
        lk.unlock();
        run_request(sv, *w, *r, *fe, build);
        lk.lock();
        fe->users -= 1;
        if (fe->users == 0 && (fe->failed || fe->growth.tc_timeout)) {
            // a failed build (or a tensor-core wait that gave up) must not serve later
            // requests: drop it so that the next one rebuilds
            for (auto it = sv->cache.begin(); it != sv->cache.end(); ++it)
                if (&it->second == fe) {
                    drop_entry(sv, it);
                    break;
                }
        }
        r->done = true;
        sv->cv.notify_all();
        if (w->stop_after) break;
    }
    w->alive = false;
}

// Starts the thread of every worker found stopped (server lock held).  A worker stops
// only between requests, so nothing it had admitted is lost; the queued requests wait
// for the restarted (or any other) worker.
void respawn_workers(expm_server_s *sv) {
    if (sv->stop) return;
    for (auto &w : sv->workers) {
        if (w->alive) continue;
        if (w->th.joinable()) w->th.join();  // it has left worker_loop: returns at once
        w->stop_after = false;
        w->alive = true;
        w->th = std::thread(worker_loop, sv, w.get());
    }
}

}  // namespace

extern "C" {

expm_status expm_server_create(size_t hbm_budget_bytes, int max_inflight, expm_server *out) {
    if (!out) return set_error(EXPM_EINVAL, "server_create: out is NULL");
    *out = nullptr;
    if (hbm_budget_bytes == 0 || max_inflight < 1 || max_inflight > 64)
        return set_error(EXPM_EINVAL, "server_create: need a budget > 0 and 1 <= max_inflight <= 64");
    auto sv = new (std::nothrow) expm_server_s();
    if (!sv) return set_error(EXPM_ENOMEM, "server_create: host allocation");
    sv->budget = hbm_budget_bytes;
    sv->max_inflight = max_inflight;
    sv->t0 = Clock::now();
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sv->sm_count, cudaDevAttrMultiProcessorCount, sv->device);
    for (int i = 0; i < max_inflight && e == cudaSuccess; ++i) {
        auto w = std::make_unique<Worker>();
        e = cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking);
        sv->workers.push_back(std::move(w));
    }
    if (e != cudaSuccess) {
        for (auto &w : sv->workers)
            if (w->stream) cudaStreamDestroy(w->stream);
        delete sv;
        return cuda_error(e, "server_create");
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (auto &w : sv->workers) {
            w->alive = true;
            w->th = std::thread(worker_loop, sv, w.get());
        }
    }
    *out = sv;
    return EXPM_OK;
}

expm_status expm_server_register_op(expm_server sv, const expm_op_desc *desc, uint64_t *op_id) {
    if (!sv || !desc || !op_id) return set_error(EXPM_EINVAL, "server_register_op: NULL argument");
    if (desc->n < 1) return set_error(EXPM_EINVAL, "server_register_op: n must be >= 1");
    Op op;
    op.kind = desc->kind;
    op.n = desc->n;
    DeviceGuard guard(sv->device);
    cudaError_t e = cudaSuccess;
    if (desc->kind == EXPM_OP_TRIDIAG) {
        if (!desc->d || (desc->n > 1 && !desc->e)) return set_error(EXPM_EINVAL, "server_register_op: NULL d or e");
        op.herm = desc->e_is_complex ? 1 : 0;
        op.bytes = sizeof(double) * ((op.herm ? 4 : 2) * (size_t)desc->n);
        e = cudaMalloc(&op.data, op.bytes);
        if (e == cudaSuccess) e = cudaMemcpy(op.data, desc->d, sizeof(double) * desc->n, cudaMemcpyDefault);
        if (e == cudaSuccess && desc->n > 1 && !op.herm)
            e = cudaMemcpy((double *)op.data + desc->n, desc->e, sizeof(double) * (desc->n - 1), cudaMemcpyDefault);
        if (e == cudaSuccess && op.herm) {  // |e| and phi once per operator (D^H T D real symmetric)
            void *tmp = nullptr;
            const size_t eb = 2 * sizeof(double) * (size_t)std::max<int64_t>(desc->n - 1, 1);
            e = cudaMalloc(&tmp, eb + herm_part_bytes(desc->n));
            if (e == cudaSuccess && desc->n > 1) e = cudaMemcpy(tmp, desc->e, eb, cudaMemcpyDefault);
            double *dd = (double *)op.data;
            if (e == cudaSuccess)
                e = herm_phases(desc->n, (const double *)tmp, dd + desc->n, dd + 2 * desc->n,
                                (double *)((unsigned char *)tmp + eb), nullptr);
            if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
            if (tmp) cudaFree(tmp);
        }
    } else if (desc->kind == EXPM_OP_DENSE) {
        if (!desc->A || desc->lda < desc->n) return set_error(EXPM_EINVAL, "server_register_op: bad A or lda");
        op.a_cplx = desc->a_is_complex ? 1 : 0;
        const size_t ew = op.a_cplx ? 2 : 1;
        op.bytes = sizeof(double) * ew * (size_t)desc->n * desc->n;
        e = cudaMalloc(&op.data, op.bytes);
        if (e == cudaSuccess)
            e = cudaMemcpy2D(op.data, sizeof(double) * ew * desc->n, desc->A, sizeof(double) * ew * desc->lda,
                             sizeof(double) * ew * desc->n, desc->n, cudaMemcpyDefault);
    } else {
        return set_error(EXPM_EINVAL, "server_register_op: unknown kind");
    }
    if (e != cudaSuccess) {
        if (op.data) cudaFree(op.data);
        cudaGetLastError();
        return cuda_error(e, "server_register_op");
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    *op_id = sv->next_op++;
    sv->ops[*op_id] = op;
    return EXPM_OK;
}

expm_status expm_server_submit(expm_server sv, uint64_t op_id, const expm_plan plan, const void *V, int k,
                               int v_is_complex, void *Y, const expm_opts *opts_in, uint64_t *ticket) {
    if (!sv || !plan || !V || !Y || !ticket) return set_error(EXPM_EINVAL, "server_submit: NULL argument");
    if (k < 1 || k > 64) return set_error(EXPM_EINVAL, "server_submit: k must be in 1..64");
    expm_opts opts;
    if (opts_in) opts = *opts_in; else expm_opts_default(&opts);
    const bool tri_mixed = opts.prec == EXPM_MIXED_FP32;  // meaningful for tridiagonal operators
    if ((opts.flags != 0 && opts.flags != EXPM_FLAG_SKIP_FINAL_RESIDUAL) || !std::isfinite(opts.t) ||
        !std::isfinite(opts.shift_c))
        return set_error(EXPM_EINVAL, "server_submit: bad options");
    {
        DeviceGuard guard(sv->device);
        if (!is_device_ptr(V) || !is_device_ptr(Y))
            return set_error(EXPM_EINVAL, "server_submit: V and Y must be device memory");
    }
    auto r = std::make_unique<Request>();
    r->op = op_id;
    r->plan = plan;
    r->V = V;
    r->Y = Y;
    r->k = k;
    r->v_cplx = v_is_complex ? 1 : 0;
    r->opts = opts;
    std::lock_guard<std::mutex> lk(sv->mu);
    respawn_workers(sv);
    auto oi = sv->ops.find(op_id);
    if (oi == sv->ops.end()) return set_error(EXPM_ENOTFOUND, "server_submit: unknown operator id");
    const Op &op = oi->second;
    r->opv = op;
    const bool ff = opts.prec != EXPM_FP64;
    if (op.kind == EXPM_OP_TRIDIAG) {
        if (opts.prec != EXPM_FP64 && opts.prec != EXPM_MIXED_F32X2 && opts.prec != EXPM_MIXED_FP32)
            return set_error(EXPM_EINVAL, "server_submit: tridiagonal precision must be FP64, MIXED_F32X2 or MIXED_FP32");
        if (tri_mixed && (opts.max_refine < 0 || opts.max_refine > 64 || !(opts.tol >= 0.0)))
            return set_error(EXPM_EINVAL, "server_submit: need 0 <= max_refine <= 64 and tol >= 0");
        const int Rc = op.herm ? 2 * k : k * (v_is_complex ? 2 : 1);
        if (tri_mixed) {
            const TriGeom g = tri_mixed_geometry(op.n, plan->degree / 2, Rc, sv->sm_count);
            r->solve_bytes = tri_mixed_solve_bytes(g, opts.max_refine);
            r->factor_bytes = tri_mixed_factor_bytes(g);
        } else {
            const TriGeom g = tri_geometry(op.n, plan->degree / 2, Rc, ff, sv->sm_count);
            r->solve_bytes = tri_solve_bytes(g, ff);
            r->factor_bytes = tri_factor_bytes(g, ff);
        }
        if (op.herm)  // D^H V past the solve part
            r->solve_bytes = ((r->solve_bytes + 255) & ~(size_t)255) + 2 * sizeof(double) * (size_t)op.n * k;
    } else {
        if (opts.prec != EXPM_FP64 && opts.prec != EXPM_MIXED_FP32 && opts.prec != EXPM_MIXED_F32X2)
            return set_error(EXPM_EINVAL, "server_submit: dense precision must be FP64 or mixed");
        if (opts.flags != 0) return set_error(EXPM_EINVAL, "server_submit: flags apply to tridiagonal operators only");
        const DenseGeom g = dense_geom(op, plan, opts, k, v_is_complex);
        r->solve_bytes = dense_solve_bytes(g);
        r->factor_bytes = dense_factor_bytes(g);
    }
    if (r->solve_bytes + r->factor_bytes > sv->budget)
        return set_error(EXPM_ENOMEM, "server_submit: request larger than the whole HBM budget");
    if ((int)sv->queue.size() >= sv->max_queue) return EXPM_EAGAIN;
    r->ticket = sv->next_ticket++;
    r->ts[0] = sv->now();
    *ticket = r->ticket;
    sv->queue.push_back(r.get());
    sv->requests[r->ticket] = std::move(r);
    sv->cv.notify_all();
    return EXPM_OK;
}

expm_status expm_server_poll(expm_server sv, uint64_t ticket, expm_info *info, double ts[4]) {
    if (!sv) return set_error(EXPM_EINVAL, "server_poll: NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    respawn_workers(sv);
    auto it = sv->requests.find(ticket);
    if (it == sv->requests.end()) return EXPM_ENOTFOUND;
    Request &r = *it->second;
    if (!r.done) return EXPM_EAGAIN;
    if (info) *info = r.info;
    if (ts) std::memcpy(ts, r.ts, sizeof(r.ts));
    const expm_status s = r.status;
    sv->requests.erase(it);
    return s;
}

expm_status expm_server_set_queue_limit(expm_server sv, int max_queue) {
    if (!sv) return set_error(EXPM_EINVAL, "server_set_queue_limit: NULL server");
    if (max_queue < 1 || max_queue > (1 << 20))
        return set_error(EXPM_EINVAL, "server_set_queue_limit: need 1 <= max_queue <= 2^20");
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->max_queue = max_queue;
    return EXPM_OK;
}

// Test hooks (not declared in include/expm.h): make the next factor build report a
// failure; make worker `idx` leave its loop after its current request.
int expm_internal_server_fail_next_factor(expm_server sv) {
    if (!sv) return 1;
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->fail_next_factor = true;
    return 0;
}
int expm_internal_server_stop_worker(expm_server sv, int idx) {
    if (!sv || idx < 0 || idx >= (int)sv->workers.size()) return 1;
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->workers[idx]->stop_after = true;
    sv->cv.notify_all();
    return 0;
}
int expm_internal_server_workers_alive(expm_server sv) {
    if (!sv) return -1;
    std::lock_guard<std::mutex> lk(sv->mu);
    int n = 0;
    for (auto &w : sv->workers) n += w->alive ? 1 : 0;
    return n;
}

expm_status expm_server_destroy(expm_server sv) {
    if (!sv) return EXPM_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->queue.clear();
    }
    sv->cv.notify_all();
    for (auto &w : sv->workers)
        if (w->th.joinable()) w->th.join();
    DeviceGuard guard(sv->device);
    for (auto &w : sv->workers) {
        cudaStreamSynchronize(w->stream);
        if (w->work) cudaFree(w->work);
        cudaStreamDestroy(w->stream);
    }
    for (auto &c : sv->cache) {
        if (c.second.done) cudaEventDestroy(c.second.done);
        if (c.second.buf) cudaFree(c.second.buf);
    }
    for (auto &o : sv->ops)
        if (o.second.data) cudaFree(o.second.data);
    delete sv;
    return EXPM_OK;
}

}  // extern "C"
