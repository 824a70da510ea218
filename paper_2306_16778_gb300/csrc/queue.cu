// queue.cu -- device-fed work queue of small dense evaluations (expm_queue_*).
//
// Each request is one small instance of eq. expAx (n <= 64, at most 4 right-hand sides):
// Y = e^c R_n(tA - cI) V.  Instead of one kernel launch per request, a persistent kernel
// of thread-block clusters (dense_small.cu: one cluster per request in flight, one CTA per
// solved system, the same evaluation as the one-launch path) consumes requests that the
// host publishes in a ring of slots in mapped (pinned, device-visible) host memory:
//   submit  writes the slot (geometry, pointers, poles and weights with e^c folded in, as
//           expm_apply_dense forms them) and then the slot's sequence word, ticket + 1,
//           with a release store;
//   kernel  a cluster claims ticket t (atomic counter), waits until seq[t % cap] = t + 1,
//           evaluates, and stores done[t % cap] = t + 1 after a system-scope fence;
//   poll    reads done with an acquire load; the statistics (growth, residual, sweeps)
//           are in the slot's stat entry; the ticket is then released.
// Waits are bounded: a cluster that sees no request for idle_ms makes the whole kernel
// exit with the ETIMEOUT exit status (reported by expm_queue_state); the next submit or
// poll that finds the kernel finished launches it again, with the claim counter at the
// oldest unreleased ticket (completed tickets are skipped).  A ticket's slot is reused
// only after that ticket was polled, so a restarted kernel never meets a slot that holds
// a later ticket than the one it claimed.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/expm.h"
#include "dense.cuh"
#include "plan.cuh"

namespace {

struct QueueShared {  // mapped host memory: host <-> kernel flags
    unsigned stop;
    unsigned exit_status;
    unsigned long long restart_at;  // source of the claim counter's reset (pinned)
};

template <class T> void store_release(T *p, T v) { __atomic_store_n(p, v, __ATOMIC_RELEASE); }
template <class T> T load_acquire(const T *p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }

}  // namespace

using namespace expm;

struct expm_queue_s {
    int device = 0;
    int degree = 0;
    std::vector<double> lam, w;  // the plan's poles and weights (copied at creation)
    int complex_a = 0, k = 0, v_cplx = 0, split_v = 0, kc = 0, nsys = 0, mixed = 0, max_refine = 0, mode = 0;
    double tol = 0.0, growth_max = 0.0;
    int cap = 0, nclusters = 0;
    long long idle_ns = 0;
    void *mapped = nullptr;  // one cudaHostAlloc block: slots, seq, done, stat, shared flags
    SmallQueueSlot *slots = nullptr;
    unsigned long long *seq = nullptr, *done = nullptr;
    double *stat = nullptr;
    QueueShared *sh = nullptr;
    SmallQueueArgs args{};  // device views
    void *dmem = nullptr;   // claim counter and halt flag
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool launched = false;
    unsigned long long launches = 0;
    std::mutex mu;
    unsigned long long head = 0, tail = 0;  // next ticket; oldest ticket not yet released
    std::vector<unsigned char> released;    // per slot: its ticket was polled after completion
};

namespace {

size_t al64(size_t b) { return (b + 63) & ~(size_t)63; }

// (Re)launches the consumer kernel if it is not running.  Called with q->mu held.
expm_status ensure_running(expm_queue q) {
    if (q->launched) {
        const cudaError_t e = cudaEventQuery(q->ev);
        if (e == cudaErrorNotReady) return EXPM_OK;
        if (e != cudaSuccess) return cuda_error(e, "queue: consumer kernel");
    }
    q->sh->restart_at = q->tail;
    q->sh->exit_status = 0;
    cudaError_t e = cudaMemcpyAsync(q->args.claim, &q->sh->restart_at, sizeof(unsigned long long),
                                    cudaMemcpyHostToDevice, q->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(q->args.halt, 0, sizeof(unsigned), q->st);
    if (e == cudaSuccess) e = dense_small_queue_launch(q->args, q->mode, q->nclusters, q->st);
    if (e == cudaSuccess) e = cudaEventRecord(q->ev, q->st);
    if (e != cudaSuccess) return cuda_error(e, "queue: consumer launch");
    q->launched = true;
    ++q->launches;
    return EXPM_OK;
}

void advance_tail(expm_queue q) {
    while (q->tail < q->head && q->released[q->tail % q->cap]) ++q->tail;
}

void free_queue(expm_queue q) {
    if (q->st) cudaStreamSynchronize(q->st);
    if (q->ev) cudaEventDestroy(q->ev);
    if (q->st) cudaStreamDestroy(q->st);
    if (q->dmem) cudaFree(q->dmem);
    if (q->mapped) cudaFreeHost(q->mapped);
    delete q;
}

}  // namespace

extern "C" expm_status expm_queue_create(expm_plan p, int a_is_complex, int k, int v_is_complex,
                                         const expm_opts *opts_in, int capacity, int max_clusters, double idle_ms,
                                         expm_queue *out) {
    if (!out) return set_error(EXPM_EINVAL, "queue_create: out is NULL");
    *out = nullptr;
    if (!p) return set_error(EXPM_EINVAL, "queue_create: NULL plan");
    expm_opts opts;
    if (opts_in) opts = *opts_in; else expm_opts_default(&opts);
    if (opts.prec < EXPM_FP64 || opts.prec > EXPM_MIXED_BF16X3)
        return set_error(EXPM_EINVAL, "queue_create: unknown precision");
    if (!(opts.tol > 0) || opts.max_refine < 0) return set_error(EXPM_EINVAL, "queue_create: bad tol or max_refine");
    if (capacity < 1 || capacity > 65536) return set_error(EXPM_EINVAL, "queue_create: capacity must be 1..65536");
    if (max_clusters < 0) return set_error(EXPM_EINVAL, "queue_create: max_clusters must be >= 0");
    if (!(idle_ms > 0.0) || idle_ms > 600000.0) return set_error(EXPM_EINVAL, "queue_create: idle_ms must be in (0, 6e5]");
    const int S = p->degree / 2;
    const int complex_a = a_is_complex ? 1 : 0;
    const int split_v = (!complex_a && v_is_complex) ? 1 : 0;  // real A, complex V: parts as columns
    const int kc = split_v ? 2 * k : k;
    const int nsys = complex_a ? 2 * S : S;
    if (k < 1 || kc > 4) return set_error(EXPM_EINVAL, "queue_create: need 1 <= k and at most 4 solved columns");
    if (nsys > 16) return set_error(EXPM_EINVAL, "queue_create: at most 16 solved systems (degree too high)");

    expm_queue q = new (std::nothrow) expm_queue_s();
    if (!q) return set_error(EXPM_ENOMEM, "queue_create: host allocation");
    q->device = p->device;
    q->degree = p->degree;
    q->lam = p->lam;
    q->w = p->w;
    q->complex_a = complex_a;
    q->k = k;
    q->v_cplx = v_is_complex ? 1 : 0;
    q->split_v = split_v;
    q->kc = kc;
    q->nsys = nsys;
    q->mixed = opts.prec != EXPM_FP64;
    q->mode = q->mixed ? kc : 0;
    q->max_refine = opts.max_refine;
    q->tol = opts.tol;
    q->growth_max = opts.growth_max;
    q->cap = capacity;
    q->idle_ns = (long long)(idle_ms * 1e6);
    q->released.assign(capacity, 0);
    DeviceGuard guard(q->device);
    const int fit = dense_small_queue_max_clusters(q->mode, nsys);
    if (fit < 1) {
        delete q;
        cudaGetLastError();
        return set_error(EXPM_ECUDA, "queue_create: no cluster of the consumer kernel fits on the device");
    }
    q->nclusters = max_clusters > 0 ? std::min(max_clusters, fit) : fit;

    const size_t b_slots = al64(sizeof(SmallQueueSlot) * capacity), b_words = al64(sizeof(unsigned long long) * capacity),
                 b_stat = al64(3 * sizeof(double) * capacity), b_sh = al64(sizeof(QueueShared));
    cudaError_t e = cudaHostAlloc(&q->mapped, b_slots + 2 * b_words + b_stat + b_sh,
                                  cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) {
        unsigned char *m = (unsigned char *)q->mapped;
        std::memset(m, 0, b_slots + 2 * b_words + b_stat + b_sh);
        q->slots = (SmallQueueSlot *)m;
        q->seq = (unsigned long long *)(m + b_slots);
        q->done = (unsigned long long *)(m + b_slots + b_words);
        q->stat = (double *)(m + b_slots + 2 * b_words);
        q->sh = (QueueShared *)(m + b_slots + 2 * b_words + b_stat);
        void *dm = nullptr;
        e = cudaHostGetDevicePointer(&dm, q->mapped, 0);
        if (e == cudaSuccess) {
            unsigned char *d = (unsigned char *)dm;
            q->args.slots = (SmallQueueSlot *)d;
            q->args.seq = (unsigned long long *)(d + b_slots);
            q->args.done = (unsigned long long *)(d + b_slots + b_words);
            q->args.stat = (double *)(d + b_slots + 2 * b_words);
            QueueShared *dsh = (QueueShared *)(d + b_slots + 2 * b_words + b_stat);
            q->args.stop = &dsh->stop;
            q->args.exit_status = &dsh->exit_status;
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&q->dmem, 256);
    if (e == cudaSuccess) {
        q->args.claim = (unsigned long long *)q->dmem;
        q->args.halt = (unsigned *)((unsigned char *)q->dmem + 64);
        q->args.cap = capacity;
        q->args.nsys = nsys;
        q->args.idle_ns = q->idle_ns;
        e = cudaStreamCreateWithFlags(&q->st, cudaStreamNonBlocking);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_queue(q);
        cudaGetLastError();
        return cuda_error(e, "queue_create");
    }
    *out = q;
    return EXPM_OK;
}

extern "C" expm_status expm_queue_submit(expm_queue q, int n, const void *A, int lda, const void *V, int ldv, void *Y,
                                         int ldy, double t, double shift_c, uint64_t *ticket) {
    if (!q || !ticket) return set_error(EXPM_EINVAL, "queue_submit: NULL argument");
    if (n < 1 || n > 64) return set_error(EXPM_EINVAL, "queue_submit: n must be 1..64");
    if (lda < n || ldv < q->k || ldy < q->k) return set_error(EXPM_EINVAL, "queue_submit: leading dimension too small");
    if (!A || !V || !Y) return set_error(EXPM_EINVAL, "queue_submit: NULL data pointer");
    if (!std::isfinite(t) || !std::isfinite(shift_c)) return set_error(EXPM_EINVAL, "queue_submit: t and shift_c must be finite");
    DeviceGuard guard(q->device);
    if (!is_device_ptr(A) || !is_device_ptr(V) || !is_device_ptr(Y))
        return set_error(EXPM_EINVAL, "queue_submit: A, V and Y must be device memory");
    SmallQueueSlot r{};
    r.a.n = n;
    r.a.kc = q->kc;
    r.a.nsys = q->nsys;
    r.a.complex_a = q->complex_a;
    r.a.v_cplx = (q->complex_a && q->v_cplx) ? 1 : 0;
    r.a.y_real = q->complex_a ? 0 : 1;
    r.a.mixed = q->mixed;
    r.a.max_refine = q->max_refine;
    r.a.t = t;
    r.a.tol = q->tol;
    r.a.A = (const double *)A;
    r.a.lda = lda;
    r.a.V = (const double *)V;
    r.a.ldv = q->split_v ? 2 * (int64_t)ldv : ldv;
    r.a.Y = (double *)Y;
    r.a.ldy = q->split_v ? 2 * (int64_t)ldy : ldy;
    // poles and weights as expm_apply_dense forms them (same expressions)
    DenseSystems &sys = r.sys;
    sys.cshift = shift_c;
    const double ec = std::exp(shift_c);
    for (int s = 0; s < q->degree / 2; ++s) {
        const double tr = -q->lam[4 * s], ti = -q->lam[4 * s + 1];
        const double ar = q->w[4 * s], ai = q->w[4 * s + 1];
        if (q->complex_a) {
            sys.th_re[2 * s] = tr; sys.th_im[2 * s] = ti; sys.w_re[2 * s] = ec * ar; sys.w_im[2 * s] = ec * ai;
            sys.th_re[2 * s + 1] = tr; sys.th_im[2 * s + 1] = -ti;
            sys.w_re[2 * s + 1] = ec * ar; sys.w_im[2 * s + 1] = -ec * ai;
        } else {
            sys.th_re[s] = tr; sys.th_im[s] = ti; sys.w_re[s] = 2 * ec * ar; sys.w_im[s] = 2 * ec * ai;
        }
    }
    std::lock_guard<std::mutex> lk(q->mu);
    advance_tail(q);
    if (q->head - q->tail >= (unsigned long long)q->cap) return EXPM_EAGAIN;
    const unsigned long long tk = q->head;
    const int slot = (int)(tk % q->cap);
    std::memcpy(&q->slots[slot], &r, sizeof(r));
    q->released[slot] = 0;
    store_release(&q->seq[slot], tk + 1);
    ++q->head;
    *ticket = tk;
    return ensure_running(q);
}

extern "C" expm_status expm_queue_poll(expm_queue q, uint64_t ticket, expm_info *info) {
    if (!q) return set_error(EXPM_EINVAL, "queue_poll: NULL queue");
    DeviceGuard guard(q->device);
    std::lock_guard<std::mutex> lk(q->mu);
    const int slot = (int)(ticket % q->cap);
    if (ticket >= q->head || ticket < q->tail || q->released[slot]) return EXPM_ENOTFOUND;
    if (load_acquire(&q->done[slot]) != ticket + 1) {
        const expm_status s = ensure_running(q);  // a kernel that ended on an idle wait restarts
        return s == EXPM_OK ? EXPM_EAGAIN : s;
    }
    const double g = q->stat[3 * slot], r = q->stat[3 * slot + 1], sw = q->stat[3 * slot + 2];
    q->released[slot] = 1;
    advance_tail(q);
    expm_status st = EXPM_OK;
    if (g > q->growth_max) st = EXPM_EGROWTH;
    else if (q->mixed && !(r <= q->tol)) st = EXPM_ENOCONV;
    if (info) {
        info->refine_iters_max = (int)sw;
        info->growth_max_seen = g;
        info->resid_rel_max = r;
        info->status_worst = st;
    }
    return st;
}

extern "C" expm_status expm_queue_state(expm_queue q, int *running, int *last_exit, uint64_t *launches, int *clusters) {
    if (!q) return set_error(EXPM_EINVAL, "queue_state: NULL queue");
    DeviceGuard guard(q->device);
    std::lock_guard<std::mutex> lk(q->mu);
    int run = 0;
    if (q->launched) {
        const cudaError_t e = cudaEventQuery(q->ev);
        if (e == cudaErrorNotReady) run = 1;
        else if (e != cudaSuccess) return cuda_error(e, "queue_state: consumer kernel");
    }
    if (running) *running = run;
    if (last_exit) *last_exit = run ? EXPM_OK : (int)load_acquire(&q->sh->exit_status);
    if (launches) *launches = q->launches;
    if (clusters) *clusters = q->nclusters;
    return EXPM_OK;
}

extern "C" expm_status expm_queue_destroy(expm_queue q) {
    if (!q) return EXPM_OK;
    DeviceGuard guard(q->device);
    store_release(&q->sh->stop, 1u);  // every cluster leaves at its next claim or wait poll
    free_queue(q);
    return EXPM_OK;
}
