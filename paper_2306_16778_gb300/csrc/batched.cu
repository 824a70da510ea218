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

// Padded order of a bucket.  Scheme 0 (the default): multiples of 32 up to 128, then
// steps of about 1/4.  Scheme 1 (fine): multiples of 32 throughout -- least padding,
// most buckets.  Scheme 2 (coarse): powers of two and their midpoints -- fewest,
// largest launches.  The graph path can time all three and keep the fastest.
int bucket_order(int n, int scheme = 0) {
    if (scheme == 1) return (n + 31) / 32 * 32;
    if (scheme == 2) {
        static const int edges2[] = {64, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048};
        for (int e : edges2)
            if (n <= e) return e;
        return (n + 511) / 512 * 512;
    }
    static const int edges[] = {32, 64, 96, 128, 160, 192, 256, 320, 384, 448, 512, 640, 768, 896, 1024,
                                1280, 1536, 1792, 2048};
    for (int e : edges)
        if (n <= e) return e;
    return (n + 255) / 256 * 256;
}

}  // namespace expm

using namespace expm;

// Tensor-core trailing updates (EXPM_MIXED_TF32X3 / EXPM_MIXED_BF16X3) for buckets whose
// padded order exceeds one outer panel of the tensor-core LU; smaller buckets factor on
// the FP32 pipe (their updates are too small to fill a 128-row tile per step).
static int batch_tc(int prec, int nb) {
    if (nb <= 256) return 0;
    return prec == EXPM_MIXED_TF32X3 ? 1 : prec == EXPM_MIXED_BF16X3 ? 2 : 0;
}
static bool batch_prec_ok(int prec) {
    return prec == EXPM_FP64 || prec == EXPM_MIXED_FP32 || prec == EXPM_MIXED_F32X2 || prec == EXPM_MIXED_TF32X3 ||
           prec == EXPM_MIXED_BF16X3;
}

extern "C" expm_status expm_apply_batched(expm_plan p, int count, const int *n, const void *const *A, int a_is_complex,
                                          const void *const *V, const int *k, int v_is_complex, void *const *Y,
                                          const expm_opts *opts_in, expm_info *per_instance) {
    if (!p) return set_error(EXPM_EINVAL, "apply_batched: NULL plan");
    if (count < 0 || (count > 0 && (!n || !A || !V || !k || !Y)))
        return set_error(EXPM_EINVAL, "apply_batched: NULL array argument");
    if (count == 0) return EXPM_OK;
    expm_opts opts;
    if (opts_in) opts = *opts_in; else expm_opts_default(&opts);
    if (!batch_prec_ok(opts.prec)) return set_error(EXPM_EINVAL, "apply_batched: unknown precision");
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
        g.tc = batch_tc(opts.prec, nb);
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
            if (res.tc_timeout) return set_error(EXPM_ETIMEOUT, "apply_batched: a tensor-core wait gave up");
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

// ------------------------------------------------------------------ captured graph
// expm_batched_capture records the whole batched evaluation -- every bucket's gather,
// factorization, device-controlled refinement and scatter -- into one CUDA graph over
// the caller's buffers; expm_batched_replay launches it with a single call.  The graph
// owns its device memory (workspace, staging, pointer tables, per-instance results).

namespace expm {
namespace {

struct GraphChunk {
    DenseGeom g;
    int nb, kb;
    double tile_ms[2] = {-1.0, -1.0};  // factorization time with each trailing-update tile shape (tuned)
    std::vector<int> inst;  // original instance indices, in batch order
    size_t ptr_off, res_off;  // offsets of the pointer table and of the results in the graph memory
};

struct BatchSpec {
    int count, complex_a, v_cplx, aw, vw, yw, nsys, S;
    const int *n, *k;
    const void *const *A;
    const void *const *V;
    void *const *Y;
    expm_opts opts;
    DenseSystems sys;
};

std::vector<GraphChunk> plan_chunks(const BatchSpec &b, int scheme) {
    std::vector<int> order(b.count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return bucket_order(b.n[x], scheme) > bucket_order(b.n[y], scheme); });
    std::vector<GraphChunk> out;
    size_t pos = 0;
    while (pos < order.size()) {
        const int nb = bucket_order(b.n[order[pos]], scheme);
        size_t end = pos;
        int kb = 1;
        while (end < order.size() && bucket_order(b.n[order[end]], scheme) == nb) kb = std::max(kb, b.k[order[end++]]);
        DenseGeom g{};
        g.n = nb;
        g.kc = kb;
        g.npairs = b.S;
        g.nsys = b.nsys;
        g.complex_a = b.complex_a;
        g.mixed = b.opts.prec != EXPM_FP64;
        g.t = b.opts.t;
        g.tol = b.opts.tol;
        g.max_refine = b.opts.max_refine;
        g.tc = batch_tc(b.opts.prec, nb);
        g.devctl = 1;
        g.ninst = 1;
        const size_t per_inst = dense_workspace_bytes(g) + sizeof(double) * ((size_t)nb * nb * b.aw + 2 * (size_t)nb * kb * 2);
        size_t chunk = std::max<size_t>(1, ((size_t)8 << 30) / per_inst);
        chunk = std::min<size_t>(chunk, 65535 / b.nsys);
        for (size_t c0 = pos; c0 < end; c0 += chunk) {
            GraphChunk c;
            c.nb = nb;
            c.kb = kb;
            c.g = g;
            c.g.ninst = (int)(std::min(end, c0 + chunk) - c0);
            for (size_t z = c0; z < c0 + (size_t)c.g.ninst; ++z) c.inst.push_back(order[z]);
            out.push_back(std::move(c));
        }
        pos = end;
    }
    return out;
}

}  // namespace
}  // namespace expm

struct expm_batch_graph_s {
    int device = 0;
    int scheme = 0;
    // one instance small enough for the one-launch kernel (dense_small.cu): the graph is
    // that launch on the caller's buffers, its status block at the start of mem
    bool small = false;
    expm::DenseGeom sg{};
    double ms_per_scheme[3] = {-1.0, -1.0, -1.0};
    expm::BatchSpec spec{};
    std::vector<expm::GraphChunk> chunks;
    void *mem = nullptr;
    size_t mem_bytes = 0, work_off = 0, stage_off = 0, res_bytes = 0, res_base = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace expm {
namespace {

static inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// The padded staging buffers of chunk c as the dense kernels' input/output.
DenseIO chunk_io(const expm_batch_graph_s *G, const GraphChunk &c) {
    const BatchSpec &b = G->spec;
    unsigned char *m = (unsigned char *)G->mem;
    const int nb = c.nb, kb = c.kb, ni = c.g.ninst;
    const size_t bytesA = sizeof(double) * (size_t)ni * nb * nb * b.aw;
    const size_t bytesV = sizeof(double) * (size_t)ni * nb * kb * b.vw;
    DenseIO io{};
    io.A = (double *)(m + G->stage_off);
    io.lda = nb;
    io.astride = (int64_t)nb * nb;
    io.V = (double *)(m + G->stage_off + bytesA);
    io.ldv = kb;
    io.vstride = (int64_t)nb * kb;
    io.v_cplx = b.v_cplx;
    io.Y = (double *)(m + G->stage_off + bytesA + bytesV);
    io.ldy = kb;
    io.ystride = (int64_t)nb * kb;
    io.y_real = b.yw == 1 ? 1 : 0;
    return io;
}
void enqueue_gather(const expm_batch_graph_s *G, const GraphChunk &c, const DenseIO &io, cudaStream_t st) {
    const BatchSpec &b = G->spec;
    const InstPtr *dptr = (const InstPtr *)((unsigned char *)G->mem + c.ptr_off);
    const unsigned gx = (unsigned)std::min<int64_t>(((int64_t)c.nb * c.nb * b.aw + 255) / 256, 1024);
    gather_pad<<<dim3(gx, 1, c.g.ninst), 256, 0, st>>>(dptr, c.nb, c.kb, b.aw, b.vw, const_cast<double *>(io.A),
                                                     const_cast<double *>(io.V));
}

// Per-bucket tuning of the binary32 trailing updates' tile shape: each chunk's gather and
// factorization run with 128 x 64 and with 64 x 64 output tiles (the second run of each
// timed), and the faster shape is kept for the capture.
cudaError_t tune_tiles(expm_batch_graph_s *G, cudaStream_t st) {
    Profiler off;
    cudaEvent_t e0, e1;
    cudaError_t err = cudaEventCreate(&e0);
    if (err != cudaSuccess) return err;
    if ((err = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return err;
    }
    const DenseSystems &sys = G->spec.sys;
    for (GraphChunk &c : G->chunks) {
        if (!c.g.mixed || c.g.tc) continue;  // binary64 has one shape; tensor-core buckets use no SIMT tile
        const DenseIO io = chunk_io(G, c);
        for (int tile = 0; tile < 2 && err == cudaSuccess; ++tile) {
            c.g.tile = tile;
            for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {
                if (rep == 1) err = cudaEventRecord(e0, st);
                enqueue_gather(G, c, io, st);
                if (err == cudaSuccess) err = cudaGetLastError();
                if (err == cudaSuccess) err = dense_factor(c.g, io, sys, (unsigned char *)G->mem + G->work_off, st, off);
                if (err == cudaSuccess && rep == 1) err = cudaEventRecord(e1, st);
            }
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            c.tile_ms[tile] = ms;
        }
        c.g.tile = (c.tile_ms[1] >= 0.0 && c.tile_ms[1] < c.tile_ms[0]) ? 1 : 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return err;
}

// Enqueues the whole evaluation of graph object G on st (used for the warm-up run and
// inside the capture).
cudaError_t enqueue_batched(expm_batch_graph_s *G, cudaStream_t st) {
    Profiler off;
    const BatchSpec &b = G->spec;
    unsigned char *m = (unsigned char *)G->mem;
    if (G->small) {
        DenseIO io{};
        io.A = (const double *)b.A[0];
        io.lda = G->sg.n;
        io.V = (const double *)b.V[0];
        io.ldv = G->sg.kc;
        io.v_cplx = b.v_cplx;
        io.Y = (double *)b.Y[0];
        io.ldy = G->sg.kc;
        io.y_real = b.yw == 1 ? 1 : 0;
        return dense_small_launch(G->sg, io, b.sys, (double *)m, st, off);
    }
    for (const GraphChunk &c : G->chunks) {
        const int nb = c.nb, kb = c.kb, ni = c.g.ninst;
        const DenseIO io = chunk_io(G, c);
        const InstPtr *dptr = (const InstPtr *)(m + c.ptr_off);
        enqueue_gather(G, c, io, st);
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        unsigned char *r = m + c.res_off;
        DenseDevOut out{(int *)r, (double *)(r + 256), (double *)(r + 256 + al256(sizeof(double) * ni))};
        err = dense_run_devctl(c.g, io, b.sys, m + G->work_off, st, off, out);
        if (err != cudaSuccess) return err;
        if (c.g.tc) {  // the tensor-core updates' time-out flag, next to the sweep count
            err = cudaMemcpyAsync(r + sizeof(int), m + G->work_off + dense_tc_flag_offset(c.g), sizeof(int),
                                  cudaMemcpyDeviceToDevice, st);
            if (err != cudaSuccess) return err;
        } else {
            err = cudaMemsetAsync(r + sizeof(int), 0, sizeof(int), st);
            if (err != cudaSuccess) return err;
        }
        scatter_unpad<<<dim3((unsigned)std::min<int64_t>(((int64_t)nb * kb * b.yw + 255) / 256, 1024), 1, ni), 256, 0,
                        st>>>(dptr, nb, kb, b.yw, io.Y);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    return cudaSuccess;
}

void destroy_graph(expm_batch_graph_s *G) {
    if (!G) return;
    DeviceGuard guard(G->device);
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    if (G->mem) cudaFree(G->mem);
    delete G;
}

// Builds, warms up and captures the graph for one bucket scheme (or, with `small`, the
// one-launch kernel for the single instance of geometry sg); with `tune`, each bucket's
// trailing-update tile shape is chosen by timing first.
expm_status build_graph(const BatchSpec &b, int scheme, int device, expm_batch_graph_s **out,
                        const DenseGeom *sg = nullptr, bool tune = false) {
    auto G = new expm_batch_graph_s();
    G->device = device;
    G->scheme = scheme;
    G->spec = b;
    if (sg) {
        G->small = true;
        G->sg = *sg;
    } else {
        G->chunks = plan_chunks(b, scheme);
    }
    size_t work = 0, stage = 0, ptrs = 0, res = G->small ? 256 : 0;
    for (GraphChunk &c : G->chunks) {
        const int ni = c.g.ninst;
        work = std::max(work, dense_workspace_bytes(c.g));
        stage = std::max(stage, sizeof(double) * ((size_t)ni * c.nb * c.nb * b.aw + (size_t)ni * c.nb * c.kb * (b.vw + b.yw)));
        c.ptr_off = ptrs;
        ptrs += al256(sizeof(InstPtr) * ni);
        c.res_off = res;
        res += 256 + 2 * al256(sizeof(double) * ni);
    }
    G->work_off = 0;
    G->stage_off = al256(work);
    const size_t ptr_base = G->stage_off + al256(stage);
    G->res_base = ptr_base + ptrs;
    G->res_bytes = res;
    G->mem_bytes = G->res_base + res;
    for (GraphChunk &c : G->chunks) {
        c.ptr_off += ptr_base;
        c.res_off += G->res_base;
    }
    cudaError_t err = cudaMalloc(&G->mem, G->mem_bytes);
    if (err != cudaSuccess) {
        cudaGetLastError();
        G->mem = nullptr;
        destroy_graph(G);
        return set_error(EXPM_ENOMEM, "batched_capture: device memory for the graph");
    }
    for (const GraphChunk &c : G->chunks) {  // pointer tables, uploaded once (outside the graph)
        std::vector<InstPtr> hp(c.g.ninst);
        for (int z = 0; z < c.g.ninst; ++z) {
            const int i = c.inst[z];
            hp[z] = InstPtr{(const double *)b.A[i], (const double *)b.V[i], (double *)b.Y[i], b.n[i], b.k[i]};
        }
        err = cudaMemcpy((unsigned char *)G->mem + c.ptr_off, hp.data(), sizeof(InstPtr) * hp.size(),
                         cudaMemcpyHostToDevice);
        if (err != cudaSuccess) break;
    }
    cudaStream_t st = nullptr;
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (err == cudaSuccess && tune && !G->small) err = tune_tiles(G, st);
    // one plain run first: sets kernel attributes and checks every launch outside capture
    if (err == cudaSuccess) err = enqueue_batched(G, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err == cudaSuccess) err = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
        cudaError_t e1 = enqueue_batched(G, st);
        cudaError_t e2 = cudaStreamEndCapture(st, &G->graph);
        err = e1 != cudaSuccess ? e1 : e2;
    }
    if (err == cudaSuccess) err = cudaGraphInstantiate(&G->exec, G->graph, 0);
    if (st) cudaStreamDestroy(st);
    if (err != cudaSuccess) {
        cudaGetLastError();
        destroy_graph(G);
        return cuda_error(err, "batched_capture");
    }
    *out = G;
    return EXPM_OK;
}

// Average time of `reps` launches after one untimed launch (ms).
double time_graph(expm_batch_graph_s *G, int reps) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return 1e30;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaGraphLaunch(G->exec, st);
    cudaEventRecord(a, st);
    for (int r = 0; r < reps; ++r) cudaGraphLaunch(G->exec, st);
    cudaEventRecord(b, st);
    float ms = 0.f;
    const bool ok = cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(st);
    return ok ? ms / reps : 1e30;
}

}  // namespace
}  // namespace expm

extern "C" expm_status expm_batched_capture(expm_plan p, int count, const int *n, const void *const *A,
                                            int a_is_complex, const void *const *V, const int *k, int v_is_complex,
                                            void *const *Y, const expm_opts *opts_in, int scheme,
                                            expm_batch_graph *out) {
    if (!p || !out) return set_error(EXPM_EINVAL, "batched_capture: NULL plan or output");
    *out = nullptr;
    if (count < 1 || !n || !A || !V || !k || !Y) return set_error(EXPM_EINVAL, "batched_capture: empty or NULL arrays");
    if (scheme < -1 || scheme > 2) return set_error(EXPM_EINVAL, "batched_capture: scheme must be -1 (tune), 0, 1 or 2");
    expm_opts opts;
    if (opts_in) opts = *opts_in; else expm_opts_default(&opts);
    if (!batch_prec_ok(opts.prec)) return set_error(EXPM_EINVAL, "batched_capture: unknown precision");
    if (opts.flags != 0) return set_error(EXPM_EINVAL, "batched_capture: opts.flags must be 0");
    if (!std::isfinite(opts.t) || !std::isfinite(opts.shift_c) || !(opts.tol > 0) || opts.max_refine < 0 ||
        opts.max_refine > 64)
        return set_error(EXPM_EINVAL, "batched_capture: bad t, shift_c, tol or max_refine");
    const bool complex_a = a_is_complex != 0;
    if (!complex_a && v_is_complex)
        return set_error(EXPM_ENOTSUP, "batched_capture: complex V with real A (use complex A or split V)");
    DeviceGuard guard(p->device);
    for (int i = 0; i < count; ++i) {
        if (n[i] < 1 || k[i] < 1 || k[i] > 8) return set_error(EXPM_EINVAL, "batched_capture: need n[i] >= 1, 1 <= k[i] <= 8");
        if (!A[i] || !V[i] || !Y[i] || !is_device_ptr(A[i]) || !is_device_ptr(V[i]) || !is_device_ptr(Y[i]))
            return set_error(EXPM_EINVAL, "batched_capture: instance data must be device memory");
        if (!dense_narrow_fits(bucket_order(n[i], 2), k[i]))
            return set_error(EXPM_EINVAL, "batched_capture: an instance is too large for the graph path");
    }
    BatchSpec b{};
    b.count = count;
    b.complex_a = complex_a;
    b.v_cplx = v_is_complex ? 1 : 0;
    b.aw = complex_a ? 2 : 1;
    b.vw = v_is_complex ? 2 : 1;
    b.yw = (complex_a || v_is_complex) ? 2 : 1;
    b.S = p->degree / 2;
    b.nsys = complex_a ? 2 * b.S : b.S;
    b.n = n;
    b.k = k;
    b.A = A;
    b.V = V;
    b.Y = Y;
    b.opts = opts;
    b.sys.cshift = opts.shift_c;
    const double ec = std::exp(opts.shift_c);
    for (int s = 0; s < b.S; ++s) {
        const double tr = -p->lam[4 * s], ti = -p->lam[4 * s + 1];
        const double ar = p->w[4 * s], ai = p->w[4 * s + 1];
        if (complex_a) {
            b.sys.th_re[2 * s] = tr; b.sys.th_im[2 * s] = ti; b.sys.w_re[2 * s] = ec * ar; b.sys.w_im[2 * s] = ec * ai;
            b.sys.th_re[2 * s + 1] = tr; b.sys.th_im[2 * s + 1] = -ti;
            b.sys.w_re[2 * s + 1] = ec * ar; b.sys.w_im[2 * s + 1] = -ec * ai;
        } else {
            b.sys.th_re[s] = tr; b.sys.th_im[s] = ti; b.sys.w_re[s] = 2 * ec * ar; b.sys.w_im[s] = 2 * ec * ai;
        }
    }
    // the pointer arrays are read again at capture time only: keep nothing of the caller's
    // host arrays (the graph captured their values)
    if (count == 1) {  // one small instance: the graph is the one-launch kernel
        DenseGeom g{};
        g.n = n[0];
        g.kc = k[0];
        g.ninst = 1;
        g.complex_a = complex_a;
        g.npairs = b.S;
        g.nsys = b.nsys;
        g.mixed = opts.prec != EXPM_FP64;
        g.t = opts.t;
        g.tol = opts.tol;
        g.max_refine = opts.max_refine;
        if (dense_small_fits(g)) {
            expm_batch_graph_s *G = nullptr;
            expm_status s = build_graph(b, 0, p->device, &G, &g);
            if (s != EXPM_OK) return s;
            *out = G;
            return EXPM_OK;
        }
    }
    if (scheme >= 0) {
        expm_batch_graph_s *G = nullptr;
        expm_status s = build_graph(b, scheme, p->device, &G);
        if (s != EXPM_OK) return s;
        G->spec.n = G->spec.k = nullptr;
        G->spec.A = G->spec.V = nullptr;
        G->spec.Y = nullptr;
        *out = G;
        return EXPM_OK;
    }
    // autotune: capture every scheme, time each, keep the fastest
    expm_batch_graph_s *best = nullptr;
    double ms[3] = {-1.0, -1.0, -1.0};
    for (int sc = 0; sc < 3; ++sc) {
        expm_batch_graph_s *G = nullptr;
        expm_status s = build_graph(b, sc, p->device, &G, nullptr, true);
        if (s != EXPM_OK) {
            if (best) destroy_graph(best);
            return s;
        }
        ms[sc] = time_graph(G, 2);
        if (!best || ms[sc] < ms[best->scheme]) {
            if (best) destroy_graph(best);
            best = G;
        } else {
            destroy_graph(G);
        }
    }
    for (int sc = 0; sc < 3; ++sc) best->ms_per_scheme[sc] = ms[sc];
    best->spec.n = best->spec.k = nullptr;
    best->spec.A = best->spec.V = nullptr;
    best->spec.Y = nullptr;
    *out = best;
    return EXPM_OK;
}

extern "C" expm_status expm_batched_replay(expm_batch_graph G, void *stream, expm_info *per_instance) {
    if (!G) return set_error(EXPM_EINVAL, "batched_replay: NULL graph");
    DeviceGuard guard(G->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t err = cudaGraphLaunch(G->exec, st);
    if (err != cudaSuccess) return cuda_error(err, "batched_replay: launch");
    if (!per_instance) return EXPM_OK;
    std::vector<unsigned char> h(G->res_bytes);
    err = cudaMemcpyAsync(h.data(), (unsigned char *)G->mem + G->res_base, G->res_bytes, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return cuda_error(err, "batched_replay: results");
    const expm_opts &o = G->spec.opts;
    expm_status worst = EXPM_OK;
    if (G->small) {  // growth, residual, sweeps of the one-launch kernel
        double r3[3];
        std::memcpy(r3, h.data(), sizeof(r3));
        if (r3[0] > o.growth_max) worst = EXPM_EGROWTH;
        else if (G->sg.mixed && !(r3[1] <= o.tol)) worst = EXPM_ENOCONV;
        per_instance[0] = expm_info{(int)r3[2], r3[0], r3[1], worst};
    }
    for (const GraphChunk &c : G->chunks) {
        const unsigned char *r = h.data() + (c.res_off - G->res_base);
        int iters, tc_timeout;
        std::memcpy(&iters, r, sizeof(int));
        std::memcpy(&tc_timeout, r + sizeof(int), sizeof(int));
        if (tc_timeout) return set_error(EXPM_ETIMEOUT, "batched_replay: a tensor-core wait gave up");
        const double *resid = (const double *)(r + 256);
        const double *growth = (const double *)(r + 256 + al256(sizeof(double) * c.g.ninst));
        for (int z = 0; z < c.g.ninst; ++z) {
            expm_status si = EXPM_OK;
            if (growth[z] > o.growth_max) si = EXPM_EGROWTH;
            else if (c.g.mixed && !(resid[z] <= o.tol)) si = EXPM_ENOCONV;
            if (si != EXPM_OK && worst == EXPM_OK) worst = si;
            per_instance[c.inst[z]] = expm_info{iters, growth[z], resid[z], si};
        }
    }
    if (worst == EXPM_EGROWTH) return set_error(worst, "batched_replay: LU growth exceeds opts.growth_max");
    if (worst == EXPM_ENOCONV) return set_error(worst, "batched_replay: refinement did not reach opts.tol");
    return EXPM_OK;
}

extern "C" expm_status expm_batched_graph_info(expm_batch_graph G, int *scheme, int *launch_groups,
                                               size_t *device_bytes, double ms_per_scheme[3]) {
    if (!G) return set_error(EXPM_EINVAL, "batched_graph_info: NULL graph");
    if (scheme) *scheme = G->scheme;
    if (launch_groups) *launch_groups = G->small ? 1 : (int)G->chunks.size();
    if (device_bytes) *device_bytes = G->mem_bytes;
    if (ms_per_scheme)
        for (int i = 0; i < 3; ++i) ms_per_scheme[i] = G->ms_per_scheme[i];
    return EXPM_OK;
}

extern "C" int expm_batched_graph_buckets(expm_batch_graph G, int max, int *order, int *ninst, int *tile,
                                          double *ms_tile0, double *ms_tile1) {
    if (!G) return -1;
    const int nc = (int)G->chunks.size();
    for (int i = 0; i < nc && i < max; ++i) {
        const expm::GraphChunk &c = G->chunks[i];
        if (order) order[i] = c.nb;
        if (ninst) ninst[i] = c.g.ninst;
        if (tile) tile[i] = c.g.tile;
        if (ms_tile0) ms_tile0[i] = c.tile_ms[0];
        if (ms_tile1) ms_tile1[i] = c.tile_ms[1];
    }
    return nc;
}

extern "C" expm_status expm_batched_graph_destroy(expm_batch_graph G) {
    destroy_graph(G);
    return EXPM_OK;
}
