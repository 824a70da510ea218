// dense.cuh -- geometry and launcher of the pole-batched dense path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

namespace expm {

struct Profiler;

constexpr int DENSE_MAXSYS = 64;

// One "system" per solved pole: real data solves the Im(theta) > 0 member of each
// pair (weight 2 e^c a); complex Hermitian A solves both members (weights e^c a,
// e^c conj(a)), systems 2s and 2s+1 sharing the factorization of pair s.
struct DenseSystems {
    double th_re[DENSE_MAXSYS], th_im[DENSE_MAXSYS];  // theta of each system
    double w_re[DENSE_MAXSYS], w_im[DENSE_MAXSYS];    // weight of each system
    double cshift;                                    // c
};

// A batch of `ninst` problems of the same (padded) order n.  Instance i uses
// A + i*astride, V + i*vstride, Y + i*ystride (strides in elements of each array).
struct DenseGeom {
    int n;          // matrix order
    int kc;         // complex right-hand-side columns solved per system
    int ninst;      // instances
    int npairs;     // factorizations per instance
    int nsys;       // solved systems per instance
    int complex_a;  // A complex Hermitian (else real symmetric)
    int mixed;      // binary32 factorization + binary64 refinement
    int tc;         // mixed only: LU trailing updates on the tensor cores (1: 3xTF32, 2: bf16x3)
    int tile = 0;   // binary32 SIMT trailing updates: 0 = 128 x 64 output tiles, 1 = 64 x 64
    double t;       // time factor
    double tol;     // refinement tolerance
    int max_refine;
    int devctl = 0;  // mixed, kc <= 8 only: refinement decided on the device (no host
                     // synchronisation; every sweep is launched and skips itself once the
                     // stopping test has passed), so the whole solve can be captured in a graph
};

// Device-side results of a devctl solve, written where these point (device memory).
struct DenseDevOut {
    int *iters;          // refinement sweeps applied (one int)
    double *inst_resid;  // per instance: the last relative residual formed
    double *inst_growth; // per instance: growth factor of its pairs' LUs
};

struct DenseIO {
    const double *A;
    int64_t lda, astride;
    const double *V;
    int64_t ldv, vstride;  // in loaded elements (real doubles, or complex when v_cplx)
    int v_cplx;
    double *Y;
    int64_t ldy, ystride;  // in stored elements (real when y_real, else complex)
    int y_real;
};

struct DenseResult {
    int tc_timeout = 0;          // a bounded wait inside the tensor-core kernel gave up
    int iters;                   // refinement sweeps (max over the batch)
    double resid_rel_max;        // worst final relative residual
    double growth_max;           // worst growth factor
    std::vector<int> inst_iters;         // per instance
    std::vector<double> inst_resid;      // per instance
    std::vector<double> inst_growth;     // per instance
};

size_t dense_workspace_bytes(const DenseGeom &g);  // one call (factor + solve)
size_t dense_factor_bytes(const DenseGeom &g);     // reusable factor part
size_t dense_solve_bytes(const DenseGeom &g);      // per-call solve part
// factor part: tA - cI + theta I per pair, its unpivoted LU and growth data
cudaError_t dense_factor(const DenseGeom &g, const DenseIO &io, const DenseSystems &sys, void *fwork, cudaStream_t st,
                         Profiler &prof);
// solve part (triangular solves, refinement, residue sum) with factors from dense_factor
cudaError_t dense_solve(const DenseGeom &g, const DenseIO &io, const DenseSystems &sys, const void *fwork, void *swork,
                        cudaStream_t st, Profiler &prof, DenseResult *res);
// growth factors of a factor part (synchronises st)
cudaError_t dense_growth(const DenseGeom &g, const void *fwork, cudaStream_t st, DenseResult *res);
cudaError_t dense_run(const DenseGeom &g, const DenseIO &io, const DenseSystems &sys, void *work, cudaStream_t st,
                      Profiler &prof, DenseResult *res);
// whether the fused narrow triangular solve (kc <= 8, solution in shared memory) takes
// an n x kc right-hand side in binary32 -- the requirement of a devctl solve
bool dense_narrow_fits(int n, int kc);
// whether the solves of geometry g multiply by explicit inverses of the LU's diagonal
// panels (kept in the factor part: factor parts with and without them differ)
bool dense_uses_inv(const DenseGeom &g);
// small problems in one cluster launch (dense_small.cu): one instance, n <= 64, kc <= 4,
// at most 16 solved systems; binary64, or the binary32 inverse with binary64-residual
// refinement for every mixed precision.  dense_small_launch only enqueues (growth,
// residual and sweeps land in out[0..2], device memory; usable under stream capture);
// dense_small_run also synchronises st to read them.
bool dense_small_fits(const DenseGeom &g);
// one small problem for the kernels of dense_small.cu (n <= 64, kc <= 4, nsys <= 16)
struct SmallReq {
    int n, kc, nsys, complex_a, v_cplx, y_real, mixed, max_refine;
    double t, tol;
    const double *A;
    int64_t lda;
    const double *V;
    int64_t ldv;
    double *Y;
    int64_t ldy;
    double *out;  // worst growth, worst residual, sweeps (3 doubles)
};
// Device-fed work queue of small problems (queue.cu): a persistent cluster kernel whose
// clusters claim tickets, wait (bounded) for the host to publish each ticket's request in
// mapped host memory, evaluate it and publish its completion.
struct SmallQueueSlot {
    SmallReq a;        // out is set on the device (the slot's stat entry)
    DenseSystems sys;  // poles and weights (e^c folded in), shift c
};
struct SmallQueueArgs {
    SmallQueueSlot *slots;       // cap slots (mapped host memory, device view)
    unsigned long long *seq;     // cap: ticket + 1 once the slot holds that ticket's request
    unsigned long long *done;    // cap: ticket + 1 once that ticket is evaluated
    double *stat;                // cap x 3: growth, residual, sweeps of the slot's last request
    unsigned *stop;              // set by the host: exit after the current request
    unsigned *exit_status;       // set by the kernel: EXPM_ETIMEOUT when an idle wait ran out
    unsigned long long *claim;   // next ticket to claim (device memory)
    unsigned *halt;              // a cluster timed out or saw stop: the others exit too (device memory)
    int cap, nsys;
    long long idle_ns;           // longest wait for a request before the kernel exits
};
// mode 0: binary64; 1..4: mixed with that many columns
cudaError_t dense_small_queue_launch(const SmallQueueArgs &q, int mode, int nclusters, cudaStream_t st);
int dense_small_queue_max_clusters(int mode, int nsys);  // co-resident clusters (0 on error)
size_t dense_small_workspace_bytes();
cudaError_t dense_small_launch(const DenseGeom &g, const DenseIO &io, const DenseSystems &sys, double *out,
                               cudaStream_t st, Profiler &prof);
cudaError_t dense_small_run(const DenseGeom &g, const DenseIO &io, const DenseSystems &sys, void *work,
                            cudaStream_t st, Profiler &prof, DenseResult *res);
// offset in the workspace of the tensor-core updates' time-out flag (an int; g.tc != 0)
size_t dense_tc_flag_offset(const DenseGeom &g);
// devctl form: factor + growth + solve fully enqueued on st (nothing read back); results to out
cudaError_t dense_run_devctl(const DenseGeom &g, const DenseIO &io, const DenseSystems &sys, void *work,
                             cudaStream_t st, Profiler &prof, const DenseDevOut &out);

}  // namespace expm
