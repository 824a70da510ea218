// dense.cuh -- geometry and launcher of the pole-batched dense path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

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

struct DenseGeom {
    int n;          // matrix order
    int kc;         // complex right-hand-side columns solved per system
    int npairs;     // factorizations
    int nsys;       // solved systems
    int complex_a;  // A complex Hermitian (else real symmetric)
    int mixed;      // binary32 factorization + binary64 refinement
    double t;       // time factor
    double tol;     // refinement tolerance
    int max_refine;
};

struct DenseResult {
    int iters;
    double resid_rel_max;
    double growth_max;
};

size_t dense_workspace_bytes(const DenseGeom &g);
cudaError_t dense_run(const DenseGeom &g, const double *A, int64_t lda, const double *V, int64_t ldv, int v_cplx,
                      double *Y, int64_t ldy, const DenseSystems &sys, void *work, cudaStream_t st, Profiler &prof,
                      DenseResult *res);

}  // namespace expm
