// tridiag.cuh -- geometry and launcher of the pole-batched tridiagonal path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <algorithm>

namespace expm {

struct Profiler;

constexpr int TRI_PF = 8;       // rows kept in flight by the factor kernel's backward pass
constexpr int TRI_PMAX = 3000;  // max blocks: the reduced system (P-1 rows) lives in shared memory
constexpr int TRI_MMIN = 8;     // min interior rows per block
constexpr int TRI_MAXSYS = 32;  // real data: one system per conjugate pair, degree <= 64

// Row partition: P blocks; block b starts at row b*B, has m interior rows
// (the last block has N - (P-1)*B rows) and, for b < P-1, is followed by the
// separator row b*B + m.
struct TriGeom {
    int64_t N;
    int m, B, P;
    int S;       // systems (shifted matrices)
    int LG;      // lanes per (block, column) group in the solve kernel: power of two >= S
    int Rc;      // real right-hand-side columns
    double t;    // time factor
    double cshift;
};

// Shifts theta_s (paper's notation: the system is t T - cI + theta_s I) and the
// weights W_s multiplying Re(W_s x_s) in the sum.
struct TriPoles {
    double th_re[TRI_MAXSYS], th_im[TRI_MAXSYS];
    double w_re[TRI_MAXSYS], w_im[TRI_MAXSYS];
};

TriGeom tri_geometry(int64_t N, int S, int Rc, bool ff, int sm_count);
size_t tri_workspace_bytes(const TriGeom &g, bool ff);  // one call (factor + solve)
size_t tri_factor_bytes(const TriGeom &g, bool ff);     // the reusable factor part
size_t tri_solve_bytes(const TriGeom &g, bool ff);      // the per-call solve part
// factor part: d' = t d - c, e' = t e, the block LUs and spikes (depends on T, t, c, poles)
cudaError_t tri_factor(const TriGeom &g, bool ff, const double *d, const double *e, const TriPoles &ps, void *fwork,
                       cudaStream_t st, Profiler &prof);
// solve part for a block of right-hand sides, with a factor part made by tri_factor
cudaError_t tri_solve(const TriGeom &g, bool ff, const double *V, double *Y, const TriPoles &ps, const void *fwork,
                      void *swork, cudaStream_t st, Profiler &prof);
// v_ready (optional): an event that st waits for between the factorization and the
// first kernel that reads V (V copied on another stream meanwhile)
cudaError_t tri_run(const TriGeom &g, bool ff, const double *d, const double *e, const double *V, double *Y,
                    const TriPoles &ps, void *work, cudaStream_t st, Profiler &prof, cudaEvent_t v_ready = nullptr);

// binary32 factors + refinement (EXPM_MIXED_FP32), tridiag_mixed.cu.  The factor part
// (prep + binary32 block LUs and spikes) depends on T, t, c and the poles only.
struct MixOpts {
    int max_refine;  // correction passes at most (0: the binary32 solve alone)
    int verify;      // form the residual after the last pass too (stopping test / report)
    double tol;      // stop when max_s ||r_s|| / ((beta + |theta_s|) ||x_s||) <= tol
};
struct MixResult {
    bool converged;  // the last residual formed met tol
    int iters;       // correction passes applied
    double resid;    // the last relative residual formed
};
TriGeom tri_mixed_geometry(int64_t N, int S, int Rc, int sm_count);
size_t tri_mixed_factor_bytes(const TriGeom &g);
size_t tri_mixed_solve_bytes(const TriGeom &g, int max_refine);
cudaError_t tri_mixed_factor(const TriGeom &g, const double *d, const double *e, const TriPoles &ps, void *fwork,
                             cudaStream_t st, Profiler &prof);
cudaError_t tri_mixed_solve(const TriGeom &g, const double *V, double *Y, const TriPoles &ps, const void *fwork,
                            void *swork, const MixOpts &mo, cudaStream_t st, Profiler &prof);
// copies the device-side refinement state back (synchronises the stream)
cudaError_t tri_mixed_read_state(const TriGeom &g, const void *swork, int max_refine, MixResult *out, cudaStream_t st);

// complex Hermitian T (tridiag_herm.cu): D^H T D is real symmetric with off-diagonal |e|
// for a diagonal unitary D = diag(phi).  herm_prepare forms |e| (N-1 doubles), phi (N
// complex) and V' = D^H V (N x r complex) in the scratch; the real-off-diagonal kernels
// then solve with |e| and V' into the complex Y, and herm_finish multiplies row i of Y
// by phi_i in place.
struct HermWork {
    double *eabs;  // |e_i|, N-1 doubles
    double *phi;   // phi_i, N complex
    double *Vp;    // D^H V, N x r complex
    double *part;  // block products (scan scratch)
};
size_t herm_scratch_bytes(int64_t N, int r);
size_t herm_part_bytes(int64_t N);  // scan scratch of herm_phases
// |e| (N-1 doubles) and phi (N complex) of complex e (N-1 complex)
cudaError_t herm_phases(int64_t N, const double *e, double *eabs, double *phi, double *part, cudaStream_t st);
// Out = s(phi) X row by row (s = conj with conj_phi); X real or complex, Out complex; Out
// may equal X when X is complex
cudaError_t herm_scale(int64_t N, int r, const double *phi, const double *X, int x_cplx, double *Out, int conj_phi,
                       int sm_count, cudaStream_t st);
HermWork herm_carve(void *scratch, int64_t N, int r);
cudaError_t herm_prepare(int64_t N, const double *e, const double *V, int r, int v_cplx, const HermWork &w,
                         int sm_count, cudaStream_t st);
cudaError_t herm_finish(int64_t N, int r, const HermWork &w, double *Y, int sm_count, cudaStream_t st);

}  // namespace expm
