// tridiag_herm.cu -- complex Hermitian tridiagonal matrices through a diagonal unitary
// similarity onto a real symmetric one.
//
// T has real diagonal d, T_{i,i+1} = e_i and T_{i+1,i} = conj(e_i) (Sec. 3: A Hermitian).
// With D = diag(phi), phi_0 = 1 and phi_{i+1} = phi_i conj(e_i) / |e_i| (phi_{i+1} = phi_i
// where e_i = 0), every |phi_i| = 1 and
//   (D^H T D)_{i,i+1} = conj(phi_i) e_i phi_{i+1} = |e_i|,
// so T~ = D^H T D is the real symmetric tridiagonal matrix with diagonal d and
// off-diagonal |e|.  Since D is unitary and diagonal it commutes with the shifts:
//   (tT - cI + theta I)^{-1} = D (tT~ - cI + theta I)^{-1} D^H
// for every pole, hence for the partial-fraction sum of eq. expAx:
//   Y = D [ e^c R_n(tT~ - cI) ] (D^H V).
// The complex case therefore runs the real-off-diagonal kernels on D^H V and multiplies
// row i of their result by phi_i.  The same identity leaves the refinement's stopping
// test unchanged: residual and solution norms are invariant under D.
//
// phi is a prefix product of unit complex numbers u_i = conj(e_{i-1}) / |e_{i-1}|
// (u_0 = 1).  It is formed as a three-level scan (4 rows serially per thread, the
// block's 256 threads by warp shuffles, the blocks' products by one scanning block), so
// the tree adds at most about 30 rounded complex products to each phi_i; but phi_i also
// carries the rounding errors of all u_j, j <= i (a few units each).  Their phases add
// up as a random walk (about sqrt(i) units: the result's error is 1.2e-13 at N = 2^20,
// measured), and their moduli would drift further, so phi_i is renormalised to unit
// modulus (without it the error was 4e-11 at N = 2^20).  For a real e every factor is
// exactly +-1 (products of +-1 and 0 imaginary parts are exact), so the result is then
// bit-identical to that of the real-off-diagonal path on the same data.
#include "tridiag.cuh"

#include <cuda_runtime.h>
#include <stdint.h>

namespace expm {
namespace {

constexpr int HB_THREADS = 256;
constexpr int HB_ROWS = 4;                        // rows per thread
constexpr int HB_SPAN = HB_THREADS * HB_ROWS;     // rows per block
constexpr int HT_THREADS = 1024;                  // the blocks' scan: one block

struct C2 {
    double re, im;
};
__device__ __forceinline__ C2 cmul(C2 a, C2 b) { return C2{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ C2 shfl_up(C2 a, int k) {
    return C2{__shfl_up_sync(0xffffffffu, a.re, k), __shfl_up_sync(0xffffffffu, a.im, k)};
}

// u_i for row i (conj(e_{i-1}) / |e_{i-1}|; 1 for row 0 and rows past the end), writing
// |e_{i-1}| when eabs is given
__device__ __forceinline__ C2 unit_of(const double *__restrict__ e, int64_t N, int64_t i, double *__restrict__ eabs) {
    if (i < 1 || i >= N) return C2{1.0, 0.0};
    const double re = e[2 * (i - 1)], im = e[2 * (i - 1) + 1];
    const double h = hypot(re, im);
    if (eabs) eabs[i - 1] = h;
    if (h == 0.0) return C2{1.0, 0.0};
    return C2{re / h, -im / h};  // divisions: a real e gives exactly +-1
}

// inclusive scan (product) of one value per thread over a block of HB_THREADS or
// HT_THREADS threads; returns the thread's exclusive prefix and the block total
template <int NT>
__device__ __forceinline__ C2 block_exclusive(C2 v, C2 *total) {
    __shared__ C2 warp_tot[NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    C2 inc = v;
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        const C2 o = shfl_up(inc, k);
        if (lane >= k) inc = cmul(o, inc);
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        C2 t = lane < NT / 32 ? warp_tot[lane] : C2{1.0, 0.0};
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const C2 o = shfl_up(t, k);
            if (lane >= k) t = cmul(o, t);
        }
        if (lane < NT / 32) warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    C2 exc = shfl_up(inc, 1);
    if (lane == 0) exc = C2{1.0, 0.0};
    if (w > 0) exc = cmul(warp_tot[w - 1], exc);
    *total = warp_tot[NT / 32 - 1];
    __syncthreads();  // warp_tot is reused by the next call
    return exc;
}

// per block of HB_SPAN rows: the product of its u_i (and |e| for its rows)
__global__ void __launch_bounds__(HB_THREADS) herm_block_prod(const double *__restrict__ e, int64_t N,
                                                              double *__restrict__ eabs, double *__restrict__ part) {
    const int64_t r0 = (int64_t)blockIdx.x * HB_SPAN + (int64_t)threadIdx.x * HB_ROWS;
    C2 p{1.0, 0.0};
#pragma unroll
    for (int j = 0; j < HB_ROWS; ++j) p = cmul(p, unit_of(e, N, r0 + j, eabs));
    C2 tot;
    block_exclusive<HB_THREADS>(p, &tot);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = tot.re;
        part[2 * blockIdx.x + 1] = tot.im;
    }
}

// exclusive scan of the nb block products, in place (one block)
__global__ void __launch_bounds__(HT_THREADS) herm_top_scan(double *__restrict__ part, int nb) {
    const int seg = (nb + HT_THREADS - 1) / HT_THREADS;
    const int b0 = threadIdx.x * seg, b1 = min(nb, b0 + seg);
    C2 p{1.0, 0.0};
    for (int b = b0; b < b1; ++b) p = cmul(p, C2{part[2 * b], part[2 * b + 1]});
    C2 tot;
    C2 run = block_exclusive<HT_THREADS>(p, &tot);
    for (int b = b0; b < b1; ++b) {
        const C2 v{part[2 * b], part[2 * b + 1]};
        part[2 * b] = run.re;
        part[2 * b + 1] = run.im;
        run = cmul(run, v);
    }
}

// phi_i for every row: the block's prefix times the in-block prefix, renormalised
__global__ void __launch_bounds__(HB_THREADS) herm_phase(const double *__restrict__ e, int64_t N,
                                                         const double *__restrict__ part, double *__restrict__ phi) {
    const int64_t r0 = (int64_t)blockIdx.x * HB_SPAN + (int64_t)threadIdx.x * HB_ROWS;
    C2 u[HB_ROWS];
    C2 p{1.0, 0.0};
#pragma unroll
    for (int j = 0; j < HB_ROWS; ++j) {
        u[j] = unit_of(e, N, r0 + j, nullptr);
        p = cmul(p, u[j]);
    }
    C2 tot;
    C2 run = cmul(C2{part[2 * blockIdx.x], part[2 * blockIdx.x + 1]}, block_exclusive<HB_THREADS>(p, &tot));
#pragma unroll
    for (int j = 0; j < HB_ROWS; ++j) {
        run = cmul(run, u[j]);
        if (r0 + j < N) {
            const double m = hypot(run.re, run.im);
            phi[2 * (r0 + j)] = run.re / m;
            phi[2 * (r0 + j) + 1] = run.im / m;
        }
    }
}

// Out[i, c] = s(phi_i) X[i, c] over N rows of r columns; s = conj when conj_phi; X real
// (x_cplx == 0, r doubles per row) or complex; Out complex.  Out may equal X when X is
// complex (each element is read before it is written by the same thread).
__global__ void __launch_bounds__(256) herm_scale_rows(const double *__restrict__ phi, int64_t N, int r,
                                                       const double *X, int x_cplx, double *Out, int conj_phi) {
    const int64_t total = N * (int64_t)r;
    const double sg = conj_phi ? -1.0 : 1.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / r;
        const double pr = phi[2 * i], pi = sg * phi[2 * i + 1];
        double xr, xi;
        if (x_cplx) {
            xr = X[2 * k];
            xi = X[2 * k + 1];
        } else {
            xr = X[k];
            xi = 0.0;
        }
        Out[2 * k] = pr * xr - pi * xi;
        Out[2 * k + 1] = pr * xi + pi * xr;
    }
}

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

size_t herm_scratch_bytes(int64_t N, int r) {
    const int64_t nb = (N + HB_SPAN - 1) / HB_SPAN;
    return al256(sizeof(double) * (size_t)N) + al256(2 * sizeof(double) * (size_t)N) +
           al256(2 * sizeof(double) * (size_t)N * r) + al256(2 * sizeof(double) * (size_t)nb);
}

HermWork herm_carve(void *scratch, int64_t N, int r) {
    unsigned char *m = (unsigned char *)scratch;
    HermWork w;
    w.eabs = (double *)m;
    m += al256(sizeof(double) * (size_t)N);
    w.phi = (double *)m;
    m += al256(2 * sizeof(double) * (size_t)N);
    w.Vp = (double *)m;
    m += al256(2 * sizeof(double) * (size_t)N * r);
    w.part = (double *)m;
    return w;
}

size_t herm_part_bytes(int64_t N) { return 2 * sizeof(double) * (size_t)((N + HB_SPAN - 1) / HB_SPAN); }

cudaError_t herm_phases(int64_t N, const double *e, double *eabs, double *phi, double *part, cudaStream_t st) {
    const int64_t nb = (N + HB_SPAN - 1) / HB_SPAN;
    if (nb > (int64_t)1 << 30) return cudaErrorInvalidValue;
    herm_block_prod<<<(unsigned)nb, HB_THREADS, 0, st>>>(e, N, eabs, part);
    herm_top_scan<<<1, HT_THREADS, 0, st>>>(part, (int)nb);
    herm_phase<<<(unsigned)nb, HB_THREADS, 0, st>>>(e, N, part, phi);
    return cudaGetLastError();
}

cudaError_t herm_scale(int64_t N, int r, const double *phi, const double *X, int x_cplx, double *Out, int conj_phi,
                       int sm_count, cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>((N * r + 255) / 256, (int64_t)sm_count * 8);
    herm_scale_rows<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(phi, N, r, X, x_cplx, Out, conj_phi);
    return cudaGetLastError();
}

cudaError_t herm_prepare(int64_t N, const double *e, const double *V, int r, int v_cplx, const HermWork &w,
                         int sm_count, cudaStream_t st) {
    cudaError_t err = herm_phases(N, e, w.eabs, w.phi, w.part, st);
    if (err == cudaSuccess) err = herm_scale(N, r, w.phi, V, v_cplx, w.Vp, 1, sm_count, st);
    return err;
}

cudaError_t herm_finish(int64_t N, int r, const HermWork &w, double *Y, int sm_count, cudaStream_t st) {
    return herm_scale(N, r, w.phi, Y, 1, Y, 0, sm_count, st);
}

}  // namespace expm
