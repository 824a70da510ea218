// dense.cu -- pole-batched dense path: exp(tA)V ~ e^c sum_k a_k (tA - cI + theta_k I)^{-1} V.
//
// Eqs. ExpoMatRat / expAx of the paper with one unpivoted LU per conjugate pole
// pair.  Real A and real V: only the Im(theta) > 0 member of each pair is solved and
// the sum is 2 Re(a X) (Remark 5.1).  Complex Hermitian A: the conjugate pole's
// matrix is the conjugate transpose, tA - cI + conj(theta) I = (tA - cI + theta I)^H
// = U^H L^H, so one factorization serves both poles of a pair.
//
// Precision (opts.prec):
//   binary64      factor, solve and sum in binary64;
//   mixed         factor and solve in binary32; the solution is kept in binary64 and
//                 refined with binary64 residuals R = V - (tA - cI + theta I) X until
//                 ||R||_F <= tol (||tA||_F + |theta - c|) ||X||_F or max_refine sweeps;
//                 the residue sum is binary64.
//
// Blocked right-looking LU, panel width DN_NB, per step: diagonal-block LU,
// the two panel triangular solves, and the trailing update as a batched complex
// GEMM (all pole pairs in one launch).  Triangular solves with more than 8 columns
// multiply each 128-row diagonal panel by its explicit inverse (formed once per
// factorization, all panels of all factors as one batch) and update the rows past the
// panel with one batched GEMM; up to 8 columns, one fused kernel per system.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <vector>

#include "arith.cuh"
#include "dense.cuh"
#include "oz_gemm.cuh"
#include "dense_kernels.cuh"
#include "plan.cuh"
#include "tc_gemm.cuh"

namespace expm {

// ------------------------------------------------------------------ small kernels

// X[z] (n x kc, cx<T>) = V of instance z / per_inst as complex; V real (v_cplx = 0)
// or complex (v_cplx = 1).
template <class T>
__global__ void load_rhs(int n, int kc, DenseIO io, int per_inst, cx<T> *X, int64_t xstride) {
    const int z = blockIdx.z;
    const double *V = io.V + (int64_t)(z / per_inst) * io.vstride * (io.v_cplx ? 2 : 1);
    const int64_t total = (int64_t)n * kc;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / kc, j = idx % kc;
        cx<T> v;
        if (io.v_cplx) v = {(T)V[2 * (i * io.ldv + j)], (T)V[2 * (i * io.ldv + j) + 1]};
        else v = {(T)V[i * io.ldv + j], (T)0};
        X[(int64_t)z * xstride + idx] = v;
    }
}

// R[z] = V - (theta_sys - c) X[z]   (the diagonal part of the residual; the tA X part
// is subtracted by a GEMM afterwards).  z = instance * nsys + sys.
__global__ void residual_diag(int n, int kc, DenseIO io, int nsys, const cx<double> *X, cx<double> *R, int64_t stride,
                              DenseSystems sys, const int *skip) {
    if (skip != nullptr && *skip) return;
    const int z = blockIdx.z;
    const int b = z % nsys;
    const double *V = io.V + (int64_t)(z / nsys) * io.vstride * (io.v_cplx ? 2 : 1);
    const cx<double> sh = {sys.th_re[b] - sys.cshift, sys.th_im[b]};
    const int64_t total = (int64_t)n * kc;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / kc, j = idx % kc;
        cx<double> v;
        if (io.v_cplx) v = {V[2 * (i * io.ldv + j)], V[2 * (i * io.ldv + j) + 1]};
        else v = {V[i * io.ldv + j], 0.0};
        R[(int64_t)z * stride + idx] = v - sh * X[(int64_t)z * stride + idx];
    }
}

// R[z] -= (theta_b - c) D[z]: the diagonal part of the residual update for a correction D
// (binary32) that has just been added to X
__global__ void residual_diag_step(int64_t total, int nsys, cx<double> *R, const cx<float> *D, int64_t stride,
                                   DenseSystems sys) {
    const int z = blockIdx.z, b = z % nsys;
    const cx<double> sh = {sys.th_re[b] - sys.cshift, sys.th_im[b]};
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const cx<float> d = D[(int64_t)z * stride + idx];
        cx<double> &r = R[(int64_t)z * stride + idx];
        r = r - sh * cx<double>{(double)d.re, (double)d.im};
    }
}

// Xc (binary32) = R (binary64) and sums of |R|^2, |X|^2 per batch entry
__global__ void demote_and_norms(int64_t total, const cx<double> *R, const cx<double> *X, cx<float> *Xc,
                                 int64_t stride, double *rn2, double *xn2, const int *skip) {
    if (skip != nullptr && *skip) return;
    const int b = blockIdx.z;
    double r2 = 0.0, x2 = 0.0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const cx<double> r = R[(int64_t)b * stride + idx];
        const cx<double> x = X[(int64_t)b * stride + idx];
        Xc[(int64_t)b * stride + idx] = {(float)r.re, (float)r.im};
        r2 += r.re * r.re + r.im * r.im;
        x2 += x.re * x.re + x.im * x.im;
    }
    for (int o = 16; o > 0; o >>= 1) {
        r2 += __shfl_xor_sync(0xffffffffu, r2, o);
        x2 += __shfl_xor_sync(0xffffffffu, x2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(rn2 + b, r2);
        atomicAdd(xn2 + b, x2);
    }
}

// X (binary64) += D (binary32 correction)
__global__ void add_correction(int64_t total, const cx<float> *D, cx<double> *X, int64_t stride, const int *skip) {
    if (skip != nullptr && *skip) return;
    const int b = blockIdx.z;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const cx<float> d = D[(int64_t)b * stride + idx];
        cx<double> &x = X[(int64_t)b * stride + idx];
        x.re += (double)d.re;
        x.im += (double)d.im;
    }
}

// Device-side stopping test after sweep `it` (devctl): per instance the largest
// ||R||_F / ((||tA||_F + |theta - c|) ||X||_F) over its systems; all <= tol sets *done.
// One block; z = instance * nsys + system.
__global__ void refine_check(int ninst, int nsys, const double *rn2, const double *xn2, const double *an2, double t,
                             DenseSystems sys, double tol, int it, int *done, int *iters, double *inst_resid) {
    if (*done) return;
    int bad = 0;
    for (int inst = threadIdx.x; inst < ninst; inst += blockDim.x) {
        double worst = 0.0;
        for (int b = 0; b < nsys; ++b) {
            const int z = inst * nsys + b;
            const double shift = hypot(sys.th_re[b] - sys.cshift, sys.th_im[b]);
            const double den = (sqrt(an2[inst]) * fabs(t) + shift) * sqrt(xn2[z]);
            const double rel = den > 0.0 ? sqrt(rn2[z]) / den : 0.0;
            worst = fmax(worst, rel);
            if (!(rel <= tol)) bad = 1;
        }
        inst_resid[inst] = worst;
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        *iters = it - 1;
        if (!bad) *done = 1;
    }
}

// Per instance the largest growth max|U| / max|M| over its pairs (devctl); one block.
__global__ void growth_dev(int ninst, int npairs, const unsigned *amax, const unsigned *umax, double *inst_growth) {
    for (int inst = threadIdx.x; inst < ninst; inst += blockDim.x) {
        double gmax = 0.0;
        for (int s = 0; s < npairs; ++s) {
            const float a = __uint_as_float(amax[inst * npairs + s]), u = __uint_as_float(umax[inst * npairs + s]);
            if (a > 0.f) gmax = fmax(gmax, (double)u / (double)a);
        }
        inst_growth[inst] = gmax;
    }
}

// Residue-weighted sum (a8) per instance z: Y = sum_sys W_sys X[z, sys], real part
// only when y_real.  The sum over systems is taken in a fixed order per element.
__global__ void accumulate(int n, int kc, int nsys, const cx<double> *__restrict__ X, int64_t stride,
                           DenseSystems sys, DenseIO io) {
    const int z = blockIdx.z;
    double *Y = io.Y + (int64_t)z * io.ystride * (io.y_real ? 1 : 2);
    const int64_t total = (int64_t)n * kc;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / kc, j = idx % kc;
        cx<double> acc = {0.0, 0.0};
        for (int b = 0; b < nsys; ++b) {
            const cx<double> w = {sys.w_re[b], sys.w_im[b]};
            acc = acc + w * X[((int64_t)z * nsys + b) * stride + idx];
        }
        if (io.y_real) Y[i * io.ldy + j] = acc.re;
        else {
            Y[2 * (i * io.ldy + j)] = acc.re;
            Y[2 * (i * io.ldy + j) + 1] = acc.im;
        }
    }
}

// sum of |A_ij|^2 (binary64) of instance z into out[z]
__global__ void frob2(int n, const double *__restrict__ A, int64_t lda, int64_t astride, int cplx, double *out) {
    A += (int64_t)blockIdx.z * astride * (cplx ? 2 : 1);
    out += blockIdx.z;
    double acc = 0.0;
    // rows blockIdx.x, blockIdx.x + gridDim.x, ...; threads over the columns
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        if (cplx) {
            const double re = A[2 * (i * lda + j)], im = A[2 * (i * lda + j) + 1];
            acc += re * re + im * im;
        } else {
            const double v = A[i * lda + j];
            acc += v * v;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// Operands of the tensor-core trailing update C -= L21 U12 (complex, binary32), laid out
// for the real K-major product C_real -= A' B'^T with the 3xTF32 split:
//   L21 (rest x nb complex) is the real rest x 2nb matrix A (re, im interleaved);
//   U12 (nb x rest complex) becomes the real 2rest x 2nb matrix BT with rows
//       BT[2j] = (.. ur_kj, -ui_kj ..),  BT[2j+1] = (.. ui_kj, ur_kj ..),
//   so that (A BT^T)[i][2j] = Re(L21 U12)_ij and [i][2j+1] = Im(L21 U12)_ij;
//   A' = [A_lo | A_hi | A_hi] and B' = [BT_hi | BT_lo | BT_hi] (K = 6 nb), with x_hi
//   x rounded to TF32 and x_lo = x - x_hi (exact in binary32).  The small products come
//   first along K: the tensor cores' fp32 accumulation truncates, so each addition loses
//   up to an ulp of the running sum, and the running sum is kept small while the small
//   terms go in.
// Batch z of A' occupies rows z*rest_a .. of a stacked matrix, likewise B' (2 rest rows).
EXPM_D float tf32_hi(float x) { return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u); }

__global__ void split_tc_operands(int rest, int nb, const cx<float> *__restrict__ F, int n, int64_t fstride,
                                  float *__restrict__ Ap, float *__restrict__ Bp) {
    const int z = blockIdx.z;
    const cx<float> *L21 = F + (int64_t)z * fstride + (int64_t)nb * n;  // relative to the diagonal block
    const cx<float> *U12 = F + (int64_t)z * fstride + nb;
    const int K6 = 6 * nb;
    const int64_t na = (int64_t)rest * nb;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < na; idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / nb), k = (int)(idx % nb);
        const cx<float> a = L21[(int64_t)i * n + k];
        float *row = Ap + ((int64_t)z * rest + i) * K6;
        const float hr = tf32_hi(a.re), hi = tf32_hi(a.im);
        row[2 * k] = a.re - hr;        row[2 * k + 1] = a.im - hi;
        row[2 * nb + 2 * k] = hr;      row[2 * nb + 2 * k + 1] = hi;
        row[4 * nb + 2 * k] = hr;      row[4 * nb + 2 * k + 1] = hi;
        // the U12 entry (k, i) of the same index range (rest x nb pairs, transposed)
        const cx<float> u = U12[(int64_t)k * n + i];
        float *r0 = Bp + ((int64_t)z * 2 * rest + 2 * i) * K6;
        float *r1 = r0 + K6;
        const float ur = u.re, ui = -u.im, uh = tf32_hi(ur), vh = tf32_hi(ui);
        // row 2j: (ur, -ui); row 2j+1: (ui, ur)
        r0[2 * k] = uh;                r0[2 * k + 1] = vh;
        r0[2 * nb + 2 * k] = ur - uh;  r0[2 * nb + 2 * k + 1] = ui - vh;
        r0[4 * nb + 2 * k] = uh;       r0[4 * nb + 2 * k + 1] = vh;
        const float wr = u.im, wh = tf32_hi(wr);
        r1[2 * k] = wh;                r1[2 * k + 1] = uh;
        r1[2 * nb + 2 * k] = wr - wh;  r1[2 * nb + 2 * k + 1] = ur - uh;
        r1[4 * nb + 2 * k] = wh;       r1[4 * nb + 2 * k + 1] = uh;
    }
}

// The same update with the bf16x3 split: x = h + m + l, each part bf16 (h = bf16(x),
// m = bf16(x - h), l = bf16(x - h - m); the differences are exact in binary32), 24 bits
// in all.  A' = [A_l | A_m | A_h | A_m | A_h | A_h] and B' = [BT_h | BT_m | BT_l | BT_h |
// BT_m | BT_h] (K = 12 nb), so A' B'^T sums the six products with p + q <= 2, the
// smallest first (see the TF32 split above).
EXPM_D uint16_t bf16_rn_bits(float x) {  // round to nearest even (finite x)
    const unsigned u = __float_as_uint(x);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}
EXPM_D float bf16_val(uint16_t b) { return __uint_as_float((unsigned)b << 16); }
EXPM_D void bf16x3(float x, uint16_t &h, uint16_t &m, uint16_t &l) {
    h = bf16_rn_bits(x);
    const float r1 = __fsub_rn(x, bf16_val(h));
    m = bf16_rn_bits(r1);
    l = bf16_rn_bits(__fsub_rn(r1, bf16_val(m)));
}

__global__ void split_tc_operands_bf16(int rest, int nb, const cx<float> *__restrict__ F, int n, int64_t fstride,
                                       uint16_t *__restrict__ Ap, uint16_t *__restrict__ Bp) {
    const int z = blockIdx.z;
    const cx<float> *L21 = F + (int64_t)z * fstride + (int64_t)nb * n;
    const cx<float> *U12 = F + (int64_t)z * fstride + nb;
    const int K12 = 12 * nb, w = 2 * nb;  // one segment: nb complex = 2 nb values
    const int64_t na = (int64_t)rest * nb;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < na; idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / nb), k = (int)(idx % nb);
        const cx<float> a = L21[(int64_t)i * n + k];
        uint16_t rh, rm, rl, ih, im, il;
        bf16x3(a.re, rh, rm, rl);
        bf16x3(a.im, ih, im, il);
        uint16_t *row = Ap + ((int64_t)z * rest + i) * K12 + 2 * k;
        const uint16_t segr[6] = {rl, rm, rh, rm, rh, rh}, segi[6] = {il, im, ih, im, ih, ih};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            row[q * w] = segr[q];
            row[q * w + 1] = segi[q];
        }
        // U12 entry (k, i): rows 2i (Re output: (ur, -ui)) and 2i+1 (Im output: (ui, ur))
        const cx<float> u = U12[(int64_t)k * n + i];
        uint16_t uh, um, ul, vh, vm, vl, wh, wm, wl;
        bf16x3(u.re, uh, um, ul);
        bf16x3(-u.im, vh, vm, vl);
        bf16x3(u.im, wh, wm, wl);
        uint16_t *r0 = Bp + ((int64_t)z * 2 * rest + 2 * i) * K12 + 2 * k;
        uint16_t *r1 = r0 + K12;
        const uint16_t s0r[6] = {uh, um, ul, uh, um, uh}, s0i[6] = {vh, vm, vl, vh, vm, vh};
        const uint16_t s1r[6] = {wh, wm, wl, wh, wm, wh}, s1i[6] = {uh, um, ul, uh, um, uh};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            r0[q * w] = s0r[q];
            r0[q * w + 1] = s0i[q];
            r1[q * w] = s1r[q];
            r1[q * w + 1] = s1i[q];
        }
    }
}

// Operands of a triangular-solve update X[r0 .. r0+m) -= op(F)[r0.., k0 .. k0+K) X[k0 .. k0+K)
// on the tensor cores with the bf16x3 split (same segment order as above).  A' rows
// i < m: op(F) = F (conj = false) or the conjugate transpose of F (conj = true: entry
// (i, k) is conj F[k0+k][r0+i]), K-major, 12 K bf16 per row; batch z at Ap + z m 12K.
__global__ void split_solve_a_bf16(int m, int K, const cx<float> *__restrict__ F, int n, int64_t fstride, int r0,
                                   int k0, int conj, uint16_t *__restrict__ Ap) {
    const int z = blockIdx.z;
    const cx<float> *f = F + (int64_t)z * fstride;
    const int K12 = 12 * K;
    const int64_t na = (int64_t)m * K;
    // consecutive threads write consecutive (re, im) pairs of a row (one 4-byte store per
    // segment); the transposed reads of the conjugate case are the strided side
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < na; idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / K), k = (int)(idx % K);
        cx<float> a = conj ? f[(int64_t)(k0 + k) * n + r0 + i] : f[(int64_t)(r0 + i) * n + k0 + k];
        if (conj) a.im = -a.im;
        uint16_t rh, rm, rl, ih, im, il;
        bf16x3(a.re, rh, rm, rl);
        bf16x3(a.im, ih, im, il);
        uint32_t *row = reinterpret_cast<uint32_t *>(Ap + ((int64_t)z * m + i) * K12 + 2 * k);
        const uint16_t segr[6] = {rl, rm, rh, rm, rh, rh}, segi[6] = {il, im, ih, im, ih, ih};
#pragma unroll
        for (int q = 0; q < 6; ++q) row[q * K] = (uint32_t)segr[q] | ((uint32_t)segi[q] << 16);
    }
}

// B' of that update from X rows k0 .. k0+K (kc complex columns, batch stride xstride):
// row 2c (real output): (Re x, -Im x), row 2c+1 (imaginary output): (Im x, Re x); batch z
// at Bp + z 2kc 12K.
__global__ void split_solve_b_bf16(int K, int kc, const cx<float> *__restrict__ X, int64_t xstride, int k0,
                                   uint16_t *__restrict__ Bp) {
    const int z = blockIdx.z;
    const cx<float> *x = X + (int64_t)z * xstride;
    const int K12 = 12 * K;
    const int64_t na = (int64_t)K * kc;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < na; idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / K), k = (int)(idx % K);  // consecutive threads: consecutive k of a row
        const cx<float> u = x[(int64_t)(k0 + k) * kc + c];
        uint16_t uh, um, ul, vh, vm, vl, wh, wm, wl;
        bf16x3(u.re, uh, um, ul);
        bf16x3(-u.im, vh, vm, vl);
        bf16x3(u.im, wh, wm, wl);
        uint32_t *r0 = reinterpret_cast<uint32_t *>(Bp + ((int64_t)z * 2 * kc + 2 * c) * K12 + 2 * k);
        uint32_t *r1 = r0 + K12 / 2;
        const uint16_t s0r[6] = {uh, um, ul, uh, um, uh}, s0i[6] = {vh, vm, vl, vh, vm, vh};
        const uint16_t s1r[6] = {wh, wm, wl, wh, wm, wh}, s1i[6] = {uh, um, ul, uh, um, uh};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            r0[q * K] = (uint32_t)s0r[q] | ((uint32_t)s0i[q] << 16);
            r1[q * K] = (uint32_t)s1r[q] | ((uint32_t)s1i[q] << 16);
        }
    }
}

// ------------------------------------------------------------------ host helpers

static unsigned grid1d(int64_t total, int threads = 256) {
    int64_t g = (total + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

template <class K> static cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define EXPM_TRY(x)                               \
    do {                                          \
        cudaError_t _e = (x);                     \
        if (_e != cudaSuccess) return _e;         \
    } while (0)

// Tensor-core scratch of the trailing update (binary32 LU with the TF32 split).
struct TcScratch {
    float *Ap = nullptr, *Bp = nullptr;  // bf16 operands in the same bytes when bf16
    int *err = nullptr;
    bool bf16 = false;
};

constexpr int DN_PNB = 4 * DN_NB;  // outer panel of the tensor-core LU

// C_z -= A_z B_z^T for z < batch (A_z: M x K, B_z: N x K, K-major with ld K; batch
// strides in elements) on the tensor cores: one launch when the strides meet the TMA
// rules, else one launch per product.
static cudaError_t tc_update(bool bf16, int M, int N, int K, const void *A, int64_t sA, const void *B, int64_t sB,
                             float *C, int ldc, int64_t sC, int batch, int *err, cudaStream_t st) {
    if (tc_gemm_supported(M, N, K, A, K, B, K, C, ldc, bf16, sA, sB, sC))
        return tc_gemm_batched(bf16, M, N, K, A, K, sA, B, K, sB, C, ldc, sC, batch, err, st);
    const size_t es = bf16 ? 2 : 4;
    for (int z = 0; z < batch; ++z) {
        const void *Az = (const unsigned char *)A + (size_t)z * sA * es;
        const void *Bz = (const unsigned char *)B + (size_t)z * sB * es;
        cudaError_t e = tc_gemm_batched(bf16, M, N, K, Az, K, 0, Bz, K, 0, C + (int64_t)z * sC, ldc, 0, 1, err, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Binary32 LU with the trailing updates on the tensor cores (bf16x3), in 256-column outer panels:
// inside a panel, 64-column steps (diagonal LU, L21 for every row below, U12 and the
// update restricted to the panel's columns, on the CUDA cores); then the panel's row
// block to the right, U12 = L11^{-1} A12, by the same 64-row steps, and one trailing
// update A22 -= L21 U12 with K = 256 complex on the tensor cores -- a 128 x 128 C tile
// is read and written once per 256 columns instead of once per 64, which bounds these
// updates (the tile traffic, not the tensor pipe).
static cudaError_t lu_panels_tc(int n, int batch, cx<float> *F, cudaStream_t st, Profiler &prof,
                                const TcScratch *tc) {
    const int64_t bs = (int64_t)n * n;
    const size_t sm1 = tri_smem_bytes<float>(), sm2 = 2 * tri_smem_bytes<float>();
    EXPM_TRY(set_smem(lu_diag<float>, sm1));
    EXPM_TRY(set_smem(trsm_left<float, true, true, false>, sm2));
    EXPM_TRY(set_smem(trsm_right_upper<float>, sm2));
    const cx<float> mone = {-1.f, 0.f};
    for (int p0 = 0; p0 < n; p0 += DN_PNB) {
        const int pe = std::min(n, p0 + DN_PNB), pw = pe - p0;
        for (int p = p0; p < pe; p += DN_NB) {
            const int nb = std::min(DN_NB, pe - p);
            const int below = n - p - nb, inpanel = pe - p - nb;
            cx<float> *diag = F + (int64_t)p * n + p;
            EXPM_TRY(prof.timed("lu_diag<f32>", st, [&] {
                lu_diag<float><<<dim3(1, 1, batch), 256, sm1, st>>>(nb, diag, n, bs);
                return cudaGetLastError();
            }));
            if (below <= 0) break;
            EXPM_TRY(prof.timed("trsm_panels<f32>", st, [&] {
                trsm_right_upper<float><<<dim3((below + 63) / 64, 1, batch), 64, sm2, st>>>(
                    nb, below, diag, n, bs, diag + (int64_t)nb * n, n, bs);
                if (inpanel > 0)
                    trsm_left<float, true, true, false><<<dim3((inpanel + 63) / 64, 1, batch), 64, sm2, st>>>(
                        nb, inpanel, diag, n, bs, diag + nb, n, bs);
                return cudaGetLastError();
            }));
            if (inpanel > 0)
                EXPM_TRY(prof.timed("cgemm_update<f32>", st, [&] {
                    cgemm_launch<float, cx<float>, false, false>(below, inpanel, nb, mone, 1.f, diag + (int64_t)nb * n,
                                                                 n, bs, diag + nb, n, bs, diag + (int64_t)nb * n + nb,
                                                                 n, bs, 1, batch, st);
                    return cudaGetLastError();
                }));
        }
        const int right = n - pe;
        if (right <= 0) continue;
        for (int p = p0; p < pe; p += DN_NB) {  // U12 = L11^{-1} A12 for the panel's rows
            const int nb = std::min(DN_NB, pe - p);
            cx<float> *diag = F + (int64_t)p * n + p;
            cx<float> *a12 = F + (int64_t)p * n + pe;
            EXPM_TRY(prof.timed("trsm_panels<f32>", st, [&] {
                trsm_left<float, true, true, false><<<dim3((right + 63) / 64, 1, batch), 64, sm2, st>>>(
                    nb, right, diag, n, bs, a12, n, bs);
                return cudaGetLastError();
            }));
            if (pe - p - nb > 0)
                EXPM_TRY(prof.timed("cgemm_update<f32>", st, [&] {
                    cgemm_launch<float, cx<float>, false, false>(pe - p - nb, right, nb, mone, 1.f,
                                                                 diag + (int64_t)nb * n, n, bs, a12, n, bs,
                                                                 a12 + (int64_t)nb * n, n, bs, 1, batch, st);
                    return cudaGetLastError();
                }));
        }
        // A22 -= L21 U12 (K = pw complex) on the tensor cores, one real product per matrix
        cx<float> *pdiag = F + (int64_t)p0 * n + p0;
        float *C0 = reinterpret_cast<float *>(F + (int64_t)pe * n + pe);
        const int kr = (tc->bf16 ? 12 : 6) * pw;  // real K of the split product
        if (!tc_gemm_supported(right, 2 * right, kr, tc->Ap, kr, tc->Bp, kr, C0, 2 * n, tc->bf16)) {
            EXPM_TRY(prof.timed("cgemm_update<f32>", st, [&] {
                cgemm_launch<float, cx<float>, false, false>(right, right, pw, mone, 1.f, pdiag + (int64_t)pw * n, n,
                                                             bs, pdiag + pw, n, bs, pdiag + (int64_t)pw * n + pw, n,
                                                             bs, 1, batch, st);
                return cudaGetLastError();
            }));
            continue;
        }
        EXPM_TRY(prof.timed("split_tc_operands", st, [&] {
            if (tc->bf16)
                split_tc_operands_bf16<<<dim3(grid1d((int64_t)right * pw), 1, batch), 256, 0, st>>>(
                    right, pw, pdiag, n, bs, reinterpret_cast<uint16_t *>(tc->Ap), reinterpret_cast<uint16_t *>(tc->Bp));
            else
                split_tc_operands<<<dim3(grid1d((int64_t)right * pw), 1, batch), 256, 0, st>>>(right, pw, pdiag, n, bs,
                                                                                             tc->Ap, tc->Bp);
            return cudaGetLastError();
        }));
        EXPM_TRY(prof.timed(tc->bf16 ? "tc_gemm_bf16x3" : "tc_gemm_tf32x3", st, [&] {
            return tc_update(tc->bf16, right, 2 * right, kr, tc->Ap, (int64_t)right * kr, tc->Bp,
                             (int64_t)2 * right * kr, C0, 2 * n, 2 * bs, batch, tc->err, st);
        }));
    }
    return cudaSuccess;
}

// Unpivoted blocked LU of `batch` n x n matrices F (ld n, batch stride n*n).  With
// tc (binary32 only) the trailing updates run on the tensor cores.
template <class T>
static cudaError_t lu_blocked(int n, int batch, cx<T> *F, cudaStream_t st, Profiler &prof,
                              const TcScratch *tc = nullptr, int tile = 0) {
    // bf16x3 only: with 3xTF32 (twice the truncated accumulation steps per unit of K, 22
    // split bits instead of 24) the K = 256 updates cost a second refinement sweep
    // (measured), so 3xTF32 keeps the rank-64 updates
    if constexpr (std::is_same<T, float>::value)
        if (tc != nullptr && tc->bf16 && n > DN_PNB) return lu_panels_tc(n, batch, F, st, prof, tc);
    const int64_t bs = (int64_t)n * n;
    const size_t sm1 = tri_smem_bytes<T>(), sm2 = 2 * tri_smem_bytes<T>();
    EXPM_TRY(set_smem(lu_diag<T>, sm1));
    EXPM_TRY(set_smem(trsm_left<T, true, true, false>, sm2));
    EXPM_TRY(set_smem(trsm_right_upper<T>, sm2));
    const char *tag = sizeof(T) == 8 ? "f64" : "f32";
    (void)tag;
    for (int p = 0; p < n; p += DN_NB) {
        const int nb = std::min(DN_NB, n - p);
        const int rest = n - p - nb;
        cx<T> *diag = F + (int64_t)p * n + p;
        EXPM_TRY(prof.timed(sizeof(T) == 8 ? "lu_diag<f64>" : "lu_diag<f32>", st, [&] {
            lu_diag<T><<<dim3(1, 1, batch), 256, sm1, st>>>(nb, diag, n, bs);
            return cudaGetLastError();
        }));
        if (rest <= 0) break;
        EXPM_TRY(prof.timed(sizeof(T) == 8 ? "trsm_panels<f64>" : "trsm_panels<f32>", st, [&] {
            // U12 = L11^{-1} A12 and L21 = A21 U11^{-1}
            trsm_left<T, true, true, false><<<dim3((rest + 63) / 64, 1, batch), 64, sm2, st>>>(
                nb, rest, diag, n, bs, diag + nb, n, bs);
            trsm_right_upper<T><<<dim3((rest + 63) / 64, 1, batch), 64, sm2, st>>>(nb, rest, diag, n, bs,
                                                                                 diag + (int64_t)nb * n, n, bs);
            return cudaGetLastError();
        }));
        if (tc != nullptr && tc->bf16 && sizeof(T) == 4 && rest >= 128 &&
            tc_gemm_supported(rest, 2 * rest, 12 * nb, tc->Ap, 12 * nb, tc->Bp, 12 * nb,
                              F + (int64_t)(p + nb) * n + p + nb, 2 * n, true)) {
            // A22 -= L21 U12 as one real product per matrix, bf16x3 split
            uint16_t *Ab = reinterpret_cast<uint16_t *>(tc->Ap), *Bb = reinterpret_cast<uint16_t *>(tc->Bp);
            EXPM_TRY(prof.timed("split_tc_operands", st, [&] {
                split_tc_operands_bf16<<<dim3(grid1d((int64_t)rest * nb), 1, batch), 256, 0, st>>>(
                    rest, nb, reinterpret_cast<const cx<float> *>(diag), n, bs, Ab, Bb);
                return cudaGetLastError();
            }));
            EXPM_TRY(prof.timed("tc_gemm_bf16x3", st, [&] {
                float *C0 = reinterpret_cast<float *>(F + (int64_t)(p + nb) * n + p + nb);
                return tc_update(true, rest, 2 * rest, 12 * nb, Ab, (int64_t)rest * 12 * nb, Bb,
                                 (int64_t)2 * rest * 12 * nb, C0, 2 * n, 2 * bs, batch, tc->err, st);
            }));
            continue;
        }
        if (tc != nullptr && !tc->bf16 && sizeof(T) == 4 && rest >= 128 &&
            tc_gemm_supported(rest, 2 * rest, 6 * nb, tc->Ap, 6 * nb, tc->Bp, 6 * nb,
                              F + (int64_t)(p + nb) * n + p + nb, 2 * n)) {
            // A22 -= L21 U12 as one real product per matrix on the tensor cores
            EXPM_TRY(prof.timed("split_tc_operands", st, [&] {
                split_tc_operands<<<dim3(grid1d((int64_t)rest * nb), 1, batch), 256, 0, st>>>(
                    rest, nb, reinterpret_cast<const cx<float> *>(diag), n, bs, tc->Ap, tc->Bp);
                return cudaGetLastError();
            }));
            EXPM_TRY(prof.timed("tc_gemm_tf32x3", st, [&] {
                float *C0 = reinterpret_cast<float *>(F + (int64_t)(p + nb) * n + p + nb);
                return tc_update(false, rest, 2 * rest, 6 * nb, tc->Ap, (int64_t)rest * 6 * nb, tc->Bp,
                                 (int64_t)2 * rest * 6 * nb, C0, 2 * n, 2 * bs, batch, tc->err, st);
            }));
            continue;
        }
        EXPM_TRY(prof.timed(sizeof(T) == 8 ? "cgemm_update<f64>" : "cgemm_update<f32>", st, [&] {
            // A22 -= L21 U12
            cgemm_launch<T, cx<T>, false, false>(rest, rest, nb, cx<T>{T(-1), T(0)}, T(1), diag + (int64_t)nb * n, n,
                                                 bs, diag + nb, n, bs, diag + (int64_t)nb * n + nb, n, bs, 1, batch,
                                                 st, tile);
            return cudaGetLastError();
        }));
    }
    return cudaSuccess;
}

// Tensor-core scratch of the binary32 triangular solves (bf16x3 mode): the split operands
// of one panel update for every batch entry, and the kernel's time-out flag.
struct SolveTc {
    uint16_t *Ap = nullptr, *Bp = nullptr;
    int *err = nullptr;
};

// Explicit inverses of the diagonal panels for the wide solves: Inv[z][q][0] = L_q^{-1},
// Inv[z][q][1] = U_q^{-1} (B x B each, z the factor, q the panel), and the scratch T
// (batch x B x kc) that one panel's product goes through.
struct SolveInv {
    const void *inv = nullptr;
    void *T = nullptr;
    int B = 0, npan = 0;
};

// In-place solve of the kc columns of X[b] (n x kc) with the factors in F[b].
// conj = false: L U x = b (forward unit-lower, back upper).
// conj = true : U^H L^H x = b (forward with U^H, back with unit L^H).
// sweeps: 1 forward only, 2 backward only, 3 both.  With `inv`, each diagonal panel is
// applied as one product by its inverse (or the inverse's conjugate transpose);
// without it, as 64-row triangular solves and the updates inside the panel.
template <class T>
static cudaError_t lu_solve(int n, int kc, int batch, const cx<T> *F, int64_t fstride, bool conj, cx<T> *X,
                            int64_t xstride, cudaStream_t st, Profiler &prof, const int *skip = nullptr,
                            const SolveTc *tcs = nullptr, Profiler *parts = nullptr, const SolveInv *inv = nullptr,
                            int sweeps = 3) {
    const size_t smn = narrow_smem_bytes<T>(n, kc);
    if (sweeps == 3 && kc <= 8 && smn <= (200u << 10)) {  // few right-hand sides: one fused kernel per batch entry
        // the attribute is a ceiling, set to the largest size used so that concurrent
        // callers (server workers) never lower it under one another's launch
        EXPM_TRY(set_smem(lu_solve_narrow<T, false>, 200u << 10));
        EXPM_TRY(set_smem(lu_solve_narrow<T, true>, 200u << 10));
        return prof.timed(sizeof(T) == 8 ? "lu_solve<f64>" : "lu_solve<f32>", st, [&]() -> cudaError_t {
            if (conj) lu_solve_narrow<T, true><<<batch, 256, smn, st>>>(n, kc, F, fstride, X, xstride, skip);
            else lu_solve_narrow<T, false><<<batch, 256, smn, st>>>(n, kc, F, fstride, X, xstride, skip);
            return cudaGetLastError();
        });
    }
    if (skip != nullptr) return cudaErrorInvalidValue;  // device-side control needs the narrow kernel
    const size_t sm2 = 2 * tri_smem_bytes<T>();
    const int cb = (kc + 63) / 64;
    EXPM_TRY(set_smem(trsm_left<T, true, true, false>, sm2));
    EXPM_TRY(set_smem(trsm_left<T, false, false, false>, sm2));
    EXPM_TRY(set_smem(trsm_left<T, true, false, true>, sm2));
    EXPM_TRY(set_smem(trsm_left<T, false, true, true>, sm2));
    auto ones = cx<T>{T(-1), T(0)};
    // Two-level blocking: 64-row diagonal blocks (triangular solve, then the update of the
    // rest of their 256-row panel), and one update with K = 256 of everything past the
    // panel -- a quarter of the passes over X that rank-64 updates would make.
    constexpr int PNB = 4 * DN_NB;
    auto trsm = [&](int p, int nb, bool lower) {
        const cx<T> *dg = F + (int64_t)p * n + p;
        cx<T> *xp = X + (int64_t)p * kc;
        const dim3 grid(cb, 1, batch);
        if (lower) {
            if (!conj) trsm_left<T, true, true, false><<<grid, 64, sm2, st>>>(nb, kc, dg, n, fstride, xp, kc, xstride);
            else trsm_left<T, true, false, true><<<grid, 64, sm2, st>>>(nb, kc, dg, n, fstride, xp, kc, xstride);
        } else {
            if (!conj) trsm_left<T, false, false, false><<<grid, 64, sm2, st>>>(nb, kc, dg, n, fstride, xp, kc, xstride);
            else trsm_left<T, false, true, true><<<grid, 64, sm2, st>>>(nb, kc, dg, n, fstride, xp, kc, xstride);
        }
    };
    // X[r0 : r0+m] -= op(factor block rows r0.., columns k0 .. k0+K) X[k0 : k0+K], where the
    // block is L or U of the non-conjugate solve, or the conjugate transpose of U (forward)
    // or L (backward) of the conjugate one -- all read from the one stored factor
    auto update = [&](int r0, int m, int k0, int K) {
        cx<T> *xk = X + (int64_t)k0 * kc, *xr = X + (int64_t)r0 * kc;
        if (!conj)
            cgemm_launch<T, cx<T>, false, false>(m, kc, K, ones, T(1), F + (int64_t)r0 * n + k0, n, fstride, xk, kc,
                                                 xstride, xr, kc, xstride, 1, batch, st);
        else
            cgemm_launch<T, cx<T>, true, false>(m, kc, K, ones, T(1), F + (int64_t)k0 * n + r0, n, fstride, xk, kc,
                                                xstride, xr, kc, xstride, 1, batch, st);
    };
    // the K = 256 updates past a panel: on the tensor cores with the bf16x3 split when
    // scratch is given (binary32 only) and the shapes meet the TMA rules, else as above
    auto big_update = [&](int r0, int m, int k0, int K) -> cudaError_t {
        if constexpr (std::is_same<T, float>::value) {
            const int kr = 12 * K;
            float *C0 = reinterpret_cast<float *>(X + (int64_t)r0 * kc);
            if (tcs != nullptr && tc_gemm_supported(m, 2 * kc, kr, tcs->Ap, kr, tcs->Bp, kr, C0, 2 * kc, true)) {
                split_solve_a_bf16<<<dim3(grid1d((int64_t)m * K), 1, batch), 256, 0, st>>>(
                    m, K, F, n, fstride, r0, k0, conj ? 1 : 0, tcs->Ap);
                split_solve_b_bf16<<<dim3(grid1d((int64_t)K * kc), 1, batch), 256, 0, st>>>(K, kc, X, xstride, k0,
                                                                                         tcs->Bp);
                EXPM_TRY(cudaGetLastError());
                return tc_update(true, m, 2 * kc, kr, tcs->Ap, (int64_t)m * kr, tcs->Bp, (int64_t)2 * kc * kr, C0,
                                 2 * kc, 2 * xstride, batch, tcs->err, st);
            }
        }
        update(r0, m, k0, K);
        return cudaGetLastError();
    };
    // optional per-part timing (diagonal blocks, in-panel updates, updates past a panel)
    Profiler none;
    Profiler &pp = parts ? *parts : none;
    const bool f64 = sizeof(T) == 8;
    auto t_trsm = [&](int p, int nb, bool lower) {
        return pp.timed(f64 ? "solve_diag<f64>" : "solve_diag<f32>", st, [&] {
            trsm(p, nb, lower);
            return cudaGetLastError();
        });
    };
    auto t_update = [&](int r0, int m, int k0, int K) {
        return pp.timed(f64 ? "solve_panel_update<f64>" : "solve_panel_update<f32>", st, [&] {
            update(r0, m, k0, K);
            return cudaGetLastError();
        });
    };
    auto t_big = [&](int r0, int m, int k0, int K) {
        return pp.timed(f64 ? "solve_big_update<f64>" : "solve_big_update<f32>", st,
                        [&] { return big_update(r0, m, k0, K); });
    };
    if (inv != nullptr) {
        // X[p0 : pe] <- op(Inv_q) X[p0 : pe] through the scratch T.  Non-conjugate: forward
        // by L_q^{-1} (slot 0), backward by U_q^{-1} (slot 1); conjugate: forward by
        // (U_q^H)^{-1} = (U_q^{-1})^H, backward by (L_q^{-1})^H.  A padded panel's inverse
        // is block diagonal with the identity, so its leading nb x nb block is the inverse
        // of the panel itself.
        const int B = inv->B;
        const int64_t bb = (int64_t)B * B, dstride = (int64_t)inv->npan * 2 * bb;
        cx<T> *Ts = static_cast<cx<T> *>(inv->T);
        const cx<T> one{T(1), T(0)};
        auto apply = [&](int q, bool lower) -> cudaError_t {
            const int p0 = q * B, nb = std::min(B, n - p0);
            const cx<T> *D = static_cast<const cx<T> *>(inv->inv) + (int64_t)q * 2 * bb + ((lower != conj) ? 0 : bb);
            cx<T> *xp = X + (int64_t)p0 * kc;
            return pp.timed(f64 ? "solve_diag<f64>" : "solve_diag<f32>", st, [&]() -> cudaError_t {
                if (!conj)
                    cgemm_launch<T, cx<T>, false, false>(nb, kc, nb, one, T(0), D, B, dstride, xp, kc, xstride, Ts, kc,
                                                         (int64_t)B * kc, 1, batch, st);
                else
                    cgemm_launch<T, cx<T>, true, false>(nb, kc, nb, one, T(0), D, B, dstride, xp, kc, xstride, Ts, kc,
                                                        (int64_t)B * kc, 1, batch, st);
                EXPM_TRY(cudaGetLastError());
                const size_t w = (size_t)nb * kc * sizeof(cx<T>), dp = (size_t)xstride * sizeof(cx<T>),
                             sp = (size_t)B * kc * sizeof(cx<T>);
                if (dp <= (size_t)INT32_MAX)
                    return cudaMemcpy2DAsync(xp, dp, Ts, sp, w, (size_t)batch, cudaMemcpyDeviceToDevice, st);
                for (int z = 0; z < batch; ++z)  // pitches past the 2-D copy's limit: one copy per entry
                    EXPM_TRY(cudaMemcpyAsync(xp + z * xstride, Ts + (int64_t)z * B * kc, w, cudaMemcpyDeviceToDevice,
                                             st));
                return cudaSuccess;
            });
        };
        const int npan = (n + B - 1) / B;
        if (sweeps & 1)
            for (int q = 0; q < npan; ++q) {
                const int p0 = q * B, pe = std::min(n, p0 + B);
                EXPM_TRY(apply(q, true));
                if (n - pe > 0) EXPM_TRY(t_big(pe, n - pe, p0, pe - p0));
            }
        if (sweeps & 2)
            for (int q = npan - 1; q >= 0; --q) {
                const int p0 = q * B, pe = std::min(n, p0 + B);
                EXPM_TRY(apply(q, false));
                if (p0 > 0) EXPM_TRY(t_big(0, p0, p0, pe - p0));
            }
        return cudaGetLastError();
    }
    // forward sweep (unit L, or U^H)
    if (sweeps & 1)
        for (int p0 = 0; p0 < n; p0 += PNB) {
            const int pe = std::min(n, p0 + PNB);
            for (int p = p0; p < pe; p += DN_NB) {
                const int nb = std::min(DN_NB, pe - p);
                EXPM_TRY(t_trsm(p, nb, true));
                if (pe - p - nb > 0) EXPM_TRY(t_update(p + nb, pe - p - nb, p, nb));
            }
            if (n - pe > 0) EXPM_TRY(t_big(pe, n - pe, p0, pe - p0));
        }
    // backward sweep (U, or unit L^H), panels from the bottom
    if (sweeps & 2)
        for (int pe = n; pe > 0; pe -= PNB) {
            const int p0 = std::max(0, pe - PNB);
            const int nblk = (pe - p0 + DN_NB - 1) / DN_NB;
            for (int bi = nblk - 1; bi >= 0; --bi) {
                const int p = p0 + bi * DN_NB, nb = std::min(DN_NB, pe - p);
                EXPM_TRY(t_trsm(p, nb, false));
                if (p > p0) EXPM_TRY(t_update(p0, p - p0, p, nb));
            }
            if (p0 > 0) EXPM_TRY(t_big(0, p0, p0, pe - p0));
        }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ driver

// Workspace = factor part [amax, umax, factors] + solve part [norms, X binary64,
// R binary64 and D binary32 (mixed)].  The factor part depends only on A, t, c and
// the poles and can be kept for later right-hand sides.
struct DenseLayout {
    size_t amax, umax, F, tcA, tcB, tcflag, P, inv, factor_total;             // factor part
    size_t rn2, xn2, an2, ctl, X, R, D, oz, stA, stB, sterr, Ts, solve_total;  // solve part (offsets from its own base)
};
static inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// The refinement residual of a single problem with more than 8 right-hand-side columns
// runs on the tensor cores (binary64-accurate slice products, oz_gemm.cu); batches of
// instances keep the float-pair GEMM.
static bool dense_uses_oz(const DenseGeom &g) {
    return g.mixed && g.kc > 8 && g.ninst == 1 && oz_resid_supported(g.n, g.kc, g.nsys);
}

// Binary32 triangular solves with many columns in bf16x3 mode: panel updates on the
// tensor cores.
static bool dense_tc_solves(const DenseGeom &g) { return g.mixed && g.tc == 2 && g.kc > 8; }

// Diagonal-panel inverses of the wide solves: panels of B = min(n, 128) rows, used for
// every solve that does not take the fused narrow kernel (as long as the (factor, panel)
// pairs fit one grid dimension of the inversion).  128 rather than 256: the residual a
// product by an explicit inverse leaves grows with the inverted block's condition, and
// with 128-row blocks the binary32 solves refine as well as substitution does.
constexpr int DN_IB = 128;
static int inv_block(int n) { return std::min(n, DN_IB); }

bool dense_uses_inv(const DenseGeom &g) {
    const size_t smn = g.mixed ? narrow_smem_bytes<float>(g.n, g.kc) : narrow_smem_bytes<double>(g.n, g.kc);
    if (g.kc <= 8 && smn <= (200u << 10)) return false;
    const int B = inv_block(g.n);
    return (int64_t)g.ninst * g.npairs * ((g.n + B - 1) / B) <= 65535;
}

static DenseLayout dense_layout(const DenseGeom &g) {
    DenseLayout L{};
    const size_t nn = (size_t)g.n * g.n, nk = (size_t)g.n * g.kc;
    const size_t npz = (size_t)g.ninst * g.npairs, nsz = (size_t)g.ninst * g.nsys;
    size_t off = 0;
    L.amax = off; off += align_up(npz * sizeof(unsigned));
    L.umax = off; off += align_up(npz * sizeof(unsigned));
    L.F = off; off += align_up(npz * nn * (g.mixed ? sizeof(cx<float>) : sizeof(cx<double>)));
    L.tcA = L.tcB = L.tcflag = off;
    if (g.mixed && g.tc) {  // trailing-update operands for the largest step (rest < n)
        const size_t kw = g.tc == 2 ? DN_PNB : DN_NB;  // bf16x3: 256-column panels
        L.tcA = off; off += align_up(npz * (size_t)g.n * 6 * kw * sizeof(float));
        L.tcB = off; off += align_up(npz * (size_t)g.n * 2 * 6 * kw * sizeof(float));
        L.tcflag = off; off += align_up(sizeof(int));
    }
    const size_t es = g.mixed ? sizeof(cx<float>) : sizeof(cx<double>);
    L.P = L.inv = off;
    if (dense_uses_inv(g)) {  // the gathered panels, then the two inverses of each
        const size_t B = inv_block(g.n), blocks = npz * ((g.n + B - 1) / B);
        L.P = off; off += align_up(blocks * B * B * es);
        L.inv = off; off += align_up(2 * blocks * B * B * es);
    }
    L.factor_total = off;
    off = 0;
    L.rn2 = off; off += align_up(nsz * sizeof(double));
    L.xn2 = off; off += align_up(nsz * sizeof(double));
    L.an2 = off; off += align_up((size_t)g.ninst * sizeof(double));
    L.ctl = off; off += align_up(sizeof(int));
    L.X = off; off += align_up(nsz * nk * sizeof(cx<double>));
    L.R = off;
    L.D = off;
    if (g.mixed) {
        off += align_up(nsz * nk * sizeof(cx<double>));
        L.D = off;
        off += align_up(nsz * nk * sizeof(cx<float>));
    }
    L.oz = off;
    if (dense_uses_oz(g)) off += align_up(oz_resid_bytes(g.n, g.kc, g.nsys, g.complex_a));
    L.stA = L.stB = L.sterr = off;
    if (dense_tc_solves(g)) {  // two sets (the plain and the conjugate half run concurrently)
        const size_t batch = (size_t)g.ninst * g.npairs, kr = 12 * DN_PNB;
        L.stA = off; off += 2 * align_up(batch * (size_t)g.n * kr * sizeof(uint16_t));
        L.stB = off; off += 2 * align_up(batch * 2 * (size_t)g.kc * kr * sizeof(uint16_t));
        L.sterr = off; off += align_up(sizeof(int));
    }
    L.Ts = off;
    if (dense_uses_inv(g))  // one product scratch per concurrently running half
        off += 2 * align_up((size_t)g.ninst * g.npairs * inv_block(g.n) * g.kc * es);
    L.solve_total = off;
    return L;
}

size_t dense_factor_bytes(const DenseGeom &g) { return dense_layout(g).factor_total; }
size_t dense_solve_bytes(const DenseGeom &g) { return dense_layout(g).solve_total; }
size_t dense_workspace_bytes(const DenseGeom &g) {
    const DenseLayout L = dense_layout(g);
    return L.factor_total + L.solve_total;
}

template <class T>
static cudaError_t factor_pairs(const DenseGeom &g, const DenseIO &io, const DenseSystems &sys, cx<T> *F,
                                unsigned *amax, unsigned *umax, cudaStream_t st, Profiler &prof,
                                const TcScratch *tc = nullptr) {
    // pair s uses system 2s (complex A) or s (real data); both carry the Im(theta) > 0 member
    DenseSystems pairs = sys;
    for (int s = 0; s < g.npairs; ++s) {
        const int b = g.complex_a ? 2 * s : s;
        pairs.th_re[s] = sys.th_re[b];
        pairs.th_im[s] = sys.th_im[b];
    }
    const int batch = g.ninst * g.npairs;
    EXPM_TRY(cudaMemsetAsync(amax, 0, sizeof(unsigned) * batch, st));
    EXPM_TRY(cudaMemsetAsync(umax, 0, sizeof(unsigned) * batch, st));
    EXPM_TRY(prof.timed(sizeof(T) == 8 ? "form_shifted<f64>" : "form_shifted<f32>", st, [&] {
        form_shifted<T><<<dim3((g.n + 7) / 8, 1, g.ninst), 256, 0, st>>>(
            g.n, io.A, (int)io.lda, io.astride, g.complex_a, g.npairs, g.t, pairs, F, amax);
        return cudaGetLastError();
    }));
    EXPM_TRY(lu_blocked<T>(g.n, batch, F, st, prof, tc, g.tile));
    max_abs_upper<T><<<dim3((g.n + 7) / 8, 1, batch), 256, 0, st>>>(g.n, F, g.n, (int64_t)g.n * g.n, umax);
    return cudaGetLastError();
}

// A second stream per host thread and device for the conjugate half of a complex solve
// (created on first use, destroyed when the thread exits).
static cudaStream_t aux_stream() {
    struct Holder {
        cudaStream_t s[16] = {};
        ~Holder() {
            for (cudaStream_t x : s)
                if (x) cudaStreamDestroy(x);
        }
    };
    static thread_local Holder h;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return nullptr;
    if (!h.s[dev] && cudaStreamCreateWithFlags(&h.s[dev], cudaStreamNonBlocking) != cudaSuccess) h.s[dev] = nullptr;
    return h.s[dev];
}

template <class T>
static cudaError_t solve_systems(const DenseGeom &g, const cx<T> *F, cx<T> *X, int64_t xstride, cudaStream_t st,
                                 Profiler &prof, const int *skip = nullptr, const SolveTc *tcs = nullptr,
                                 const SolveInv *inv = nullptr) {
    const int64_t fs = (int64_t)g.n * g.n;
    const int batch = g.ninst * g.npairs;
    const char *name = sizeof(T) == 8 ? "lu_solve<f64>" : "lu_solve<f32>";
    Profiler quiet;  // the whole solve is timed here, its parts by lu_solve
    // tcs (optional): two scratch sets, one per concurrently running half
    const SolveTc *tc0 = tcs, *tc1 = tcs != nullptr ? tcs + 1 : nullptr;
    const SolveInv *iv0 = inv, *iv1 = inv != nullptr ? inv + 1 : nullptr;  // likewise the inverse scratch
    if (!g.complex_a)
        return prof.timed(name, st, [&] {
            return lu_solve<T>(g.n, g.kc, batch, F, fs, false, X, xstride, st, quiet, skip, tc0, &prof, iv0);
        });
    // systems 2s (theta) and 2s+1 (conj theta) of every instance share factor s: the
    // even and the odd systems each form a batch with stride 2*xstride
    cudaStream_t aux = aux_stream();
    if (!aux)
        return prof.timed(name, st, [&]() -> cudaError_t {
            EXPM_TRY(lu_solve<T>(g.n, g.kc, batch, F, fs, false, X, 2 * xstride, st, quiet, skip, tc0, &prof, iv0));
            return lu_solve<T>(g.n, g.kc, batch, F, fs, true, X + xstride, 2 * xstride, st, quiet, skip, tc0,
                               &prof, iv0);
        });
    // the two halves are independent and run concurrently (fork / join through events,
    // so the work stays ordered on st for the caller; also inside a stream capture)
    return prof.timed(name, st, [&]() -> cudaError_t {
        cudaEvent_t fork, join;
        EXPM_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        cudaError_t e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, fork, 0);
        if (e == cudaSuccess)
            e = lu_solve<T>(g.n, g.kc, batch, F, fs, false, X, 2 * xstride, st, quiet, skip, tc0, &prof, iv0);
        if (e == cudaSuccess)
            e = lu_solve<T>(g.n, g.kc, batch, F, fs, true, X + xstride, 2 * xstride, aux, quiet, skip, tc1, &prof, iv1);
        if (e == cudaSuccess) e = cudaEventRecord(join, aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, join, 0);
        cudaEventDestroy(fork);
        cudaEventDestroy(join);
        return e;
    });
}

// L_q^{-1} and U_q^{-1} of every diagonal panel of every factor: the panels gathered
// into B x B blocks (identity-padded), then one forward and one backward blocked solve
// on identities, all (factor, panel) blocks as one batch.
template <class T>
static cudaError_t invert_panels(const DenseGeom &g, const cx<T> *F, cx<T> *P, cx<T> *Inv, cudaStream_t st,
                                 Profiler &prof) {
    const int B = inv_block(g.n), npan = (g.n + B - 1) / B, npz = g.ninst * g.npairs;
    const int64_t bb = (int64_t)B * B;
    return prof.timed(sizeof(T) == 8 ? "invert_panels<f64>" : "invert_panels<f32>", st, [&]() -> cudaError_t {
        const unsigned gx = (unsigned)std::min<int64_t>((bb + 255) / 256, 64);
        gather_diag_panels<T><<<dim3(gx, npan, npz), 256, 0, st>>>(g.n, B, npan, F, (int64_t)g.n * g.n, P, Inv);
        EXPM_TRY(cudaGetLastError());
        Profiler quiet;
        const int batch = npz * npan;
        EXPM_TRY(lu_solve<T>(B, B, batch, P, bb, false, Inv, 2 * bb, st, quiet, nullptr, nullptr, nullptr, nullptr, 1));
        return lu_solve<T>(B, B, batch, P, bb, false, Inv + bb, 2 * bb, st, quiet, nullptr, nullptr, nullptr, nullptr,
                           2);
    });
}

cudaError_t dense_factor(const DenseGeom &g, const DenseIO &io, const DenseSystems &sys, void *fwork, cudaStream_t st,
                         Profiler &prof) {
    const DenseLayout L = dense_layout(g);
    unsigned char *p = (unsigned char *)fwork;
    unsigned *amax = (unsigned *)(p + L.amax);
    unsigned *umax = (unsigned *)(p + L.umax);
    const bool inv = dense_uses_inv(g);
    if (g.mixed) {
        cx<float> *F = (cx<float> *)(p + L.F);
        if (g.tc) {
            TcScratch tc{(float *)(p + L.tcA), (float *)(p + L.tcB), (int *)(p + L.tcflag), g.tc == 2};
            EXPM_TRY(cudaMemsetAsync(tc.err, 0, sizeof(int), st));
            EXPM_TRY(factor_pairs<float>(g, io, sys, F, amax, umax, st, prof, &tc));
        } else {
            EXPM_TRY(factor_pairs<float>(g, io, sys, F, amax, umax, st, prof));
        }
        if (inv) EXPM_TRY(invert_panels<float>(g, F, (cx<float> *)(p + L.P), (cx<float> *)(p + L.inv), st, prof));
        return cudaSuccess;
    }
    cx<double> *F = (cx<double> *)(p + L.F);
    EXPM_TRY(factor_pairs<double>(g, io, sys, F, amax, umax, st, prof));
    if (inv) EXPM_TRY(invert_panels<double>(g, F, (cx<double> *)(p + L.P), (cx<double> *)(p + L.inv), st, prof));
    return cudaSuccess;
}

// the inverse part of a solve: the factor's inverses and this solve's two scratch halves
static const SolveInv *solve_inv(const DenseGeom &g, const DenseLayout &L, const void *fwork, void *swork,
                                 SolveInv out[2]) {
    if (!dense_uses_inv(g)) return nullptr;
    const int B = inv_block(g.n);
    const size_t es = g.mixed ? sizeof(cx<float>) : sizeof(cx<double>);
    const size_t half = align_up((size_t)g.ninst * g.npairs * B * g.kc * es);
    for (int h = 0; h < 2; ++h) {
        out[h].inv = (const unsigned char *)fwork + L.inv;
        out[h].T = (unsigned char *)swork + L.Ts + h * half;
        out[h].B = B;
        out[h].npan = (g.n + B - 1) / B;
    }
    return out;
}

cudaError_t dense_growth(const DenseGeom &g, const void *fwork, cudaStream_t st, DenseResult *res) {
    const DenseLayout L = dense_layout(g);
    const unsigned char *p = (const unsigned char *)fwork;
    const int npz = g.ninst * g.npairs;
    std::vector<unsigned> hm(2 * (size_t)npz);
    int tcflag = 0;
    EXPM_TRY(cudaMemcpyAsync(hm.data(), p + L.amax, sizeof(unsigned) * npz, cudaMemcpyDeviceToHost, st));
    EXPM_TRY(cudaMemcpyAsync(hm.data() + npz, p + L.umax, sizeof(unsigned) * npz, cudaMemcpyDeviceToHost, st));
    if (g.mixed && g.tc) EXPM_TRY(cudaMemcpyAsync(&tcflag, p + L.tcflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    EXPM_TRY(cudaStreamSynchronize(st));
    res->tc_timeout = res->tc_timeout || tcflag;  // keeps a time-out of the solve's residual kernel
    res->growth_max = 0.0;
    res->inst_growth.assign(g.ninst, 0.0);
    for (int z = 0; z < npz; ++z) {
        float a, u;
        std::memcpy(&a, &hm[z], 4);
        std::memcpy(&u, &hm[npz + z], 4);
        if (a > 0) {
            const double gz = (double)u / (double)a;
            res->growth_max = std::max(res->growth_max, gz);
            res->inst_growth[z / g.npairs] = std::max(res->inst_growth[z / g.npairs], gz);
        }
    }
    return cudaSuccess;
}

cudaError_t dense_solve(const DenseGeom &g, const DenseIO &io, const DenseSystems &sys, const void *fwork, void *swork,
                        cudaStream_t st, Profiler &prof, DenseResult *res) {
    const int64_t nk = (int64_t)g.n * g.kc;
    const DenseLayout L = dense_layout(g);
    const void *F = (const unsigned char *)fwork + L.F;
    unsigned char *p = (unsigned char *)swork;
    double *rn2 = (double *)(p + L.rn2);
    double *xn2 = (double *)(p + L.xn2);
    double *an2 = (double *)(p + L.an2);
    cx<double> *X = (cx<double> *)(p + L.X);
    const int nsz = g.ninst * g.nsys;
    const unsigned gx = grid1d(nk);
    res->iters = 0;
    res->resid_rel_max = 0.0;
    res->inst_iters.assign(g.ninst, 0);
    res->inst_resid.assign(g.ninst, 0.0);
    if (!g.mixed) {
        load_rhs<double><<<dim3(gx, 1, nsz), 256, 0, st>>>(g.n, g.kc, io, g.nsys, X, nk);
        EXPM_TRY(cudaGetLastError());
        SolveInv sv[2];
        EXPM_TRY(solve_systems<double>(g, (const cx<double> *)F, X, nk, st, prof, nullptr, nullptr,
                                       solve_inv(g, L, fwork, swork, sv)));
    } else {
        cx<double> *R = (cx<double> *)(p + L.R);
        cx<float> *D = (cx<float> *)(p + L.D);
        const bool use_oz = dense_uses_oz(g);
        void *oz_ws = p + L.oz;
        bool oz_a_ready = false;  // A's slices are formed at the first residual product
        SolveTc stc[2];
        const SolveTc *tcs = nullptr;
        if (dense_tc_solves(g)) {
            const size_t batch = (size_t)g.ninst * g.npairs, kr = 12 * DN_PNB;
            const size_t ab = align_up(batch * (size_t)g.n * kr * sizeof(uint16_t));
            const size_t bb = align_up(batch * 2 * (size_t)g.kc * kr * sizeof(uint16_t));
            int *flag = (int *)(p + L.sterr);
            stc[0] = {(uint16_t *)(p + L.stA), (uint16_t *)(p + L.stB), flag};
            stc[1] = {(uint16_t *)(p + L.stA + ab), (uint16_t *)(p + L.stB + bb), flag};
            EXPM_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
            tcs = stc;
        }
        SolveInv siv[2];
        const SolveInv *sinv = solve_inv(g, L, fwork, swork, siv);
        EXPM_TRY(cudaMemsetAsync(X, 0, (size_t)nsz * nk * sizeof(cx<double>), st));
        std::vector<double> h(2 * (size_t)nsz), an(g.ninst);
        // ||tA||_F of every instance for the relative residual of the stopping test
        EXPM_TRY(cudaMemsetAsync(an2, 0, sizeof(double) * g.ninst, st));
        frob2<<<dim3((unsigned)std::min(g.n, 1024), 1, g.ninst), 256, 0, st>>>(g.n, io.A, io.lda, io.astride,
                                                                           g.complex_a, an2);
        EXPM_TRY(cudaGetLastError());
        EXPM_TRY(cudaMemcpyAsync(an.data(), an2, sizeof(double) * g.ninst, cudaMemcpyDeviceToHost, st));
        EXPM_TRY(cudaStreamSynchronize(st));
        // it = 0: initial solve; it = 1 .. max_refine: refinement sweeps; the residual
        // of the current X is checked before every sweep and once after the last one
        for (int it = 0;; ++it) {
            if (use_oz && it >= 2) {
                // after a correction D (~1e-6 of X): R -= (tA - cI + theta I) D, the product
                // on the tensor cores in its light form (four slices of A and of D)
                EXPM_TRY(prof.timed("residual_diag", st, [&] {
                    residual_diag_step<<<dim3(gx, 1, nsz), 256, 0, st>>>(nk, g.nsys, R, D, nk, sys);
                    return cudaGetLastError();
                }));
                int to = 0;
                EXPM_TRY(prof.timed("oz_split_d", st, [&] {
                    return oz_split_d(g.n, g.kc, g.nsys, g.complex_a, D, nk, oz_ws, st);
                }));
                EXPM_TRY(prof.timed("oz_gemm_light", st, [&] {
                    return oz_product_light(g.n, g.kc, g.nsys, g.complex_a, g.t, nk, R, oz_ws, st, nullptr);
                }));
                EXPM_TRY(oz_read_timeout(g.n, g.kc, g.nsys, g.complex_a, oz_ws, st, &to));
                if (to) {
                    res->tc_timeout = 1;
                    return cudaSuccess;
                }
            } else {
            // R = V - (tA - cI + theta I) X, binary64
            EXPM_TRY(prof.timed("residual_diag", st, [&] {
                residual_diag<<<dim3(gx, 1, nsz), 256, 0, st>>>(g.n, g.kc, io, g.nsys, X, R, nk, sys, nullptr);
                return cudaGetLastError();
            }));
            if (it > 0) {
                if (use_oz) {
                    if (!oz_a_ready) {
                        EXPM_TRY(prof.timed("oz_split_a", st, [&] {
                            return oz_split_a(g.n, io.A, io.lda, g.complex_a, oz_ws, st);
                        }));
                        oz_a_ready = true;
                    }
                    int to = 0;
                    EXPM_TRY(prof.timed("oz_split_x", st, [&] {
                        return oz_split_x(g.n, g.kc, g.nsys, g.complex_a, X, nk, oz_ws, st);
                    }));
                    EXPM_TRY(prof.timed("oz_gemm", st, [&] {
                        return oz_product(g.n, g.kc, g.nsys, g.complex_a, g.t, nk, R, oz_ws, st, nullptr);
                    }));
                    EXPM_TRY(oz_read_timeout(g.n, g.kc, g.nsys, g.complex_a, oz_ws, st, &to));
                    if (to) {
                        res->tc_timeout = 1;
                        return cudaSuccess;
                    }
                } else if (g.kc <= 8) {
                    EXPM_TRY(prof.timed("resid_gemv<f32x2>", st, [&] {
                        if (g.complex_a)
                            resid_gemv_f32x2_launch<cx<double>>(g.n, g.kc, g.nsys, g.ninst, g.t,
                                                                (const cx<double> *)io.A, (int)io.lda, io.astride, X,
                                                                nk, R, nullptr, st);
                        else
                            resid_gemv_f32x2_launch<double>(g.n, g.kc, g.nsys, g.ninst, g.t, io.A, (int)io.lda,
                                                            io.astride, X, nk, R, nullptr, st);
                        return cudaGetLastError();
                    }));
                } else EXPM_TRY(prof.timed("resid_gemm<f32x2>", st, [&] {
                    dim3 gg((g.kc + 63) / 64, (g.n + 63) / 64, nsz);
                    cudaError_t e;
                    if (g.complex_a) {
                        e = set_smem(resid_gemm_f32x2<cx<double>>, RESID_GEMM_SMEM);
                        if (e == cudaSuccess)
                            resid_gemm_f32x2<cx<double>><<<gg, 256, RESID_GEMM_SMEM, st>>>(
                                g.n, g.kc, g.n, g.t, (const cx<double> *)io.A, (int)io.lda, io.astride, X, g.kc, nk, R,
                                g.kc, nk, g.nsys);
                    } else {
                        e = set_smem(resid_gemm_f32x2<double>, RESID_GEMM_SMEM);
                        if (e == cudaSuccess)
                            resid_gemm_f32x2<double><<<gg, 256, RESID_GEMM_SMEM, st>>>(g.n, g.kc, g.n, g.t, io.A,
                                                                                       (int)io.lda, io.astride, X, g.kc,
                                                                                       nk, R, g.kc, nk, g.nsys);
                    }
                    return e != cudaSuccess ? e : cudaGetLastError();
                }));
            }
            }
            EXPM_TRY(cudaMemsetAsync(rn2, 0, sizeof(double) * nsz, st));
            EXPM_TRY(cudaMemsetAsync(xn2, 0, sizeof(double) * nsz, st));
            EXPM_TRY(prof.timed("demote_and_norms", st, [&] {
                demote_and_norms<<<dim3(gx, 1, nsz), 256, 0, st>>>(nk, R, X, D, nk, rn2, xn2, nullptr);
                return cudaGetLastError();
            }));
            if (it > 0) {
                EXPM_TRY(cudaMemcpyAsync(h.data(), rn2, sizeof(double) * nsz, cudaMemcpyDeviceToHost, st));
                EXPM_TRY(cudaMemcpyAsync(h.data() + nsz, xn2, sizeof(double) * nsz, cudaMemcpyDeviceToHost, st));
                EXPM_TRY(cudaStreamSynchronize(st));
                bool done = true;
                double worst = 0.0;
                std::fill(res->inst_resid.begin(), res->inst_resid.end(), 0.0);  // this sweep's residuals
                for (int z = 0; z < nsz; ++z) {
                    const int inst = z / g.nsys, b = z % g.nsys;
                    const double shift = std::hypot(sys.th_re[b] - sys.cshift, sys.th_im[b]);
                    const double den = (std::sqrt(an[inst]) * std::fabs(g.t) + shift) * std::sqrt(h[nsz + z]);
                    const double rel = den > 0 ? std::sqrt(h[z]) / den : 0.0;
                    worst = std::max(worst, rel);
                    res->inst_resid[inst] = std::max(res->inst_resid[inst], rel);
                    if (!(rel <= g.tol)) done = false;
                }
                res->resid_rel_max = worst;
                res->iters = it - 1;
                for (int i = 0; i < g.ninst; ++i) res->inst_iters[i] = it - 1;
                if (done || it > g.max_refine) break;
            }
            EXPM_TRY(solve_systems<float>(g, (const cx<float> *)F, D, nk, st, prof, nullptr, tcs, sinv));
            EXPM_TRY(prof.timed("add_correction", st, [&] {
                add_correction<<<dim3(gx, 1, nsz), 256, 0, st>>>(nk, D, X, nk, nullptr);
                return cudaGetLastError();
            }));
        }
    }
    if (dense_tc_solves(g)) {  // a bounded wait in a tensor-core solve update gave up
        int flag = 0;
        EXPM_TRY(cudaMemcpyAsync(&flag, p + L.sterr, sizeof(int), cudaMemcpyDeviceToHost, st));
        EXPM_TRY(cudaStreamSynchronize(st));
        if (flag) res->tc_timeout = 1;
    }
    EXPM_TRY(prof.timed("accumulate", st, [&] {
        accumulate<<<dim3(gx, 1, g.ninst), 256, 0, st>>>(g.n, g.kc, g.nsys, X, nk, sys, io);
        return cudaGetLastError();
    }));
    return cudaSuccess;
}

bool dense_narrow_fits(int n, int kc) { return kc <= 8 && narrow_smem_bytes<float>(n, kc) <= (200u << 10); }

// Device-controlled refinement (mixed, kc <= 8): the same sweeps as dense_solve, all
// enqueued up front -- 1 + max_refine solves and max_refine + 1 residual checks -- each
// kernel returning at once after refine_check has found every instance converged.  The
// result is bit-identical to dense_solve's, which stops launching at that point.
static cudaError_t dense_solve_devctl(const DenseGeom &g, const DenseIO &io, const DenseSystems &sys,
                                      const void *fwork, void *swork, cudaStream_t st, Profiler &prof,
                                      const DenseDevOut &out) {
    if (!g.mixed || g.kc > 8 || narrow_smem_bytes<float>(g.n, g.kc) > (200u << 10)) return cudaErrorInvalidValue;
    const int64_t nk = (int64_t)g.n * g.kc;
    const DenseLayout L = dense_layout(g);
    const cx<float> *F = (const cx<float> *)((const unsigned char *)fwork + L.F);
    unsigned char *p = (unsigned char *)swork;
    double *rn2 = (double *)(p + L.rn2);
    double *xn2 = (double *)(p + L.xn2);
    double *an2 = (double *)(p + L.an2);
    int *done = (int *)(p + L.ctl);
    cx<double> *X = (cx<double> *)(p + L.X);
    cx<double> *R = (cx<double> *)(p + L.R);
    cx<float> *D = (cx<float> *)(p + L.D);
    const int nsz = g.ninst * g.nsys;
    const unsigned gx = grid1d(nk);
    EXPM_TRY(cudaMemsetAsync(X, 0, (size_t)nsz * nk * sizeof(cx<double>), st));
    EXPM_TRY(cudaMemsetAsync(done, 0, sizeof(int), st));
    EXPM_TRY(cudaMemsetAsync(out.iters, 0, sizeof(int), st));
    EXPM_TRY(cudaMemsetAsync(an2, 0, sizeof(double) * g.ninst, st));
    frob2<<<dim3((unsigned)std::min(g.n, 1024), 1, g.ninst), 256, 0, st>>>(g.n, io.A, io.lda, io.astride, g.complex_a,
                                                                          an2);
    EXPM_TRY(cudaGetLastError());
    for (int it = 0; it <= g.max_refine + 1; ++it) {
        residual_diag<<<dim3(gx, 1, nsz), 256, 0, st>>>(g.n, g.kc, io, g.nsys, X, R, nk, sys, done);
        EXPM_TRY(cudaGetLastError());
        if (it > 0) {
            EXPM_TRY(prof.timed("resid_gemv<f32x2>", st, [&] {
                if (g.complex_a)
                    resid_gemv_f32x2_launch<cx<double>>(g.n, g.kc, g.nsys, g.ninst, g.t, (const cx<double> *)io.A,
                                                        (int)io.lda, io.astride, X, nk, R, done, st);
                else
                    resid_gemv_f32x2_launch<double>(g.n, g.kc, g.nsys, g.ninst, g.t, io.A, (int)io.lda, io.astride, X,
                                                    nk, R, done, st);
                return cudaGetLastError();
            }));
        }
        EXPM_TRY(cudaMemsetAsync(rn2, 0, sizeof(double) * nsz, st));
        EXPM_TRY(cudaMemsetAsync(xn2, 0, sizeof(double) * nsz, st));
        demote_and_norms<<<dim3(gx, 1, nsz), 256, 0, st>>>(nk, R, X, D, nk, rn2, xn2, done);
        EXPM_TRY(cudaGetLastError());
        if (it > 0) {
            refine_check<<<1, 1024, 0, st>>>(g.ninst, g.nsys, rn2, xn2, an2, g.t, sys, g.tol, it, done, out.iters,
                                             out.inst_resid);
            EXPM_TRY(cudaGetLastError());
        }
        if (it <= g.max_refine) {
            EXPM_TRY(solve_systems<float>(g, F, D, nk, st, prof, done));
            add_correction<<<dim3(gx, 1, nsz), 256, 0, st>>>(nk, D, X, nk, done);
            EXPM_TRY(cudaGetLastError());
        }
    }
    return prof.timed("accumulate", st, [&] {
        accumulate<<<dim3(gx, 1, g.ninst), 256, 0, st>>>(g.n, g.kc, g.nsys, X, nk, sys, io);
        return cudaGetLastError();
    });
}

size_t dense_tc_flag_offset(const DenseGeom &g) { return dense_layout(g).tcflag; }

cudaError_t dense_run_devctl(const DenseGeom &g, const DenseIO &io, const DenseSystems &sys, void *work,
                             cudaStream_t st, Profiler &prof, const DenseDevOut &out) {
    const DenseLayout L = dense_layout(g);
    unsigned char *p = (unsigned char *)work;
    EXPM_TRY(dense_factor(g, io, sys, p, st, prof));
    growth_dev<<<1, 1024, 0, st>>>(g.ninst, g.npairs, (const unsigned *)(p + L.amax), (const unsigned *)(p + L.umax),
                                   out.inst_growth);
    EXPM_TRY(cudaGetLastError());
    if (g.mixed) return dense_solve_devctl(g, io, sys, p, p + L.factor_total, st, prof, out);
    // binary64: no refinement, and its solve reads nothing back
    EXPM_TRY(cudaMemsetAsync(out.iters, 0, sizeof(int), st));
    EXPM_TRY(cudaMemsetAsync(out.inst_resid, 0, sizeof(double) * g.ninst, st));
    DenseResult unused;
    return dense_solve(g, io, sys, p, p + L.factor_total, st, prof, &unused);
}

cudaError_t dense_run(const DenseGeom &g, const DenseIO &io, const DenseSystems &sys, void *work, cudaStream_t st,
                      Profiler &prof, DenseResult *res) {
    const DenseLayout L = dense_layout(g);
    unsigned char *p = (unsigned char *)work;
    EXPM_TRY(dense_factor(g, io, sys, p, st, prof));
    EXPM_TRY(dense_solve(g, io, sys, p, p + L.factor_total, st, prof, res));
    return dense_growth(g, p, st, res);
}

}  // namespace expm
