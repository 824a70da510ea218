// tridiag_kernels.cuh -- kernels shared by the binary64 / float-float and the
// binary32-with-refinement tridiagonal paths: the prep pass, the block LUs with
// their spikes, the block end dots, the reduced separator system, and the warp
// helpers of the solve kernels.  See tridiag.cu for the separator partition.
//
// Everything here has internal linkage (anonymous namespace): each translation
// unit instantiates its own real types, so no kernel is registered twice.
#pragma once
#include <cstdint>

#include "arith.cuh"
#include "tridiag.cuh"

namespace expm {
namespace {

// ------------------------------------------------------------------ conversions

template <class R> struct Store;
template <> struct Store<double> {
    static EXPM_D double split(double x) { return x; }
};
template <> struct Store<f32x2> {
    static EXPM_D f32x2 split(double x) { return split_bits(x); }
};

// ------------------------------------------------------------------ K0
// Either part may be skipped by passing null outputs (dP/eP, or VP).
template <class R>
__global__ void tri_prep(TriGeom g, const double *__restrict__ d, const double *__restrict__ e,
                         const double *__restrict__ V, R *__restrict__ dP, R *__restrict__ eP, R *__restrict__ VP) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (dP != nullptr) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += stride) {
            dP[i] = Store<R>::split(g.t * d[i] - g.cshift);
            eP[i] = Store<R>::split(i + 1 < g.N ? g.t * e[i] : 0.0);
        }
    }
    if (VP != nullptr) {
        const int64_t nv = g.N * g.Rc;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride)
            VP[i] = Store<R>::split(V[i]);
    }
}

// ------------------------------------------------------------------ K1a
// One thread per (system, block): LU of M_b and the two unit spikes.  The loads of
// the next row are issued one iteration ahead so the serial factorization chain
// does not wait on memory.
template <class R>
__global__ void __launch_bounds__(128) tri_block_factor(TriGeom g, const R *__restrict__ dP,
                                                        const R *__restrict__ eP, TriPoles ps,
                                                        cx<R> *__restrict__ fact, cx<R> *__restrict__ us,
                                                        cx<R> *__restrict__ wsp, cx<R> *__restrict__ spk) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)g.S * g.P) return;
    const int b = (int)(tid % g.P);
    const int s = (int)(tid / g.P);
    const int64_t first = (int64_t)b * g.B;
    const int len = (b < g.P - 1) ? g.m : (int)(g.N - first);
    const cx<R> theta = cx_from<R>(ps.th_re[s], ps.th_im[s]);
    const cx<R> wgt = cx_from<R>(ps.w_re[s], ps.w_im[s]);
    cx<R> *F = fact + ((int64_t)s * g.N) * 3;  // per row: c', a = W g, b = g e'_{q-1}
    cx<R> *U = us + (int64_t)s * g.N;
    cx<R> *W = wsp + (int64_t)s * g.N;

    // forward: LU of M_b (c'_i, g_i = 1/w_i) and the forward-eliminated eps_first.
    // The solve kernel runs the forward substitution on z = W d' (W the system's residue
    // weight): z_i = a_i v_i - b_i z_{i-1} with a_i = W g_i, b_i = g_i e'_{i-1}, so that
    // its back substitution yields W x directly and Re(W x) costs nothing.
    cx<R> cprev = cxz<R>(), hprev = cxz<R>(), glast = cxz<R>();
    R dn = dP[first], en = eP[first];
    R eprev = RealOps<R>::zero();  // e'[q-1]
    for (int i = 0; i < len; ++i) {
        const int64_t q = first + i;
        const R dq = dn, eq = en;  // d'[q], e'[q]
        if (i + 1 < len) {
            dn = dP[q + 1];
            en = eP[q + 1];
        }
        cx<R> w = {dq + theta.re, theta.im};
        if (i > 0) w = w - scale(eprev, cprev);
        const cx<R> gi = cinv(w);
        const cx<R> cp = (i < len - 1) ? scale(eq, gi) : cxz<R>();
        const cx<R> h = (i == 0) ? gi : -(gi * scale(eprev, hprev));
        F[3 * q] = cp;
        F[3 * q + 1] = wgt * gi;
        F[3 * q + 2] = (i > 0) ? scale(eprev, gi) : cxz<R>();
        eprev = eq;
        glast = gi;
        U[q] = h;
        cprev = cp;
        hprev = h;
    }
    // backward: u = M_b^{-1} eps_first, w = M_b^{-1} eps_last.  The chain per row is
    // short, so the (h, c') of the next TRI_PF rows are kept in flight.
    const int64_t last = first + len - 1;
    cx<R> un = U[last], wn = glast;
    const cx<R> uL = un, wL = wn;
    W[last] = wn;
    cx<R> hq[TRI_PF], cq[TRI_PF];
#pragma unroll
    for (int r = 0; r < TRI_PF; ++r) {
        const int i = len - 2 - r;
        hq[r] = (i >= 0) ? U[first + i] : cxz<R>();
        cq[r] = (i >= 0) ? F[3 * (first + i)] : cxz<R>();
    }
    for (int i0 = len - 2; i0 >= 0; i0 -= TRI_PF) {
#pragma unroll
        for (int r = 0; r < TRI_PF; ++r) {
            const int i = i0 - r;
            if (i >= 0) {
                const cx<R> h = hq[r], cp = cq[r];
                const int ipf = i - TRI_PF;  // refill this slot for the next round
                if (ipf >= 0) {
                    hq[r] = U[first + ipf];
                    cq[r] = F[3 * (first + ipf)];
                }
                un = csub_mul(h, cp, un);
                wn = -(cp * wn);
                U[first + i] = un;
                W[first + i] = wn;
            }
        }
    }
    cx<R> *SP = spk + ((int64_t)s * g.P + b) * 4;
    SP[0] = un;  // u_b[first]
    SP[1] = uL;  // u_b[last]
    SP[2] = wn;  // w_b[first]
    SP[3] = wL;  // w_b[last]
}

// ------------------------------------------------------------------ K1b
// One thread per (system, block, column): y_b[first] = u_b^T v_b, y_b[last] = w_b^T v_b.
template <class R>
__global__ void __launch_bounds__(128) tri_block_dots(TriGeom g, const R *__restrict__ VP,
                                                      const cx<R> *__restrict__ us, const cx<R> *__restrict__ wsp,
                                                      cx<R> *__restrict__ yend) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)g.S * g.P * g.Rc) return;
    const int j = (int)(tid % g.Rc);
    const int64_t sb = tid / g.Rc;
    const int b = (int)(sb % g.P);
    const int s = (int)(sb / g.P);
    const int64_t first = (int64_t)b * g.B;
    const int len = (b < g.P - 1) ? g.m : (int)(g.N - first);
    const cx<R> *U = us + (int64_t)s * g.N;
    const cx<R> *W = wsp + (int64_t)s * g.N;
    cx<R> yu = cxz<R>(), yw = cxz<R>();
    cx<R> un = U[first], wn = W[first];
    R vn = VP[first * g.Rc + j];
    for (int i = 0; i < len; ++i) {
        const int64_t q = first + i;
        const cx<R> u = un, w = wn;
        const R v = vn;
        if (i + 1 < len) {
            un = U[q + 1];
            wn = W[q + 1];
            vn = VP[(q + 1) * g.Rc + j];
        }
        yu = yu + scale(v, u);
        yw = yw + scale(v, w);
    }
    cx<R> *YE = yend + ((int64_t)s * g.P + b) * g.Rc * 2;
    YE[2 * j] = yu;
    YE[2 * j + 1] = yw;
}

// ------------------------------------------------------------------ K2
// Reduced system for the separators of one (system, column):
//   A_b sigma_{b-1} + B_b sigma_b + C_b sigma_{b+1} = D_b,   b = 0 .. P-2
// solved by cyclic reduction (odd-even elimination) in shared memory.
// Shared-memory layout of the reduced system's arrays: entry i at cr_ix(i), one padding
// entry after every 128 bytes, so that the strided accesses of the deeper reduction
// levels (i = 2^k t + const) spread over the banks; cr_len(n) entries per array.
template <class R> __host__ __device__ constexpr int cr_shift() { return sizeof(cx<R>) == 8 ? 4 : 3; }
template <class R> EXPM_D int cr_ix(int i) { return i + (i >> cr_shift<R>()); }
template <class R> __host__ __device__ inline size_t cr_len(int64_t n) { return (size_t)(n + (n >> cr_shift<R>()) + 1); }

// Cyclic reduction of the tridiagonal system  A_i x_{i-1} + Bc_i x_i + C_i x_{i+1} = D_i
// (i < n) held in shared memory (entry i at cr_ix(i)); every thread of the CTA takes part
// and the solution overwrites D.  Forward: odd levels eliminated into their neighbours
// level by level; back: substitution from the top level down.
template <class R>
EXPM_D void cr_solve_smem(cx<R> *A, cx<R> *Bc, cx<R> *C, cx<R> *D, int n) {
    for (int stride = 1; 2 * stride - 1 < n; stride *= 2) {
        for (int i = 2 * stride - 1 + 2 * stride * threadIdx.x; i < n; i += 2 * stride * blockDim.x) {
            const int lo = i - stride, hi = i + stride;
            const cx<R> k1 = A[cr_ix<R>(i)] * cinv(Bc[cr_ix<R>(lo)]);
            cx<R> nb = Bc[cr_ix<R>(i)] - k1 * C[cr_ix<R>(lo)];
            cx<R> nd = D[cr_ix<R>(i)] - k1 * D[cr_ix<R>(lo)];
            cx<R> na = -(k1 * A[cr_ix<R>(lo)]);
            cx<R> nc = cxz<R>();
            if (hi < n) {
                const cx<R> k2 = C[cr_ix<R>(i)] * cinv(Bc[cr_ix<R>(hi)]);
                nb = nb - k2 * A[cr_ix<R>(hi)];
                nd = nd - k2 * D[cr_ix<R>(hi)];
                nc = -(k2 * C[cr_ix<R>(hi)]);
            }
            A[cr_ix<R>(i)] = na;
            Bc[cr_ix<R>(i)] = nb;
            C[cr_ix<R>(i)] = nc;
            D[cr_ix<R>(i)] = nd;
        }
        __syncthreads();
    }
    int top = 1;
    while (top * 2 <= n) top *= 2;
    for (int st = top; st >= 1; st /= 2) {
        for (int i = st - 1 + 2 * st * threadIdx.x; i < n; i += 2 * st * blockDim.x) {
            cx<R> rhs = D[cr_ix<R>(i)];
            if (i - st >= 0) rhs = rhs - A[cr_ix<R>(i)] * D[cr_ix<R>(i - st)];
            if (i + st < n) rhs = rhs - C[cr_ix<R>(i)] * D[cr_ix<R>(i + st)];
            D[cr_ix<R>(i)] = rhs * cinv(Bc[cr_ix<R>(i)]);  // D now holds the solution at index i
        }
        __syncthreads();
    }
}

template <class R>
__global__ void __launch_bounds__(1024) tri_reduced_cr(TriGeom g, const R *__restrict__ dP,
                                                       const R *__restrict__ eP, const R *__restrict__ VP,
                                                       const cx<R> *__restrict__ sepRhs,
                                                       TriPoles ps, const cx<R> *__restrict__ spk,
                                                       const cx<R> *__restrict__ yend, cx<R> *__restrict__ sigma,
                                                       const int *skip) {
    if (skip != nullptr && *skip) return;  // refinement already converged (uniform over the launch)
    extern __shared__ unsigned char smem_raw[];
    const int n = g.P - 1;
    const int np = (int)cr_len<R>(n);
    cx<R> *A = reinterpret_cast<cx<R> *>(smem_raw);
    cx<R> *Bc = A + np;
    cx<R> *C = Bc + np;
    cx<R> *D = C + np;
    const int s = blockIdx.x / g.Rc;
    const int j = blockIdx.x % g.Rc;
    const cx<R> theta = cx_from<R>(ps.th_re[s], ps.th_im[s]);
    const cx<R> *SP = spk + (int64_t)s * g.P * 4;
    const cx<R> *YE = yend + (int64_t)s * g.P * g.Rc * 2;

    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        const int64_t r = (int64_t)b * g.B + g.m;  // separator row
        const R el = eP[r - 1];                    // couples sigma_b and the last row of block b
        const R er = eP[r];                        // couples sigma_b and the first row of block b+1
        const cx<R> uL = SP[4 * b + 1], wL = SP[4 * b + 3];
        const cx<R> u0n = SP[4 * (b + 1) + 0], w0n = SP[4 * (b + 1) + 2];
        cx<R> Ab = cxz<R>(), Cb = cxz<R>();
        if (b >= 1) Ab = -scale(el * eP[r - g.B], uL);               // e' at the previous separator's right
        if (b + 1 <= n - 1) Cb = -scale(er * eP[r + g.B - 1], w0n);  // e' at the next separator's left
        cx<R> Bb = {dP[r] + theta.re, theta.im};
        Bb = Bb - scale(el * el, wL) - scale(er * er, u0n);
        const cx<R> yL = YE[(int64_t)b * g.Rc * 2 + 2 * j + 1];        // y_b[last]
        const cx<R> y0n = YE[(int64_t)(b + 1) * g.Rc * 2 + 2 * j + 0];  // y_{b+1}[first]
        // right-hand side at the separator: V's entry, or a per-system complex value
        // (refinement passes) when sepRhs is given, laid out [system][separator][column]
        cx<R> Db = sepRhs != nullptr ? sepRhs[((int64_t)s * g.P + b) * g.Rc + j]
                                     : cx<R>{VP[r * g.Rc + j], RealOps<R>::zero()};
        Db = Db - scale(el, yL) - scale(er, y0n);
        A[cr_ix<R>(b)] = Ab;
        Bc[cr_ix<R>(b)] = Bb;
        C[cr_ix<R>(b)] = Cb;
        D[cr_ix<R>(b)] = Db;
    }
    __syncthreads();
    cr_solve_smem<R>(A, Bc, C, D, n);
    cx<R> *SG = sigma + (int64_t)s * g.P * g.Rc;
    for (int b = threadIdx.x; b < n; b += blockDim.x) SG[(int64_t)b * g.Rc + j] = D[cr_ix<R>(b)];
}

// ------------------------------------------------------------------ K4: float pairs of Y to binary64
__global__ void tri_finish(int64_t n, double *__restrict__ Y) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const f32x2 v = reinterpret_cast<const f32x2 *>(Y)[i];
        Y[i] = widen_bits(v.hi) + widen_bits(v.lo);
    }
}

// ------------------------------------------------------------------ warp helpers
template <class T> EXPM_D T shfl_xor(unsigned mask, T v, int off) { return __shfl_xor_sync(mask, v, off); }
template <> EXPM_D f32x2 shfl_xor<f32x2>(unsigned mask, f32x2 v, int off) {
    return {__shfl_xor_sync(mask, v.hi, off), __shfl_xor_sync(mask, v.lo, off)};
}


// Reduce-scatter of LG values per lane over the LG lanes of a group by recursive
// halving: afterwards lane l holds the sum over the group of everyone's v[l] in v[0].
// LG-1 additions per lane for LG rows (instead of log2(LG) per row for a per-row tree).
template <int LG, class R> EXPM_D void reduce_scatter(unsigned gmask, int sl, R (&v)[LG]) {
#pragma unroll
    for (int off = LG / 2; off > 0; off >>= 1) {
        const bool upper = (sl & off) != 0;
#pragma unroll
        for (int idx = 0; idx < off; ++idx) {
            const R send = upper ? v[idx] : v[idx + off];
            const R keep = upper ? v[idx + off] : v[idx];
            v[idx] = keep + shfl_xor(gmask, send, off);
        }
    }
}

}  // namespace
}  // namespace expm
