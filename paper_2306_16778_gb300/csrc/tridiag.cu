// tridiag.cu -- pole-batched shifted tridiagonal solves with the fused residue sum.
//
// Computes Y = sum_s Re(W_s X_s) (real data) where X_s solves
//     (t T - c I + theta_s I) X_s = V,     T real symmetric tridiagonal,
// for every "system" s (one member of each conjugate pole pair, Remark 5.1) and
// every right-hand-side column j.  This is eq. expAx of the paper with the
// 2 Re halving of Remark 5.1; W_s = 2 e^c a_s is folded in by the host.
//
// Parallel structure (separator partition of the rows).  Rows are cut into P
// blocks of `m` interior rows, each followed by one separator row (the last block
// has no separator).  With M_b the block's shifted matrix, the interior solution is
//     x_b = M_b^{-1} v_b - (t e_{first-1}) sigma_{b-1} u_b - (t e_{last}) sigma_b w_b
// with the unit spikes u_b = M_b^{-1} eps_first, w_b = M_b^{-1} eps_last.  Eliminating
// the interiors leaves a tridiagonal system for the separator values sigma_b.
// Because M_b is complex symmetric, the two end values of y_b = M_b^{-1} v_b that
// this system needs are dot products: y_b[first] = u_b^T v_b, y_b[last] = w_b^T v_b.
//
//   K1 tri_block_factor   one thread per (system, block): unpivoted LU of M_b
//                         (stored), spikes u_b and w_b, the end values y_b.
//   K2 tri_reduced_cr     one CTA per (system, column): the reduced system by
//                         cyclic reduction in shared memory.
//   K3 tri_block_solve    one thread per (block, column): forward and back
//                         substitution of every system with the separator values as
//                         boundary data, and the weighted sum over systems.
//
// No pivoting: for Im(theta) != 0, (-i sign(Im theta)) M has Hermitian part
// |Im theta| I, positive definite, so every leading block and every Schur
// complement (including the reduced system) is non-singular and unpivoted
// elimination is stable.
//
// Templated on the real type R: double (binary64) or f32x2 (float-float).
#include <cstdio>
#include <cstdint>
#include <type_traits>

#include "arith.cuh"
#include "tridiag.cuh"
#include "plan.cuh"

namespace expm {

template <class R>
__global__ void __launch_bounds__(128) tri_block_factor(TriGeom g, const double *__restrict__ d,
                                                        const double *__restrict__ e,
                                                        const double *__restrict__ V, TriPoles ps,
                                                        cx<R> *__restrict__ fact, cx<R> *__restrict__ us,
                                                        cx<R> *__restrict__ wsp, cx<R> *__restrict__ spk,
                                                        cx<R> *__restrict__ yend) {
    using O = RealOps<R>;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)g.S * g.P) return;
    const int b = (int)(tid % g.P);
    const int s = (int)(tid / g.P);
    const int64_t first = (int64_t)b * g.B;
    const int len = (b < g.P - 1) ? g.m : (int)(g.N - first);
    const cx<R> theta = cx_from<R>(ps.th_re[s] - g.cshift, ps.th_im[s]);
    const R tt = O::from(g.t);
    cx<R> *F = fact + ((int64_t)s * g.N) * 2;
    cx<R> *U = us + (int64_t)s * g.N;
    cx<R> *W = wsp + (int64_t)s * g.N;

    // forward: LU of M_b (c'_i, g_i = 1/w_i) and the forward-eliminated eps_first
    cx<R> cprev = cxz<R>(), hprev = cxz<R>();
    for (int i = 0; i < len; ++i) {
        const int64_t q = first + i;
        cx<R> w = {tt * O::from(d[q]) + theta.re, theta.im};
        R elow = O::zero();
        if (i > 0) {
            elow = tt * O::from(e[q - 1]);
            w = w - scale(elow, cprev);
        }
        const cx<R> gi = cinv(w);
        cx<R> cp = cxz<R>();
        if (i < len - 1) cp = scale(tt * O::from(e[q]), gi);
        const cx<R> h = (i == 0) ? gi : -(gi * scale(elow, hprev));
        F[2 * q] = cp;
        F[2 * q + 1] = gi;
        U[q] = h;
        cprev = cp;
        hprev = h;
    }
    // backward: u = M_b^{-1} eps_first, w = M_b^{-1} eps_last
    cx<R> un = cxz<R>(), wn = cxz<R>();
    cx<R> u0, uL, w0, wL;
    for (int i = len - 1; i >= 0; --i) {
        const int64_t q = first + i;
        cx<R> u, w;
        if (i == len - 1) {
            u = U[q];
            w = F[2 * q + 1];
            uL = u;
            wL = w;
        } else {
            const cx<R> cp = F[2 * q];
            u = U[q] - cp * un;
            w = -(cp * wn);
        }
        U[q] = u;
        W[q] = w;
        un = u;
        wn = w;
    }
    u0 = un;
    w0 = wn;
    cx<R> *SP = spk + ((int64_t)s * g.P + b) * 4;
    SP[0] = u0;
    SP[1] = uL;
    SP[2] = w0;
    SP[3] = wL;
    // end values of y_b = M_b^{-1} v_b for every column: u^T v and w^T v
    cx<R> *YE = yend + ((int64_t)s * g.P + b) * g.Rc * 2;
    for (int j0 = 0; j0 < g.Rc; j0 += TRI_RCH) {
        cx<R> yu[TRI_RCH], yw[TRI_RCH];
#pragma unroll
        for (int jj = 0; jj < TRI_RCH; ++jj) yu[jj] = yw[jj] = cxz<R>();
        for (int i = 0; i < len; ++i) {
            const int64_t q = first + i;
            const cx<R> u = U[q], w = W[q];
            const double *vr = V + q * g.Rc + j0;
#pragma unroll
            for (int jj = 0; jj < TRI_RCH; ++jj) {
                if (j0 + jj < g.Rc) {
                    const R v = O::from(vr[jj]);
                    yu[jj] = yu[jj] + scale(v, u);
                    yw[jj] = yw[jj] + scale(v, w);
                }
            }
        }
#pragma unroll
        for (int jj = 0; jj < TRI_RCH; ++jj)
            if (j0 + jj < g.Rc) {
                YE[2 * (j0 + jj)] = yu[jj];
                YE[2 * (j0 + jj) + 1] = yw[jj];
            }
    }
}

// Reduced system for the separators of one (system, column):
//   A_b sigma_{b-1} + B_b sigma_b + C_b sigma_{b+1} = D_b,   b = 0 .. P-2
// solved by cyclic reduction (odd-even elimination) in shared memory.
template <class R>
__global__ void __launch_bounds__(1024) tri_reduced_cr(TriGeom g, const double *__restrict__ d,
                                                       const double *__restrict__ e,
                                                       const double *__restrict__ V, TriPoles ps,
                                                       const cx<R> *__restrict__ spk,
                                                       const cx<R> *__restrict__ yend,
                                                       cx<R> *__restrict__ sigma) {
    using O = RealOps<R>;
    extern __shared__ unsigned char smem_raw[];
    const int n = g.P - 1;
    cx<R> *A = reinterpret_cast<cx<R> *>(smem_raw);
    cx<R> *Bc = A + n;
    cx<R> *C = Bc + n;
    cx<R> *D = C + n;
    const int s = blockIdx.x / g.Rc;
    const int j = blockIdx.x % g.Rc;
    const cx<R> theta = cx_from<R>(ps.th_re[s] - g.cshift, ps.th_im[s]);
    const R tt = O::from(g.t);
    const cx<R> *SP = spk + (int64_t)s * g.P * 4;
    const cx<R> *YE = yend + (int64_t)s * g.P * g.Rc * 2;

    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        const int64_t r = (int64_t)b * g.B + g.m;  // separator row
        const R el = tt * O::from(e[r - 1]);       // couples sigma_b and the last row of block b
        const R er = tt * O::from(e[r]);           // couples sigma_b and the first row of block b+1
        const cx<R> uL = SP[4 * b + 1], wL = SP[4 * b + 3];
        const cx<R> u0n = SP[4 * (b + 1) + 0], w0n = SP[4 * (b + 1) + 2];
        cx<R> Ab = cxz<R>(), Cb = cxz<R>();
        if (b >= 1) {
            const R erp = tt * O::from(e[r - g.B]);  // t e at the previous separator's right side
            Ab = -scale(el * erp, uL);
        }
        if (b + 1 <= n - 1) {
            const R eln = tt * O::from(e[r + g.B - 1]);  // t e at the next separator's left side
            Cb = -scale(er * eln, w0n);
        }
        cx<R> Bb = {tt * O::from(d[r]) + theta.re, theta.im};
        Bb = Bb - scale(el * el, wL) - scale(er * er, u0n);
        const cx<R> yL = YE[(int64_t)b * g.Rc * 2 + 2 * j + 1];        // y_b[last]
        const cx<R> y0n = YE[(int64_t)(b + 1) * g.Rc * 2 + 2 * j + 0];  // y_{b+1}[first]
        cx<R> Db = {O::from(V[r * g.Rc + j]), O::zero()};
        Db = Db - scale(el, yL) - scale(er, y0n);
        A[b] = Ab;
        Bc[b] = Bb;
        C[b] = Cb;
        D[b] = Db;
    }
    __syncthreads();
    int stride = 1;
    for (; 2 * stride - 1 < n; stride *= 2) {
        for (int i = 2 * stride - 1 + 2 * stride * threadIdx.x; i < n; i += 2 * stride * blockDim.x) {
            const int lo = i - stride, hi = i + stride;
            const cx<R> k1 = A[i] * cinv(Bc[lo]);
            cx<R> nb = Bc[i] - k1 * C[lo];
            cx<R> nd = D[i] - k1 * D[lo];
            cx<R> na = -(k1 * A[lo]);
            cx<R> nc = cxz<R>();
            if (hi < n) {
                const cx<R> k2 = C[i] * cinv(Bc[hi]);
                nb = nb - k2 * A[hi];
                nd = nd - k2 * D[hi];
                nc = -(k2 * C[hi]);
            }
            A[i] = na;
            Bc[i] = nb;
            C[i] = nc;
            D[i] = nd;
        }
        __syncthreads();
    }
    int top = 1;
    while (top * 2 <= n) top *= 2;
    for (int st = top; st >= 1; st /= 2) {
        for (int i = st - 1 + 2 * st * threadIdx.x; i < n; i += 2 * st * blockDim.x) {
            cx<R> rhs = D[i];
            if (i - st >= 0) rhs = rhs - A[i] * D[i - st];
            if (i + st < n) rhs = rhs - C[i] * D[i + st];
            D[i] = rhs * cinv(Bc[i]);  // D now holds the solution at index i
        }
        __syncthreads();
    }
    cx<R> *SG = sigma + (int64_t)s * g.P * g.Rc;
    for (int b = threadIdx.x; b < n; b += blockDim.x) SG[(int64_t)b * g.Rc + j] = D[b];
}

// K3: one thread per (block, column).  Systems are processed in groups of
// TRI_SG; the forward sweep of a group stores d'_i in `scr`, the back sweep
// forms x_i for every system of the group and adds Re(W_s x_i) into Y.
template <class R>
__global__ void __launch_bounds__(128) tri_block_solve(TriGeom g, const double *__restrict__ e,
                                                       const double *__restrict__ V, TriPoles ps,
                                                       const cx<R> *__restrict__ fact,
                                                       const cx<R> *__restrict__ sigma,
                                                       cx<R> *__restrict__ scr, double *__restrict__ Y) {
    using O = RealOps<R>;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)g.P * g.Rc) return;
    const int j = (int)(tid % g.Rc);
    const int b = (int)(tid / g.Rc);
    const int64_t first = (int64_t)b * g.B;
    const int len = (b < g.P - 1) ? g.m : (int)(g.N - first);
    const R tt = O::from(g.t);
    const bool has_left = b > 0, has_right = b < g.P - 1;
    const R eleft = has_left ? tt * O::from(e[first - 1]) : O::zero();
    const R eright = has_right ? tt * O::from(e[first + len - 1]) : O::zero();

    for (int s0 = 0; s0 < g.S; s0 += TRI_SG) {
        const int ns = min(TRI_SG, g.S - s0);
        cx<R> sl[TRI_SG], sr[TRI_SG], dp[TRI_SG];
#pragma unroll
        for (int k = 0; k < TRI_SG; ++k) {
            sl[k] = sr[k] = dp[k] = cxz<R>();
            if (k < ns) {
                const cx<R> *SG = sigma + (int64_t)(s0 + k) * g.P * g.Rc;
                if (has_left) sl[k] = SG[(int64_t)(b - 1) * g.Rc + j];
                if (has_right) sr[k] = SG[(int64_t)b * g.Rc + j];
            }
        }
        // forward substitution, all systems of the group together
        for (int i = 0; i < len; ++i) {
            const int64_t q = first + i;
            const R v = O::from(V[q * g.Rc + j]);
            const R elow = (i > 0) ? tt * O::from(e[q - 1]) : O::zero();
            cx<R> *SC = scr + (((int64_t)q * TRI_SG) * g.Rc + j);
#pragma unroll
            for (int k = 0; k < TRI_SG; ++k) {
                if (k < ns) {
                    cx<R> rhs = {v, O::zero()};
                    if (i == 0 && has_left) rhs = rhs - scale(eleft, sl[k]);
                    if (i == len - 1 && has_right) rhs = rhs - scale(eright, sr[k]);
                    if (i > 0) rhs = rhs - scale(elow, dp[k]);
                    const cx<R> gi = fact[((int64_t)(s0 + k) * g.N + q) * 2 + 1];
                    dp[k] = gi * rhs;
                    SC[(int64_t)k * g.Rc] = dp[k];
                }
            }
        }
        // back substitution and weighted sum
        cx<R> xn[TRI_SG];
#pragma unroll
        for (int k = 0; k < TRI_SG; ++k) xn[k] = cxz<R>();
        for (int i = len - 1; i >= 0; --i) {
            const int64_t q = first + i;
            const cx<R> *SC = scr + (((int64_t)q * TRI_SG) * g.Rc + j);
            R acc = O::zero();
#pragma unroll
            for (int k = 0; k < TRI_SG; ++k) {
                if (k < ns) {
                    cx<R> x = SC[(int64_t)k * g.Rc];
                    if (i < len - 1) x = x - fact[((int64_t)(s0 + k) * g.N + q) * 2] * xn[k];
                    xn[k] = x;
                    acc = acc + re_mul(cx_from<R>(ps.w_re[s0 + k], ps.w_im[s0 + k]), x);
                }
            }
            double out = O::todbl(acc);
            if (s0 > 0) out += Y[q * g.Rc + j];
            Y[q * g.Rc + j] = out;
        }
        // the separator row that follows this block
        if (has_right) {
            const int64_t r = first + len;
            R acc = O::zero();
#pragma unroll
            for (int k = 0; k < TRI_SG; ++k)
                if (k < ns) acc = acc + re_mul(cx_from<R>(ps.w_re[s0 + k], ps.w_im[s0 + k]), sr[k]);
            double out = O::todbl(acc);
            if (s0 > 0) out += Y[r * g.Rc + j];
            Y[r * g.Rc + j] = out;
        }
    }
}

// ------------------------------------------------------------------ host side

TriGeom tri_geometry(int64_t N, int S, int Rc, bool ff, int sm_count) {
    TriGeom g{};
    g.N = N;
    g.S = S;
    g.Rc = Rc;
    // enough (system, block) threads to keep every SM sub-partition busy in K1
    const int64_t warps_per_sm = ff ? 8 : 4;
    const int64_t target = (int64_t)sm_count * warps_per_sm * 32;
    int64_t P = (target + S - 1) / S;
    P = std::max<int64_t>(1, std::min<int64_t>(P, TRI_PMAX));
    int64_t m = (N - P + 1 + P - 1) / P;  // ceil((N - (P-1)) / P)
    m = std::max<int64_t>(m, TRI_MMIN);
    const int64_t B = m + 1;
    P = (N + B - 1) / B;  // last block length N - (P-1) B lies in [1, B]
    if (P > TRI_PMAX) {   // very long systems: grow the blocks instead
        const int64_t Bmin = (N + TRI_PMAX - 1) / TRI_PMAX;
        m = Bmin;  // B = m + 1 >= Bmin guarantees P <= TRI_PMAX
        P = (N + m) / (m + 1);
    }
    g.m = (int)m;
    g.B = (int)(m + 1);
    g.P = (int)P;
    return g;
}

size_t tri_workspace_bytes(const TriGeom &g, bool ff) {
    const size_t c = 16;  // sizeof(cx<double>) == sizeof(cx<f32x2>)
    (void)ff;
    size_t fact = (size_t)g.S * g.N * 2 * c;
    size_t us = (size_t)g.S * g.N * c, ws = us;
    size_t spk = (size_t)g.S * g.P * 4 * c;
    size_t yend = (size_t)g.S * g.P * g.Rc * 2 * c;
    size_t sig = (size_t)g.S * g.P * g.Rc * c;
    size_t scr = (size_t)g.N * TRI_SG * g.Rc * c;
    size_t k1 = us + ws;
    return fact + spk + yend + sig + std::max(k1, scr) + 6 * 256;
}

static inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

template <class R>
static cudaError_t tri_run_t(const TriGeom &g, const double *d, const double *e, const double *V,
                             double *Y, const TriPoles &ps, void *work, cudaStream_t st, Profiler &prof) {
    const size_t c = sizeof(cx<R>);
    unsigned char *p = (unsigned char *)work;
    cx<R> *fact = (cx<R> *)p;
    p += align_up((size_t)g.S * g.N * 2 * c);
    cx<R> *spk = (cx<R> *)p;
    p += align_up((size_t)g.S * g.P * 4 * c);
    cx<R> *yend = (cx<R> *)p;
    p += align_up((size_t)g.S * g.P * g.Rc * 2 * c);
    cx<R> *sig = (cx<R> *)p;
    p += align_up((size_t)g.S * g.P * g.Rc * c);
    // K1's spike scratch and K3's forward scratch share one region
    cx<R> *us = (cx<R> *)p;
    cx<R> *wsp = us + (size_t)g.S * g.N;
    cx<R> *scr = (cx<R> *)p;

    const bool ff = sizeof(R) != sizeof(double) || !std::is_same<R, double>::value;
    const int64_t n1 = (int64_t)g.S * g.P;
    cudaError_t err = prof.timed(ff ? "tri_block_factor<f32x2>" : "tri_block_factor<f64>", st, [&] {
        tri_block_factor<R><<<(unsigned)((n1 + 127) / 128), 128, 0, st>>>(g, d, e, V, ps, fact, us, wsp, spk,
                                                                            yend);
        return cudaGetLastError();
    });
    if (err != cudaSuccess) return err;
    if (g.P > 1) {
        const size_t smem = (size_t)4 * (g.P - 1) * c;
        err = cudaFuncSetAttribute(tri_reduced_cr<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        err = prof.timed(ff ? "tri_reduced_cr<f32x2>" : "tri_reduced_cr<f64>", st, [&] {
            tri_reduced_cr<R><<<g.S * g.Rc, 512, smem, st>>>(g, d, e, V, ps, spk, yend, sig);
            return cudaGetLastError();
        });
        if (err != cudaSuccess) return err;
    }
    const int64_t n3 = (int64_t)g.P * g.Rc;
    return prof.timed(ff ? "tri_block_solve<f32x2>" : "tri_block_solve<f64>", st, [&] {
        tri_block_solve<R><<<(unsigned)((n3 + 127) / 128), 128, 0, st>>>(g, e, V, ps, fact, sig, scr, Y);
        return cudaGetLastError();
    });
}

cudaError_t tri_run(const TriGeom &g, bool ff, const double *d, const double *e, const double *V, double *Y,
                    const TriPoles &ps, void *work, cudaStream_t st, Profiler &prof) {
    return ff ? tri_run_t<f32x2>(g, d, e, V, Y, ps, work, st, prof)
              : tri_run_t<double>(g, d, e, V, Y, ps, work, st, prof);
}

}  // namespace expm
