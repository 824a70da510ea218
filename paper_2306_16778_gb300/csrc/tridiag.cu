// tridiag.cu -- pole-batched shifted tridiagonal solves with the fused residue sum.
//
// Computes Y = sum_s Re(W_s X_s) where X_s solves
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
//   K0 tri_prep          d' = t d - c and e' = t e (and, for float-float, V split
//                        into float pairs) -- once per call, so no kernel below
//                        repeats the scaling or a binary64 conversion per system.
//   K1a tri_block_factor one thread per (system, block): unpivoted LU of M_b
//                        (stored) and the unit spikes u_b, w_b.
//   K1b tri_block_dots   one thread per (system, block, column): y_b end values.
//   K2 tri_reduced_cr    one CTA per (system, column): the reduced system by cyclic
//                        reduction in shared memory.
//   K3 tri_block_solve   one thread per (block, column, system): forward and back
//                        substitution with the separator values as boundary data;
//                        Re(W_s x_s) summed over the systems by a reduce-scatter
//                        across the system lanes, one chunk of rows at a time.
//   K4 tri_finish        float-float only: the float pairs of Y to binary64.
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
#include "tridiag_kernels.cuh"
#include "plan.cuh"

namespace expm {

// ------------------------------------------------------------------ K3
// One thread per (block, column, system).  The systems of one (block, column) sit in
// LG consecutive lanes (LG = power of two >= S, <= 32); each lane runs the forward
// and back substitution of its system, and Re(W_s x_s) is summed over the LG lanes
// by a reduce-scatter over chunks of LG rows in a fixed order (the result does not
// depend on scheduling).
// The next row's loads are issued one iteration ahead.  Output: binary64 Y, or for
// float-float the unrounded pair (hi, lo) stored in Y's 8 bytes, finished by K4.
template <class R> EXPM_D void store_out(double *Y, int64_t idx, R v);
template <> EXPM_D void store_out<double>(double *Y, int64_t idx, double v) { Y[idx] = v; }
template <> EXPM_D void store_out<f32x2>(double *Y, int64_t idx, f32x2 v) {
    reinterpret_cast<f32x2 *>(Y)[idx] = v;
}

// z = a v - b z_prev  (a, b, z_prev complex; v real): one row of the weighted forward
// substitution, two multiplies and four FMAs in binary64
template <class R> EXPM_D cx<R> zstep(cx<R> a, cx<R> b, R v, cx<R> zp) {
    return {a.re * v - b.re * zp.re + b.im * zp.im, a.im * v - b.re * zp.im - b.im * zp.re};
}
template <> EXPM_D cx<double> zstep<double>(cx<double> a, cx<double> b, double v, cx<double> zp) {
    return {fma(b.im, zp.im, fma(-b.re, zp.re, a.re * v)), fma(-b.im, zp.re, fma(-b.re, zp.im, a.im * v))};
}

template <class R, int LG>
__global__ void __launch_bounds__(128) tri_block_solve(TriGeom g, const R *__restrict__ eP,
                                                       const R *__restrict__ VP, TriPoles ps,
                                                       const cx<R> *__restrict__ fact,
                                                       const cx<R> *__restrict__ sigma,
                                                       cx<R> *__restrict__ scr, double *__restrict__ Y) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = (int)(tid % LG);
    const int64_t bj = tid / LG;
    // groups past the end leave as a whole (LG divides the CTA size); the shuffles
    // use the group's own lane mask
    if (bj >= (int64_t)g.P * g.Rc) return;
    const unsigned lane = threadIdx.x & 31;
    const unsigned gmask = (LG == 32) ? 0xffffffffu : (((1u << LG) - 1u) << (lane & ~(unsigned)(LG - 1)));
    const int j = (int)(bj % g.Rc);
    const int b = (int)(bj / g.Rc);
    const bool active = sl < g.S;
    const int s = active ? sl : 0;  // idle lanes shadow system 0 and contribute zero
    const int64_t first = (int64_t)b * g.B;
    const int len = (b < g.P - 1) ? g.m : (int)(g.N - first);
    const bool has_left = b > 0, has_right = b < g.P - 1;
    const cx<R> wgt = active ? cx_from<R>(ps.w_re[s], ps.w_im[s]) : cxz<R>();
    const cx<R> *SG = sigma + (int64_t)s * g.P * g.Rc;
    const cx<R> sl_v = has_left ? SG[(int64_t)(b - 1) * g.Rc + j] : cxz<R>();
    const cx<R> sr_v = has_right ? SG[(int64_t)b * g.Rc + j] : cxz<R>();
    const R eleft = has_left ? eP[first - 1] : RealOps<R>::zero();
    const R eright = has_right ? eP[first + len - 1] : RealOps<R>::zero();
    const cx<R> *F = fact + (int64_t)s * g.N * 3;  // per row: c', a = W g, b = g e'_{q-1}
    cx<R> *SC = scr + (((int64_t)first * g.Rc + j) * LG + sl);  // this lane's column
    const int64_t sstride = (int64_t)g.Rc * LG;

    // forward substitution on z = W d' (the factor kernel folded W into a and b):
    // z_i = a_i (v_i - boundary terms) - b_i z_{i-1}; the back substitution then gives W x
    cx<R> dz = cxz<R>();
    R vn = VP[first * g.Rc + j];
    cx<R> an = F[3 * first + 1], bn = F[3 * first + 2];
    for (int i = 0; i < len; ++i) {
        const int64_t q = first + i;
        const R vq = vn;
        const cx<R> aq = an, bq = bn;
        if (i + 1 < len) {
            vn = VP[(q + 1) * g.Rc + j];
            an = F[3 * (q + 1) + 1];
            bn = F[3 * (q + 1) + 2];
        }
        if ((i == 0 && has_left) || (i == len - 1 && has_right)) {  // a separator value enters
            cx<R> rhs = {vq, RealOps<R>::zero()};
            if (i == 0 && has_left) rhs = rhs - scale(eleft, sl_v);
            if (i == len - 1 && has_right) rhs = rhs - scale(eright, sr_v);
            dz = aq * rhs - bq * dz;
        } else {
            dz = zstep(aq, bq, vq, dz);  // b = 0 on a block's first row
        }
        SC[(int64_t)i * sstride] = dz;
    }
    // back substitution in chunks of LG rows; each chunk's weighted contributions
    // are reduce-scattered so lane l writes row (i0 - l) of column j
    cx<R> xn = cxz<R>();
    cx<R> scn = SC[(int64_t)(len - 1) * sstride];
    cx<R> cn = (len > 1) ? F[3 * (first + len - 2)] : cxz<R>();  // c' of row last-1
    for (int i0 = len - 1; i0 >= 0; i0 -= LG) {
        R v[LG];
#pragma unroll
        for (int r = 0; r < LG; ++r) {
            const int i = i0 - r;
            v[r] = RealOps<R>::zero();
            if (i >= 0) {
                const cx<R> sc = scn;
                if (i > 0) scn = SC[(int64_t)(i - 1) * sstride];
                cx<R> x = sc;
                if (i < len - 1) {
                    x = csub_mul(sc, cn, xn);            // cn is c'[row i]
                    if (i > 0) cn = F[3 * (first + i - 1)];  // c'[row i-1] for the next row
                }
                xn = x;
                v[r] = active ? x.re : RealOps<R>::zero();  // x is W x_s: its real part is the term
            }
        }
        reduce_scatter<LG>(gmask, sl, v);
        const int i = i0 - sl;
        if (i >= 0) store_out<R>(Y, (first + i) * g.Rc + j, v[0]);
    }
    // the separator row that follows this block
    R acc = re_mul(wgt, sr_v);
#pragma unroll
    for (int off = LG / 2; off > 0; off >>= 1) acc = acc + shfl_xor(gmask, acc, off);
    if (sl == 0 && has_right) store_out<R>(Y, (first + len) * g.Rc + j, acc);
}

// ------------------------------------------------------------------ host side

TriGeom tri_geometry(int64_t N, int S, int Rc, bool ff, int sm_count) {
    TriGeom g{};
    g.N = N;
    g.S = S;
    g.Rc = Rc;
    // enough (system, block) threads to keep every SM sub-partition busy in K1a
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
    int lg = 1;
    while (lg < S) lg *= 2;
    g.LG = lg;
    return g;
}

static inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Buffers of one evaluation.  The factor part (dP, eP, fact, us, ws, spk) depends
// only on T, t, c and the poles and can be kept for later right-hand sides; the
// solve part (VP, yend, sig, scr) is per call.  In a single call scr overlays us/ws,
// which are dead once K1b has run.
struct TriLayout {
    size_t fact, spk, us, prepd, prepe, factor_total;  // factor part
    size_t yend, sig, scr, prepv, solve_total;          // solve part (offsets from its own base)
};

static TriLayout tri_layout(const TriGeom &g, bool ff) {
    const size_t c = 16;  // sizeof(cx<double>) == sizeof(cx<f32x2>)
    TriLayout L{};
    size_t off = 0;
    L.fact = off; off += align_up((size_t)g.S * g.N * 3 * c);
    L.spk = off; off += align_up((size_t)g.S * g.P * 4 * c);
    L.prepd = off; off += align_up((size_t)g.N * 8);
    L.prepe = off; off += align_up((size_t)g.N * 8);
    L.us = off; off += align_up((size_t)g.S * g.N * 2 * c);  // us then ws
    L.factor_total = off;
    off = 0;
    L.yend = off; off += align_up((size_t)g.S * g.P * g.Rc * 2 * c);
    L.sig = off; off += align_up((size_t)g.S * g.P * g.Rc * c);
    L.prepv = off; if (ff) off += align_up((size_t)g.N * g.Rc * 8);
    L.scr = off; off += align_up((size_t)g.N * g.LG * g.Rc * c);
    L.solve_total = off;
    return L;
}

size_t tri_factor_bytes(const TriGeom &g, bool ff) { return tri_layout(g, ff).factor_total; }
size_t tri_solve_bytes(const TriGeom &g, bool ff) { return tri_layout(g, ff).solve_total; }

// A single call uses one workspace: [factor part | overflow | yend, sig, prepv].  The K3
// scratch starts at the spikes (dead after K1b) and runs into the overflow area when
// it is larger than them.
static size_t tri_overflow(const TriGeom &g) {
    const size_t scr = (size_t)g.N * g.LG * g.Rc * 16;
    const size_t spikes = (size_t)g.S * g.N * 2 * 16;
    return scr > spikes ? align_up(scr - spikes) : 0;
}

size_t tri_workspace_bytes(const TriGeom &g, bool ff) {
    const TriLayout L = tri_layout(g, ff);
    return L.factor_total + tri_overflow(g) + L.scr;  // L.scr = bytes of yend, sig, prepv
}

template <class R>
static cudaError_t tri_factor_t(const TriGeom &g, const double *d, const double *e, const TriPoles &ps,
                                void *fwork, cudaStream_t st, Profiler &prof) {
    const bool ff = !std::is_same<R, double>::value;
    const TriLayout L = tri_layout(g, ff);
    unsigned char *p = (unsigned char *)fwork;
    cx<R> *fact = (cx<R> *)(p + L.fact);
    cx<R> *spk = (cx<R> *)(p + L.spk);
    cx<R> *us = (cx<R> *)(p + L.us);
    cx<R> *wsp = us + (size_t)g.S * g.N;
    R *dP = (R *)(p + L.prepd);
    R *eP = (R *)(p + L.prepe);
    const unsigned pgrid = (unsigned)std::min<int64_t>((g.N + 255) / 256, 152 * 8);
    cudaError_t err = prof.timed(ff ? "tri_prep<f32x2>" : "tri_prep<f64>", st, [&] {
        tri_prep<R><<<pgrid, 256, 0, st>>>(g, d, e, nullptr, dP, eP, (R *)nullptr);
        return cudaGetLastError();
    });
    if (err != cudaSuccess) return err;
    const int64_t n1 = (int64_t)g.S * g.P;
    return prof.timed(ff ? "tri_block_factor<f32x2>" : "tri_block_factor<f64>", st, [&] {
        tri_block_factor<R><<<(unsigned)((n1 + 127) / 128), 128, 0, st>>>(g, dP, eP, ps, fact, us, wsp, spk);
        return cudaGetLastError();
    });
}

template <class R>
static cudaError_t tri_solve_t(const TriGeom &g, const double *V, double *Y, const TriPoles &ps, const void *fwork,
                               void *swork, void *scr_override, cudaStream_t st, Profiler &prof) {
    const bool ff = !std::is_same<R, double>::value;
    const TriLayout L = tri_layout(g, ff);
    const unsigned char *p = (const unsigned char *)fwork;
    const cx<R> *fact = (const cx<R> *)(p + L.fact);
    const cx<R> *spk = (const cx<R> *)(p + L.spk);
    const cx<R> *us = (const cx<R> *)(p + L.us);
    const cx<R> *wsp = us + (size_t)g.S * g.N;
    const R *dP = (const R *)(p + L.prepd);
    const R *eP = (const R *)(p + L.prepe);
    unsigned char *q = (unsigned char *)swork;
    cx<R> *yend = (cx<R> *)(q + L.yend);
    cx<R> *sig = (cx<R> *)(q + L.sig);
    R *VP = ff ? (R *)(q + L.prepv) : nullptr;
    cx<R> *scr = scr_override ? (cx<R> *)scr_override : (cx<R> *)(q + L.scr);
    const R *Vuse = ff ? VP : reinterpret_cast<const R *>(V);
    cudaError_t err = cudaSuccess;
    if (ff) {
        const unsigned pgrid = (unsigned)std::min<int64_t>((g.N * g.Rc + 255) / 256, 152 * 8);
        err = prof.timed("tri_prep_rhs<f32x2>", st, [&] {
            tri_prep<R><<<pgrid, 256, 0, st>>>(g, nullptr, nullptr, V, nullptr, nullptr, VP);
            return cudaGetLastError();
        });
        if (err != cudaSuccess) return err;
    }
    const int64_t n1b = (int64_t)g.S * g.P * g.Rc;
    err = prof.timed(ff ? "tri_block_dots<f32x2>" : "tri_block_dots<f64>", st, [&] {
        tri_block_dots<R><<<(unsigned)((n1b + 127) / 128), 128, 0, st>>>(g, Vuse, us, wsp, yend);
        return cudaGetLastError();
    });
    if (err != cudaSuccess) return err;
    if (g.P > 1) {
        const size_t smem = 4 * cr_len<R>(g.P - 1) * sizeof(cx<R>);
        // the attribute is a ceiling: set it to the largest reduced system (TRI_PMAX) so
        // that concurrent callers (server workers) never lower it under another's launch
        err = cudaFuncSetAttribute(tri_reduced_cr<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(4 * cr_len<R>(TRI_PMAX - 1) * sizeof(cx<R>)));
        if (err != cudaSuccess) return err;
        err = prof.timed(ff ? "tri_reduced_cr<f32x2>" : "tri_reduced_cr<f64>", st, [&] {
            tri_reduced_cr<R><<<g.S * g.Rc, 512, smem, st>>>(g, dP, eP, Vuse, nullptr, ps, spk, yend, sig, nullptr);
            return cudaGetLastError();
        });
        if (err != cudaSuccess) return err;
    }
    const int64_t n3 = (int64_t)g.P * g.Rc * g.LG;  // LG divides 128: groups never straddle CTAs
    err = prof.timed(ff ? "tri_block_solve<f32x2>" : "tri_block_solve<f64>", st, [&] {
        const unsigned grid = (unsigned)((n3 + 127) / 128);
        switch (g.LG) {
            case 1: tri_block_solve<R, 1><<<grid, 128, 0, st>>>(g, eP, Vuse, ps, fact, sig, scr, Y); break;
            case 2: tri_block_solve<R, 2><<<grid, 128, 0, st>>>(g, eP, Vuse, ps, fact, sig, scr, Y); break;
            case 4: tri_block_solve<R, 4><<<grid, 128, 0, st>>>(g, eP, Vuse, ps, fact, sig, scr, Y); break;
            case 8: tri_block_solve<R, 8><<<grid, 128, 0, st>>>(g, eP, Vuse, ps, fact, sig, scr, Y); break;
            case 16: tri_block_solve<R, 16><<<grid, 128, 0, st>>>(g, eP, Vuse, ps, fact, sig, scr, Y); break;
            default: tri_block_solve<R, 32><<<grid, 128, 0, st>>>(g, eP, Vuse, ps, fact, sig, scr, Y); break;
        }
        return cudaGetLastError();
    });
    if (err != cudaSuccess || !ff) return err;
    return prof.timed("tri_finish<f32x2>", st, [&] {
        const int64_t ny = g.N * g.Rc;
        tri_finish<<<(unsigned)std::min<int64_t>((ny + 255) / 256, 152 * 8), 256, 0, st>>>(ny, Y);
        return cudaGetLastError();
    });
}

cudaError_t tri_factor(const TriGeom &g, bool ff, const double *d, const double *e, const TriPoles &ps, void *fwork,
                       cudaStream_t st, Profiler &prof) {
    return ff ? tri_factor_t<f32x2>(g, d, e, ps, fwork, st, prof) : tri_factor_t<double>(g, d, e, ps, fwork, st, prof);
}

cudaError_t tri_solve(const TriGeom &g, bool ff, const double *V, double *Y, const TriPoles &ps, const void *fwork,
                      void *swork, cudaStream_t st, Profiler &prof) {
    return ff ? tri_solve_t<f32x2>(g, V, Y, ps, fwork, swork, nullptr, st, prof)
              : tri_solve_t<double>(g, V, Y, ps, fwork, swork, nullptr, st, prof);
}

cudaError_t tri_run(const TriGeom &g, bool ff, const double *d, const double *e, const double *V, double *Y,
                    const TriPoles &ps, void *work, cudaStream_t st, Profiler &prof, cudaEvent_t v_ready) {
    const TriLayout L = tri_layout(g, ff);
    unsigned char *p = (unsigned char *)work;
    void *scr = p + L.us;
    unsigned char *solve_base = p + L.factor_total + tri_overflow(g);
    cudaError_t err = ff ? tri_factor_t<f32x2>(g, d, e, ps, p, st, prof) : tri_factor_t<double>(g, d, e, ps, p, st, prof);
    if (err == cudaSuccess && v_ready) err = cudaStreamWaitEvent(st, v_ready, 0);  // V arrives on another stream
    if (err != cudaSuccess) return err;
    return ff ? tri_solve_t<f32x2>(g, V, Y, ps, p, solve_base, scr, st, prof)
              : tri_solve_t<double>(g, V, Y, ps, p, solve_base, scr, st, prof);
}

}  // namespace expm
