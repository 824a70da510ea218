// tridiag_mixed.cu -- the tridiagonal path in binary32 with iterative refinement
// (EXPM_MIXED_FP32).
//
// Same problem as tridiag.cu: Y = sum_s Re(W_s X_s) with (t T - c I + theta_s I) X_s = V
// (eq. expAx, conjugate pairs folded by Remark 5.1).  The shifted matrices M_s are
// factored once in binary32 by the separator partition of tridiag.cu (block LUs,
// spikes, reduced system), and every solve with those factors (written M~^{-1}) is
// binary32 arithmetic.  Accuracy is won back by refinement:
//     pass 0:   x_0 = M~^{-1} v,          r_1     = v   - M x_0
//     pass k:   d_k = M~^{-1} r_k,        r_{k+1} = r_k - M d_k
//     Y = sum_s Re(W_s x_0) + sum_k sum_s Re(W_s d_k).
// Each pass contracts the error by about kappa(M_s) u_32.  Only the first residual
// needs more than binary32: r_1 = v - M x_0 cancels down to ~u_32 |M| |x|, so it is
// formed from the binary64 entries of t T - c I split into float pairs (d' = dPf + dPl,
// e' = ePf + ePl), theta_s split the same way, error-free products (one FMA gives the
// rounding error of a binary32 product) and compensated sums (Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 2005): float-float accuracy on
// the FP32 pipe only.  Later residuals r_{k+1} = r_k - M d_k only cancel from |r_k|,
// so binary32 arithmetic leaves an error of order u_32 |r_k| <= u_32^2 |M| |x|.
//
// Kernels (every launch of a pass after the first returns at once when the
// stopping test has already passed, so the launch sequence is fixed):
//   mx_prep / mx_prep_v      split d', e' and V into float pairs; beta = max row sum
//   mx_factor                binary32 block LUs and spikes, stored [row][system]
//   mx_dots                  pass 0 block end values y_b = u_b^T v_b, w_b^T v_b
//   tri_reduced_cr<float>    reduced separator system of the pass
//   mx_solve                 one thread per (block, column, system), system lanes of a
//                            (block, column) adjacent: forward substitution keeping a
//                            checkpoint every CK rows; then chunk by chunk (last first)
//                            the forward values recomputed into registers and the
//                            back substitution.  Fused: the Y update (reduce-scatter
//                            over the system lanes), the next residual on the block's
//                            rows with its block end dots for the next pass, norms.
//   mx_sep_resid             the residual at the separator rows
//   mx_check                 stopping test  ||r_s||_F <= tol (beta + |theta_s|) ||x_s||_F
//   tri_finish               the float pairs of Y to binary64
#include <cmath>
#include <cstdint>
#include <cstring>

#include "arith.cuh"
#include "plan.cuh"
#include "tridiag.cuh"
#include "tridiag_kernels.cuh"

namespace expm {

namespace {

constexpr int MX_CTA = 128;

enum : int { MX_RESID = 1, MX_STORE = 2, MX_COMP = 4, MX_LO_IN = 8, MX_LO_OUT = 16 };

struct MixState {
    int done;   // stopping test passed: later passes return at once
    int iters;  // correction passes applied
    double resid;
    double xnorm2[TRI_MAXSYS];
};

struct MxArgs {
    const float *dPf, *dPl, *ePf, *ePl;  // t d - c and t e as float pairs
    const float *VPf, *VPl;              // V as float pairs
    const cx<float> *fact, *us, *ws, *sig;
    cx<float> *R, *Rlo;  // interior residuals (binary32 part, low part), [row][column][lane]
    cx<float> *X;        // the pass's solution, [row][column][lane]
    cx<float> *yend, *ckpt;
    cx<float> *sepR, *sepLo;  // separator residuals, [system][separator][column]
    double *Y;                 // float pairs during the passes
    double *part3, *partS;     // per-CTA partial norms of mx_solve and mx_sep_resid
    MixState *state;
    const unsigned *beta_bits;
};

// ------------------------------------------------------------------ prep
__global__ void mx_prep(TriGeom g, const double *__restrict__ d, const double *__restrict__ e, float *dPf,
                        float *dPl, float *ePf, float *ePl, unsigned *beta_bits) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float bmax = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += stride) {
        const double dv = g.t * d[i] - g.cshift;
        const double ev = i + 1 < g.N ? g.t * e[i] : 0.0;
        const double evp = i > 0 ? g.t * e[i - 1] : 0.0;
        const f32x2 ds = split_bits(dv), es = split_bits(ev);
        dPf[i] = ds.hi;
        dPl[i] = ds.lo;
        ePf[i] = es.hi;
        ePl[i] = es.lo;
        bmax = fmaxf(bmax, __double2float_ru(fabs(dv) + fabs(ev) + fabs(evp)));
    }
    for (int off = 16; off > 0; off >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, off));
    if ((threadIdx.x & 31) == 0) atomicMax(beta_bits, __float_as_uint(bmax));  // non-negative: bit order = value order
}

__global__ void mx_prep_v(int64_t n, const double *__restrict__ V, float *VPf, float *VPl) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const f32x2 v = split_bits(V[i]);
        VPf[i] = v.hi;
        VPl[i] = v.lo;
    }
}

// ------------------------------------------------------------------ residual arithmetic
// s + c  -=  (ah + al) x : the binary32 product ah x split exactly by an FMA, the
// rounding error of the running sum s collected in c.
EXPM_D void csum_sub(float &s, float &c, float ah, float al, float x) {
    const float p = __fmul_rn(ah, x);
    float pe = __fmaf_rn(ah, x, -p);
    pe = __fmaf_rn(al, x, pe);
    const f32x2 t = two_sum(s, -p);
    s = t.hi;
    c = __fadd_rn(c, __fsub_rn(t.lo, pe));
}

// Pass 0:  r = v - [ (d_q + theta) x_q + e_{q-1} x_{q-1} + e_q x_{q+1} ]  for one row, with
// x_0 in binary32, v, d', e', theta as float pairs; float-float accurate, returned as
// (hi, lo) per component.
EXPM_D void mx_resid_first(f32x2 v, f32x2 dq, f32x2 el, f32x2 er, f32x2 thr, f32x2 thi, cx<float> xl,
                           cx<float> xs, cx<float> xr, cx<float> &hi, cx<float> &lo) {
    const f32x2 t = two_sum(dq.hi, thr.hi);  // a = d_q + Re theta as an (unnormalised) pair
    const float alo = __fadd_rn(t.lo, __fadd_rn(dq.lo, thr.lo));
    float sr = v.hi, cr = v.lo;
    csum_sub(sr, cr, t.hi, alo, xs.re);
    csum_sub(sr, cr, -thi.hi, -thi.lo, xs.im);
    csum_sub(sr, cr, el.hi, el.lo, xl.re);
    csum_sub(sr, cr, er.hi, er.lo, xr.re);
    const float p = __fmul_rn(t.hi, xs.im);  // imaginary part: v is real
    float pe = __fmaf_rn(t.hi, xs.im, -p);
    pe = __fmaf_rn(alo, xs.im, pe);
    float si = -p, ci = -pe;
    csum_sub(si, ci, thi.hi, thi.lo, xs.re);
    csum_sub(si, ci, el.hi, el.lo, xl.im);
    csum_sub(si, ci, er.hi, er.lo, xr.im);
    const f32x2 a = two_sum(sr, cr), b = two_sum(si, ci);
    hi = {a.hi, b.hi};
    lo = {a.lo, b.lo};
}

// Later stored residuals:  r_{k+1} = r_k - M d_k  with r_k = rh + rl, float-float accurate.
EXPM_D void mx_resid_comp(cx<float> rh, cx<float> rl, f32x2 dq, f32x2 el, f32x2 er, f32x2 thr, f32x2 thi,
                          cx<float> xl, cx<float> xs, cx<float> xr, cx<float> &hi, cx<float> &lo) {
    const f32x2 t = two_sum(dq.hi, thr.hi);
    const float alo = __fadd_rn(t.lo, __fadd_rn(dq.lo, thr.lo));
    float sr = rh.re, cr = rl.re, si = rh.im, ci = rl.im;
    csum_sub(sr, cr, t.hi, alo, xs.re);
    csum_sub(sr, cr, -thi.hi, -thi.lo, xs.im);
    csum_sub(sr, cr, el.hi, el.lo, xl.re);
    csum_sub(sr, cr, er.hi, er.lo, xr.re);
    csum_sub(si, ci, t.hi, alo, xs.im);
    csum_sub(si, ci, thi.hi, thi.lo, xs.re);
    csum_sub(si, ci, el.hi, el.lo, xl.im);
    csum_sub(si, ci, er.hi, er.lo, xr.im);
    const f32x2 a = two_sum(sr, cr), b = two_sum(si, ci);
    hi = {a.hi, b.hi};
    lo = {a.lo, b.lo};
}

// The verification residual r_{K+1} = r_K - M d_K in binary32: its terms are already
// small, so the rounding is O(u_32 |r_K|) -- enough for a norm.
EXPM_D cx<float> mx_resid_corr(cx<float> rk, float dq, float el, float er, float thr, float thi, cx<float> xl,
                               cx<float> xs, cx<float> xr) {
    const float a = __fadd_rn(dq, thr);
    float re = __fmaf_rn(-a, xs.re, rk.re);
    re = __fmaf_rn(thi, xs.im, re);
    re = __fmaf_rn(-el, xl.re, re);
    re = __fmaf_rn(-er, xr.re, re);
    float im = __fmaf_rn(-a, xs.im, rk.im);
    im = __fmaf_rn(-thi, xs.re, im);
    im = __fmaf_rn(-el, xl.im, im);
    im = __fmaf_rn(-er, xr.im, im);
    return {re, im};
}

// Fire-and-forget prefetch of one line into L2: the per-thread row walks below issue
// these MX_PD rows ahead, so the loads of a chunk find their lines in L2 without
// holding registers for loads in flight.
constexpr int MX_PD = 32;
constexpr int MX_RING_BYTES = 4 * 4 * 3 * MX_CTA * 8;  // mx_resid: NST x RK x 3 slots x threads x 8 B
EXPM_D void pf_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Per-thread asynchronous copies global -> shared (8 bytes each), committed in groups:
// a thread streams its own future rows into its shared-memory slots without holding
// registers for the loads in flight.
EXPM_D void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
EXPM_D void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> EXPM_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

EXPM_D cx<float> cmul_rn(cx<float> a, cx<float> b) {
    return {__fmaf_rn(a.re, b.re, -__fmul_rn(a.im, b.im)), __fmaf_rn(a.re, b.im, __fmul_rn(a.im, b.re))};
}
EXPM_D cx<float> cfms_rn(cx<float> s, cx<float> c, cx<float> x) {  // s - c x
    return {__fmaf_rn(c.im, x.im, __fmaf_rn(-c.re, x.re, s.re)), __fmaf_rn(-c.im, x.re, __fmaf_rn(-c.re, x.im, s.im))};
}
EXPM_D cx<float> cfma_rn(cx<float> s, cx<float> c, cx<float> x) {  // s + c x
    return {__fmaf_rn(-c.im, x.im, __fmaf_rn(c.re, x.re, s.re)), __fmaf_rn(c.im, x.re, __fmaf_rn(c.re, x.im, s.im))};
}

// Re(W x): float pair for pass 0 (x_0 carries the full solution), binary32 afterwards
// (the corrections are small, their rounding is below the pair's).
// A float pair summed with the "sloppy" double-word addition (one TwoSum of the high
// parts): its error is O(u_32^2 (|a| + |b|)), which is what the weighted sum over the
// poles needs -- the bound is on the terms, the cancellation is not amplified further.
struct f32x2s {
    float hi, lo;
};
EXPM_D f32x2s operator+(f32x2s a, f32x2s b) {
    const f32x2 s = two_sum(a.hi, b.hi);
    const f32x2 r = fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
    return {r.hi, r.lo};
}
template <> EXPM_D f32x2s shfl_xor<f32x2s>(unsigned mask, f32x2s v, int off) {
    return {__shfl_xor_sync(mask, v.hi, off), __shfl_xor_sync(mask, v.lo, off)};
}

template <bool FIRST> struct WeightT;
template <> struct WeightT<true> {
    using T = f32x2s;
    static EXPM_D T zero() { return {0.f, 0.f}; }
    static EXPM_D T re_wx(f32x2 wr, f32x2 wi, cx<float> x) {
        const float p1 = __fmul_rn(wr.hi, x.re);
        float e1 = __fmaf_rn(wr.hi, x.re, -p1);
        e1 = __fmaf_rn(wr.lo, x.re, e1);
        const float p2 = __fmul_rn(wi.hi, x.im);
        float e2 = __fmaf_rn(wi.hi, x.im, -p2);
        e2 = __fmaf_rn(wi.lo, x.im, e2);
        const f32x2 s = two_sum(p1, -p2);
        const f32x2 r = fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(e1, e2)));
        return {r.hi, r.lo};
    }
    static EXPM_D void update(double *Y, int64_t idx, T v) { reinterpret_cast<f32x2 *>(Y)[idx] = f32x2{v.hi, v.lo}; }
};
template <> struct WeightT<false> {
    using T = float;
    static EXPM_D T zero() { return 0.f; }
    static EXPM_D T re_wx(f32x2 wr, f32x2 wi, cx<float> x) { return __fmaf_rn(wr.hi, x.re, -__fmul_rn(wi.hi, x.im)); }
    static EXPM_D void update(double *Y, int64_t idx, T v) {
        f32x2 *p = reinterpret_cast<f32x2 *>(Y) + idx;
        const f32x2 y = *p;
        const f32x2 s = two_sum(y.hi, v);
        *p = fast_two_sum(s.hi, __fadd_rn(s.lo, y.lo));
    }
};

// Sum per system lane over the CTA into part[blockIdx][lane][2] (fixed order).
template <int LG>
EXPM_D void cta_norms(float rn2, float xn2, double *part) {
    __shared__ float red[MX_CTA / 32][LG][2];
#pragma unroll
    for (int off = 16; off >= LG; off >>= 1) {
        rn2 += __shfl_xor_sync(0xffffffffu, rn2, off);
        xn2 += __shfl_xor_sync(0xffffffffu, xn2, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < LG) {
        red[warp][lane][0] = rn2;
        red[warp][lane][1] = xn2;
    }
    __syncthreads();
    if (threadIdx.x < 2 * LG) {
        const int l = threadIdx.x >> 1, c = threadIdx.x & 1;
        double acc = 0.0;
        for (int w = 0; w < MX_CTA / 32; ++w) acc += (double)red[w][l][c];
        part[((int64_t)blockIdx.x * LG + l) * 2 + c] = acc;
    }
}

// ------------------------------------------------------------------ factor (binary32)
// The binary32 factors and spikes are stored system-interleaved, [row][system]: the S
// systems of one block run in adjacent lanes, so every per-row load and store of the
// factor, dots and solve kernels touches S consecutive elements.
constexpr int MX_FCK = 8;  // rows whose loads are issued together in the factor/dots loops

EXPM_D cx<float> cinv_fast(cx<float> w) {  // 1/w = conj(w)/|w|^2 (binary32, ~2 ulp)
    const float n2 = __fmaf_rn(w.re, w.re, __fmul_rn(w.im, w.im));
    const float r = __fdividef(1.0f, n2);
    return {__fmul_rn(w.re, r), -__fmul_rn(w.im, r)};
}

// One thread per (block, system): unpivoted LU of M_b = (t T - c I + theta_s I)_b in
// binary32 (c'_i, g_i = 1/w_i) and the unit spikes u_b = M_b^{-1} eps_first,
// w_b = M_b^{-1} eps_last; spike end values to spk[system][block][4] for the reduced system.
__global__ void __launch_bounds__(128) mx_factor(TriGeom g, const float *__restrict__ dPf,
                                                 const float *__restrict__ ePf, TriPoles ps, cx<float> *fact,
                                                 cx<float> *us, cx<float> *ws, cx<float> *__restrict__ spk) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)g.S * g.P) return;
    const int s = (int)(tid % g.S);
    const int b = (int)(tid / g.S);
    const int64_t S = g.S;
    const int64_t first = (int64_t)b * g.B;
    const int len = (b < g.P - 1) ? g.m : (int)(g.N - first);
    const cx<float> theta = {__double2float_rn(ps.th_re[s]), __double2float_rn(ps.th_im[s])};
    cx<float> cprev = {0.f, 0.f}, hprev = {0.f, 0.f};
    float eprev = 0.f;
    for (int i0 = 0; i0 < len; i0 += MX_FCK) {
        float dv[MX_FCK], ev[MX_FCK];
#pragma unroll
        for (int r = 0; r < MX_FCK; ++r) {
            const int i = i0 + r;
            dv[r] = i < len ? dPf[first + i] : 0.f;
            ev[r] = i < len ? ePf[first + i] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < MX_FCK; ++r) {
            const int i = i0 + r;
            if (i < len) {
                const int64_t q = first + i;
                cx<float> w = {__fadd_rn(dv[r], theta.re), theta.im};
                if (i > 0) {
                    w.re = __fmaf_rn(-eprev, cprev.re, w.re);
                    w.im = __fmaf_rn(-eprev, cprev.im, w.im);
                }
                const cx<float> gi = cinv_fast(w);
                const cx<float> cp = (i < len - 1) ? cx<float>{__fmul_rn(ev[r], gi.re), __fmul_rn(ev[r], gi.im)}
                                                   : cx<float>{0.f, 0.f};
                const cx<float> h =
                    (i == 0) ? gi : -cmul_rn(gi, cx<float>{__fmul_rn(eprev, hprev.re), __fmul_rn(eprev, hprev.im)});
                fact[(q * S + s) * 2] = cp;
                fact[(q * S + s) * 2 + 1] = gi;
                us[q * S + s] = h;
                eprev = ev[r];
                cprev = cp;
                hprev = h;
            }
        }
    }
    const int64_t last = first + len - 1;
    cx<float> un = us[last * S + s], wn = fact[(last * S + s) * 2 + 1];
    const cx<float> uL = un, wL = wn;
    ws[last * S + s] = wn;
    for (int i1 = len - 2; i1 >= 0; i1 -= MX_FCK) {
        cx<float> hv[MX_FCK], cv[MX_FCK];
#pragma unroll
        for (int r = 0; r < MX_FCK; ++r) {
            const int i = i1 - r;
            if (i >= 0) {
                hv[r] = us[(first + i) * S + s];
                cv[r] = fact[((first + i) * S + s) * 2];
            }
        }
#pragma unroll
        for (int r = 0; r < MX_FCK; ++r) {
            const int i = i1 - r;
            if (i >= 0) {
                un = cfms_rn(hv[r], cv[r], un);
                wn = -cmul_rn(cv[r], wn);
                us[(first + i) * S + s] = un;
                ws[(first + i) * S + s] = wn;
            }
        }
    }
    cx<float> *SP = spk + ((int64_t)s * g.P + b) * 4;
    SP[0] = un;  // u_b[first]
    SP[1] = uL;  // u_b[last]
    SP[2] = wn;  // w_b[first]
    SP[3] = wL;  // w_b[last]
}

// Pass 0 block end values y_b[first] = u_b^T v_b, y_b[last] = w_b^T v_b; one thread per
// (block, column, system) with the system lanes of a (block, column) adjacent.
template <int LG>
__global__ void __launch_bounds__(128) mx_dots(TriGeom g, const float *__restrict__ VPf,
                                               const cx<float> *__restrict__ us, const cx<float> *__restrict__ ws,
                                               cx<float> *__restrict__ yend) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = (int)(tid % LG);
    const int64_t bj = tid / LG;
    if (bj >= (int64_t)g.P * g.Rc || sl >= g.S) return;
    const int j = (int)(bj % g.Rc);
    const int b = (int)(bj / g.Rc);
    const int64_t S = g.S;
    const int64_t first = (int64_t)b * g.B;
    const int len = (b < g.P - 1) ? g.m : (int)(g.N - first);
    cx<float> yu = {0.f, 0.f}, yw = {0.f, 0.f};
    for (int i0 = 0; i0 < len; i0 += MX_FCK) {
        float vv[MX_FCK];
        cx<float> uv[MX_FCK], wv[MX_FCK];
#pragma unroll
        for (int r = 0; r < MX_FCK; ++r) {
            const int64_t q = first + i0 + r;
            const bool in = i0 + r < len;
            vv[r] = in ? VPf[q * g.Rc + j] : 0.f;
            uv[r] = in ? us[q * S + sl] : cx<float>{0.f, 0.f};
            wv[r] = in ? ws[q * S + sl] : cx<float>{0.f, 0.f};
        }
#pragma unroll
        for (int r = 0; r < MX_FCK; ++r) {
            yu = {__fmaf_rn(vv[r], uv[r].re, yu.re), __fmaf_rn(vv[r], uv[r].im, yu.im)};
            yw = {__fmaf_rn(vv[r], wv[r].re, yw.re), __fmaf_rn(vv[r], wv[r].im, yw.im)};
        }
    }
    cx<float> *YE = yend + (((int64_t)sl * g.P + b) * g.Rc + j) * 2;
    YE[0] = yu;
    YE[1] = yw;
}

// ------------------------------------------------------------------ solve pass
// One thread per (block, column, system); the LG system lanes of a (block, column) are
// adjacent, so per-row loads of the [row][system] factors and the [row][column][lane]
// right-hand sides and solutions are contiguous across a group.  The forward
// substitution runs once keeping a checkpoint every CK rows; the back substitution
// then walks the chunks from the last, recomputing each chunk's forward values into
// registers (binary32 arithmetic is cheap; the scratch traffic it replaces is not).
// Y += sum_s Re(W_s x_s) is summed over the system lanes by a reduce-scatter; pass 0
// (FIRST, x_0 the full solution) in float pairs, later passes (small corrections) in
// binary32 added to the pairs.  The solution is stored for the residual kernel when
// mode has MX_RESID.
template <int LG, int CK, bool FIRST>
__global__ void __launch_bounds__(MX_CTA, 4) mx_solve(TriGeom g, MxArgs a, TriPoles ps, int mode) {
    using WT = WeightT<FIRST>;
    using VT = typename WT::T;
    if (!FIRST && a.state->done) return;  // uniform over the launch
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = (int)(tid % LG);
    const int64_t bj = tid / LG;
    if (bj >= (int64_t)g.P * g.Rc) return;  // whole groups leave (LG divides the CTA)
    const unsigned lane = threadIdx.x & 31;
    const unsigned gmask = (LG == 32) ? 0xffffffffu : (((1u << LG) - 1u) << (lane & ~(unsigned)(LG - 1)));
    const int j = (int)(bj % g.Rc);
    const int b = (int)(bj / g.Rc);
    const bool active = sl < g.S;
    const int s = active ? sl : 0;  // idle lanes shadow system 0 (its data, its slots) with zero weight
    const int64_t first = (int64_t)b * g.B;
    const int len = (b < g.P - 1) ? g.m : (int)(g.N - first);
    const bool has_left = b > 0, has_right = b < g.P - 1;
    const bool keep_x = (mode & MX_RESID) != 0 && active;
    const f32x2 wr = active ? split_bits(ps.w_re[s]) : f32x2{0.f, 0.f};
    const f32x2 wi = active ? split_bits(ps.w_im[s]) : f32x2{0.f, 0.f};
    const cx<float> *SG = a.sig + (int64_t)s * g.P * g.Rc;
    const cx<float> zero = {0.f, 0.f};
    const cx<float> sl_v = has_left ? SG[(int64_t)(b - 1) * g.Rc + j] : zero;
    const cx<float> sr_v = has_right ? SG[(int64_t)b * g.Rc + j] : zero;
    const float eleft = has_left ? a.ePf[first - 1] : 0.f;
    const float eright = has_right ? a.ePf[first + len - 1] : 0.f;
    const int S2 = 2 * g.S, Rc = g.Rc, RL = g.Rc * LG;
    const cx<float> *F = a.fact + (first * g.S + s) * 2;   // (c', g) of row i at F[i*S2], F[i*S2+1]
    const float *vf = a.VPf + first * g.Rc + j;             // row i at [i * Rc]
    const cx<float> *Rr = a.R != nullptr ? a.R + (first * g.Rc + j) * LG + s : nullptr;  // row i at [i * RL]
    cx<float> *Xw = a.X + (first * g.Rc + j) * LG + s;
    const float *epf = a.ePf + first;
    cx<float> *ck = a.ckpt + bj * LG + sl;
    const int64_t ckstride = (int64_t)g.P * g.Rc * LG;

    struct FwdIn {
        cx<float> rhs[CK], gq[CK];
        float el[CK];
    };
    auto load_chunk = [&](int i0, FwdIn &in) {
#pragma unroll
        for (int r = 0; r < CK; ++r) {
            const int i = i0 + r;
            if (i < len) {
                in.rhs[r] = FIRST ? cx<float>{vf[i * Rc], 0.f} : Rr[i * RL];
                in.gq[r] = F[i * S2 + 1];
                in.el[r] = i > 0 ? epf[i - 1] : eleft;
            }
        }
    };
    auto fwd = [&](int i, cx<float> rhs, cx<float> gq, float el, cx<float> dprev) -> cx<float> {
        const cx<float> xb = i > 0 ? dprev : sl_v;  // el is 0 for the first row of block 0
        rhs.re = __fmaf_rn(-el, xb.re, rhs.re);
        rhs.im = __fmaf_rn(-el, xb.im, rhs.im);
        if (i == len - 1 && has_right) {
            rhs.re = __fmaf_rn(-eright, sr_v.re, rhs.re);
            rhs.im = __fmaf_rn(-eright, sr_v.im, rhs.im);
        }
        return cmul_rn(gq, rhs);
    };

    // forward run with checkpoints: slot c holds the forward value of row (c+1)*CK - 1
    const int nch = (len + CK - 1) / CK;
    cx<float> dp = zero;
    for (int c = 0; c < nch; ++c) {
        FwdIn in;
#pragma unroll
        for (int r = 0; r < CK; ++r) {  // rows MX_PD ahead into L2
            const int ip = c * CK + MX_PD + r;
            if (ip < len) {
                pf_l2(F + ip * S2);
                if (!FIRST) pf_l2(Rr + ip * RL);
            }
        }
        load_chunk(c * CK, in);
#pragma unroll
        for (int r = 0; r < CK; ++r)
            if (c * CK + r < len) dp = fwd(c * CK + r, in.rhs[r], in.gq[r], in.el[r], dp);
        if (c + 1 < nch) ck[(int64_t)c * ckstride] = dp;
    }
    // back substitution, chunk by chunk from the last
    cx<float> xn = zero;
    for (int c = nch - 1; c >= 0; --c) {
        const int i0 = c * CK;
        cx<float> buf[CK];
        cx<float> dcur = (c == 0) ? zero : ck[(int64_t)(c - 1) * ckstride];
        {
            FwdIn in;
#pragma unroll
            for (int r = 0; r < CK; ++r) {  // the chunk MX_PD rows earlier into L2
                const int ip = i0 - MX_PD + r;
                if (ip >= 0) {
                    pf_l2(F + ip * S2);
                    if (!FIRST) pf_l2(Rr + ip * RL);
                }
            }
            load_chunk(i0, in);
#pragma unroll
            for (int r = 0; r < CK; ++r) {
                if (i0 + r < len) {
                    dcur = fwd(i0 + r, in.rhs[r], in.gq[r], in.el[r], dcur);
                    buf[r] = dcur;
                }
            }
        }
        VT v[LG];
#pragma unroll
        for (int r = CK - 1; r >= 0; --r) {
            const int i = i0 + r;
            if ((r % LG) == LG - 1) {
#pragma unroll
                for (int k = 0; k < LG; ++k) v[k] = WT::zero();
            }
            if (i < len) {
                cx<float> x = buf[r];
                if (i < len - 1) x = cfms_rn(x, F[i * S2], xn);
                v[r % LG] = WT::re_wx(wr, wi, x);
                if (keep_x) Xw[i * RL] = x;
                xn = x;
            }
            if ((r % LG) == 0) {
                reduce_scatter<LG>(gmask, sl, v);
                const int row = i0 + r + sl;  // lane sl now holds row i0 + r + sl
                if (row < len) WT::update(a.Y, (first + row) * g.Rc + j, v[0]);
            }
        }
    }
    // the separator row after this block
    VT acc = WT::re_wx(wr, wi, sr_v);
#pragma unroll
    for (int off = LG / 2; off > 0; off >>= 1) acc = acc + shfl_xor(gmask, acc, off);
    if (sl == 0 && has_right) WT::update(a.Y, (first + len) * g.Rc + j, acc);
}

// ------------------------------------------------------------------ residual pass
// Same thread layout.  r = rhs - M x on the block's rows from the stored solution x of
// the pass (x_{-1} and x_len are the separator values), in one of three forms:
//   FIRST          rhs = V:   float-float (mx_resid_first)
//   CORR, comp     rhs = r_k given as (hi, lo): float-float (mx_resid_comp)
//   CORR, !comp    binary32 (mx_resid_corr) -- the final verification residual
// The stored residual overwrites r_k in place; the block end dots of the next pass and
// the per-CTA norms are formed on the way.
template <int LG, bool FIRST>
__global__ void __launch_bounds__(MX_CTA, 5) mx_resid(TriGeom g, MxArgs a, TriPoles ps, int mode) {
    if (!FIRST && a.state->done) return;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = (int)(tid % LG);
    const int64_t bj = tid / LG;
    float rn2 = 0.f, xn2 = 0.f;
    if (bj < (int64_t)g.P * g.Rc && sl < g.S) {
        const int j = (int)(bj % g.Rc);
        const int b = (int)(bj / g.Rc);
        const int s = sl;
        const int64_t first = (int64_t)b * g.B;
        const int len = (b < g.P - 1) ? g.m : (int)(g.N - first);
        const bool has_left = b > 0, has_right = b < g.P - 1;
        const bool store = (mode & MX_STORE) != 0, comp = (mode & MX_COMP) != 0;
        const bool lo_in = (mode & MX_LO_IN) != 0, lo_out = (mode & MX_LO_OUT) != 0;
        const f32x2 thr = split_bits(ps.th_re[s]), thi = split_bits(ps.th_im[s]);
        const cx<float> *SG = a.sig + (int64_t)s * g.P * g.Rc;
        const cx<float> zero = {0.f, 0.f};
        const int Rc = g.Rc, RL = g.Rc * LG, S = g.S;
        const cx<float> *Xr = a.X + (first * g.Rc + j) * LG + s;
        cx<float> *Rw = a.R != nullptr ? a.R + (first * g.Rc + j) * LG + s : nullptr;
        cx<float> *Rlw = a.Rlo != nullptr ? a.Rlo + (first * g.Rc + j) * LG + s : nullptr;
        const float *vf = a.VPf + first * g.Rc + j, *vl = a.VPl + first * g.Rc + j;
        const float *dpf = a.dPf + first, *dpl = a.dPl + first;
        const float *epf = a.ePf + first - 1, *epl = a.ePl + first - 1;  // e'_{first+i-1} at [i]
        const cx<float> *U = a.us + first * S + s, *Wsp = a.ws + first * S + s;
        cx<float> xl = has_left ? SG[(int64_t)(b - 1) * g.Rc + j] : zero;
        cx<float> xs = Xr[0];
        const cx<float> xend = has_right ? SG[(int64_t)b * g.Rc + j] : zero;
        float ecur = (first > 0) ? epf[0] : 0.f, ecur_l = (first > 0) ? epl[0] : 0.f;  // e'_{q-1}
        cx<float> yu = zero, yw = zero;
        // shared-memory ring: NST stages of RK rows; per row the next x, r_k and its low part
        constexpr int RK = 4, NST = 4;
        extern __shared__ cx<float> ring[];  // [NST][RK][3][MX_CTA]
        auto slot = [&](int st, int r, int arr) -> cx<float> * {
            return ring + ((st * RK + r) * 3 + arr) * MX_CTA + threadIdx.x;
        };
        const int nck = (len + RK - 1) / RK;
        auto issue = [&](int c) {
            if (c < nck) {
                const int st = c % NST;
#pragma unroll
                for (int r = 0; r < RK; ++r) {
                    const int i = c * RK + r;
                    if (i + 1 < len) cp_async8(slot(st, r, 0), Xr + (i + 1) * RL);
                    if (!FIRST && i < len) {
                        cp_async8(slot(st, r, 1), Rw + i * RL);
                        if (lo_in) cp_async8(slot(st, r, 2), Rlw + i * RL);
                    }
                }
            }
            cp_async_commit();  // possibly empty: keeps the group count uniform
        };
#pragma unroll
        for (int c = 0; c < NST; ++c) issue(c);
        for (int c = 0; c < nck; ++c) {
            cp_async_wait<NST - 1>();  // group c has landed
            const int st = c % NST, i0 = c * RK;
            if (store) {
#pragma unroll
                for (int r = 0; r < RK; ++r) {  // spikes of rows MX_PD ahead into L2
                    const int ip = i0 + MX_PD + r;
                    if (ip < len) {
                        pf_l2(U + ip * S);
                        pf_l2(Wsp + ip * S);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < RK; ++r) {
                const int i = i0 + r;
                if (i < len) {
                    const cx<float> xr = i + 1 < len ? *slot(st, r, 0) : xend;
                    const float dh = dpf[i], dl = dpl[i], eh = epf[i + 1], elo = epl[i + 1];
                    cx<float> hi, lo = zero;
                    if (FIRST) {
                        mx_resid_first(f32x2{vf[i * Rc], vl[i * Rc]}, f32x2{dh, dl}, f32x2{ecur, ecur_l},
                                       f32x2{eh, elo}, thr, thi, xl, xs, xr, hi, lo);
                        xn2 = __fmaf_rn(xs.re, xs.re, __fmaf_rn(xs.im, xs.im, xn2));
                    } else if (comp) {
                        mx_resid_comp(*slot(st, r, 1), lo_in ? *slot(st, r, 2) : zero, f32x2{dh, dl},
                                      f32x2{ecur, ecur_l}, f32x2{eh, elo}, thr, thi, xl, xs, xr, hi, lo);
                    } else {
                        hi = mx_resid_corr(*slot(st, r, 1), dh, ecur, eh, thr.hi, thi.hi, xl, xs, xr);
                    }
                    rn2 = __fmaf_rn(hi.re, hi.re, __fmaf_rn(hi.im, hi.im, rn2));
                    if (store) {
                        Rw[i * RL] = hi;
                        if (lo_out) Rlw[i * RL] = lo;
                        yu = cfma_rn(yu, U[i * S], hi);
                        yw = cfma_rn(yw, Wsp[i * S], hi);
                    }
                    xl = xs;
                    xs = xr;
                    ecur = eh;
                    ecur_l = elo;
                }
            }
            issue(c + NST);  // refill the stage just consumed (its values are all used above)
        }
        cp_async_wait<0>();
        if (store) {
            const int64_t e = ((int64_t)s * g.P + b) * g.Rc + j;
            a.yend[2 * e] = yu;
            a.yend[2 * e + 1] = yw;
        }
    }
    cta_norms<LG>(rn2, xn2, a.part3);
}

// ------------------------------------------------------------------ separator residuals
// grid (ceil((P-1) Rc / MX_CTA), S): one thread per (separator, column) of system blockIdx.y.
template <int LG, bool FIRST>
__global__ void __launch_bounds__(MX_CTA) mx_sep_resid(TriGeom g, MxArgs a, TriPoles ps, int mode) {
    if (!FIRST && a.state->done) return;
    const int s = blockIdx.y;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float rn2 = 0.f, xn2 = 0.f;
    if (t < (int64_t)(g.P - 1) * g.Rc) {
        const int j = (int)(t % g.Rc);
        const int b = (int)(t / g.Rc);
        const int64_t p = (int64_t)b * g.B + g.m;
        const int64_t e = ((int64_t)s * g.P + b) * g.Rc + j;
        const cx<float> xs = a.sig[e];
        const cx<float> xl = a.X[((p - 1) * g.Rc + j) * LG + s];
        const cx<float> xr = a.X[((p + 1) * g.Rc + j) * LG + s];
        const f32x2 thr = split_bits(ps.th_re[s]), thi = split_bits(ps.th_im[s]);
        const f32x2 dq = {a.dPf[p], a.dPl[p]}, el = {a.ePf[p - 1], a.ePl[p - 1]}, er = {a.ePf[p], a.ePl[p]};
        cx<float> hi, lo = {0.f, 0.f};
        if (FIRST) {
            mx_resid_first(f32x2{a.VPf[p * g.Rc + j], a.VPl[p * g.Rc + j]}, dq, el, er, thr, thi, xl, xs, xr, hi, lo);
            xn2 = __fmaf_rn(xs.re, xs.re, xs.im * xs.im);
        } else if (mode & MX_COMP) {
            const cx<float> rl = (mode & MX_LO_IN) ? a.sepLo[e] : cx<float>{0.f, 0.f};
            mx_resid_comp(a.sepR[e], rl, dq, el, er, thr, thi, xl, xs, xr, hi, lo);
        } else {
            hi = mx_resid_corr(a.sepR[e], dq.hi, el.hi, er.hi, thr.hi, thi.hi, xl, xs, xr);
        }
        rn2 = __fmaf_rn(hi.re, hi.re, hi.im * hi.im);
        if (mode & MX_STORE) {
            a.sepR[e] = hi;
            if (mode & MX_LO_OUT) a.sepLo[e] = lo;
        }
    }
    // CTA sum (all threads of the CTA belong to system s)
    __shared__ float red[MX_CTA / 32][2];
    for (int off = 16; off > 0; off >>= 1) {
        rn2 += __shfl_xor_sync(0xffffffffu, rn2, off);
        xn2 += __shfl_xor_sync(0xffffffffu, xn2, off);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = rn2;
        red[threadIdx.x >> 5][1] = xn2;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double acc = 0.0;
        for (int w = 0; w < MX_CTA / 32; ++w) acc += (double)red[w][threadIdx.x];
        a.partS[((int64_t)s * gridDim.x + blockIdx.x) * 2 + threadIdx.x] = acc;
    }
}

// ------------------------------------------------------------------ stopping test
// One warp per system.  After pass `pass`: iters = pass; with a residual, the relative
// residual max_s ||r_s|| / ((beta + |theta_s|) ||x_s||) and the stopping decision.
__global__ void mx_check(MxArgs a, TriPoles ps, int S, int LG, int n3, int nS, int pass, int has_resid, int first,
                         double tol) {
    __shared__ double rel[TRI_MAXSYS];
    MixState *st = a.state;
    if (st->done) return;
    const int s = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double r2 = 0.0, x2 = 0.0;
    if (has_resid) {
        for (int i = lane; i < n3; i += 32) {
            r2 += a.part3[((int64_t)i * LG + s) * 2];
            x2 += a.part3[((int64_t)i * LG + s) * 2 + 1];
        }
        for (int i = lane; i < nS; i += 32) {
            r2 += a.partS[((int64_t)s * nS + i) * 2];
            x2 += a.partS[((int64_t)s * nS + i) * 2 + 1];
        }
        for (int off = 16; off > 0; off >>= 1) {
            r2 += __shfl_xor_sync(0xffffffffu, r2, off);
            x2 += __shfl_xor_sync(0xffffffffu, x2, off);
        }
        if (lane == 0) {
            if (first) st->xnorm2[s] = x2;
            const double xn = sqrt(first ? x2 : st->xnorm2[s]);
            const double beta = (double)__uint_as_float(*a.beta_bits);
            const double den = (beta + hypot(ps.th_re[s], ps.th_im[s])) * xn;
            rel[s] = den > 0.0 ? sqrt(r2) / den : (r2 > 0.0 ? INFINITY : 0.0);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st->iters = pass;
        if (has_resid) {
            double m = 0.0;
            for (int k = 0; k < S; ++k) m = fmax(m, rel[k]);
            st->resid = m;
            if (m <= tol) st->done = 1;
        }
    }
}

struct MixLayout {
    size_t dPf, dPl, ePf, ePl, fact, us, ws, spk, beta, factor_total;
    size_t VPf, VPl, yend, sig, sepR, sepLo, R, Rlo, X, ckpt, part3, partS, state, solve_total;
    int CK, nchk, n3, nSx;
};

static inline size_t al(size_t x) { return (x + 255) & ~size_t(255); }

static MixLayout mx_layout(const TriGeom &g, int max_refine) {
    MixLayout L{};
    const size_t N = (size_t)g.N, S = (size_t)g.S, P = (size_t)g.P, Rc = (size_t)g.Rc, LG = (size_t)g.LG;
    size_t off = 0;
    L.dPf = off; off += al(N * 4);
    L.dPl = off; off += al(N * 4);
    L.ePf = off; off += al(N * 4);
    L.ePl = off; off += al(N * 4);
    L.fact = off; off += al(S * N * 2 * 8);
    L.us = off; off += al(S * N * 8);
    L.ws = off; off += al(S * N * 8);
    L.spk = off; off += al(S * P * 4 * 8);
    L.beta = off; off += 256;
    L.factor_total = off;
    L.CK = g.LG < 8 ? 8 : g.LG;
    L.nchk = (g.B + L.CK - 1) / L.CK;
    L.n3 = (int)((P * Rc * LG + MX_CTA - 1) / MX_CTA);
    L.nSx = g.P > 1 ? (int)(((P - 1) * Rc + MX_CTA - 1) / MX_CTA) : 0;
    off = 0;
    L.VPf = off; off += al(N * Rc * 4);
    L.VPl = off; off += al(N * Rc * 4);
    L.yend = off; off += al(S * P * Rc * 2 * 8);
    L.sig = off; off += al(S * P * Rc * 8);
    L.sepR = off; off += al(S * P * Rc * 8);
    L.sepLo = off; off += al(S * P * Rc * 8);
    L.R = off; off += max_refine >= 1 ? al(N * Rc * LG * 8) : 0;
    L.Rlo = off; off += max_refine >= 2 ? al(N * Rc * LG * 8) : 0;
    L.X = off; off += al(N * Rc * LG * 8);
    L.ckpt = off; off += al((size_t)L.nchk * P * Rc * LG * 8);
    L.part3 = off; off += al((size_t)L.n3 * LG * 2 * 8);
    L.partS = off; off += al((size_t)std::max(L.nSx, 1) * S * 2 * 8);
    L.state = off; off += al(sizeof(MixState));
    L.solve_total = off;
    return L;
}

template <int LG, int CK>
static cudaError_t launch_solve(bool first_pass, const TriGeom &g, const MxArgs &a, const TriPoles &ps, int mode,
                                unsigned grid, cudaStream_t st) {
    if (first_pass) mx_solve<LG, CK, true><<<grid, MX_CTA, 0, st>>>(g, a, ps, mode);
    else mx_solve<LG, CK, false><<<grid, MX_CTA, 0, st>>>(g, a, ps, mode);
    return cudaGetLastError();
}

template <int LG>
static cudaError_t launch_resid(bool first_pass, const TriGeom &g, const MxArgs &a, const TriPoles &ps, int mode,
                                unsigned grid, unsigned sgrid, cudaStream_t st) {
    // the ring plus the kernel's static shared memory exceeds the 48 KB default
    cudaError_t err = cudaFuncSetAttribute(mx_resid<LG, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           MX_RING_BYTES);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(mx_resid<LG, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MX_RING_BYTES);
    if (err != cudaSuccess) return err;
    if (first_pass) mx_resid<LG, true><<<grid, MX_CTA, MX_RING_BYTES, st>>>(g, a, ps, mode);
    else mx_resid<LG, false><<<grid, MX_CTA, MX_RING_BYTES, st>>>(g, a, ps, mode);
    if (g.P > 1) {
        const dim3 sg(sgrid, (unsigned)g.S);
        if (first_pass) mx_sep_resid<LG, true><<<sg, MX_CTA, 0, st>>>(g, a, ps, mode);
        else mx_sep_resid<LG, false><<<sg, MX_CTA, 0, st>>>(g, a, ps, mode);
    }
    return cudaGetLastError();
}

}  // namespace

TriGeom tri_mixed_geometry(int64_t N, int S, int Rc, int sm_count) { return tri_geometry(N, S, Rc, false, sm_count); }
size_t tri_mixed_factor_bytes(const TriGeom &g) { return mx_layout(g, 0).factor_total; }
size_t tri_mixed_solve_bytes(const TriGeom &g, int max_refine) { return mx_layout(g, max_refine).solve_total; }

cudaError_t tri_mixed_factor(const TriGeom &g, const double *d, const double *e, const TriPoles &ps, void *fwork,
                             cudaStream_t st, Profiler &prof) {
    const MixLayout L = mx_layout(g, 0);
    unsigned char *p = (unsigned char *)fwork;
    float *dPf = (float *)(p + L.dPf), *dPl = (float *)(p + L.dPl), *ePf = (float *)(p + L.ePf),
          *ePl = (float *)(p + L.ePl);
    unsigned *beta = (unsigned *)(p + L.beta);
    cudaError_t err = cudaMemsetAsync(beta, 0, sizeof(unsigned), st);
    if (err != cudaSuccess) return err;
    const unsigned pgrid = (unsigned)std::min<int64_t>((g.N + 255) / 256, 152 * 8);
    err = prof.timed("tri_prep<mixed>", st, [&] {
        mx_prep<<<pgrid, 256, 0, st>>>(g, d, e, dPf, dPl, ePf, ePl, beta);
        return cudaGetLastError();
    });
    if (err != cudaSuccess) return err;
    const int64_t n1 = (int64_t)g.S * g.P;
    return prof.timed("tri_mixed_factor", st, [&] {
        mx_factor<<<(unsigned)((n1 + 127) / 128), 128, 0, st>>>(g, dPf, ePf, ps, (cx<float> *)(p + L.fact),
                                                               (cx<float> *)(p + L.us), (cx<float> *)(p + L.ws),
                                                               (cx<float> *)(p + L.spk));
        return cudaGetLastError();
    });
}

cudaError_t tri_mixed_solve(const TriGeom &g, const double *V, double *Y, const TriPoles &ps, const void *fwork,
                            void *swork, const MixOpts &mo, cudaStream_t st, Profiler &prof) {
    const MixLayout L = mx_layout(g, mo.max_refine);
    const unsigned char *p = (const unsigned char *)fwork;
    unsigned char *q = (unsigned char *)swork;
    MxArgs a{};
    a.dPf = (const float *)(p + L.dPf);
    a.dPl = (const float *)(p + L.dPl);
    a.ePf = (const float *)(p + L.ePf);
    a.ePl = (const float *)(p + L.ePl);
    a.fact = (const cx<float> *)(p + L.fact);
    a.us = (const cx<float> *)(p + L.us);
    a.ws = (const cx<float> *)(p + L.ws);
    a.beta_bits = (const unsigned *)(p + L.beta);
    const cx<float> *spk = (const cx<float> *)(p + L.spk);
    float *VPf = (float *)(q + L.VPf), *VPl = (float *)(q + L.VPl);
    a.VPf = VPf;
    a.VPl = VPl;
    cx<float> *sig = (cx<float> *)(q + L.sig);
    a.sig = sig;
    a.yend = (cx<float> *)(q + L.yend);
    a.sepR = (cx<float> *)(q + L.sepR);
    a.sepLo = (cx<float> *)(q + L.sepLo);
    a.R = mo.max_refine >= 1 ? (cx<float> *)(q + L.R) : nullptr;
    a.Rlo = mo.max_refine >= 2 ? (cx<float> *)(q + L.Rlo) : nullptr;
    a.X = (cx<float> *)(q + L.X);
    a.ckpt = (cx<float> *)(q + L.ckpt);
    a.part3 = (double *)(q + L.part3);
    a.partS = (double *)(q + L.partS);
    a.state = (MixState *)(q + L.state);
    a.Y = Y;

    cudaError_t err = cudaMemsetAsync(a.state, 0, sizeof(MixState), st);
    if (err != cudaSuccess) return err;
    const int64_t nv = g.N * g.Rc;
    err = prof.timed("tri_prep_rhs<mixed>", st, [&] {
        mx_prep_v<<<(unsigned)std::min<int64_t>((nv + 255) / 256, 152 * 8), 256, 0, st>>>(nv, V, VPf, VPl);
        return cudaGetLastError();
    });
    if (err != cudaSuccess) return err;
    err = prof.timed("tri_mixed_dots", st, [&] {
        const unsigned grid = (unsigned)L.n3;
        switch (g.LG) {
            case 1: mx_dots<1><<<grid, MX_CTA, 0, st>>>(g, VPf, a.us, a.ws, a.yend); break;
            case 2: mx_dots<2><<<grid, MX_CTA, 0, st>>>(g, VPf, a.us, a.ws, a.yend); break;
            case 4: mx_dots<4><<<grid, MX_CTA, 0, st>>>(g, VPf, a.us, a.ws, a.yend); break;
            case 8: mx_dots<8><<<grid, MX_CTA, 0, st>>>(g, VPf, a.us, a.ws, a.yend); break;
            case 16: mx_dots<16><<<grid, MX_CTA, 0, st>>>(g, VPf, a.us, a.ws, a.yend); break;
            default: mx_dots<32><<<grid, MX_CTA, 0, st>>>(g, VPf, a.us, a.ws, a.yend); break;
        }
        return cudaGetLastError();
    });
    if (err != cudaSuccess) return err;
    const size_t smem = g.P > 1 ? (size_t)4 * (g.P - 1) * sizeof(cx<float>) : 0;
    if (g.P > 1) {
        // a ceiling for the largest reduced system, never lowered under a concurrent launch
        err = cudaFuncSetAttribute(tri_reduced_cr<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(4 * (size_t)(TRI_PMAX - 1) * sizeof(cx<float>)));
        if (err != cudaSuccess) return err;
    }
    const int npass = 1 + mo.max_refine;
    for (int k = 0; k < npass; ++k) {
        const bool last = k == npass - 1;
        const bool resid = !last || mo.verify;
        // stored residuals are float-float (pass 0 always; later passes from r_k's low
        // part when the pass before kept it); the final verification residual is binary32
        int mode = 0;
        if (resid) mode |= MX_RESID;
        if (!last) mode |= MX_STORE;
        if (k >= 1 && !last) mode |= MX_COMP | MX_LO_IN;
        if (!last && k + 1 < npass - 1) mode |= MX_LO_OUT;
        if (g.P > 1) {
            err = prof.timed("tri_reduced_cr<f32>", st, [&] {
                tri_reduced_cr<float><<<g.S * g.Rc, 512, smem, st>>>(g, a.dPf, a.ePf, VPf, k == 0 ? nullptr : a.sepR,
                                                                      ps, spk, a.yend, sig, k == 0 ? nullptr : &a.state->done);
                return cudaGetLastError();
            });
            if (err != cudaSuccess) return err;
        }
        err = prof.timed("tri_mixed_solve", st, [&] {
            const unsigned grid = (unsigned)L.n3;
            switch (g.LG) {
                case 1: return launch_solve<1, 8>(k == 0, g, a, ps, mode, grid, st);
                case 2: return launch_solve<2, 8>(k == 0, g, a, ps, mode, grid, st);
                case 4: return launch_solve<4, 8>(k == 0, g, a, ps, mode, grid, st);
                case 8: return launch_solve<8, 8>(k == 0, g, a, ps, mode, grid, st);
                case 16: return launch_solve<16, 16>(k == 0, g, a, ps, mode, grid, st);
                default: return launch_solve<32, 32>(k == 0, g, a, ps, mode, grid, st);
            }
        });
        if (err != cudaSuccess) return err;
        if (resid) {
            err = prof.timed("tri_mixed_resid", st, [&] {
                const unsigned grid = (unsigned)L.n3, sgrid = (unsigned)L.nSx;
                switch (g.LG) {
                    case 1: return launch_resid<1>(k == 0, g, a, ps, mode, grid, sgrid, st);
                    case 2: return launch_resid<2>(k == 0, g, a, ps, mode, grid, sgrid, st);
                    case 4: return launch_resid<4>(k == 0, g, a, ps, mode, grid, sgrid, st);
                    case 8: return launch_resid<8>(k == 0, g, a, ps, mode, grid, sgrid, st);
                    case 16: return launch_resid<16>(k == 0, g, a, ps, mode, grid, sgrid, st);
                    default: return launch_resid<32>(k == 0, g, a, ps, mode, grid, sgrid, st);
                }
            });
            if (err != cudaSuccess) return err;
        }
        err = prof.timed("tri_mixed_check", st, [&] {
            mx_check<<<1, 32 * g.S, 0, st>>>(a, ps, g.S, g.LG, L.n3, g.P > 1 ? L.nSx : 0, k, resid ? 1 : 0,
                                             k == 0 ? 1 : 0, mo.tol);
            return cudaGetLastError();
        });
        if (err != cudaSuccess) return err;
    }
    return prof.timed("tri_finish<mixed>", st, [&] {
        tri_finish<<<(unsigned)std::min<int64_t>((nv + 255) / 256, 152 * 8), 256, 0, st>>>(nv, Y);
        return cudaGetLastError();
    });
}

cudaError_t tri_mixed_read_state(const TriGeom &g, const void *swork, int max_refine, MixResult *out,
                                 cudaStream_t st) {
    const MixLayout L = mx_layout(g, max_refine);
    MixState h{};
    cudaError_t err = cudaMemcpyAsync(&h, (const unsigned char *)swork + L.state, sizeof(MixState),
                                      cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return err;
    out->converged = h.done != 0;
    out->iters = h.iters;
    out->resid = h.resid;
    return cudaSuccess;
}

}  // namespace expm
