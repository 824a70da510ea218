// tridiag_mixed.cu -- the tridiagonal path in binary32 with iterative refinement
// (EXPM_MIXED_FP32).
//
// Same problem as tridiag.cu: Y = sum_s Re(W_s X_s) with (t T - c I + theta_s I) X_s = V
// (eq. expAx, conjugate pairs folded by Remark 5.1).  Every solve with the shifted
// matrices M_s is binary32 arithmetic on the separator partition of tridiag.cu (block
// LUs, a reduced system for the separator rows); write M~^{-1} for that approximate
// inverse.  Accuracy is won back by refinement:
//     pass 0:   x_0 = M~^{-1} v,          r_1     = v   - M x_0
//     pass k:   d_k = M~^{-1} r_k,        r_{k+1} = r_k - M d_k
//     Y = sum_s Re(W_s x_0) + sum_k sum_s Re(W_s d_k).
// Each pass contracts the error by about kappa(M_s) u_32.  Only the first residual
// needs more than binary32: r_1 = v - M x_0 cancels down to ~u_32 |M| |x|, so it is
// formed from the binary64 entries of t T - c I split into float pairs (d' = dPf + dPl,
// e' = ePf + ePl), theta_s split the same way, error-free products (one FMA gives the
// rounding error of a binary32 product) and compensated sums (Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 2005): float-float accuracy on
// the FP32 pipe only.  Later residuals r_{k+1} = r_k - M d_k only cancel from |r_k|;
// they are float-float when another correction follows and binary32 for the final
// verification (an error of order u_32 |r_k|, enough for a norm).
//
// Nothing that grows with rows x systems x columns is stored except the residual
// itself.  The binary32 pivots (per row and system, shared by all columns) are computed
// once per factorization and read, like d', e' and V, from a tile of the CTA's rows in
// shared memory; each block solve keeps only a checkpoint of its forward recurrence every
// MX_CK rows and recomputes each chunk of forward values for the back substitution, and
// the residual, the Y update and the next pass's block end values are formed on the
// same walk (no solution vector goes through HBM).  The kernels:
//   mx_prep / mx_prep_v   split d', e' and V into float pairs; beta = max row sum
//   mx_pivots             per (block, system): the binary32 pivots of the block LU
//                         top-down and bottom-up, stored per (row, system), and the
//                         corner entries of M~_b^{-1} (factor part: T, t, c, poles only)
//   mx_ends               pass 0 end values of M~_b^{-1} v_b: a top-down sweep gives
//                         the last row, a bottom-up (UL) sweep the first
//   mx_cr_coef            the reduced separator system's coefficients (factor part)
//   mx_cr                 reduced separator system of a pass (cyclic reduction)
//   mx_main               pass 0, one thread per (block, column, system): the block
//                         solve for x_0, then, walking the rows bottom-up, the
//                         float-float residual r_1 (stored), Re(W x_0) summed over the
//                         system lanes into Y (float pairs), the end values of
//                         M~_b^{-1} r_1 for the next pass (a dot with the last-row
//                         spike and a bottom-up sweep) and the norms of the stopping test
//   mx_pass               pass k >= 1: the block solve for d_k from r_k, Y += Re(W d_k),
//                         and r_{k+1} (stored, with the next end values) or the final
//                         verification residual; the last pass writes binary64 Y
//   mx_sep_resid          residuals at the separator rows
//   mx_check              stopping test  ||r_s||_F <= tol (beta + |theta_s|) ||x_s||_F
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>

#include "arith.cuh"
#include "plan.cuh"
#include "tridiag.cuh"
#include "tridiag_kernels.cuh"

namespace expm {

namespace {

#ifndef EXPM_MX_WAVES
#define EXPM_MX_WAVES 4
#endif
constexpr int MX_CTA = 128;
constexpr int MX_CK = 8;            // rows per forward-recurrence checkpoint
constexpr int MX_PMAX = 6144;       // blocks: the binary32 reduced system (32 B per separator) in shared memory
#ifndef EXPM_MX_CTAS_SM
#define EXPM_MX_CTAS_SM 3
#endif
#ifndef EXPM_MX_SMEM_KB
#define EXPM_MX_SMEM_KB 72
#endif
constexpr int MX_THREADS_SM = 128 * EXPM_MX_CTAS_SM;  // resident (block, column, system) threads per SM
constexpr int MX_WAVES = EXPM_MX_WAVES;
constexpr int MX_SMEM_MAX = EXPM_MX_SMEM_KB * 1024;  // shared-memory tile per CTA of the solve kernels

enum : int { MX_STORE = 1, MX_LO_OUT = 2, MX_FINAL = 4, MX_COMP = 8, MX_LO_IN = 16, MX_RESID = 32 };

struct MixState {
    int done;   // stopping test passed: later passes return at once
    int iters;  // correction passes applied
    double resid;
    double xnorm2[TRI_MAXSYS];
};

struct MxArgs {
    const float *dPf, *dPl, *ePf, *ePl;  // t d - c and t e as float pairs
    const float *VPf, *VPl;              // V as float pairs
    const cx<float> *pg, *pu;            // pivots g (top-down) and g^ (bottom-up), [row][LG]
    const cx<float> *spk;                // corner entries of M~_b^{-1}, [system][block][4]
    const struct MxCrc *crc;             // reduced-system coefficients, [system][separator]
    cx<float> *yend;                     // block end values of the pass's right-hand side, [system][column][block][2]
    cx<float> *sig;                      // separator values of the pass, [system][block][column]
    cx<float> *xb;                       // first / last row of the pass's block solutions, [system][block][column][2]
    cx<float> *sepR, *sepLo;             // separator residuals, [system][block][column]
    cx<float> *R, *Rlo;                  // interior residuals, [row][column][lane]
    float2 *ckpt;                        // forward checkpoints z, [chunk][thread]
    double *Y;                           // float pairs during the passes, binary64 at the end
    float *part3;                        // per-CTA partial norms of mx_main / mx_pass
    double *partS;                       // per-CTA partial norms of mx_sep_resid
    MixState *state;
    const unsigned *beta_bits;
};

// ------------------------------------------------------------------ prep
__global__ void mx_prep(TriGeom g, const double *__restrict__ d, const double *__restrict__ e, float *dPf,
                        float *dPl, float *ePf, float *ePl, unsigned *beta_bits) {
    // d' = t d - c and e' = t e as float pairs, formed in float-float arithmetic from the
    // pairs of d, e, t and c (binary32 and integer operations only: this part's FP64 unit
    // would bind), and the row sums |d'| + |e'_i| + |e'_{i-1}| bounded in binary32 rounded
    // upwards
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const f32x2 t2 = split_bits(g.t), c2 = split_bits(g.cshift);
    const bool plain = g.t == 1.0 && g.cshift == 0.0;  // t T - c I = T: the splits as they are
    auto bound = [](f32x2 v) { return __fadd_ru(fabsf(v.hi), fabsf(v.lo)); };
    float bmax = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += stride) {
        f32x2 ds = split_bits(d[i]);
        f32x2 es = i + 1 < g.N ? split_bits(e[i]) : f32x2{0.f, 0.f};
        f32x2 esp = i > 0 ? split_bits(e[i - 1]) : f32x2{0.f, 0.f};
        if (!plain) {
            ds = dd_fma(t2, ds, -c2);
            es = t2 * es;
            esp = t2 * esp;
        }
        dPf[i] = ds.hi;
        dPl[i] = ds.lo;
        ePf[i] = es.hi;
        ePl[i] = es.lo;
        bmax = fmaxf(bmax, __fadd_ru(__fadd_ru(bound(ds), bound(es)), bound(esp)));
    }
    // one atomic per CTA (one per warp serialises thousands of them on one address)
    __shared__ float wmax[32];
    for (int off = 16; off > 0; off >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, off));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = bmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) bmax = fmaxf(bmax, wmax[w]);
        atomicMax(beta_bits, __float_as_uint(bmax));  // non-negative: bit order = value order
    }
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
// The residual of a row pairs its two components term by term, each term a real
// coefficient (a float pair) times a binary32 pair of x entries:
//   (a, a)(xs.re, xs.im), (-Im theta, Im theta)(xs.im, xs.re), (e_l, e_l)(xl.re, xl.im),
//   (e_r, e_r)(xr.re, xr.im),   a = d_q + Re theta,
// so both components run through one packed (two-lane) instruction stream.
// s + c  -=  (ah + al) x  on pairs: the binary32 product ah x split exactly by an FMA,
// the rounding error of the running sum s (TwoSum of s and -p) collected in c.
EXPM_D void pcsum_sub(uint64_t &s, uint64_t &c, uint64_t ah, uint64_t al, uint64_t x) {
    const uint64_t p = pmul2(ah, x);
    const uint64_t pe = ffma2(al, x, ffma2(ah, x, pneg2(p)));
    const uint64_t t = psub2(s, p);
    const uint64_t bb = psub2(t, s);
    const uint64_t err = psub2(psub2(s, psub2(t, bb)), padd2(p, bb));
    s = t;
    c = padd2(c, psub2(err, pe));
}
// the four terms of a row, then the pair (s, c) renormalised by TwoSum
EXPM_D void mx_resid_terms(uint64_t s, uint64_t c, f32x2 dq, f32x2 el, f32x2 er, f32x2 thr, f32x2 thi, cx<float> xl,
                           cx<float> xs, cx<float> xr, cx<float> &hi, cx<float> &lo) {
    const f32x2 t = two_sum(dq.hi, thr.hi);  // a = d_q + Re theta as an (unnormalised) pair
    const float alo = __fadd_rn(t.lo, __fadd_rn(dq.lo, thr.lo));
    pcsum_sub(s, c, pk2(t.hi, t.hi), pk2(alo, alo), pk2(xs.re, xs.im));
    pcsum_sub(s, c, pk2(-thi.hi, thi.hi), pk2(-thi.lo, thi.lo), pk2(xs.im, xs.re));
    pcsum_sub(s, c, pk2(el.hi, el.hi), pk2(el.lo, el.lo), pk2(xl.re, xl.im));
    pcsum_sub(s, c, pk2(er.hi, er.hi), pk2(er.lo, er.lo), pk2(xr.re, xr.im));
    const uint64_t h = padd2(s, c);
    const uint64_t bb = psub2(h, s);
    const uint64_t l = padd2(psub2(s, psub2(h, bb)), psub2(c, bb));
    upk2(h, hi.re, hi.im);
    upk2(l, lo.re, lo.im);
}

// Pass 0:  r = v - [ (d_q + theta) x_q + e_{q-1} x_{q-1} + e_q x_{q+1} ]  for one row, with
// x_0 in binary32, v, d', e', theta as float pairs; float-float accurate, returned as
// (hi, lo) per component.
EXPM_D void mx_resid_first(f32x2 v, f32x2 dq, f32x2 el, f32x2 er, f32x2 thr, f32x2 thi, cx<float> xl,
                           cx<float> xs, cx<float> xr, cx<float> &hi, cx<float> &lo) {
    mx_resid_terms(pk2(v.hi, 0.f), pk2(v.lo, 0.f), dq, el, er, thr, thi, xl, xs, xr, hi, lo);
}

// Later stored residuals:  r_{k+1} = r_k - M d_k  with r_k = rh + rl, float-float accurate.
EXPM_D void mx_resid_comp(cx<float> rh, cx<float> rl, f32x2 dq, f32x2 el, f32x2 er, f32x2 thr, f32x2 thi,
                          cx<float> xl, cx<float> xs, cx<float> xr, cx<float> &hi, cx<float> &lo) {
    mx_resid_terms(pk2(rh.re, rh.im), pk2(rl.re, rl.im), dq, el, er, thr, thi, xl, xs, xr, hi, lo);
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

EXPM_D cx<float> cmul_rn(cx<float> a, cx<float> b) {
    return {__fmaf_rn(a.re, b.re, -__fmul_rn(a.im, b.im)), __fmaf_rn(a.re, b.im, __fmul_rn(a.im, b.re))};
}
EXPM_D cx<float> cfms_rn(cx<float> s, cx<float> c, cx<float> x) {  // s - c x
    return {__fmaf_rn(c.im, x.im, __fmaf_rn(-c.re, x.re, s.re)), __fmaf_rn(-c.im, x.re, __fmaf_rn(-c.re, x.im, s.im))};
}
EXPM_D cx<float> cfma_rn(cx<float> s, cx<float> c, cx<float> x) {  // s + c x
    return {__fmaf_rn(-c.im, x.im, __fmaf_rn(c.re, x.re, s.re)), __fmaf_rn(c.im, x.re, __fmaf_rn(c.re, x.im, s.im))};
}
EXPM_D cx<float> cscale(float e, cx<float> a) { return {__fmul_rn(e, a.re), __fmul_rn(e, a.im)}; }
EXPM_D cx<float> cinv_fast(cx<float> w) {  // 1/w = conj(w)/|w|^2 (binary32, ~2 ulp)
    const float n2 = __fmaf_rn(w.re, w.re, __fmul_rn(w.im, w.im));
    const float r = __fdividef(1.0f, n2);
    return {__fmul_rn(w.re, r), -__fmul_rn(w.im, r)};
}
EXPM_D float cnorm2(cx<float> a) { return __fmaf_rn(a.re, a.re, __fmul_rn(a.im, a.im)); }

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
EXPM_D f32x2s re_wx_pair(f32x2 wr, f32x2 wi, cx<float> x) {
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
EXPM_D float re_wx_f32(float wr, float wi, cx<float> x) { return __fmaf_rn(wr, x.re, -__fmul_rn(wi, x.im)); }
EXPM_D void y_store_pair(double *Y, int64_t idx, f32x2s v, bool final_) {  // Y[idx]
    if (final_) Y[idx] = widen_bits(v.hi) + widen_bits(v.lo);
    else reinterpret_cast<f32x2 *>(Y)[idx] = f32x2{v.hi, v.lo};
}
// Y (float pair) += v; the last pass writes the binary64 sum
EXPM_D void y_add(double *Y, int64_t idx, float v, bool final_) {
    f32x2 *p = reinterpret_cast<f32x2 *>(Y) + idx;
    const f32x2 y = *p;
    if (final_) {  // the three terms added in float-float, one binary64 addition for the pair
        const f32x2 s = two_sum(y.hi, v);
        const f32x2 r = fast_two_sum(s.hi, __fadd_rn(s.lo, y.lo));
        Y[idx] = widen_bits(r.hi) + widen_bits(r.lo);
    } else {
        const f32x2 s = two_sum(y.hi, v);
        *p = fast_two_sum(s.hi, __fadd_rn(s.lo, y.lo));
    }
}

// Sum per system lane over the CTA into part[blockIdx][lane][2] (binary32, fixed order:
// these feed only the stopping test's norms).
template <int LG>
EXPM_D void cta_norms(float rn2, float xn2, float *part) {
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
        float acc = 0.f;
        for (int w = 0; w < MX_CTA / 32; ++w) acc += red[w][l][c];
        part[((int64_t)blockIdx.x * LG + l) * 2 + c] = acc;
    }
}

// ------------------------------------------------------------------ thread layout
// One thread per (block b, column j, system lane sl); the LG lanes of a (block, column)
// are adjacent and consecutive groups are consecutive columns of one block, so a
// warp's per-row loads of V and stores of Y and R touch contiguous bytes, and the
// block's rows of d' and e' are read by the whole group at once.
struct MxLane {
    int64_t bj, first;
    int sl, s, j, b, len;
    bool active, has_left, has_right;
    unsigned gmask;
};
template <int LG> EXPM_D bool mx_lane(const TriGeom &g, MxLane &t) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    t.sl = (int)(tid % LG);
    t.bj = tid / LG;
    if (t.bj >= (int64_t)g.P * g.Rc) return false;  // whole groups (LG divides the CTA)
    const unsigned lane = threadIdx.x & 31;
    t.gmask = (LG == 32) ? 0xffffffffu : (((1u << LG) - 1u) << (lane & ~(unsigned)(LG - 1)));
    t.j = (int)(t.bj % g.Rc);
    t.b = (int)(t.bj / g.Rc);
    t.active = t.sl < g.S;
    t.s = t.active ? t.sl : 0;  // idle lanes shadow system 0 with zero weight
    t.first = (int64_t)t.b * g.B;
    t.len = (t.b < g.P - 1) ? g.m : (int)(g.N - t.first);
    t.has_left = t.b > 0;
    t.has_right = t.b < g.P - 1;
    return true;
}

// ------------------------------------------------------------------ shared-memory tile
// The rows of the blocks a CTA's threads walk are copied once into shared memory with
// asynchronous copies (no registers held for loads in flight): d' and e' as float
// pairs and, for the kernels that read V, the CTA's columns of V's float pairs, stored
// column by column (a thread's column is then contiguous, and the odd column stride
// keeps the four columns of a warp in different banks).  The row walks then read
// shared memory only; every block is walked several times (two sweeps, or a sweep and
// a recompute), so each byte comes from HBM once.
EXPM_D void cp_async4(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
EXPM_D void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
EXPM_D void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
EXPM_D void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
EXPM_D void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> EXPM_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// n floats from g to s by the whole CTA; s and g must be congruent modulo 16 bytes
EXPM_D void cta_copy(float *s, const float *g, int64_t n) {
    const int nt = blockDim.x;
    int64_t head = (int64_t)(((16u - ((unsigned)(uintptr_t)g & 15u)) & 15u) >> 2);
    head = head < n ? head : n;
    for (int64_t i = threadIdx.x; i < head; i += nt) cp_async4(s + i, g + i);
    const int64_t body = (n - head) >> 2;
    for (int64_t i = threadIdx.x; i < body; i += nt) cp_async16(s + head + 4 * i, g + head + 4 * i);
    for (int64_t i = head + 4 * body + threadIdx.x; i < n; i += nt) cp_async4(s + i, g + i);
}
// A region of shared memory for n floats copied from g: regions start on 16-byte
// boundaries (region_floats(n) floats each, a multiple of 4) and the copy is shifted
// inside its region so that it is congruent with g modulo 16 bytes.
EXPM_HD int64_t region_floats(int64_t n) { return ((n + 3) & ~(int64_t)3) + 4; }
EXPM_D float *congruent(float *region, const float *g) {
    return region + (((unsigned)(uintptr_t)g & 15u) >> 2);
}
// odd column stride of the column-major V tile
EXPM_HD int64_t col_stride(int64_t rows) { return rows | 1; }

// The rows and columns one CTA covers: its (block, column) groups run from bj_lo to
// bj_hi - 1, i.e. blocks b_lo .. b_hi; all columns when it spans several blocks, else
// the columns c0 .. c0 + nc - 1 of its one block.
struct MxTile {
    int64_t row0;
    int nrows, c0, nc;
};
EXPM_D MxTile mx_tile(const TriGeom &g, int LG) {
    MxTile T;
    const int64_t groups = MX_CTA / LG;
    const int64_t bj_lo = (int64_t)blockIdx.x * groups;
    int64_t bj_hi = bj_lo + groups;
    if (bj_hi > (int64_t)g.P * g.Rc) bj_hi = (int64_t)g.P * g.Rc;
    const int64_t b_lo = bj_lo / g.Rc, b_hi = (bj_hi - 1) / g.Rc;
    T.row0 = b_lo * g.B;
    const int64_t row1 = (b_hi + 1) * g.B < g.N ? (b_hi + 1) * g.B : g.N;
    T.nrows = (int)(row1 - T.row0);
    if (b_lo == b_hi) {
        T.c0 = (int)(bj_lo % g.Rc);
        T.nc = (int)((bj_hi - 1) % g.Rc) - T.c0 + 1;
    } else {
        T.c0 = 0;
        T.nc = g.Rc;
    }
    return T;
}
// Floats of shared memory a tile needs (host and device agree on this bound): 4 arrays
// of rows for d', e'; 2 column-major arrays of rows x columns for V (`with_v`); the
// pivot tables g (`npiv` >= 1) and g^ (`npiv` == 2), rows x LG complex each.
EXPM_HD int64_t mx_tile_floats(int64_t rows, int64_t cols, int LG, bool with_v, int npiv) {
    return 4 * region_floats(rows) + (with_v ? 2 * region_floats(col_stride(rows) * cols) : 0) +
           npiv * region_floats(2 * rows * LG);
}
// Largest tile over the CTAs of a launch.  A CTA's groups start at a multiple of
// `groups`: with Rc a multiple of `groups` they stay inside one block (`groups`
// columns); with `groups` a multiple of Rc they cover whole blocks; otherwise they
// span at most (groups - 1) / Rc + 2 blocks, all columns.
static inline void mx_tile_bound(const TriGeom &g, int64_t &rows, int64_t &cols) {
    const int64_t groups = MX_CTA / g.LG;
    int64_t nb;
    if (g.Rc % groups == 0) {
        nb = 1;
        cols = groups;
    } else if (groups % g.Rc == 0) {
        nb = groups / g.Rc;
        cols = g.Rc;
    } else {
        nb = (groups - 1) / g.Rc + 2;
        cols = g.Rc;
    }
    if (nb > g.P) nb = g.P;
    rows = nb * g.B;
    if (rows > g.N) rows = g.N;
}

// Where a thread reads its block's rows: the tile in shared memory (ST, V's column
// contiguous) or global memory (V's rows Rc apart).  Pivots of the thread's system:
// row i at [i * LG].
template <bool ST> struct MxRows {
    const float *dh, *dl, *eh, *el;  // row i of the block at [i]
    const float *vh, *vl;            // row i, this thread's column
    const cx<float> *g, *u;          // pivots g_i and g^_i
    int vs;                          // V's row stride (global memory only)
    EXPM_D float v_hi(int i) const { return ST ? vh[i] : vh[(int64_t)i * vs]; }
    EXPM_D float v_lo(int i) const { return ST ? vl[i] : vl[(int64_t)i * vs]; }
};
// Copies the tile (all threads of the CTA take part, before any of them returns) and
// points `R` at the rows of block `b`, column `j`, system lane `s`.
template <int LG, bool ST>
EXPM_D void mx_stage(const TriGeom &g, const MxArgs &a, bool with_v, int npiv, float *smem, int64_t first, int j,
                     int s, MxRows<ST> &R) {
    if (!ST) {
        R.dh = a.dPf + first;
        R.dl = a.dPl + first;
        R.eh = a.ePf + first;
        R.el = a.ePl + first;
        R.vh = with_v ? a.VPf + first * g.Rc + j : nullptr;
        R.vl = with_v ? a.VPl + first * g.Rc + j : nullptr;
        R.g = a.pg + first * LG + s;
        R.u = a.pu + first * LG + s;
        R.vs = g.Rc;
        return;
    }
    const MxTile T = mx_tile(g, LG);
    const int64_t nr = T.nrows, cs = col_stride(nr), nv = nr * T.nc;
    float *base[4];
    float *p = smem;
    const float *src[4] = {a.dPf + T.row0, a.dPl + T.row0, a.ePf + T.row0, a.ePl + T.row0};
    for (int k = 0; k < 4; ++k) {
        base[k] = congruent(p, src[k]);
        cta_copy(base[k], src[k], nr);
        p += region_floats(nr);
    }
    float *vh = p, *vl = p + region_floats(cs * T.nc);
    if (with_v) {
        for (int64_t i = threadIdx.x; i < nv; i += blockDim.x) {  // row-major in global, column-major here
            const int64_t r = i / T.nc, c = i - r * T.nc;
            const int64_t gi = (T.row0 + r) * g.Rc + T.c0 + c;
            cp_async4(vh + c * cs + r, a.VPf + gi);
            cp_async4(vl + c * cs + r, a.VPl + gi);
        }
        p += 2 * region_floats(cs * T.nc);
    }
    const float *pgs = nullptr, *pus = nullptr;
    if (npiv >= 1) {
        const float *src_g = reinterpret_cast<const float *>(a.pg + T.row0 * LG);
        float *dg = congruent(p, src_g);
        cta_copy(dg, src_g, 2 * nr * LG);
        pgs = dg;
        p += region_floats(2 * nr * LG);
    }
    if (npiv >= 2) {
        const float *src_u = reinterpret_cast<const float *>(a.pu + T.row0 * LG);
        float *du = congruent(p, src_u);
        cta_copy(du, src_u, 2 * nr * LG);
        pus = du;
    }
    cp_async_wait_all();
    __syncthreads();
    const int64_t off = first - T.row0;
    R.dh = base[0] + off;
    R.dl = base[1] + off;
    R.eh = base[2] + off;
    R.el = base[3] + off;
    R.vh = with_v ? vh + (j - T.c0) * cs + off : nullptr;
    R.vl = with_v ? vl + (j - T.c0) * cs + off : nullptr;
    R.g = pgs ? reinterpret_cast<const cx<float> *>(pgs) + off * LG + s : nullptr;
    R.u = pus ? reinterpret_cast<const cx<float> *>(pus) + off * LG + s : nullptr;
    R.vs = 1;
}

// ------------------------------------------------------------------ pivots (factor part)
// One thread per (block, system): the binary32 block LU of M_b = (t T - c I + theta I)_b
// top-down, w_i = d'_i + theta - e'_{i-1} c'_{i-1}, g_i = 1/w_i, c'_i = e'_i g_i (0 on the
// block's last row), and bottom-up (UL), w^_i = d'_i + theta - e'_i^2 g^_{i+1}, g^_i = 1/w^_i.
// g and g^ are stored per (row, system lane), [row][LG], for every later kernel (which
// derive c' = e' g): a pivot costs a complex reciprocal on a dependent chain, and each is
// shared by all columns.  Also the
// corner entries of M~_b^{-1} that the reduced system needs, u_b = M~_b^{-1} eps_first and
// w_b = M~_b^{-1} eps_last at the first and last rows: u_b[last] is the last forward
// value of eps_first (zeta), w_b[last] = g_last, u_b[first] = g^_0, and w_b[first] =
// u_b[last] since M_b is complex symmetric.
EXPM_D cx<float> cinv_fast(cx<float> w);
EXPM_D cx<float> cmul_rn(cx<float> a, cx<float> b);
EXPM_D cx<float> cscale(float e, cx<float> a);
template <int LG>
__global__ void __launch_bounds__(128) mx_pivots(TriGeom g, const float *__restrict__ dPf,
                                                 const float *__restrict__ ePf, TriPoles ps, cx<float> *pg,
                                                 cx<float> *pu, cx<float> *spk) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = (int)(tid % LG);
    const int b = (int)(tid / LG);
    if (b >= g.P || sl >= g.S) return;
    const int64_t first = (int64_t)b * g.B;
    const int len = (b < g.P - 1) ? g.m : (int)(g.N - first);
    const float *dp = dPf + first, *ep = ePf + first;
    const cx<float> th = {__double2float_rn(ps.th_re[sl]), __double2float_rn(ps.th_im[sl])};
    cx<float> *G = pg + first * LG + sl, *U = pu + first * LG + sl;
    cx<float> cp = {0.f, 0.f}, zeta = {0.f, 0.f}, gi = {0.f, 0.f};
    float el = 0.f;
    for (int i0 = 0; i0 < len; i0 += MX_CK) {
        float dv[MX_CK], ev[MX_CK];
#pragma unroll
        for (int r = 0; r < MX_CK; ++r) {
            dv[r] = i0 + r < len ? dp[i0 + r] : 0.f;
            ev[r] = i0 + r < len - 1 ? ep[i0 + r] : 0.f;  // 0 on the block's last row
        }
#pragma unroll
        for (int r = 0; r < MX_CK; ++r) {
            const int i = i0 + r;
            if (i < len) {
                const cx<float> w = {__fmaf_rn(-el, cp.re, __fadd_rn(dv[r], th.re)), __fmaf_rn(-el, cp.im, th.im)};
                const cx<float> zp = zeta;
                gi = cinv_fast(w);
                cp = cscale(ev[r], gi);
                zeta = (i == 0) ? gi : cmul_rn(gi, cscale(-el, zp));
                G[(int64_t)i * LG] = gi;
                el = ev[r];
            }
        }
    }
    const cx<float> uL = zeta, wL = gi;
    cx<float> k = {0.f, 0.f};
    for (int i0 = len - 1; i0 >= 0; i0 -= MX_CK) {
        float dv[MX_CK], ev[MX_CK], em[MX_CK];
#pragma unroll
        for (int r = 0; r < MX_CK; ++r) {
            const int i = i0 - r;
            dv[r] = i >= 0 ? dp[i] : 0.f;
            ev[r] = (i >= 0 && i < len - 1) ? ep[i] : 0.f;
            em[r] = i > 0 ? ep[i - 1] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < MX_CK; ++r) {
            const int i = i0 - r;
            if (i >= 0) {
                const cx<float> w = {__fmaf_rn(-ev[r], k.re, __fadd_rn(dv[r], th.re)), __fmaf_rn(-ev[r], k.im, th.im)};
                gi = cinv_fast(w);
                U[(int64_t)i * LG] = gi;
                k = cscale(em[r], gi);
            }
        }
    }
    cx<float> *SP = spk + ((int64_t)sl * g.P + b) * 4;
    SP[0] = gi;  // u_b[first]
    SP[1] = uL;  // u_b[last]
    SP[2] = uL;  // w_b[first]
    SP[3] = wL;  // w_b[last]
}

// c'_i = e'_i g_i inside the block (0 on its last row, whose e' couples to the separator)
EXPM_D cx<float> cprime(cx<float> gi, float ei) { return cscale(ei, gi); }

// z_i = g_i (f - e'_{i-1} z_{i-1}) for a complex right-hand side f (two FMAs, a complex product)
EXPM_D cx<float> zstep(cx<float> gi, float el, cx<float> f, cx<float> zp) {
    f.re = __fmaf_rn(-el, zp.re, f.re);
    f.im = __fmaf_rn(-el, zp.im, f.im);
    return cmul_rn(gi, f);
}

// ------------------------------------------------------------------ pass 0 end values
// y_b = M~_b^{-1} v_b: the top-down sweep ends at y_b[last], the bottom-up (UL) sweep,
// h_i = g^_i (v_i - e'_i h_{i+1}), at y_b[first]; nothing is stored per row.  One thread
// per (block, system, group of MX_EC columns): a row's pivot and e' serve all the
// group's columns, whose entries of V are contiguous, and the columns' recurrences are
// independent chains.  Rows are read straight from global memory MX_CK at a time, all
// loads of a chunk issued before its first use.
constexpr int MX_EC = 2;
template <int LG, bool V4>
__global__ void __launch_bounds__(128) mx_ends(TriGeom g, MxArgs a) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int Rc = g.Rc, nq = (Rc + MX_EC - 1) / MX_EC;
    const int q = (int)(tid % nq);
    const int sl = (int)((tid / nq) % LG);
    const int b = (int)(tid / ((int64_t)nq * LG));
    if (b >= g.P || sl >= g.S) return;
    const int64_t first = (int64_t)b * g.B;
    const int len = (b < g.P - 1) ? g.m : (int)(g.N - first);
    const int j0 = q * MX_EC, nc = Rc - j0 < MX_EC ? Rc - j0 : MX_EC;
    const cx<float> *G = a.pg + first * LG + sl, *U = a.pu + first * LG + sl;
    const float *ep = a.ePf + first;
    const float *vp = a.VPf + first * Rc + j0;
    auto load_v = [&](int i, float (&v)[MX_EC]) {
        if (V4) {
            const float2 w = *reinterpret_cast<const float2 *>(vp + (int64_t)i * Rc);
            v[0] = w.x;
            v[1] = w.y;
        } else {
#pragma unroll
            for (int c = 0; c < MX_EC; ++c) v[c] = c < nc ? vp[(int64_t)i * Rc + c] : 0.f;
        }
    };
    cx<float> z[MX_EC];
#pragma unroll
    for (int c = 0; c < MX_EC; ++c) z[c] = {0.f, 0.f};
    for (int i0 = 0; i0 < len; i0 += MX_CK) {
        cx<float> p[MX_CK];
        float el[MX_CK], v[MX_CK][MX_EC];
#pragma unroll
        for (int r = 0; r < MX_CK; ++r) {
            const int i = i0 + r;
            if (i < len) {
                p[r] = G[(int64_t)i * LG];
                el[r] = i > 0 ? ep[i - 1] : 0.f;
                load_v(i, v[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < MX_CK; ++r) {
            if (i0 + r < len) {
#pragma unroll
                for (int c = 0; c < MX_EC; ++c) z[c] = zstep(p[r], el[r], cx<float>{v[r][c], 0.f}, z[c]);
            }
        }
    }
    cx<float> h[MX_EC];
#pragma unroll
    for (int c = 0; c < MX_EC; ++c) h[c] = {0.f, 0.f};
    for (int i0 = len - 1; i0 >= 0; i0 -= MX_CK) {
        cx<float> p[MX_CK];
        float er[MX_CK], v[MX_CK][MX_EC];
#pragma unroll
        for (int r = 0; r < MX_CK; ++r) {
            const int i = i0 - r;
            if (i >= 0) {
                p[r] = U[(int64_t)i * LG];
                er[r] = i < len - 1 ? ep[i] : 0.f;  // the last row has no coupling inside the block
                load_v(i, v[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < MX_CK; ++r) {
            if (i0 - r >= 0) {
#pragma unroll
                for (int c = 0; c < MX_EC; ++c) h[c] = zstep(p[r], er[r], cx<float>{v[r][c], 0.f}, h[c]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < MX_EC; ++c) {
        if (c < nc) {
            cx<float> *YE = a.yend + (((int64_t)sl * Rc + j0 + c) * g.P + b) * 2;
            YE[0] = h[c];
            YE[1] = z[c];
        }
    }
}

// ------------------------------------------------------------------ block solves
// The two solve kernels share this walk over one block: a top-down pass,
//     z_i = g_i (f_i - e'_{i-1} z_{i-1}),
// keeping a checkpoint of z every MX_CK rows, then chunk by chunk from the last, the
// chunk's z recomputed into registers and back-substituted, x_i = z_i - c'_i x_{i+1},
// with per_row(i, r, x_i, f_i) called for every row i = nch*MX_CK-1 .. 0 of the
// chunks in that order (rows past the block's end included, with i >= len, so that
// every lane of a group takes part in the group's shuffles), r = i mod MX_CK and f_i
// the row's right-hand side.  fetch(step, f) supplies the right-hand sides of the
// walk's step-th chunk (steps 0 .. nch-1 are chunks 0 .. nch-1, steps nch .. 2 nch-1
// chunks nch-1 .. 0; rows past the end read as zero).  Checkpoints are read one chunk
// ahead of their use; the separators' boundary terms enter rows 0 and len-1.  The
// x_{i+1} of the block's last row is the right separator value: c'_{len-1} is 0.
template <bool B> using Bool = std::integral_constant<bool, B>;

template <int LG, bool ST, class FetchF, class RowF>
EXPM_D void mx_block_walk(const MxLane &t, const MxRows<ST> &rw, cx<float> sl_v, cx<float> sr_v, float eleft,
                          float eright, float2 *ck, int64_t ckstride, FetchF fetch, RowF per_row) {
    const int len = t.len;
    const int nch = (len + MX_CK - 1) / MX_CK;
    const cx<float> zero = {0.f, 0.f};
    const cx<float> bl = {-eleft * sl_v.re, -eleft * sl_v.im}, br = {-eright * sr_v.re, -eright * sr_v.im};
    // Interior chunks hold neither row 0 nor the block's last two rows nor rows past
    // its end: their rows (and the rows after them, which per_row's residual reaches)
    // need no test at all.  Only LG <= MX_CK keeps the reduce-scatter groups inside a
    // chunk, which the interior path relies on.
    auto interior = [&](int c) { return LG <= MX_CK && c > 0 && c * MX_CK + MX_CK + 2 <= len; };
    auto fwd_chunk = [&](auto fast, int c, const cx<float>(&f)[MX_CK], cx<float> &z, cx<float> *zb) {
        const int i0 = c * MX_CK;
#pragma unroll
        for (int r = 0; r < MX_CK; ++r) {
            const int i = i0 + r;
            if (decltype(fast)::value) {
                z = zstep(rw.g[i * LG], rw.eh[i - 1], f[r], z);
                if (zb) zb[r] = z;
            } else {
                if (i < len) {
                    cx<float> fi = f[r];
                    if (i == 0) fi = fi + bl;
                    if (i == len - 1) fi = fi + br;
                    z = zstep(rw.g[i * LG], i > 0 ? rw.eh[i - 1] : 0.f, fi, z);
                }
                if (zb) zb[r] = (i < len) ? z : zero;
            }
        }
    };
    {
        cx<float> z = zero, fc[MX_CK];
        for (int c = 0; c < nch; ++c) {
            fetch(c, fc);
            if (interior(c)) fwd_chunk(Bool<true>(), c, fc, z, nullptr);
            else fwd_chunk(Bool<false>(), c, fc, z, nullptr);
            if (c + 1 < nch) ck[(int64_t)c * ckstride] = make_float2(z.re, z.im);
        }
    }
    cx<float> fc[MX_CK], x1 = sr_v;
    float2 qc = nch > 1 ? ck[(int64_t)(nch - 2) * ckstride] : make_float2(0.f, 0.f), qn = qc;
    for (int c = nch - 1; c >= 0; --c) {
        const int i0 = c * MX_CK;
        fetch(2 * nch - 1 - c, fc);
        if (c > 1) qn = ck[(int64_t)(c - 2) * ckstride];
        cx<float> z = c > 0 ? cx<float>{qc.x, qc.y} : zero, zb[MX_CK];
        if (interior(c)) {
            fwd_chunk(Bool<true>(), c, fc, z, zb);
#pragma unroll
            for (int r = MX_CK - 1; r >= 0; --r) {
                const int i = i0 + r;
                const cx<float> x = cfms_rn(zb[r], cprime(rw.g[i * LG], rw.eh[i]), x1);
                x1 = x;
                per_row(Bool<true>(), i, r, x, fc[r]);
            }
        } else {
            fwd_chunk(Bool<false>(), c, fc, z, zb);
#pragma unroll
            for (int r = MX_CK - 1; r >= 0; --r) {
                const int i = i0 + r;
                cx<float> x = zero;
                if (i < len) {
                    x = cfms_rn(zb[r], cprime(rw.g[i * LG], i < len - 1 ? rw.eh[i] : 0.f), x1);
                    x1 = x;
                }
                per_row(Bool<false>(), i, r, x, fc[r]);
            }
        }
        qc = qn;
    }
}

// Right-hand sides of mx_pass's walk streamed from global memory into a per-thread
// ring of MX_NST chunk slots in shared memory by asynchronous copies, MX_NST - 1 steps
// ahead of their use (a thread's own slots only: no barrier needed).
constexpr int MX_NST = 4;
struct MxRing {
    cx<float> *ring;        // this thread's slot of row r, stage k at ring[(k * MX_CK + r) * MX_CTA]
    const cx<float> *src;   // row i at src[i * rs]
    int rs, len, nch;
    EXPM_D int chunk_of(int step) const { return step < nch ? step : 2 * nch - 1 - step; }
    EXPM_D void issue(int step) const {
        if (step < 2 * nch) {
            const int c = chunk_of(step), k = step % MX_NST;
#pragma unroll
            for (int r = 0; r < MX_CK; ++r) {
                const int i = c * MX_CK + r;
                if (i < len) cp_async8(ring + (k * MX_CK + r) * MX_CTA, src + (int64_t)i * rs);
            }
        }
        cp_async_commit();  // possibly empty: keeps the group count uniform
    }
    EXPM_D void prime() const {
#pragma unroll
        for (int k = 0; k < MX_NST - 1; ++k) issue(k);
    }
    EXPM_D void fetch(int step, cx<float> (&f)[MX_CK]) const {
        issue(step + MX_NST - 1);  // refills the stage read at step - 1
        cp_async_wait<MX_NST - 1>();
        const int c = chunk_of(step), k = step % MX_NST;
#pragma unroll
        for (int r = 0; r < MX_CK; ++r)
            f[r] = (c * MX_CK + r < len) ? ring[(k * MX_CK + r) * MX_CTA] : cx<float>{0.f, 0.f};
    }
};
// bytes of the ring per CTA
constexpr size_t MX_RING_BYTES = (size_t)MX_NST * MX_CK * MX_CTA * sizeof(cx<float>);

// Slot of row i in the reduce-scatter buffer of LG rows (compile-time for LG <= MX_CK,
// since chunks start at multiples of MX_CK), whether row i opens a group (the buffer
// is cleared) and whether it closes one (the group is reduced; lane sl then holds row
// i + sl).  `top` is the first row the walk visits.
template <int LG> EXPM_D int rs_slot(int i, int r) { return LG <= MX_CK ? (r % LG) : (i % LG); }
template <int LG> EXPM_D bool rs_open(int i, int r, int top) { return rs_slot<LG>(i, r) == LG - 1 || i == top; }

// ------------------------------------------------------------------ pass 0
// One thread per (block, column, system): x_0 on the block with the pass's separator
// values as boundary data, then, bottom-up, per row q (one row behind the back
// substitution, which supplies x_{q-1}):
//   r_1[q] = v_q - (M x_0)_q           float-float; with STORE (a correction follows)
//                                      stored (hi, and lo when a second one follows),
//                                      otherwise (no correction) only its norm is formed
//   Y += sum_s Re(W_s x_0)             float pairs, reduce-scatter over the system lanes
//                                      (binary64 when no correction follows)
//   next end values (STORE)            dot with w = M~_b^{-1} eps_last (w_q = -c'_q w_{q+1})
//                                      and a bottom-up sweep for the first row
//   norms                              ||r_1||^2 and ||x_0||^2 per system
template <int LG, bool ST, bool STORE>
__global__ void __launch_bounds__(MX_CTA, 4) mx_main(TriGeom g, MxArgs a, TriPoles ps, int mode) {
    extern __shared__ __align__(16) float mx_smem[];
    MxLane t;
    float rn2 = 0.f, xn2 = 0.f;
    const bool ok = mx_lane<LG>(g, t);
    MxRows<ST> rw;
    mx_stage<LG, ST>(g, a, true, 2, mx_smem, ok ? t.first : 0, ok ? t.j : 0, ok ? t.s : 0, rw);
    const bool resid = STORE || (mode & MX_RESID) != 0;
    if (ok) {
        constexpr bool final_ = !STORE;
        const int Rc = g.Rc, len = t.len;
        const int RL = Rc * LG;
        const bool lo_out = (mode & MX_LO_OUT) != 0;
        const cx<float> zero = {0.f, 0.f};
        const f32x2 thr = split_bits(ps.th_re[t.s]), thi = split_bits(ps.th_im[t.s]);
        const f32x2 wr = t.active ? split_bits(ps.w_re[t.s]) : f32x2{0.f, 0.f};
        const f32x2 wi = t.active ? split_bits(ps.w_im[t.s]) : f32x2{0.f, 0.f};
        const cx<float> *SG = a.sig + (int64_t)t.s * g.P * Rc;
        const cx<float> sl_v = t.has_left ? SG[(int64_t)(t.b - 1) * Rc + t.j] : zero;
        const cx<float> sr_v = t.has_right ? SG[(int64_t)t.b * Rc + t.j] : zero;
        const f32x2 eleft = t.has_left ? f32x2{a.ePf[t.first - 1], a.ePl[t.first - 1]} : f32x2{0.f, 0.f};
        const f32x2 eright = t.has_right ? f32x2{rw.eh[len - 1], rw.el[len - 1]} : f32x2{0.f, 0.f};
        cx<float> *Rw = STORE ? a.R + (t.first * Rc + t.j) * LG + t.sl : nullptr;
        cx<float> *Rlw = a.Rlo != nullptr ? a.Rlo + (t.first * Rc + t.j) * LG + t.sl : nullptr;
        const int64_t ckstride = (int64_t)g.P * Rc * LG;
        float2 *ck = a.ckpt + t.bj * LG + t.sl;
        const int top = ((len + MX_CK - 1) / MX_CK) * MX_CK - 1;
        double *Yb = a.Y + t.first * Rc + t.j;

        // state of the bottom-up row walk: x_{q+1}, x_{q+2} of the residual row q (x_len is
        // the right separator value), the last-row spike w, its dot, the UL sweep h, and
        // e'_q of row q (the coupling to row q+1)
        cx<float> xr_ = sr_v, xs_ = zero;
        cx<float> wsp = zero, yw = zero, h = zero, xfirst = zero, xlast = zero;
        f32x2 en = eright;
        f32x2s yv[LG];
        auto row_resid = [&](auto fast, int q, cx<float> xl, cx<float> xs, cx<float> xr) {
            constexpr bool F = decltype(fast)::value;
            const f32x2 el = (F || q > 0) ? f32x2{rw.eh[q - 1], rw.el[q - 1]} : eleft;
            const f32x2 dq = {rw.dh[q], rw.dl[q]};
            cx<float> hi, lo;
            mx_resid_first(f32x2{rw.v_hi(q), rw.v_lo(q)}, dq, el, en, thr, thi, xl, xs, xr, hi, lo);
            rn2 += cnorm2(hi);
            if (STORE) {
                Rw[q * RL] = hi;
                if (lo_out) Rlw[q * RL] = lo;
                const bool lastq = !F && q == len - 1;
                const cx<float> gq = rw.g[q * LG];
                wsp = lastq ? gq : -cmul_rn(cprime(gq, en.hi), wsp);
                yw = cfma_rn(yw, wsp, hi);
                h = zstep(rw.u[q * LG], lastq ? 0.f : en.hi, hi, h);
            }
            en = el;
        };
        auto fetch = [&](int step, cx<float> (&f)[MX_CK]) {
            const int nch = (len + MX_CK - 1) / MX_CK;
            const int c = step < nch ? step : 2 * nch - 1 - step;
#pragma unroll
            for (int r = 0; r < MX_CK; ++r)
                f[r] = (c * MX_CK + r < len) ? cx<float>{rw.v_hi(c * MX_CK + r), 0.f} : zero;
        };
        auto per_row = [&](auto fast, int i, int r, cx<float> x, cx<float>) {
            constexpr bool F = decltype(fast)::value;
            const int ix = rs_slot<LG>(i, r);
            if (rs_open<LG>(i, r, top)) {
#pragma unroll
                for (int u = 0; u < LG; ++u) yv[u] = f32x2s{0.f, 0.f};
            }
            if (F || i < len) {
                if (resid && (F || i + 1 < len)) row_resid(fast, i + 1, x, xs_, xr_);
                xr_ = xs_;
                xs_ = x;
                if (!F) {
                    if (i == len - 1) {
                        xlast = x;
                        xr_ = sr_v;
                    }
                    if (i == 0) xfirst = x;
                }
                yv[ix] = t.active ? re_wx_pair(wr, wi, x) : f32x2s{0.f, 0.f};
                xn2 += cnorm2(x);
            }
            if (ix == 0) {
                reduce_scatter<LG>(t.gmask, t.sl, yv);
                const int row = i + t.sl;  // lane sl now holds row i + sl
                if (F || row < len) y_store_pair(Yb, (int64_t)row * Rc, yv[0], final_);
            }
        };
        mx_block_walk<LG, ST>(t, rw, sl_v, sr_v, eleft.hi, eright.hi, ck, ckstride, fetch, per_row);
        // row 0: x_{-1} is the left separator value (e' = 0 without one)
        if (resid) row_resid(Bool<false>(), 0, sl_v, xs_, xr_);
        if (t.active) {
            cx<float> *XB = a.xb + (((int64_t)t.s * g.P + t.b) * Rc + t.j) * 2;
            XB[0] = xfirst;
            XB[1] = xlast;
            if (STORE) {
                cx<float> *YE = a.yend + (((int64_t)t.s * Rc + t.j) * g.P + t.b) * 2;
                YE[0] = h;
                YE[1] = yw;
            }
        }
        // the separator row after this block
        f32x2s acc = t.active ? re_wx_pair(wr, wi, sr_v) : f32x2s{0.f, 0.f};
#pragma unroll
        for (int off = LG / 2; off > 0; off >>= 1) acc = acc + shfl_xor(t.gmask, acc, off);
        if (t.sl == 0 && t.has_right) y_store_pair(Yb, (int64_t)len * Rc, acc, final_);
    }
    if (resid) cta_norms<LG>(rn2, xn2, a.part3);
}

// ------------------------------------------------------------------ pass k >= 1
// d_k on the block from the stored r_k, Y += sum_s Re(W_s d_k) (binary64 on the last
// pass, i.e. without STORE), and r_{k+1} = r_k - M d_k: with STORE (another correction
// follows) float-float and stored in place with the next end values; on the last pass
// with MX_RESID, the binary32 verification residual (its norm only).  Returns at once
// when the stopping test has passed; the last pass then only turns Y's float pairs into
// binary64.
template <int LG, bool ST, bool STORE>
__global__ void __launch_bounds__(MX_CTA, 4) mx_pass(TriGeom g, MxArgs a, TriPoles ps, int mode, int ring_off) {
    extern __shared__ __align__(16) float mx_smem[];
    constexpr bool final_ = !STORE;
    if (a.state->done) {  // uniform over the launch
        if (!final_) return;
        MxLane t;
        if (!mx_lane<LG>(g, t)) return;
        for (int i = t.sl; i <= t.len; i += LG) {  // rows of the block, then the separator after it
            if (i == t.len && !t.has_right) break;
            const int64_t idx = (t.first + i) * g.Rc + t.j;
            const f32x2 y = reinterpret_cast<const f32x2 *>(a.Y)[idx];
            a.Y[idx] = widen_bits(y.hi) + widen_bits(y.lo);
        }
        return;
    }
    MxLane t;
    float rn2 = 0.f;
    const bool ok = mx_lane<LG>(g, t);
    MxRows<ST> rw;
    mx_stage<LG, ST>(g, a, false, STORE ? 2 : 1, mx_smem, ok ? t.first : 0, ok ? t.j : 0, ok ? t.s : 0, rw);
    const bool resid = STORE || (mode & MX_RESID) != 0;
    if (ok) {
        const int Rc = g.Rc, len = t.len;
        const int RL = Rc * LG;
        const bool lo_in = (mode & MX_LO_IN) != 0, lo_out = (mode & MX_LO_OUT) != 0;
        const cx<float> zero = {0.f, 0.f};
        const f32x2 thr = split_bits(ps.th_re[t.s]), thi = split_bits(ps.th_im[t.s]);
        const float wr = t.active ? __double2float_rn(ps.w_re[t.s]) : 0.f;
        const float wi = t.active ? __double2float_rn(ps.w_im[t.s]) : 0.f;
        const cx<float> *SG = a.sig + (int64_t)t.s * g.P * Rc;
        const cx<float> sl_v = t.has_left ? SG[(int64_t)(t.b - 1) * Rc + t.j] : zero;
        const cx<float> sr_v = t.has_right ? SG[(int64_t)t.b * Rc + t.j] : zero;
        const f32x2 eleft = t.has_left ? f32x2{a.ePf[t.first - 1], a.ePl[t.first - 1]} : f32x2{0.f, 0.f};
        const f32x2 eright = t.has_right ? f32x2{rw.eh[len - 1], rw.el[len - 1]} : f32x2{0.f, 0.f};
        cx<float> *Rw = a.R + (t.first * Rc + t.j) * LG + t.sl;
        cx<float> *Rlw = a.Rlo != nullptr ? a.Rlo + (t.first * Rc + t.j) * LG + t.sl : nullptr;
        const int64_t ckstride = (int64_t)g.P * Rc * LG;
        float2 *ck = a.ckpt + t.bj * LG + t.sl;
        const int top = ((len + MX_CK - 1) / MX_CK) * MX_CK - 1;
        double *Yb = a.Y + t.first * Rc + t.j;

        cx<float> xr_ = sr_v, xs_ = zero, rs_ = zero;  // x_{q+1}, x_q and r_k[q] of the residual row q
        cx<float> wsp = zero, yw = zero, h = zero, xfirst = zero, xlast = zero;
        f32x2 en = eright;
        float yv[LG];
        auto row_resid = [&](auto fast, int q, cx<float> xl, cx<float> xs, cx<float> xr, cx<float> rk) {
            constexpr bool F = decltype(fast)::value;
            const f32x2 el = (F || q > 0) ? f32x2{rw.eh[q - 1], STORE ? rw.el[q - 1] : 0.f} : eleft;
            cx<float> hi, lo = zero;
            if (STORE) {
                const cx<float> rl = lo_in ? Rlw[q * RL] : zero;
                mx_resid_comp(rk, rl, f32x2{rw.dh[q], rw.dl[q]}, el, en, thr, thi, xl, xs, xr, hi, lo);
            } else {
                hi = mx_resid_corr(rk, rw.dh[q], el.hi, en.hi, thr.hi, thi.hi, xl, xs, xr);
            }
            rn2 += cnorm2(hi);
            if (STORE) {
                Rw[q * RL] = hi;
                if (lo_out) Rlw[q * RL] = lo;
                const bool lastq = !F && q == len - 1;
                const cx<float> gq = rw.g[q * LG];
                wsp = lastq ? gq : -cmul_rn(cprime(gq, en.hi), wsp);
                yw = cfma_rn(yw, wsp, hi);
                h = zstep(rw.u[q * LG], lastq ? 0.f : en.hi, hi, h);
            }
            en = el;
        };
        // the ring sits after the tile in dynamic shared memory
        MxRing ring{reinterpret_cast<cx<float> *>(mx_smem + ring_off) + threadIdx.x, Rw, RL, len,
                    (len + MX_CK - 1) / MX_CK};
        ring.prime();
        auto fetch = [&](int step, cx<float> (&f)[MX_CK]) { ring.fetch(step, f); };
        auto per_row = [&](auto fast, int i, int r, cx<float> x, cx<float> ri) {
            constexpr bool F = decltype(fast)::value;
            const int ix = rs_slot<LG>(i, r);
            if (rs_open<LG>(i, r, top)) {
#pragma unroll
                for (int u = 0; u < LG; ++u) yv[u] = 0.f;
            }
            if (F || i < len) {
                if (resid && (F || i + 1 < len)) row_resid(fast, i + 1, x, xs_, xr_, rs_);
                xr_ = xs_;
                xs_ = x;
                rs_ = ri;
                if (!F) {
                    if (i == len - 1) {
                        xlast = x;
                        xr_ = sr_v;
                    }
                    if (i == 0) xfirst = x;
                }
                yv[ix] = re_wx_f32(wr, wi, x);
            }
            if (ix == 0) {
                reduce_scatter<LG>(t.gmask, t.sl, yv);
                const int row = i + t.sl;
                if (F || row < len) y_add(Yb, (int64_t)row * Rc, yv[0], final_);
            }
        };
        mx_block_walk<LG, ST>(t, rw, sl_v, sr_v, eleft.hi, eright.hi, ck, ckstride, fetch, per_row);
        cp_async_wait_all();
        if (resid) row_resid(Bool<false>(), 0, sl_v, xs_, xr_, rs_);
        if (t.active) {
            cx<float> *XB = a.xb + (((int64_t)t.s * g.P + t.b) * Rc + t.j) * 2;
            XB[0] = xfirst;
            XB[1] = xlast;
            if (STORE) {
                cx<float> *YE = a.yend + (((int64_t)t.s * Rc + t.j) * g.P + t.b) * 2;
                YE[0] = h;
                YE[1] = yw;
            }
        }
        float acc = re_wx_f32(wr, wi, sr_v);
#pragma unroll
        for (int off = LG / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(t.gmask, acc, off);
        if (t.sl == 0 && t.has_right) y_add(Yb, (int64_t)len * Rc, acc, final_);
    }
    if (resid) cta_norms<LG>(rn2, 0.f, a.part3);
}

// ------------------------------------------------------------------ separator residuals
// grid (ceil((P-1) Rc / MX_CTA), S): one thread per (separator, column) of system blockIdx.y.
// x_{p-1} and x_{p+1} are the last row of block b and the first row of block b+1 of
// the pass's solution (xb), x_p the separator value.
template <bool FIRST>
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
        const int64_t e1 = ((int64_t)s * g.P + b + 1) * g.Rc + j;
        const cx<float> xs = a.sig[e];
        const cx<float> xl = a.xb[2 * e + 1];
        const cx<float> xr = a.xb[2 * e1];
        const f32x2 thr = split_bits(ps.th_re[s]), thi = split_bits(ps.th_im[s]);
        const f32x2 dq = {a.dPf[p], a.dPl[p]}, el = {a.ePf[p - 1], a.ePl[p - 1]}, er = {a.ePf[p], a.ePl[p]};
        cx<float> hi, lo = {0.f, 0.f};
        if (FIRST) {
            mx_resid_first(f32x2{a.VPf[p * g.Rc + j], a.VPl[p * g.Rc + j]}, dq, el, er, thr, thi, xl, xs, xr, hi, lo);
            xn2 = cnorm2(xs);
        } else if (mode & MX_COMP) {
            const cx<float> rl = (mode & MX_LO_IN) ? a.sepLo[e] : cx<float>{0.f, 0.f};
            mx_resid_comp(a.sepR[e], rl, dq, el, er, thr, thi, xl, xs, xr, hi, lo);
        } else {
            hi = mx_resid_corr(a.sepR[e], dq.hi, el.hi, er.hi, thr.hi, thi.hi, xl, xs, xr);
        }
        rn2 = cnorm2(hi);
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

// ------------------------------------------------------------------ reduced system
// Row b of the reduced separator system (b < P-1) couples sigma_{b-1}, sigma_b and
// sigma_{b+1} through the corner entries of the neighbouring block inverses
// (tridiag.cu's Schur complement):
//   A_b = -e'_{p-1} e'_{p-B} u_b[last],   C_b = -e'_p e'_{p+B-1} w_{b+1}[first],
//   B_b = d'_p + theta - e'_{p-1}^2 w_b[last] - e'_p^2 u_{b+1}[first],
//   D_b = rhs_p - e'_{p-1} y_b[last] - e'_p y_{b+1}[first]            (p = bB + m).
// A, B, C depend on neither the column nor the pass: mx_cr_coef forms them once per
// factorization, stored contiguously per system with e'_{p-1}, e'_p, so that the pass's
// CR reads them coalesced instead of gathering rows B apart.
struct __align__(16) MxCrc {
    cx<float> A, B, C;
    float el, er;
};

__global__ void __launch_bounds__(128) mx_cr_coef(TriGeom g, const float *__restrict__ dPf,
                                                  const float *__restrict__ ePf, TriPoles ps,
                                                  const cx<float> *__restrict__ spk, MxCrc *crc) {
    const int n = g.P - 1;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * g.S) return;
    const int s = (int)(t / n), b = (int)(t % n);
    const int64_t r = (int64_t)b * g.B + g.m;  // separator row
    const float el = ePf[r - 1], er = ePf[r];
    const cx<float> *SP = spk + (int64_t)s * g.P * 4;
    const cx<float> uL = SP[4 * b + 1], wL = SP[4 * b + 3];
    const cx<float> u0n = SP[4 * (b + 1) + 0], w0n = SP[4 * (b + 1) + 2];
    const cx<float> th = {__double2float_rn(ps.th_re[s]), __double2float_rn(ps.th_im[s])};
    MxCrc c;
    c.A = b >= 1 ? -scale(el * ePf[r - g.B], uL) : cxz<float>();
    c.C = b + 1 <= n - 1 ? -scale(er * ePf[r + g.B - 1], w0n) : cxz<float>();
    c.B = cx<float>{dPf[r] + th.re, th.im} - scale(el * el, wL) - scale(er * er, u0n);
    c.el = el;
    c.er = er;
    crc[t] = c;
}

// The pass's reduced system, one CTA of 512 threads per (system, column), solved by cyclic
// reduction in shared memory; the right-hand side is V's separator entry (pass 0) or the
// separator residual r_k (later passes).
__global__ void __launch_bounds__(512) mx_cr(TriGeom g, const MxCrc *__restrict__ crc,
                                             const float *__restrict__ VPf, const cx<float> *__restrict__ sepRhs,
                                             const cx<float> *__restrict__ yend, cx<float> *__restrict__ sigma,
                                             const int *skip) {
    if (skip != nullptr && *skip) return;  // refinement already converged (uniform over the launch)
    extern __shared__ __align__(16) unsigned char mx_cr_smem[];
    const int n = g.P - 1;
    const int np = (int)cr_len<float>(n);
    cx<float> *A = reinterpret_cast<cx<float> *>(mx_cr_smem);
    cx<float> *Bc = A + np;
    cx<float> *C = Bc + np;
    cx<float> *D = C + np;
    const int s = blockIdx.x / g.Rc;
    const int j = blockIdx.x % g.Rc;
    const MxCrc *CF = crc + (int64_t)s * n;
    const cx<float> *YE = yend + ((int64_t)s * g.Rc + j) * g.P * 2;
    // four rows per thread and round, all their loads issued before any is used
    constexpr int U = 4;
    for (int b0 = threadIdx.x; b0 < n; b0 += U * blockDim.x) {
        MxCrc c[U];
        cx<float> yL[U], y0n[U], rhs[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int b = b0 + u * blockDim.x;
            if (b < n) {
                c[u] = CF[b];
                yL[u] = YE[2 * b + 1];
                y0n[u] = YE[2 * (b + 1)];
                const int64_t r = (int64_t)b * g.B + g.m;
                rhs[u] = sepRhs != nullptr ? sepRhs[((int64_t)s * g.P + b) * g.Rc + j] : cx<float>{VPf[r * g.Rc + j], 0.f};
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int b = b0 + u * blockDim.x;
            if (b < n) {
                const int bp = cr_ix<float>(b);
                A[bp] = c[u].A;
                Bc[bp] = c[u].B;
                C[bp] = c[u].C;
                D[bp] = rhs[u] - scale(c[u].el, yL[u]) - scale(c[u].er, y0n[u]);
            }
        }
    }
    __syncthreads();
    cr_solve_smem<float>(A, Bc, C, D, n);
    cx<float> *SG = sigma + (int64_t)s * g.P * g.Rc;
    for (int b = threadIdx.x; b < n; b += blockDim.x) SG[(int64_t)b * g.Rc + j] = D[cr_ix<float>(b)];
}

// ------------------------------------------------------------------ stopping test
// One CTA of MX_CHECK_T threads.  After pass `pass`: iters = pass; with a residual, the
// relative residual max_s ||r_s|| / ((beta + |theta_s|) ||x_s||) and the stopping
// decision.  The partial sums are added in a fixed order, so the decision does not
// depend on scheduling: the solve kernels' partials [cta][lane][2] (binary32) are read coalesced,
// thread t taking entries t, t + T, ... (all of one (lane, component), since 2 LG
// divides T) into four interleaved sums, then a tree over the threads of each
// (lane, component); the separator partials [system][cta][2] by `tps` threads per system
// (a power of two), system s = t / tps, strided, then a tree.
constexpr int MX_CHECK_T = 1024;
__global__ void __launch_bounds__(MX_CHECK_T) mx_check(MxArgs a, TriPoles ps, int S, int LG, int tps, int n3, int nS,
                                                       int pass, int has_resid, int first, double tol) {
    __shared__ double red[2][MX_CHECK_T];
    __shared__ float redf[MX_CHECK_T];
    __shared__ double bins[2 * 32];  // (lane, component) sums of the solve kernels' partials
    __shared__ double rel[TRI_MAXSYS];
    MixState *st = a.state;
    if (st->done) return;
    const int t = threadIdx.x;
    if (has_resid) {
        // (binary32 here: a CTA runs on one SM, whose FP64 rate would bind)
        const int64_t n = (int64_t)n3 * LG * 2;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        int64_t e = t;
        for (; e + 3 * MX_CHECK_T < n; e += 4 * MX_CHECK_T) {
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] += a.part3[e + k * MX_CHECK_T];
        }
        for (int k = 0; e < n; e += MX_CHECK_T, ++k) acc[k] += a.part3[e];  // fewer than 4 left
        redf[t] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        __syncthreads();
        for (int h = MX_CHECK_T / 2; h >= 2 * LG; h >>= 1) {
            if (t < h) redf[t] += redf[t + h];
            __syncthreads();
        }
        if (t < 2 * LG) bins[t] = (double)redf[t];
        __syncthreads();
        const int s = t / tps, l = t % tps;
        double r2 = 0.0, x2 = 0.0;
        if (s < S) {
            for (int i = l; i < nS; i += tps) {
                r2 += a.partS[((int64_t)s * nS + i) * 2];
                x2 += a.partS[((int64_t)s * nS + i) * 2 + 1];
            }
        }
        red[0][t] = r2;
        red[1][t] = x2;
        __syncthreads();
        for (int h = tps / 2; h > 0; h >>= 1) {
            if (l < h) {
                red[0][t] += red[0][t + h];
                red[1][t] += red[1][t + h];
            }
            __syncthreads();
        }
        if (s < S && l == 0) {
            r2 = red[0][t] + bins[2 * s];
            x2 = red[1][t] + bins[2 * s + 1];
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
    size_t dPf, dPl, ePf, ePl, beta, pg, pu, spk, crc, factor_total;
    size_t VPf, VPl, yend, sig, xb, sepR, sepLo, R, Rlo, ckpt, part3, partS, state, solve_total;
    int nchk, n3, nSx;
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
    L.beta = off; off += 256;
    L.pg = off; off += al(N * LG * 8);
    L.pu = off; off += al(N * LG * 8);
    L.spk = off; off += al(S * P * 4 * 8);
    L.crc = off; off += al(S * std::max<size_t>(P - 1, 1) * sizeof(MxCrc));
    L.factor_total = off;
    L.nchk = (g.B + MX_CK - 1) / MX_CK;
    L.n3 = (int)((P * Rc * LG + MX_CTA - 1) / MX_CTA);
    L.nSx = g.P > 1 ? (int)(((P - 1) * Rc + MX_CTA - 1) / MX_CTA) : 0;
    off = 0;
    L.VPf = off; off += al(N * Rc * 4);
    L.VPl = off; off += al(N * Rc * 4);
    L.yend = off; off += al(S * P * Rc * 2 * 8);
    L.sig = off; off += al(S * P * Rc * 8);
    L.xb = off; off += al(S * P * Rc * 2 * 8);
    L.sepR = off; off += al(S * P * Rc * 8);
    L.sepLo = off; off += al(S * P * Rc * 8);
    L.R = off; off += max_refine >= 1 ? al(N * Rc * LG * 8) : 0;
    L.Rlo = off; off += max_refine >= 2 ? al(N * Rc * LG * 8) : 0;
    L.ckpt = off; off += al((size_t)std::max(L.nchk - 1, 1) * P * Rc * LG * 8);
    L.part3 = off; off += al((size_t)L.n3 * LG * 2 * 8);
    L.partS = off; off += al((size_t)std::max(L.nSx, 1) * S * 2 * 8);
    L.state = off; off += al(sizeof(MixState));
    L.solve_total = off;
    return L;
}

// Shared-memory bytes of a launch's tile (0: the tile does not fit, rows are read from
// global memory).  The attribute is a ceiling set once per kernel to MX_SMEM_MAX, never
// lowered under a concurrent launch.
static size_t mx_smem_bytes(const TriGeom &g, bool with_v, int npiv) {
    int64_t rows, cols;
    mx_tile_bound(g, rows, cols);
    const size_t bytes = 4 * (size_t)mx_tile_floats(rows, cols, g.LG, with_v, npiv);
    return bytes <= (size_t)MX_SMEM_MAX ? bytes : 0;
}
template <class K> static cudaError_t mx_attr(K kernel, size_t ceiling = MX_SMEM_MAX) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ceiling);
}
template <int LG, bool STORE>
static cudaError_t launch_main_t(const TriGeom &g, const MxArgs &a, const TriPoles &ps, int mode, unsigned grid,
                                 size_t smem, cudaStream_t st) {
    cudaError_t err = smem > 0 ? mx_attr(mx_main<LG, true, STORE>) : cudaSuccess;
    if (err != cudaSuccess) return err;
    if (smem > 0) mx_main<LG, true, STORE><<<grid, MX_CTA, smem, st>>>(g, a, ps, mode);
    else mx_main<LG, false, STORE><<<grid, MX_CTA, 0, st>>>(g, a, ps, mode);
    return cudaGetLastError();
}
template <int LG>
static cudaError_t launch_main(const TriGeom &g, const MxArgs &a, const TriPoles &ps, int mode, unsigned grid,
                               size_t smem, cudaStream_t st) {
    return (mode & MX_STORE) ? launch_main_t<LG, true>(g, a, ps, mode, grid, smem, st)
                             : launch_main_t<LG, false>(g, a, ps, mode, grid, smem, st);
}
template <int LG, bool STORE>
static cudaError_t launch_pass_t(const TriGeom &g, const MxArgs &a, const TriPoles &ps, int mode, unsigned grid,
                                 size_t tile, cudaStream_t st) {
    // the tile (0 bytes when it does not fit) then the ring of right-hand sides, 16-byte aligned
    const size_t off = (tile + 15) & ~(size_t)15;
    const size_t smem = off + MX_RING_BYTES;
    const size_t ceiling = MX_SMEM_MAX + 16 + MX_RING_BYTES;
    cudaError_t err = tile > 0 ? mx_attr(mx_pass<LG, true, STORE>, ceiling) : mx_attr(mx_pass<LG, false, STORE>, ceiling);
    if (err != cudaSuccess) return err;
    if (tile > 0) mx_pass<LG, true, STORE><<<grid, MX_CTA, smem, st>>>(g, a, ps, mode, (int)(off / 4));
    else mx_pass<LG, false, STORE><<<grid, MX_CTA, smem, st>>>(g, a, ps, mode, (int)(off / 4));
    return cudaGetLastError();
}
template <int LG>
static cudaError_t launch_pass(const TriGeom &g, const MxArgs &a, const TriPoles &ps, int mode, unsigned grid,
                               size_t tile, cudaStream_t st) {
    return (mode & MX_STORE) ? launch_pass_t<LG, true>(g, a, ps, mode, grid, tile, st)
                             : launch_pass_t<LG, false>(g, a, ps, mode, grid, tile, st);
}
template <int LG>
static cudaError_t launch_ends(const TriGeom &g, const MxArgs &a, cudaStream_t st) {
    const int64_t n = (int64_t)g.P * LG * ((g.Rc + MX_EC - 1) / MX_EC);
    const unsigned grid = (unsigned)((n + 127) / 128);
    if (g.Rc % 2 == 0) mx_ends<LG, true><<<grid, 128, 0, st>>>(g, a);  // rows of V 8-byte aligned
    else mx_ends<LG, false><<<grid, 128, 0, st>>>(g, a);
    return cudaGetLastError();
}
template <int LG>
static cudaError_t launch_pivots(const TriGeom &g, const float *dPf, const float *ePf, const TriPoles &ps,
                                 cx<float> *pg, cx<float> *pu, cx<float> *spk, cudaStream_t st) {
    const int64_t n = (int64_t)g.P * LG;
    mx_pivots<LG><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, dPf, ePf, ps, pg, pu, spk);
    return cudaGetLastError();
}

#define MX_DISPATCH(fn, ...)                                   \
    switch (g.LG) {                                            \
        case 1: return fn<1>(__VA_ARGS__);                     \
        case 2: return fn<2>(__VA_ARGS__);                     \
        case 4: return fn<4>(__VA_ARGS__);                     \
        case 8: return fn<8>(__VA_ARGS__);                     \
        case 16: return fn<16>(__VA_ARGS__);                   \
        default: return fn<32>(__VA_ARGS__);                   \
    }

}  // namespace

// Blocks long enough that the (block, column, system) threads fill MX_WAVES waves of
// MX_THREADS_SM threads per SM, at most MX_PMAX blocks (the reduced system lives in
// shared memory) and at least TRI_MMIN interior rows each; then more, shorter blocks
// until a CTA's rows of d', e', V and both pivot tables fit in MX_SMEM_MAX bytes of
// shared memory (otherwise the solve kernels read them from global memory).
static TriGeom mx_fit(int64_t N, int S, int Rc, int lg, int64_t P) {
    TriGeom g{};
    g.N = N;
    g.S = S;
    g.Rc = Rc;
    g.LG = lg;
    P = std::max<int64_t>(1, std::min<int64_t>(P, MX_PMAX));
    int64_t m = (N - P + 1 + P - 1) / P;  // ceil((N - (P-1)) / P)
    m = std::max<int64_t>(m, TRI_MMIN);
    P = (N + m) / (m + 1);  // last block length N - (P-1)(m+1) lies in [1, m+1]
    P = std::max<int64_t>(P, 1);
    if (P > MX_PMAX) {
        m = (N + MX_PMAX - 1) / MX_PMAX;
        P = (N + m) / (m + 1);
    }
    g.m = (int)m;
    g.B = (int)(m + 1);
    g.P = (int)P;
    return g;
}

TriGeom tri_mixed_geometry(int64_t N, int S, int Rc, int sm_count) {
    int lg = 1;
    while (lg < S) lg *= 2;
    const int64_t target = (int64_t)sm_count * MX_THREADS_SM * MX_WAVES;
    int64_t P = target / ((int64_t)lg * Rc);
    TriGeom g = mx_fit(N, S, Rc, lg, P);
    while (mx_smem_bytes(g, true, 2) == 0 && g.P < MX_PMAX && g.m > TRI_MMIN) {
        P = std::min<int64_t>(MX_PMAX, (int64_t)g.P * 5 / 4 + 1);
        const TriGeom h = mx_fit(N, S, Rc, lg, P);
        if (h.P <= g.P) break;  // no more blocks to be had
        g = h;
    }
    return g;
}
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
    cx<float> *pg = (cx<float> *)(p + L.pg), *pu = (cx<float> *)(p + L.pu);
    cx<float> *spk = (cx<float> *)(p + L.spk);
    err = prof.timed("tri_mixed_pivots", st, [&] { MX_DISPATCH(launch_pivots, g, dPf, ePf, ps, pg, pu, spk, st); });
    if (err != cudaSuccess || g.P <= 1) return err;
    MxCrc *crc = (MxCrc *)(p + L.crc);
    const int64_t nc = (int64_t)(g.P - 1) * g.S;
    return prof.timed("tri_mixed_cr_coef", st, [&] {
        mx_cr_coef<<<(unsigned)((nc + 127) / 128), 128, 0, st>>>(g, dPf, ePf, ps, spk, crc);
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
    a.beta_bits = (const unsigned *)(p + L.beta);
    a.pg = (const cx<float> *)(p + L.pg);
    a.pu = (const cx<float> *)(p + L.pu);
    a.spk = (const cx<float> *)(p + L.spk);
    a.crc = (const MxCrc *)(p + L.crc);
    float *VPf = (float *)(q + L.VPf), *VPl = (float *)(q + L.VPl);
    a.VPf = VPf;
    a.VPl = VPl;
    a.yend = (cx<float> *)(q + L.yend);
    a.sig = (cx<float> *)(q + L.sig);
    a.xb = (cx<float> *)(q + L.xb);
    a.sepR = (cx<float> *)(q + L.sepR);
    a.sepLo = (cx<float> *)(q + L.sepLo);
    a.R = mo.max_refine >= 1 ? (cx<float> *)(q + L.R) : nullptr;
    a.Rlo = mo.max_refine >= 2 ? (cx<float> *)(q + L.Rlo) : nullptr;
    a.ckpt = (float2 *)(q + L.ckpt);
    a.part3 = (float *)(q + L.part3);
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
    const unsigned grid = (unsigned)L.n3;
    const size_t smem_v = mx_smem_bytes(g, true, 2);
    if (g.P > 1) {
        err = prof.timed("tri_mixed_ends", st, [&] { MX_DISPATCH(launch_ends, g, a, st); });
        if (err != cudaSuccess) return err;
        // a ceiling for the largest reduced system, never lowered under a concurrent launch
        err = cudaFuncSetAttribute(mx_cr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(4 * cr_len<float>(MX_PMAX - 1) * sizeof(cx<float>)));
        if (err != cudaSuccess) return err;
    }
    const size_t smem = g.P > 1 ? 4 * cr_len<float>(g.P - 1) * sizeof(cx<float>) : 0;
    const unsigned sgrid = (unsigned)L.nSx;
    const int npass = 1 + mo.max_refine;
    for (int k = 0; k < npass; ++k) {
        const bool last = k == npass - 1;
        const bool resid = !last || mo.verify;
        // stored residuals are float-float (pass 0 always; later passes from r_k's low
        // part when the pass before kept it); the final verification residual is binary32
        int mode = 0;
        if (resid) mode |= MX_RESID;
        if (!last) mode |= MX_STORE;
        if (last) mode |= MX_FINAL;
        if (k >= 1 && !last) mode |= MX_COMP | MX_LO_IN;
        if (!last && k + 1 < npass - 1) mode |= MX_LO_OUT;
        if (g.P > 1) {
            err = prof.timed("tri_mixed_cr", st, [&] {
                mx_cr<<<g.S * g.Rc, 512, smem, st>>>(g, a.crc, VPf, k == 0 ? nullptr : a.sepR, a.yend, a.sig,
                                                     k == 0 ? nullptr : &a.state->done);
                return cudaGetLastError();
            });
            if (err != cudaSuccess) return err;
        }
        if (k == 0) {
            err = prof.timed("tri_mixed_main", st, [&] { MX_DISPATCH(launch_main, g, a, ps, mode, grid, smem_v, st); });
        } else {
            err = prof.timed("tri_mixed_pass", st, [&] { MX_DISPATCH(launch_pass, g, a, ps, mode, grid, mx_smem_bytes(g, false, (mode & MX_STORE) ? 2 : 1), st); });
        }
        if (err != cudaSuccess) return err;
        if (resid && g.P > 1) {
            err = prof.timed("tri_mixed_sep_resid", st, [&] {
                const dim3 sg(sgrid, (unsigned)g.S);
                if (k == 0) mx_sep_resid<true><<<sg, MX_CTA, 0, st>>>(g, a, ps, mode);
                else mx_sep_resid<false><<<sg, MX_CTA, 0, st>>>(g, a, ps, mode);
                return cudaGetLastError();
            });
            if (err != cudaSuccess) return err;
        }
        err = prof.timed("tri_mixed_check", st, [&] {
            int tps = 128;
            while (tps > 32 && tps * g.S > MX_CHECK_T) tps /= 2;
            mx_check<<<1, MX_CHECK_T, 0, st>>>(a, ps, g.S, g.LG, tps, L.n3, g.P > 1 ? L.nSx : 0, k, resid ? 1 : 0,
                                               k == 0 ? 1 : 0, mo.tol);
            return cudaGetLastError();
        });
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
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
