// arith.cuh -- scalar and complex arithmetic used by the device kernels.
//
// Two real types are supported by every templated kernel:
//   double  binary64 on the FP64 pipe.
//   f32x2   "float-float": an unevaluated sum hi + lo of two binary32 numbers
//           with |lo| <= ulp(hi)/2, giving a ~48-bit significand on the FP32 pipe.
//           The error-free transformations are Knuth's TwoSum, Dekker's
//           Fast2Sum and the FMA-based TwoProd (Dekker 1971; Joldes, Muller and
//           Popescu, "Tight and rigorous error bounds for basic building blocks of
//           double-word arithmetic", ACM TOMS 2017).  All float operations below use
//           the *_rn intrinsics so the compiler cannot contract or reorder them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define EXPM_HD __host__ __device__ __forceinline__
#define EXPM_D __device__ __forceinline__

// ------------------------------------------------------------------ packed binary32 pairs
// Two binary32 numbers in one 64-bit register (low half first) and the two-lane
// instructions of sm_100 and later, add/sub/mul/fma.rn.f32x2: one instruction performs
// the same operation on both halves, each rounded as the scalar *_rn operation would be.
EXPM_D uint64_t pk2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
EXPM_D void upk2(uint64_t v, float &lo, float &hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
EXPM_D uint64_t padd2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
EXPM_D uint64_t psub2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
EXPM_D uint64_t pmul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
EXPM_D uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {  // a * b + c
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
EXPM_D uint64_t pneg2(uint64_t a) { return a ^ 0x8000000080000000ull; }  // both signs flipped

// ------------------------------------------------------------------ f32x2 type
struct f32x2 {
    float hi, lo;
};

EXPM_D f32x2 two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, err};
}
EXPM_D f32x2 fast_two_sum(float a, float b) {  // requires |a| >= |b| (or a == 0)
    float s = __fadd_rn(a, b);
    float err = __fsub_rn(b, __fsub_rn(s, a));
    return {s, err};
}
// double-word + double-word, the accurate ("AccurateDWPlusDW") variant
EXPM_D f32x2 operator+(f32x2 x, f32x2 y) {
    f32x2 s = two_sum(x.hi, y.hi);
    f32x2 t = two_sum(x.lo, y.lo);
    float c = __fadd_rn(s.lo, t.hi);
    f32x2 v = fast_two_sum(s.hi, c);
    float w = __fadd_rn(t.lo, v.lo);
    return fast_two_sum(v.hi, w);
}
EXPM_D f32x2 operator-(f32x2 x) { return {-x.hi, -x.lo}; }
EXPM_D f32x2 operator-(f32x2 x, f32x2 y) { return x + (-y); }
// double-word x double-word with FMA ("DWTimesDW3"-style)
EXPM_D f32x2 operator*(f32x2 x, f32x2 y) {
    float ch = __fmul_rn(x.hi, y.hi);
    float cl = __fmaf_rn(x.hi, y.hi, -ch);
    float tl0 = __fmul_rn(x.lo, y.lo);
    float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    float cl3 = __fadd_rn(cl, cl2);
    return fast_two_sum(ch, cl3);
}
// reciprocal: binary32 seed r0 = 1/y_hi, then one Newton-Raphson step for the reciprocal,
// r1 = r0 + r0 (1 - y r0) (the correction used for division by Markstein, IBM J. Res. Dev.
// 34(1), 1990), carried out in double-word arithmetic as in the reciprocal and division
// algorithms of Joldes, Muller and Popescu (ACM TOMS 2017): one step doubles the ~24
// correct bits of the seed, which is the precision of the pair.
EXPM_D f32x2 recip(f32x2 y) {
    float r0 = __frcp_rn(y.hi);
    f32x2 r = {r0, 0.f};
    f32x2 one = {1.f, 0.f};
    f32x2 e = one - y * r;  // residual of the seed
    return r + r * e;
}

// binary64 <-> float-float.  These go through the FP64 conversion path; they
// are used only on loads of inputs and stores of outputs.
EXPM_D f32x2 to_f32x2(double x) {
    float hi = __double2float_rn(x);
    float lo = __double2float_rn(x - (double)hi);
    return {hi, lo};
}
EXPM_D double to_double(f32x2 x) { return (double)x.hi + (double)x.lo; }

// An unsigned integer m < 2^29 to binary32, rounded to nearest, on the FP32 pipe: the
// high 6 and low 23 bits become exact floats by the 2^23 bias trick (the integer in the
// significand of 2^23, then 2^23 subtracted), and one FMA rounds mh 2^23 + ml once.
// (An integer-to-float conversion instruction runs on this part's FP64 unit.)
EXPM_D float u29_to_float_rn(unsigned m) {
    const float two23 = 8388608.0f;
    const float fh = __fsub_rn(__uint_as_float(0x4b000000u | (m >> 23)), two23);
    const float fl = __fsub_rn(__uint_as_float(0x4b000000u | (m & 0x7fffffu)), two23);
    return __fmaf_rn(fh, two23, fl);
}

// the rare range of split_bits, kept out of line so that the compiler cannot turn the
// branch into a select that runs these FP64 conversions for every value
static __device__ __noinline__ f32x2 split_slow(double x) { return to_f32x2(x); }

// binary64 -> float pair with integer and binary32 operations only (no FP64-pipe work):
// hi takes the leading 24 significand bits, lo the remaining 29 bits rounded to 24; the
// pair is then renormalised.  Values outside [2^-74, 2^128) take the binary64 route.
EXPM_D f32x2 split_bits(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((u >> 52) & 0x7ff);
    if (__builtin_expect(ex < 1023 + 52 - 126 || ex > 1023 + 127, 0)) return split_slow(x);
    const unsigned sign = (unsigned)(u >> 63) << 31;
    const float hi = __uint_as_float(sign | ((unsigned)(ex - 1023 + 127) << 23) | (unsigned)((u >> 29) & 0x7fffffu));
    const float scalef = __uint_as_float((unsigned)(ex - 1023 - 52 + 127) << 23);
    float lo = __fmul_rn(u29_to_float_rn((unsigned)(u & 0x1fffffffu)), scalef);
    if (sign) lo = -lo;
    return fast_two_sum(hi, lo);
}

// float -> binary64 by bit widening
// (subnormal, infinite and NaN inputs out of line, as for split_bits; zero stays inline)
static __device__ __noinline__ double widen_slow(float f) { return (double)f; }
EXPM_D double widen_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned ex = (u >> 23) & 0xff, man = u & 0x7fffffu;
    if (__builtin_expect(ex == 0xff || (ex == 0 && man != 0), 0)) return widen_slow(f);
    const unsigned long long e64 = ex == 0 ? 0ull : (unsigned long long)(ex - 127 + 1023);  // +-0 stays +-0
    const unsigned long long b = ((unsigned long long)(u >> 31) << 63) | (e64 << 52) | ((unsigned long long)man << 29);
    return __longlong_as_double((long long)b);
}

// c + a*b in float-float: error-free product of the high parts, the cross terms,
// then one two-sum with c and a renormalisation (the "sloppy" double-word add).
EXPM_D f32x2 dd_fma(f32x2 a, f32x2 b, f32x2 c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const f32x2 s = two_sum(p, c.hi);
    const float t = __fadd_rn(s.lo, __fadd_rn(e, c.lo));
    return fast_two_sum(s.hi, t);
}

// ------------------------------------------------------------------ traits
template <class R> struct RealOps;
template <> struct RealOps<double> {
    static EXPM_D double from(double x) { return x; }
    static EXPM_D double todbl(double x) { return x; }
    static EXPM_D double zero() { return 0.0; }
    static EXPM_D double rcp(double x) { return __drcp_rn(x); }
};
template <> struct RealOps<float> {
    static EXPM_D float from(double x) { return (float)x; }
    static EXPM_D double todbl(float x) { return (double)x; }
    static EXPM_D float zero() { return 0.f; }
    static EXPM_D float rcp(float x) { return __frcp_rn(x); }
};
template <> struct RealOps<f32x2> {  // conversions by integer operations (FP64 unit only to add)
    static EXPM_D f32x2 from(double x) { return split_bits(x); }
    static EXPM_D double todbl(f32x2 x) { return widen_bits(x.hi) + widen_bits(x.lo); }
    static EXPM_D f32x2 zero() { return {0.f, 0.f}; }
    static EXPM_D f32x2 rcp(f32x2 x) { return recip(x); }
};

// ------------------------------------------------------------------ complex
template <class R> struct cx {
    R re, im;
};

template <class R> EXPM_D cx<R> cxz() { return {RealOps<R>::zero(), RealOps<R>::zero()}; }
template <class R> EXPM_D cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> EXPM_D cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> EXPM_D cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
template <class R> EXPM_D cx<R> operator*(cx<R> a, cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R> EXPM_D cx<R> scale(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <class R> EXPM_D cx<R> conj(cx<R> a) { return {a.re, -a.im}; }
// 1/w = conj(w)/|w|^2.  Inputs here are shifted matrix entries of moderate size
// (the public entry points reject non-finite data), so |w|^2 neither overflows
// nor underflows.
template <class R> EXPM_D cx<R> cinv(cx<R> w) {
    R n2 = w.re * w.re + w.im * w.im;
    R r = RealOps<R>::rcp(n2);
    return {w.re * r, -(w.im * r)};
}
// Re(a * b)
template <class R> EXPM_D R re_mul(cx<R> a, cx<R> b) { return a.re * b.re - a.im * b.im; }
// s - c*x (complex), and v - e*d for real v, e (the Thomas updates), written so
// that binary64 uses two FMAs per component.
template <class R> EXPM_D cx<R> csub_mul(cx<R> s, cx<R> c, cx<R> x) { return s - c * x; }
template <> EXPM_D cx<double> csub_mul<double>(cx<double> s, cx<double> c, cx<double> x) {
    return {fma(c.im, x.im, fma(-c.re, x.re, s.re)), fma(-c.im, x.re, fma(-c.re, x.im, s.im))};
}
template <class R> EXPM_D cx<R> real_minus_scaled(R v, R e, cx<R> d) { return {v - e * d.re, -(e * d.im)}; }
template <> EXPM_D cx<double> real_minus_scaled<double>(double v, double e, cx<double> d) {
    return {fma(-e, d.re, v), -e * d.im};
}

template <class R> EXPM_D cx<R> cx_from(double re, double im) {
    return {RealOps<R>::from(re), RealOps<R>::from(im)};
}
