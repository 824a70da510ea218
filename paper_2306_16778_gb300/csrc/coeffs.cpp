// coeffs.cpp -- poles and weights of R_n(z) = 1/exp_n(-z) in double-double arithmetic.
//
// Sec. 2.1: theta_k are the n simple roots of exp_n(z) = sum_{k<=n} z^k/k!
// (conjugate pairs, none real, for even n).  Prop. 2.1 eq. yoyo2:
//     a_k = -n! / prod_{j != k} (theta_k - theta_j).
// The roots are found with the Aberth-Ehrlich simultaneous iteration (Aberth 1973,
// Ehrlich 1967) in double-double arithmetic (Dekker 1971; Knuth TAOCP vol. 2) and
// polished with two Newton steps; the residues use the product formula, which the
// paper found the most accurate of its three formulas (Sec. 4).  Everything is
// rounded once to binary64 at the end (the Fig. 4.1 caption: values computed with
// >= 32 digits, then truncated to 16).
//
// Host-only code: no CUDA calls.
#include <cmath>
#include <algorithm>
#include <vector>

#include "../../include/expm.h"

namespace {

struct dd {
    double hi, lo;
};

inline dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double err = (a - (s - bb)) + (b - bb);
    return {s, err};
}
inline dd quick_two_sum(double a, double b) {
    double s = a + b;
    return {s, b - (s - a)};
}
inline dd two_prod(double a, double b) {
    double p = a * b;
    return {p, std::fma(a, b, -p)};
}
inline dd operator+(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
inline dd operator-(dd a) { return {-a.hi, -a.lo}; }
inline dd operator-(dd a, dd b) { return a + (-b); }
inline dd operator*(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}
inline dd operator/(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = a - b * dd{q1, 0.0};
    double q2 = r.hi / b.hi;
    r = r - b * dd{q2, 0.0};
    double q3 = r.hi / b.hi;
    dd q = quick_two_sum(q1, q2);
    return q + dd{q3, 0.0};
}
inline dd ddv(double x) { return {x, 0.0}; }

struct cdd {
    dd re, im;
};
inline cdd operator+(cdd a, cdd b) { return {a.re + b.re, a.im + b.im}; }
inline cdd operator-(cdd a, cdd b) { return {a.re - b.re, a.im - b.im}; }
inline cdd operator*(cdd a, cdd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline cdd operator/(cdd a, cdd b) {
    dd den = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den};
}
inline double cabs_d(cdd a) { return std::hypot(a.re.hi, a.im.hi); }

// p(z) = exp_n(z) and p'(z) = exp_{n-1}(z) by Horner
void eval(const std::vector<dd> &c, int n, cdd z, cdd &p, cdd &dp) {
    p = {c[n], ddv(0)};
    for (int k = n - 1; k >= 0; --k) p = p * z + cdd{c[k], ddv(0)};
    dp = {c[n - 1], ddv(0)};
    for (int k = n - 2; k >= 0; --k) dp = dp * z + cdd{c[k], ddv(0)};
}

}  // namespace

extern "C" expm_status expm_coeffs(int degree, double *poles_ri, double *residues_ri) {
    const int n = degree;
    if (n < 2 || n > 64 || (n & 1) || !poles_ri || !residues_ri) return EXPM_EINVAL;
    std::vector<dd> c(n + 1);
    c[0] = ddv(1.0);
    for (int k = 1; k <= n; ++k) c[k] = c[k - 1] / ddv((double)k);  // 1/k!

    // Aberth-Ehrlich from a circle inside the bound |theta| <= n (eq. racn),
    // rotated so that no starting point is real.
    std::vector<cdd> z(n);
    const double r0 = 0.5 * n;
    for (int k = 0; k < n; ++k) {
        double ang = 2.0 * M_PI * (k + 0.25) / n + 0.3;
        z[k] = {ddv(r0 * std::cos(ang)), ddv(r0 * std::sin(ang))};
    }
    bool converged = false;
    int quiet = 0;
    for (int it = 0; it < 400 && !converged; ++it) {
        double worst = 0.0;
        for (int k = 0; k < n; ++k) {
            cdd p, dp;
            eval(c, n, z[k], p, dp);
            cdd ratio = p / dp;
            cdd s = {ddv(0), ddv(0)};
            for (int j = 0; j < n; ++j)
                if (j != k) s = s + cdd{ddv(1), ddv(0)} / (z[k] - z[j]);
            cdd den = cdd{ddv(1), ddv(0)} - ratio * s;
            cdd w = ratio / den;
            z[k] = z[k] - w;
            worst = std::max(worst, cabs_d(w) / std::max(1.0, cabs_d(z[k])));
        }
        // converged when the corrections reach the double-double rounding level,
        // or (large n, where evaluating exp_n near its roots cancels more digits)
        // stay far below binary64 resolution for several sweeps
        quiet = (worst < 2e-18) ? quiet + 1 : 0;
        if (worst < 1e-27 || quiet >= 5) converged = true;
    }
    if (!converged) return EXPM_EINVAL;
    for (int k = 0; k < n; ++k)  // Newton polish
        for (int it = 0; it < 2; ++it) {
            cdd p, dp;
            eval(c, n, z[k], p, dp);
            z[k] = z[k] - p / dp;
        }

    // canonical order: Im > 0 members sorted by Re ascending, each followed by
    // its conjugate (exact conjugate symmetry: exp_n has real coefficients)
    std::vector<cdd> up;
    for (auto &w : z)
        if (w.im.hi > 0) up.push_back(w);
    if ((int)up.size() != n / 2) return EXPM_EINVAL;
    std::sort(up.begin(), up.end(), [](const cdd &a, const cdd &b) {
        return a.re.hi < b.re.hi || (a.re.hi == b.re.hi && a.re.lo < b.re.lo);
    });
    std::vector<cdd> th(n);
    for (int l = 0; l < n / 2; ++l) {
        th[2 * l] = up[l];
        th[2 * l + 1] = {up[l].re, -up[l].im};
    }
    dd nfact = ddv(1.0);
    for (int k = 2; k <= n; ++k) nfact = nfact * ddv((double)k);
    for (int k = 0; k < n; ++k) {
        cdd prod = {ddv(1), ddv(0)};
        for (int j = 0; j < n; ++j)
            if (j != k) prod = prod * (th[k] - th[j]);
        cdd a = cdd{-nfact, ddv(0)} / prod;
        if (k & 1) {  // exact conjugate of the partner's residue
            a.re = {residues_ri[2 * (k - 1)], 0.0};
            a.im = {-residues_ri[2 * (k - 1) + 1], 0.0};
        }
        poles_ri[2 * k] = -th[k].re.hi;  // lambda_k = -theta_k
        poles_ri[2 * k + 1] = -th[k].im.hi;
        residues_ri[2 * k] = a.re.hi;
        residues_ri[2 * k + 1] = a.im.hi;
    }
    return EXPM_OK;
}
