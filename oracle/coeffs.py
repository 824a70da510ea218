"""Oracle coefficients: roots theta_k of exp_n and residues a_k (Sec. 2).

Test infrastructure only (see the package docstring).

What is computed
----------------
* exp_n(z) = sum_{k=0..n} z^k / k!   (Sec. 2, definition of exp_n).
* theta_k, k = 1..n, the n simple roots of exp_n (Sec. 2.1).  For even n they
  come in conjugate pairs and none is real.
* a_k = -n! / prod_{j != k} (theta_k - theta_j)   (Prop. 2.1, eq. yoyo2), the
  formula the paper keeps after comparing it with eq. yoyo234 (Sec. 4).
* the two alternative formulas of eq. yoyo234, a_k = -1/exp_n'(theta_k) and
  a_k = n!/theta_k^n, for cross-checks only.

How
---
Everything is done in Python ``decimal`` arithmetic with a working precision of
at least 40 significant digits (more for large n), then rounded once to binary64.
The paper's Fig. 4.1 caption uses coefficients computed with 32 significant
digits and truncated to 16; rounding a >= 40-digit value to binary64 is that
recipe with round-to-nearest in place of truncation (the caption's "truncated" is
read as "rounded to 16 digits": truncation would bias every coefficient downward).

Root finding: the Weierstrass (Durand-Kerner) simultaneous iteration
    z_i <- z_i - q(z_i) / prod_{j != i} (z_i - z_j)
on the monic polynomial q(z) = n! exp_n(z) = sum_k (n!/k!) z^k, started from
the binary64 eigenvalues of its companion matrix (``numpy.roots``, a library
step used only as a starting guess).  Convergence is declared when every
update is below 10^-(digits-8) relative; the result is then checked for
|q(z)| small and pairwise distinctness.

Ordering (reading of Remark 5.1, which only asks that conjugates be adjacent):
pairs sorted by Re(theta) ascending; within a pair the member with Im > 0 first.
"""

from __future__ import annotations

import functools
import math
from decimal import Decimal, localcontext

import numpy as np


class DC:
    """Minimal complex number over ``decimal.Decimal`` (re, im)."""

    __slots__ = ("re", "im")

    def __init__(self, re, im=Decimal(0)):
        self.re = re if isinstance(re, Decimal) else Decimal(re)
        self.im = im if isinstance(im, Decimal) else Decimal(im)

    def __add__(self, o):
        if isinstance(o, DC):
            return DC(self.re + o.re, self.im + o.im)
        return DC(self.re + o, self.im)

    __radd__ = __add__

    def __sub__(self, o):
        if isinstance(o, DC):
            return DC(self.re - o.re, self.im - o.im)
        return DC(self.re - o, self.im)

    def __neg__(self):
        return DC(self.re.copy_negate(), self.im.copy_negate())

    def __mul__(self, o):
        if isinstance(o, DC):
            return DC(self.re * o.re - self.im * o.im, self.re * o.im + self.im * o.re)
        return DC(self.re * o, self.im * o)

    __rmul__ = __mul__

    def __truediv__(self, o):
        if isinstance(o, DC):
            den = o.re * o.re + o.im * o.im
            return DC((self.re * o.re + self.im * o.im) / den,
                      (self.im * o.re - self.re * o.im) / den)
        return DC(self.re / o, self.im / o)

    def conj(self):
        return DC(self.re, self.im.copy_negate())

    def abs2(self):
        return self.re * self.re + self.im * self.im

    def abs(self):
        return self.abs2().sqrt()

    def to_complex(self) -> complex:
        return complex(float(self.re), float(self.im))


def _digits(n: int) -> int:
    """Working precision (significant digits) used for degree n."""
    return max(40, 30 + 2 * n)


def _monic_coeffs(n: int) -> list[Decimal]:
    """q(z) = n! exp_n(z) = sum_k c_k z^k with c_k = n!/k!, c_n = 1 (exact integers)."""
    return [Decimal(math.factorial(n) // math.factorial(k)) for k in range(n + 1)]


def _horner(c: list[Decimal], z: DC) -> DC:
    acc = DC(c[-1])
    for ck in reversed(c[:-1]):
        acc = acc * z + ck
    return acc


def exp_n_decimal(z: DC, n: int) -> DC:
    """exp_n(z) = sum_{k<=n} z^k/k! in the current decimal context (definition, Sec. 2)."""
    acc = DC(Decimal(1) / Decimal(math.factorial(n)))
    for k in range(n - 1, -1, -1):
        acc = acc * z + Decimal(1) / Decimal(math.factorial(k))
    return acc


@functools.lru_cache(maxsize=None)
def roots_decimal(n: int) -> tuple:
    """The n roots theta_k of exp_n as ``DC`` values at ``_digits(n)`` digits.

    Sec. 2.1: exp_n has n simple roots; for even n they are conjugate pairs.
    Returned in the canonical order (pairs by Re ascending, Im > 0 first).
    """
    if n < 1:
        raise ValueError("degree must be >= 1")
    digits = _digits(n)
    with localcontext() as ctx:
        ctx.prec = digits + 10
        c = _monic_coeffs(n)
        # starting guess: binary64 companion eigenvalues (numpy.roots wants the
        # highest power first); nudged off the real axis so that no two
        # starting points coincide.
        start = np.roots([float(x) for x in reversed(c)])
        z = [DC(Decimal(repr(float(s.real))) + Decimal(k) * Decimal("1e-9"),
                Decimal(repr(float(s.imag))) + Decimal("3e-9"))
             for k, s in enumerate(start)]
        tol = Decimal(10) ** (-(digits - 8))
        for _ in range(500):
            biggest = Decimal(0)
            newz = []
            for i, zi in enumerate(z):
                den = DC(Decimal(1))
                for j, zj in enumerate(z):
                    if j != i:
                        den = den * (zi - zj)
                step = _horner(c, zi) / den
                newz.append(zi - step)
                rel = (step.abs2() / max(zi.abs2(), Decimal(1))).sqrt()
                biggest = max(biggest, rel)
            z = newz
            if biggest < tol:
                break
        else:
            raise RuntimeError(f"Durand-Kerner did not converge for n={n}")
        # canonical order and exact conjugate symmetry (exp_n has real
        # coefficients, so roots come in exact conjugate pairs)
        z.sort(key=lambda w: (float(w.re), -float(w.im)))
        if n % 2 == 0:
            upper = [w for w in z if w.im > 0]
            if len(upper) != n // 2:
                raise RuntimeError("even degree must give n/2 roots with Im > 0")
            upper.sort(key=lambda w: float(w.re))
            out = []
            for w in upper:
                out.append(w)
                out.append(w.conj())
        else:
            reals = [w for w in z if abs(w.im) < tol * 100]
            if len(reals) != 1:
                raise RuntimeError("odd degree must give exactly one real root")
            r = DC(reals[0].re, Decimal(0))
            upper = sorted((w for w in z if w.im > tol * 100), key=lambda w: float(w.re))
            out = [r]
            for w in upper:
                out.append(w)
                out.append(w.conj())
        # residual check: |exp_n(theta)| tiny relative to the size of its terms
        for w in out:
            val = _horner(c, w).abs()
            scale = sum(ck * (w.abs() ** k) for k, ck in enumerate(c))
            if val > scale * Decimal(10) ** (-(digits - 12)):
                raise RuntimeError(f"root check failed for n={n}")
    return tuple(out)


@functools.lru_cache(maxsize=None)
def residues_decimal(n: int) -> tuple:
    """a_k = -n!/prod_{j != k}(theta_k - theta_j)  (Prop. 2.1, eq. yoyo2)."""
    th = roots_decimal(n)
    with localcontext() as ctx:
        ctx.prec = _digits(n) + 10
        nf = Decimal(math.factorial(n))
        out = []
        for k, tk in enumerate(th):
            den = DC(Decimal(1))
            for j, tj in enumerate(th):
                if j != k:
                    den = den * (tk - tj)
            out.append(DC(-nf) / den)
    return tuple(out)


def residues_alt_derivative(n: int) -> tuple:
    """a_k = -1/exp_n'(theta_k) with exp_n' = exp_{n-1} (eq. yoyo234, first form)."""
    th = roots_decimal(n)
    with localcontext() as ctx:
        ctx.prec = _digits(n) + 10
        return tuple(DC(Decimal(-1)) / exp_n_decimal(t, n - 1) for t in th)


def residues_alt_power(n: int) -> tuple:
    """a_k = n!/theta_k^n (eq. yoyo234, second form)."""
    th = roots_decimal(n)
    with localcontext() as ctx:
        ctx.prec = _digits(n) + 10
        out = []
        for t in th:
            p = DC(Decimal(1))
            for _ in range(n):
                p = p * t
            out.append(DC(Decimal(math.factorial(n))) / p)
        return tuple(out)


def theta(n: int) -> np.ndarray:
    """Roots theta_k of exp_n rounded once to binary64 (complex128, canonical order)."""
    return np.array([w.to_complex() for w in roots_decimal(n)], dtype=np.complex128)


def residues(n: int) -> np.ndarray:
    """Residues a_k (eq. yoyo2) rounded once to binary64 (complex128, canonical order)."""
    return np.array([w.to_complex() for w in residues_decimal(n)], dtype=np.complex128)


def abi_arrays(n: int) -> tuple[np.ndarray, np.ndarray]:
    """(poles_ri, residues_ri) in the library's convention: lambda_k = -theta_k,
    w_k = a_k, each as 2n float64 values interleaved (re, im)."""
    lam = -theta(n)
    a = residues(n)
    p = np.empty(2 * n)
    p[0::2], p[1::2] = lam.real, lam.imag
    r = np.empty(2 * n)
    r[0::2], r[1::2] = a.real, a.imag
    return p, r
