"""Pins for oracle.coeffs against what the paper fixes (Sec. 2) -- CPU only.

Each test checks a property that a plausible mistake in the root finder or the
residue formula would break: a wrong sign of theta, a conjugated residue, a
dropped factor in the product of eq. yoyo2, a transposed pair ordering.
"""

import math
import os
from decimal import Decimal, localcontext

import numpy as np
import pytest

from oracle import coeffs
from oracle.coeffs import DC

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EVEN = [2, 4, 6, 8, 10, 12, 14, 16, 20, 24, 32, 40]


def test_n2_worked_example():
    """exp_2 worked by hand (golden file cites the derivation)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "coeffs_n2.txt"))
    th = coeffs.theta(2)
    a = coeffs.residues(2)
    np.testing.assert_allclose(th.real, rows[:, 1], atol=1e-15)
    np.testing.assert_allclose(th.imag, rows[:, 2], atol=1e-15)
    np.testing.assert_allclose(a.real, rows[:, 3], atol=1e-15)
    np.testing.assert_allclose(a.imag, rows[:, 4], atol=1e-15)


@pytest.mark.parametrize("n", EVEN)
def test_roots_are_roots_and_paired(n):
    """Sec. 2.1: even n gives n/2 conjugate pairs, none real; each value is a root."""
    th = coeffs.roots_decimal(n)
    assert len(th) == n
    for k in range(0, n, 2):
        assert th[k].im > 0
        assert th[k + 1].re == th[k].re and th[k + 1].im == th[k].im.copy_negate()
    with localcontext() as ctx:
        ctx.prec = 60
        for t in th:
            v = coeffs.exp_n_decimal(t, n)
            # |exp_n(theta)| must be far below the size of its largest term
            big = max(Decimal(t.abs()) ** k / math.factorial(k) for k in range(n + 1))
            assert v.abs() < big * Decimal("1e-30")


@pytest.mark.parametrize("n", EVEN)
def test_root_modulus_bounds(n):
    """eq. racn: 1 <= |theta_k| <= n."""
    r = np.abs(coeffs.theta(n))
    assert np.all(r >= 1.0) and np.all(r <= n)


@pytest.mark.parametrize("n", EVEN)
def test_root_separation(n):
    """eq. ecart: min_{j != k} |theta_j - theta_k| >= gamma = 0.29044..."""
    th = coeffs.theta(n)
    dif = np.abs(th[:, None] - th[None, :]) + np.eye(n) * 1e9
    assert dif.min() >= 0.29044


@pytest.mark.parametrize("n", EVEN)
def test_parabola_root_free(n):
    """Saff-Varga (Sec. 2.1): no root inside the parabola y^2 = 4(x + 1)."""
    th = coeffs.theta(n)
    assert np.all(th.imag ** 2 >= 4 * (th.real + 1) - 1e-12)


@pytest.mark.parametrize("n", EVEN)
def test_moments_at_infinity(n):
    """R_n(z) = n!/prod(z + theta_k) (Sec. 2.2 with Prop. 2.1) forces
    sum_k a_k theta_k^m = 0 for m <= n-2 and sum_k a_k theta_k^(n-1) = -n!."""
    th = coeffs.roots_decimal(n)
    a = coeffs.residues_decimal(n)
    with localcontext() as ctx:
        ctx.prec = coeffs._digits(n)
        tol = Decimal(10) ** (-(coeffs._digits(n) - 20))
        for m in range(n):
            s = DC(Decimal(0))
            for tk, ak in zip(th, a):
                p = DC(Decimal(1))
                for _ in range(m):
                    p = p * tk
                s = s + ak * p
            target = Decimal(-math.factorial(n)) if m == n - 1 else Decimal(0)
            scale = max(Decimal(1), abs(target))
            assert (s - target).abs() < tol * scale * Decimal(math.factorial(n)), (n, m)


@pytest.mark.parametrize("n", EVEN)
def test_taylor_derivatives_at_zero(n):
    """eq. pade and the refinement after it: R_n^(j)(0) = 1 for j <= n,
    lambda_{n,n+1} = 0 and lambda_{n,n+2} = -2(n+1), where
    R_n^(j)(0) = (-1)^j j! sum_k a_k theta_k^-(j+1)."""
    th = coeffs.roots_decimal(n)
    a = coeffs.residues_decimal(n)
    with localcontext() as ctx:
        ctx.prec = coeffs._digits(n)
        tol = Decimal(10) ** (-(coeffs._digits(n) - 25))
        inv = [DC(Decimal(1)) / t for t in th]
        for j in range(n + 3):
            s = DC(Decimal(0))
            for ik, ak in zip(inv, a):
                p = DC(Decimal(1))
                for _ in range(j + 1):
                    p = p * ik
                s = s + ak * p
            val = s * Decimal((-1) ** j * math.factorial(j))
            target = Decimal(1) if j <= n else (Decimal(0) if j == n + 1 else Decimal(-2 * (n + 1)))
            assert (val - target).abs() < tol * Decimal(math.factorial(j) + 1), (n, j)


@pytest.mark.parametrize("n", [4, 12, 16, 24])
def test_three_residue_formulas_agree(n):
    """eq. yoyo2 and both forms of eq. yoyo234 agree in exact arithmetic."""
    a = coeffs.residues_decimal(n)
    b = coeffs.residues_alt_derivative(n)
    c = coeffs.residues_alt_power(n)
    with localcontext() as ctx:
        ctx.prec = 50
        for x, y, z in zip(a, b, c):
            assert (x - y).abs() <= x.abs() * Decimal("1e-25")
            assert (x - z).abs() <= x.abs() * Decimal("1e-25")


@pytest.mark.parametrize("n", [12, 16, 32])
def test_roots_match_independent_multiprecision(n):
    """Independent check: mpmath's polynomial root finder at 50 digits."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    cs = [mpmath.mpf(1) / mpmath.factorial(k) for k in range(n, -1, -1)]
    ref = sorted((complex(r) for r in mpmath.polyroots(cs, maxsteps=200, extraprec=200)),
                 key=lambda w: (round(w.real, 9), -w.imag))
    got = sorted(coeffs.theta(n), key=lambda w: (round(w.real, 9), -w.imag))
    np.testing.assert_allclose(np.array(got), np.array(ref), rtol=0, atol=1e-14)


def test_abi_arrays_convention():
    """Library convention: poles lambda_k = -theta_k, weights w_k = a_k, interleaved."""
    p, r = coeffs.abi_arrays(12)
    th = coeffs.theta(12)
    a = coeffs.residues(12)
    np.testing.assert_array_equal(p[0::2] + 1j * p[1::2], -th)
    np.testing.assert_array_equal(r[0::2] + 1j * r[1::2], a)


def test_planted_mistakes_are_caught(monkeypatch):
    """A conjugated residue or a dropped factor in eq. yoyo2 breaks R_n(0) = 1."""
    th = coeffs.theta(12)
    a = coeffs.residues(12)
    assert abs(np.sum(a / th) - 1) < 1e-13
    bad = a.copy()
    bad[0] = np.conj(bad[0])                      # conjugated residue
    assert abs(np.sum(bad / th) - 1) > 1e-3
    bad = a * (th - th[::-1])                     # spurious extra factor
    assert abs(np.sum(bad / th) - 1) > 1e-3
    assert abs(np.sum(a / (-th)) - 1) > 1e-3      # pole sign flipped
