"""Pins for oracle.scalar against the paper's statements (Secs. 2.3 and 4) -- CPU only."""

import math
from decimal import Decimal, localcontext

import numpy as np
import pytest

from oracle import coeffs, scalar


@pytest.mark.parametrize("n", [4, 8, 12, 16, 24, 32])
def test_partial_fractions_equal_rational(n):
    """Prop. 2.1: sum_k a_k/(x+theta_k) = 1/exp_n(-x); in binary64 the gap is
    e_3 and must stay under M_2(n, 16) of Prop. 4.1 on [-100, 0]."""
    th, a = coeffs.theta(n), coeffs.residues(n)
    x = np.linspace(-100.0, 0.0, 4001)
    _, _, e3 = scalar.e_split(x, n, th, a)
    assert np.max(np.abs(e3)) <= scalar.M2(n, 16, a)
    # and it is tiny at the degrees used on the GPU path (binary64 coefficients)
    if n <= 16:
        assert np.max(np.abs(e3)) < 1e-14


@pytest.mark.parametrize("n", [4, 8, 16, 32])
def test_truncation_error_positive_and_bounded(n):
    """Prop. 2.2 (|R_n(x) - e^x| <= 2^-n on x <= 0) and Prop. 2.3 (err_n > 0 on x < 0)."""
    x = -np.geomspace(1e-3, 60.0, 3000)
    err = scalar.err_n(x, n)
    assert np.all(err <= scalar.M1(n))
    # positivity is below binary64 resolution near 0 (err_n ~ -x^{n+1}/(n+1)!):
    # check it at 200 digits
    with localcontext() as ctx:
        ctx.prec = 200
        for xv in -np.geomspace(1e-3, 60.0, 120):
            xd = Decimal(repr(float(xv)))
            en = sum((-xd) ** k / Decimal(math.factorial(k)) for k in range(n + 1))
            assert Decimal(1) / en - xd.exp() > 0


@pytest.mark.parametrize("n", [4, 8, 12, 16, 20, 32])
def test_error_maximum_location(n):
    """Prop. 2.3, ineq. loc: err_n has one maximum xi_n with n/2 <= -xi_n <= n+2,
    increasing left of it and decreasing right of it."""
    x = np.linspace(-(3 * n + 10), -1e-6, 200001)
    err = scalar.err_n(x, n)
    i = int(np.argmax(err))
    xi = x[i]
    assert n / 2 <= -xi <= n + 2
    left, right = np.diff(err[: i + 1]), np.diff(err[i:])
    tiny = 1e-15  # binary64 noise of R_n(x) - e^x near x = 0
    assert np.all(left >= -tiny) and np.all(right <= tiny)


@pytest.mark.parametrize("n", [1, 2, 5, 10, 20, 40])
def test_lemma_inequalities(n):
    """Lemma 2.1: f_n(n+1) < 1/2 and f_n(x)^2 <= (n+1)/n f_{n-1}(x) f_{n+1}(x)."""
    assert scalar.f_n(n + 1.0, n) < 0.5
    if n >= 1:
        x = np.linspace(0.01, 3.0 * n + 5, 500)
        lhs = scalar.f_n(x, n) ** 2
        rhs = (n + 1) / n * scalar.f_n(x, n - 1) * scalar.f_n(x, n + 1)
        assert np.all(lhs <= rhs * (1 + 1e-12))


def _e_norms(n):
    th, a = coeffs.theta(n), coeffs.residues(n)
    x = np.linspace(-100.0, 0.0, 20001)
    e1, e2, e3 = scalar.e_split(x, n, th, a)
    return np.max(np.abs(e1)), np.max(np.abs(e2)), np.max(np.abs(e3))


def test_binary64_error_has_a_minimum_in_n():
    """Sec. 4, Fig. 4.1: in 16-digit arithmetic e_1 on [-100, 0] decreases until
    n is about 34 and then grows, because e_3 grows with n while e_2 decays.
    The n = 30 error is of order 1e-10 with a bound of order 1e-8 (Fig. 4.2)."""
    ns = list(range(16, 52, 2))
    e1 = np.array([_e_norms(n)[0] for n in ns])
    best = ns[int(np.argmin(e1))]
    assert 28 <= best <= 40
    e1_30, e2_30, e3_30 = _e_norms(30)
    assert 1e-12 < e1_30 < 1e-8
    th, a = coeffs.theta(30), coeffs.residues(30)
    assert scalar.M2(30, 16, a) < 1e-7 and e3_30 <= scalar.M2(30, 16, a)
    # e_3 grows with n (over the even degrees sampled, trend of the right panel)
    e3 = np.array([_e_norms(n)[2] for n in (12, 24, 36, 48)])
    assert np.all(np.diff(e3) > 0)


def test_R_n_at_zero_and_taylor():
    """R_n(0) = 1 and R_n agrees with exp to O(x^{n+1}) near 0 (eq. pade)."""
    for n in (2, 8, 16):
        assert scalar.R_n(0.0, n) == 1.0
        x = 1e-2
        # next Taylor term of R_n - exp is x^{n+2} lambda_{n,n+2}/(n+2)! - x^{n+2}/(n+2)!
        # (lambda_{n,n+1} = 0 cancels against nothing but e's own x^{n+1} term)
        diff = scalar.R_n(-x, n) - math.exp(-x)
        assert abs(diff) <= 2 * x ** (n + 1) / math.factorial(n + 1) + 1e-16
