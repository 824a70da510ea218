"""Pins for oracle.matrix against closed forms and the paper's matrix results (Sec. 3).

The oracle computes sum_k a_k (A + theta_k I)^{-1} V with one pivoted solve per
pole.  None of the references below uses partial fractions or linear solves of
shifted systems: they are eigen-decompositions with R_n evaluated by Horner,
the DST-I eigenbasis of the 1D Laplacian, the product form n!/prod(z+theta_k),
and exp itself with the paper's error bounds.
"""

import math

import numpy as np
import pytest

import workloads
from oracle import coeffs, matrix, scalar


def _coeffs(n):
    return coeffs.theta(n), coeffs.residues(n)


def test_diagonal_matrix_is_exact():
    """Remark 3.1: R_n(D) is diagonal with entries R_n(D_ii)."""
    n = 12
    th, a = _coeffs(n)
    dvals = np.linspace(-30.0, 0.0, 17)
    v = workloads.rng(100).standard_normal(17)
    Y, im = matrix.apply_dense(np.diag(dvals), v[:, None], th, a)
    np.testing.assert_allclose(Y[:, 0], scalar.R_n(dvals, n) * v, rtol=1e-13, atol=1e-15)
    assert im < 1e-13


def test_zero_matrix_gives_identity():
    """Remark 3.1: R_n(0) = I."""
    th, a = _coeffs(16)
    V = workloads.rng(101).standard_normal((9, 3))
    Y, _ = matrix.apply_dense(np.zeros((9, 9)), V, th, a)
    np.testing.assert_allclose(Y, V, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("n", [12, 16])
def test_dense_matches_eigen_closed_form(n, complex_):
    """Remark 3.1 (similarity): R_n(Q L Q^H) V = Q R_n(L) Q^H V with R_n by Horner."""
    g = workloads.rng(102 + n + complex_)
    A, Q, mu, V = workloads.dense_symmetric(48, -40.0, 0.0, 3, g, complex_)
    th, a = _coeffs(n)
    Y, im = matrix.apply_dense(A, V, th, a)
    ref = matrix.eig_apply(Q, mu, V, lambda m: scalar.R_n(m, n))
    assert matrix.rel_err(Y, ref) < 1e-13
    if not complex_:
        assert im < 1e-12 * np.abs(Y).max()


def test_dense_small_workload_matches_closed_form():
    """The 64x64 real symmetric workload (degree 12) against its eigen form."""
    w = workloads.dense_small()
    th, a = _coeffs(w["degree"])
    Y, _ = matrix.apply_dense(w["A"], w["V"], th, a)
    ref = matrix.eig_apply(w["Q"], w["mu"], w["V"], lambda m: scalar.R_n(m, 12))
    assert matrix.rel_err(Y, ref) < 1e-13


def test_product_form():
    """R_n(z) = n!/prod_k (z + theta_k) for even n: no residues involved."""
    n = 12
    th, a = _coeffs(n)
    g = workloads.rng(103)
    A, Q, mu, V = workloads.dense_symmetric(24, -20.0, 0.0, 1, g, True)
    Y, _ = matrix.apply_dense(A, V, th, a)
    P = matrix.product_apply(A, V[:, 0], th, n)
    assert matrix.rel_err(Y[:, 0], P) < 1e-12


@pytest.mark.parametrize("n", [12, 16, 24])
def test_against_exp_uniform_bound(n):
    """Eq. con with kappa_2(P) = 1 (normal A) and Prop. 2.2:
    ||exp(A)v - R_n(A)v|| <= 2^-n ||v|| for spectrum in (-inf, 0]."""
    th, a = _coeffs(n)
    g = workloads.rng(104 + n)
    A, Q, mu, V = workloads.dense_symmetric(40, -60.0, 0.0, 2, g, True)
    Y, _ = matrix.apply_dense(A, V, th, a)
    E = matrix.eig_apply(Q, mu, V, np.exp)
    for j in range(V.shape[1]):
        assert np.linalg.norm(Y[:, j] - E[:, j]) <= scalar.M1(n) * np.linalg.norm(V[:, j])


def test_theorem_negative_spectrum():
    """Theorem 3.1: if n > 2 rho(A) then ||exp(A) - R_n(A)||_2 <= R_n(-rho) - e^-rho."""
    n = 16
    th, a = _coeffs(n)
    g = workloads.rng(105)
    A, Q, mu, _ = workloads.dense_symmetric(30, -7.5, 0.0, 1, g, False)
    rho = float(np.max(np.abs(mu)))
    assert n > 2 * rho
    I = np.eye(30)
    Rn, _ = matrix.apply_dense(A, I, th, a)
    E = matrix.eig_apply(Q, mu, I, np.exp)
    assert np.linalg.norm(E - Rn, 2) <= (scalar.R_n(-rho, n) - math.exp(-rho)) * (1 + 1e-9) + 1e-14


def test_semigroup():
    """exp(2A) = exp(A)^2 carried over with Prop. 2.2 (R_n <= 1 on x <= 0):
    ||R_n(2A)v - R_n(A)R_n(A)v|| <= 3 2^-n ||v||."""
    n = 12
    th, a = _coeffs(n)
    g = workloads.rng(106)
    A, Q, mu, V = workloads.dense_symmetric(32, -25.0, 0.0, 1, g, True)
    Y2, _ = matrix.apply_dense(2 * A, V, th, a)
    Y1, _ = matrix.apply_dense(A, V, th, a)
    Y11, _ = matrix.apply_dense(A, Y1, th, a)
    assert np.linalg.norm(Y2 - Y11) <= 3 * scalar.M1(n) * np.linalg.norm(V)


def test_error_independent_of_dimension():
    """Sec. 5.2 (Fig. 5.1 left): with spectra in a fixed range [-1, 0] the
    absolute error against exp does not grow with d."""
    n = 8
    th, a = _coeffs(n)
    bound = float(np.max(scalar.err_n(np.linspace(-1, 0, 10001), n)))
    for d in (16, 64, 256):
        g = workloads.rng(107 + d)
        A, Q, mu, _ = workloads.dense_symmetric(d, -1.0, 0.0, 1, g, False)
        Rn, _ = matrix.apply_dense(A, np.eye(d), th, a)
        E = matrix.eig_apply(Q, mu, np.eye(d), np.exp)
        err = np.linalg.norm(E - Rn, 2)
        # normal A: the 2-norm error is exactly max_i err_n(mu_i), whatever d is
        assert abs(err - np.max(scalar.err_n(mu, n))) < 1e-13
        assert err <= bound * (1 + 1e-6) + 1e-15


def test_shift_method_positive_spectrum():
    """Remark 3.2: for spectrum in [0, 20], exp(A) ~ e^c R_n(A - cI) with c >= alpha(A),
    and the relative error is at most e^c/||exp(A)|| * 2^-n."""
    n = 16
    th, a = _coeffs(n)
    g = workloads.rng(108)
    A, Q, mu, V = workloads.dense_symmetric(36, 0.0, 20.0, 2, g, False)
    c = 20.0
    Y, _ = matrix.apply_dense(A, V, th, a, t=1.0, c=c)
    ref = matrix.eig_apply(Q, mu, V, lambda m: math.exp(c) * scalar.R_n(m - c, n))
    assert matrix.rel_err(Y, ref) < 1e-12
    E = matrix.eig_apply(Q, mu, V, np.exp)
    alpha = float(mu.max())
    bound = math.exp(c) / math.exp(alpha) * scalar.M1(n)
    assert matrix.rel_err(Y, E) <= bound


def test_time_scaling():
    """exp(tA)V: the t argument is R_n(tA)V."""
    th, a = _coeffs(12)
    g = workloads.rng(109)
    A, Q, mu, V = workloads.dense_symmetric(20, -10.0, 0.0, 1, g, True)
    Y1, _ = matrix.apply_dense(A, V, th, a, t=0.37)
    Y2, _ = matrix.apply_dense(0.37 * A, V, th, a)
    assert matrix.rel_err(Y1, Y2) < 1e-13


@pytest.mark.parametrize("N", [1, 2, 3, 50, 1000])
def test_tridiag_laplacian_matches_dst_closed_form(N):
    """1D Laplacian T = c tridiag(1,-2,1) (Sec. 5): the banded per-pole solves
    equal the DST-I eigen closed form of R_n."""
    w = workloads.laplacian_1d(N=N, nrhs=3, offset=110)
    n = 16
    th, a = _coeffs(n)
    Y, im = matrix.apply_tridiag(w["d"], w["e"], w["V"], th, a)
    ref = matrix.laplacian_apply(w["d0"], w["e0"], w["V"], lambda m: scalar.R_n(m, n))
    # relative 1e-12, plus the absolute rounding floor of the partial-fraction
    # sum (Prop. 4.1: |e_3| <= M_2(n, 16) per eigencomponent, normal T); the
    # floor matters only when R_n(T)V is tiny (N <= 3: spectrum near -200..-400)
    err = np.linalg.norm(Y - ref)
    assert err <= 1e-12 * np.linalg.norm(ref) + scalar.M2(n, 16, a) * np.linalg.norm(w["V"])
    if N >= 50:
        assert matrix.rel_err(Y, ref) < 1e-12
    assert im <= scalar.M2(n, 16, a) * np.abs(w["V"]).max()


@pytest.mark.parametrize("complex_e", [False, True])
def test_tridiag_general_matches_dense(complex_e):
    """Non-constant Hermitian tridiagonal: banded and dense oracle solves agree
    (the banded path's lower diagonal must be conj(e))."""
    g = workloads.rng(111 + complex_e)
    N = 40
    d = g.uniform(-30.0, -1.0, N)
    e = g.uniform(0.5, 5.0, N - 1) * (np.exp(1j * g.uniform(0, 6.28, N - 1)) if complex_e else 1.0)
    V = g.standard_normal((N, 2)) + (1j * g.standard_normal((N, 2)) if complex_e else 0.0)
    th, a = _coeffs(12)
    Yt, _ = matrix.apply_tridiag(d, e, V, th, a)
    T = matrix.tridiag_to_dense(d, e)
    Yd, _ = matrix.apply_dense(T, V, th, a)
    assert matrix.rel_err(Yt, Yd) < 1e-13
    mu, Q = np.linalg.eigh(T)
    ref = matrix.eig_apply(Q, mu, V, lambda m: scalar.R_n(m, 12))
    assert matrix.rel_err(Yt, ref) < 1e-12


def test_tridiag_diagonal_unitary_gauge():
    """The identity behind the complex-off-diagonal reading (Sec. 3, A Hermitian): for a
    diagonal unitary D0 = diag(exp(i psi)), T = D0 T~ D0^H has off-diagonal
    e_i = |e_i| exp(i (psi_i - psi_{i+1})) and every resolvent, hence e^c R_n(tT - cI)V,
    equals D0 [e^c R_n(tT~ - cI)] (D0^H V).  The oracle solves both sides directly (complex
    banded systems against real ones), so a dropped conjugate on the lower diagonal or a
    swapped phase fails here."""
    g = workloads.rng(113)
    N = 257
    d = g.uniform(-12.0, -4.0, N)
    eabs = g.uniform(0.5, 2.0, N - 1)
    psi = g.uniform(0.0, 2 * np.pi, N)
    ph = np.exp(1j * psi)
    e = eabs * ph[:-1] * np.conj(ph[1:])
    V = g.standard_normal((N, 3)) + 1j * g.standard_normal((N, 3))
    th, a = _coeffs(16)
    Y, _ = matrix.apply_tridiag(d, e, V, th, a, t=0.8, c=0.5)
    Yr, _ = matrix.apply_tridiag(d, eabs, np.conj(ph)[:, None] * V, th, a, t=0.8, c=0.5)
    assert matrix.rel_err(Y, ph[:, None] * Yr) < 1e-13
    # the gauge is not a symmetry of the wrong (conjugate-free) banded matrix
    Yw, _ = matrix.apply_dense(np.diag(d) + np.diag(e, 1) + np.diag(e, -1), V, th, a, t=0.8, c=0.5)
    assert matrix.rel_err(Yw, Y) > 1e-3


@pytest.mark.parametrize("dx,dy", [(1, 1), (5, 7), (12, 9)])
def test_laplacian2d_closed_form(dx, dy):
    """2D separable operator (Sec. 5): the DST-I closed form reproduces A V itself (f = id:
    pins the eigenvalue order and both transforms) and equals the per-pole dense solves
    on the assembled matrix for f = R_n."""
    g = workloads.rng(113 + dx)
    ax, bx, ay, by = 30.0, -70.0, 25.0, -55.0
    A = matrix.laplacian2d_matrix(dx, dy, ax, bx, ay, by)
    V = g.standard_normal((dx * dy, 3))
    AV = matrix.laplacian2d_apply(dx, dy, ax, bx, ay, by, V, lambda m: m)
    assert np.allclose(AV, A @ V, rtol=1e-12, atol=1e-12 * np.abs(A @ V).max())
    n = 12
    th, a = _coeffs(n)
    Yd, im = matrix.apply_dense(A, V, th, a)
    ref = matrix.laplacian2d_apply(dx, dy, ax, bx, ay, by, V, lambda m: scalar.R_n(m, n))
    assert np.linalg.norm(Yd - ref) <= 1e-12 * np.linalg.norm(ref) + scalar.M2(n, 16, a) * np.linalg.norm(V)
    # a transposed grid (dx <-> dy, with the coefficients) is the same operator up to the
    # permutation of the unknowns
    P = np.arange(dx * dy).reshape(dy, dx).T.reshape(-1)
    ref_t = matrix.laplacian2d_apply(dy, dx, ay, by, ax, bx, V[P], lambda m: scalar.R_n(m, n))
    assert np.allclose(ref_t, ref[P], rtol=1e-12, atol=1e-14)


def test_threaded_solves_are_identical():
    """The thread pool changes nothing: the sum is always taken in pole order."""
    w = workloads.laplacian_1d(N=3000, nrhs=2, offset=112)
    th, a = _coeffs(16)
    Y1, _ = matrix.apply_tridiag(w["d"], w["e"], w["V"], th, a, workers=1)
    Y4, _ = matrix.apply_tridiag(w["d"], w["e"], w["V"], th, a, workers=4)
    np.testing.assert_array_equal(Y1, Y4)


def test_planted_mistakes_are_caught():
    """Mistakes planted on the CPU side are visible to the eigen pin:
    a transposed complex operand, a dropped pole, a flipped pole sign."""
    n = 12
    th, a = _coeffs(n)
    g = workloads.rng(113)
    A, Q, mu, V = workloads.dense_symmetric(30, -20.0, 0.0, 1, g, True)
    ref = matrix.eig_apply(Q, mu, V, lambda m: scalar.R_n(m, n))
    Yt, _ = matrix.apply_dense(A.T, V, th, a)                # transposed operand
    assert matrix.rel_err(Yt, ref) > 1e-3
    Yd, _ = matrix.apply_dense(A, V, th[1:], a[1:])          # dropped pole
    assert matrix.rel_err(Yd, ref) > 1e-3
    Ys, _ = matrix.apply_dense(A, V, -th, a)                 # wrong pole sign
    assert matrix.rel_err(Ys, ref) > 1e-3
