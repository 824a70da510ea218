"""Oracle matrix functions (Sec. 3).  Test infrastructure only.

The exact result of the method is

    Y* = e^c R_n(tA - cI) V = e^c sum_k a_k (tA - cI + theta_k I)^{-1} V

(eq. ExpoMatRat with the shift of Remark 3.2; eq. expAx for a block of vectors).
``apply_dense`` and ``apply_tridiag`` compute it by its plain definition: one
direct solve per pole for ALL n poles (no conjugate-pair halving, so nothing
here shares the GPU path's pairing), then the residue-weighted sum in pole
order, accumulated in numpy ``longdouble``.  The solves are LAPACK's pivoted
LU (``numpy.linalg.solve`` = ?gesv, ``scipy.linalg.solve_banded`` = ?gbsv),
used as library steps.  For real A and real V the result is real
(Remark 5.1); ``Y.imag`` is then returned separately as a check.

Closed forms used to pin the above (none goes through partial fractions):
* ``eig_apply``:  f(Q diag(mu) Q^H) V = Q diag(f(mu)) Q^H V for unitary Q
  (Remark 3.1: R_n(P A P^-1) = P R_n(A) P^-1 and R_n(D) = diag(R_n(D_ii))).
* ``laplacian_apply``: the same with the DST-I eigenbasis of the constant
  tridiagonal matrix tridiag(e0, d0, e0) (eigenvalues d0 + 2 e0 cos(j pi/(N+1))).
* ``laplacian2d_apply``: the same for the separable 2D operator I (x) T_x + T_y (x) I
  (the DST-I along both axes).
* ``product_apply``: R_n(A) v = n! prod_k (A + theta_k I)^{-1} v, which
  follows from R_n(z) = 1/exp_n(-z) = n!/prod_k (z + theta_k) for even n.

``workers`` runs the per-pole solves on a thread pool (the paper's own
decomposition, one solve per processor, Sec. 5); LAPACK releases the GIL.
The sum is always taken in pole order, so the result does not depend on it.
"""

from __future__ import annotations

import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import scipy.fft
import scipy.linalg


def _is_real(*xs) -> bool:
    return all(not np.iscomplexobj(x) for x in xs)


def _pool_map(fn, items, workers: int):
    if workers <= 1:
        return [fn(x) for x in items]
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(fn, items))


def _weighted_sum(X: list, a: np.ndarray, shape) -> np.ndarray:
    acc = np.zeros(shape, dtype=np.clongdouble)
    for ak, xk in zip(a, X):
        acc += np.clongdouble(ak) * xk.astype(np.clongdouble)
    return acc


def shifted_solves_dense(A, V, theta, t=1.0, c=0.0, workers=1):
    """X_k = (tA - cI + theta_k I)^{-1} V for every k (dense, pivoted LU)."""
    A = np.asarray(A)
    n = A.shape[0]
    M0 = (t * A).astype(np.complex128)
    V = np.asarray(V, dtype=np.complex128)

    def one(tk):
        M = M0.copy()
        M[np.diag_indices(n)] += (tk - c)
        return np.linalg.solve(M, V)

    return _pool_map(one, list(theta), workers)


def apply_dense(A, V, theta, a, t=1.0, c=0.0, workers=1):
    """Y* = e^c sum_k a_k (tA - cI + theta_k I)^{-1} V  (eqs. ExpoMatRat, expAx).

    Returns (Y, imag_check): Y is float64 when A and V are real (Remark 5.1,
    real part taken, imag_check = max |Im Y|), complex128 otherwise
    (imag_check = 0.0).
    """
    A = np.asarray(A)
    V = np.asarray(V)
    X = shifted_solves_dense(A, V, theta, t, c, workers)
    Y = _weighted_sum(X, a, V.shape) * np.longdouble(math.exp(c))
    if _is_real(A, V):
        return Y.real.astype(np.float64), float(np.max(np.abs(Y.imag))) if Y.size else 0.0
    return Y.astype(np.complex128), 0.0


def shifted_solves_tridiag(d, e, V, theta, t=1.0, c=0.0, workers=1):
    """X_k = (tT - cI + theta_k I)^{-1} V for the Hermitian tridiagonal T with
    diagonal d (real, length N) and superdiagonal e (length N-1, T_{i,i+1} = e_i,
    T_{i+1,i} = conj(e_i)); banded LU with partial pivoting."""
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e)
    N = d.shape[0]
    V = np.asarray(V, dtype=np.complex128)

    def one(tk):
        ab = np.zeros((3, N), dtype=np.complex128)
        if N > 1:
            ab[0, 1:] = t * e
            ab[2, :-1] = t * np.conj(e)
        ab[1, :] = t * d - c + tk
        return scipy.linalg.solve_banded((1, 1), ab, V)

    return _pool_map(one, list(theta), workers)


def apply_tridiag(d, e, V, theta, a, t=1.0, c=0.0, workers=1):
    """Y* = e^c sum_k a_k (tT - cI + theta_k I)^{-1} V for Hermitian tridiagonal T.

    Same return convention as ``apply_dense``.
    """
    V = np.asarray(V)
    X = shifted_solves_tridiag(d, e, V, theta, t, c, workers)
    Y = _weighted_sum(X, a, V.shape) * np.longdouble(math.exp(c))
    if _is_real(np.asarray(e), V):
        return Y.real.astype(np.float64), float(np.max(np.abs(Y.imag))) if Y.size else 0.0
    return Y.astype(np.complex128), 0.0


def tridiag_to_dense(d, e) -> np.ndarray:
    """Dense Hermitian matrix with diagonal d and superdiagonal e."""
    d = np.asarray(d)
    e = np.asarray(e)
    T = np.diag(d.astype(np.result_type(d, e)))
    if e.size:
        T = T + np.diag(e, 1) + np.diag(np.conj(e), -1)
    return T


# ---------------------------------------------------------------- closed forms

def eig_apply(Q, mu, V, f) -> np.ndarray:
    """f(A) V with A = Q diag(mu) Q^H, Q unitary: Q diag(f(mu)) Q^H V (Remark 3.1)."""
    Q = np.asarray(Q)
    W = Q.conj().T @ np.asarray(V)
    return Q @ (f(np.asarray(mu))[:, None] * W)


def laplacian_eigs(d0: float, e0: float, N: int) -> np.ndarray:
    """Eigenvalues of tridiag(e0, d0, e0) of size N in DST-I order: d0 + 2 e0 cos(j pi/(N+1))."""
    j = np.arange(1, N + 1)
    return d0 + 2.0 * e0 * np.cos(j * np.pi / (N + 1))


def laplacian_apply(d0: float, e0: float, V, f) -> np.ndarray:
    """f(T) V for T = tridiag(e0, d0, e0), by the orthonormal DST-I eigenbasis
    (S = S^T = S^-1): f(T) V = S diag(f(mu)) S V."""
    V = np.asarray(V)
    N = V.shape[0]
    mu = laplacian_eigs(d0, e0, N)
    W = scipy.fft.dst(V, type=1, norm="ortho", axis=0)
    fm = f(mu)
    W = (fm[:, None] if V.ndim == 2 else fm) * W
    return scipy.fft.dst(W, type=1, norm="ortho", axis=0)


def laplacian2d_matrix(dx: int, dy: int, ax: float, bx: float, ay: float, by: float) -> np.ndarray:
    """The separable operator A = I_y (x) T_x + T_y (x) I_x of the 2D finite-difference
    Laplacian (Sec. 5), T_x = tridiag(ax, bx, ax) of size dx, T_y = tridiag(ay, by, ay) of
    size dy, assembled densely (row index iy * dx + ix); small sizes only."""
    Tx = np.diag(np.full(dx, bx)) + np.diag(np.full(dx - 1, ax), 1) + np.diag(np.full(dx - 1, ax), -1)
    Ty = np.diag(np.full(dy, by)) + np.diag(np.full(dy - 1, ay), 1) + np.diag(np.full(dy - 1, ay), -1)
    return np.kron(np.eye(dy), Tx) + np.kron(Ty, np.eye(dx))


def laplacian2d_apply(dx: int, dy: int, ax: float, bx: float, ay: float, by: float, V, f) -> np.ndarray:
    """f(A) V for the separable A of laplacian2d_matrix by its eigenbasis, the orthonormal
    DST-I along both axes: eigenvalue (bx + 2 ax cos(i pi/(dx+1))) + (by + 2 ay cos(j pi/(dy+1)))."""
    V = np.asarray(V)
    r = V.shape[1] if V.ndim == 2 else 1
    W = V.reshape(dy, dx, r)
    W = scipy.fft.dst(scipy.fft.dst(W, type=1, norm="ortho", axis=0), type=1, norm="ortho", axis=1)
    lam = laplacian_eigs(by, ay, dy)[:, None] + laplacian_eigs(bx, ax, dx)[None, :]
    W = f(lam)[:, :, None] * W
    W = scipy.fft.dst(scipy.fft.dst(W, type=1, norm="ortho", axis=0), type=1, norm="ortho", axis=1)
    return W.reshape(V.shape)


def product_apply(A, v, theta, n: int) -> np.ndarray:
    """R_n(A) v = n! prod_k (A + theta_k I)^{-1} v (even n; no residues involved)."""
    A = np.asarray(A, dtype=np.complex128)
    x = np.asarray(v, dtype=np.complex128)
    I = np.eye(A.shape[0])
    for tk in theta:
        x = np.linalg.solve(A + tk * I, x)
    return math.factorial(n) * x


def rel_err(Y, Yref) -> float:
    """Relative Frobenius error ||Y - Yref||_F / ||Yref||_F (relative 2-norm for a block)."""
    Y = np.asarray(Y)
    Yref = np.asarray(Yref)
    den = np.linalg.norm(Yref.ravel())
    num = np.linalg.norm((Y - Yref).ravel())
    return float(num / den) if den > 0 else float(num)
