"""Oracle scalar functions (Secs. 2 and 4).  Test infrastructure only.

* exp_n(x)            truncated Taylor series (Sec. 2), Horner, binary64.
* R_n(x) = 1/exp_n(-x) (Sec. 2.2).  For x <= 0 every term of exp_n(-x) is
  positive, so the Horner evaluation has no cancellation.
* pf_sum(x)           sum_k a_k/(x + theta_k)   (Prop. 2.1, eq. yoyo), binary64.
* err_n(x) = R_n(x) - e^x on x <= 0 (Prop. 2.3), and the errors e_1, e_2, e_3
  of the decomposition in Sec. 4.
* M_1(n) = 2^-n (Prop. 2.2) and M_2(n, D) (Prop. 4.1, eq. upper_bound).
* f_n(x) = exp_n(x) e^-x (Lemma 2.1).
"""

from __future__ import annotations

import math

import numpy as np

#: lower bound on the root separation of exp_n over all n >= 2 (eq. ecart)
GAMMA = 0.29044


def exp_n(x, n: int):
    """sum_{k=0..n} x^k/k! by Horner (works elementwise on arrays, real or complex)."""
    x = np.asarray(x)
    acc = np.full_like(x, 1.0 / math.factorial(n), dtype=np.result_type(x, 1.0))
    for k in range(n - 1, -1, -1):
        acc = acc * x + 1.0 / math.factorial(k)
    return acc


def R_n(x, n: int):
    """R_n(x) = 1/exp_n(-x) (Sec. 2.2)."""
    return 1.0 / exp_n(-np.asarray(x), n)


def pf_sum(x, theta: np.ndarray, a: np.ndarray):
    """sum_k a_k/(x + theta_k) (eq. yoyo), evaluated in complex128, summed in index order."""
    x = np.asarray(x, dtype=np.complex128)
    acc = np.zeros_like(x)
    for tk, ak in zip(theta, a):
        acc = acc + ak / (x + tk)
    return acc


def err_n(x, n: int):
    """err_n(x) = R_n(x) - exp(x) (Prop. 2.3: positive on (-inf, 0))."""
    return R_n(x, n) - np.exp(x)


def f_n(x, n: int):
    """f_n(x) = exp_n(x) exp(-x) (Lemma 2.1)."""
    return exp_n(x, n) * np.exp(-np.asarray(x, dtype=float))


def M1(n: int) -> float:
    """Uniform truncation bound |R_n(x) - e^x| <= 2^-n for x <= 0 (Prop. 2.2)."""
    return 2.0 ** (-n)


def M2(n: int, D: int, a_tilde: np.ndarray) -> float:
    """Rounding bound of Prop. 4.1: (C_1(D) + C_2(n, D)) * sum_k |a~_k|, valid
    when gamma > n 10^(1-D) (eq. condDn)."""
    u = 10.0 ** (1 - D)
    if not GAMMA > n * u:
        raise ValueError("condition gamma > n 10^(1-D) of Prop. 4.1 violated")
    c1 = 2 * u / (GAMMA * (1 - u))
    c2 = 4 * n * u / (GAMMA * (GAMMA - n * u))
    return (c1 + c2) * float(np.sum(np.abs(a_tilde)))


def e_split(x, n: int, theta: np.ndarray, a: np.ndarray):
    """(e_1, e_2, e_3) of Sec. 4: e_1 = exp - pf, e_2 = exp - R_n, e_3 = R_n - pf (binary64)."""
    x = np.asarray(x, dtype=float)
    pf = pf_sum(x, theta, a).real
    rn = R_n(x, n)
    ex = np.exp(x)
    return ex - pf, ex - rn, rn - pf
