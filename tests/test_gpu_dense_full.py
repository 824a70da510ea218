"""GPU parity of the full-matrix entry point (expm_apply_dense_full): the matrix
e^c R_n(tA - cI) itself (eq. ExpoMatRat), against closed forms that do not go through
partial fractions (Remark 3.1: R_n(Q diag(mu) Q^H) = Q diag(R_n(mu)) Q^H), against
exp within the uniform bound 2^-n (Prop. 2.2), the semigroup property, and the
matrix-vector entry point with V = I.

Tolerances: 1e-12 relative (Frobenius) for binary64, 1e-10 for the mixed path."""

import numpy as np
import pytest

import workloads
from oracle import matrix, scalar

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2306_16778_gb300 as P  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def plans():
    return {n: P.Plan(degree=n) for n in (12, 16)}


def _full(plan, A, prec=P.EXPM_FP64, **kw):
    dA = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    dY = torch.empty(A.shape, dtype=dA.dtype, device=DEV)
    info = P.expm_apply_dense_full(plan, dA, dY, prec=prec, **kw)
    torch.cuda.synchronize()
    return dY.cpu().numpy(), info


def _eig(Q, mu, f):
    return matrix.eig_apply(Q, mu, np.eye(Q.shape[0], dtype=Q.dtype), f)


@pytest.mark.parametrize("n,complex_,deg", [(1, False, 12), (37, True, 16), (200, True, 16), (700, False, 12),
                                            (1100, True, 12)])
def test_full_matrix_closed_form(plans, n, complex_, deg):
    """Several 512-column blocks with a ragged last block (700, 1100), real and complex."""
    A, Q, mu, _ = workloads.dense_symmetric(n, -20.0, 0.0, 1, workloads.rng(800 + n), complex_)
    Y, info = _full(plans[deg], A)
    assert info.status_worst == 0
    ref = _eig(Q, mu, lambda m: scalar.R_n(m, deg))
    assert matrix.rel_err(Y, ref) <= 1e-12
    # against exp itself: sup_x |R_n(x) - e^x| <= 2^-n on x <= 0 (Prop. 2.2), so the
    # spectral-norm error is below 2^-n and the Frobenius error below sqrt(n) 2^-n
    E = _eig(Q, mu, np.exp)
    assert np.linalg.norm(Y - E) <= np.sqrt(n) * 2.0 ** -deg


def test_full_matrix_equals_apply_with_identity(plans):
    A, _, _, _ = workloads.dense_symmetric(300, -30.0, 0.0, 1, workloads.rng(811), True)
    Y, _ = _full(plans[16], A)
    dA = torch.from_numpy(A).to(DEV)
    I = torch.eye(300, dtype=torch.complex128, device=DEV)
    Yv = torch.empty_like(I)
    P.expm_apply_dense(plans[16], dA, I, Yv)
    torch.cuda.synchronize()
    assert matrix.rel_err(Y, Yv.cpu().numpy()) <= 1e-14


def test_semigroup(plans):
    """R_n(A)^2 vs R_n(2A): both within 2^-n-type bounds of exp(A)^2 = exp(2A)."""
    n = 250
    A, Q, mu, _ = workloads.dense_symmetric(n, -15.0, 0.0, 1, workloads.rng(812), False)
    E1, _ = _full(plans[16], A)
    E2, _ = _full(plans[16], A, t=2.0)
    # ||R^2 - exp(2A)|| <= ||R - e^A|| (||R|| + ||e^A||) <= 2^-n (2 + 2^-n); R_n(2A) within 2^-n
    bound = np.sqrt(n) * (2.0 ** -16 * (2 + 2.0 ** -16) + 2.0 ** -16)
    assert np.linalg.norm(E1 @ E1 - E2) <= bound
    assert matrix.rel_err(E2, _eig(Q, 2 * mu, lambda m: scalar.R_n(m, 16))) <= 1e-12


def test_shift_method_positive_spectrum(plans):
    """Remark 3.2: spectrum in [0, 20], c = 20 >= the largest eigenvalue, e^c R_n(A - cI)
    approximates exp(A) with relative error about 2^-n (Fig. 5.2, right)."""
    n = 160
    A, Q, mu, _ = workloads.dense_symmetric(n, 0.0, 20.0, 1, workloads.rng(813), True)
    Y, _ = _full(plans[16], A, shift_c=20.0)
    ref = _eig(Q, mu, lambda m: np.exp(20.0) * scalar.R_n(m - 20.0, 16))
    assert matrix.rel_err(Y, ref) <= 1e-12
    E = _eig(Q, mu, np.exp)
    assert np.linalg.norm(Y - E, 2) <= np.exp(20.0) * 2.0 ** -16 * 1.0001


@pytest.mark.parametrize("prec", [P.EXPM_MIXED_FP32, P.EXPM_MIXED_TF32X3, P.EXPM_MIXED_BF16X3])
def test_full_matrix_mixed(plans, prec):
    A, Q, mu, _ = workloads.dense_symmetric(600, -40.0, 0.0, 1, workloads.rng(814), True)
    Y, info = _full(plans[16], A, prec=prec)
    assert info.status_worst == 0 and info.refine_iters_max >= 1
    ref = _eig(Q, mu, lambda m: scalar.R_n(m, 16))
    assert matrix.rel_err(Y, ref) <= 1e-10


def test_full_matrix_host_buffers(plans):
    A, _, _, _ = workloads.dense_symmetric(90, -10.0, 0.0, 1, workloads.rng(815), False)
    Yd, _ = _full(plans[12], A)
    Yh = np.empty_like(A)
    P.expm_apply_dense_full(plans[12], A, Yh)
    np.testing.assert_array_equal(Yh, Yd)
