"""GPU parity of expm_apply_dense_reduced: dense Hermitian A reduced to real symmetric
tridiagonal form by Householder reflectors, the pole-batched tridiagonal path, and the
reflectors applied back (R_n(Q T Q^H) = Q R_n(T) Q^H, Remark 3.1).  Against the oracle
(pivoted dense solves per pole) and the eigen closed form.  Tolerances: 1e-12 with binary64
tridiagonal solves, 1e-8 with the binary32 + refinement solves."""

import numpy as np
import pytest

import workloads
from oracle import coeffs, matrix, scalar

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2306_16778_gb300 as P  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def plans():
    return {n: P.Plan(degree=n) for n in (12, 16)}


def _close(Y, Yo, V, n, tol, unit=2.0 ** -53):
    """Relative error <= tol, or below the rounding floor of the partial-fraction sum
    when R_n(A)V is tiny next to V (Sec. 4: the terms a_k/(x + theta_k) are
    O(|a_k|/|Im theta_k|) and their rounding errors do not cancel)."""
    th, a = coeffs.theta(n), coeffs.residues(n)
    floor = 64 * unit * float(np.sum(np.abs(a) / np.abs(th.imag))) * np.linalg.norm(V)
    return np.linalg.norm(Y - Yo) <= tol * np.linalg.norm(Yo) + floor


def _run(plan, A, V, **kw):
    dA = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    dV = torch.from_numpy(np.ascontiguousarray(V)).to(DEV)
    out = torch.complex128 if (np.iscomplexobj(A) or np.iscomplexobj(V)) else torch.float64
    dY = torch.empty(V.shape, dtype=out, device=DEV)
    info = P.expm_apply_dense_reduced(plan, dA, dV, dY, **kw)
    torch.cuda.synchronize()
    return dY.cpu().numpy(), info


@pytest.mark.parametrize("n,k,complex_,deg", [(1, 1, True, 12), (2, 3, True, 16), (37, 5, True, 16),
                                              (300, 17, True, 12), (513, 40, False, 16), (700, 3, True, 16)])
def test_reduced_matches_oracle(plans, n, k, complex_, deg):
    A, Q, mu, V = workloads.dense_symmetric(n, -40.0, 0.0, k, workloads.rng(900 + n), complex_)
    Y, _ = _run(plans[deg], A, V)
    Yo, _ = matrix.apply_dense(A, V, coeffs.theta(deg), coeffs.residues(deg), workers=8)
    assert _close(Y, Yo, V, deg, 1e-12), matrix.rel_err(Y, Yo)
    ref = matrix.eig_apply(Q, mu, V, lambda m: scalar.R_n(m, deg))
    assert _close(Y, ref, V, deg, 1e-12), matrix.rel_err(Y, ref)


def test_reduced_matches_lu_path_with_time_and_shift(plans):
    """Spectrum in [0, 20] with t = 0.5 and c = 10 (Remark 3.2), against expm_apply_dense."""
    A, Q, mu, V = workloads.dense_symmetric(257, 0.0, 20.0, 4, workloads.rng(910), True)
    Y, _ = _run(plans[16], A, V, t=0.5, shift_c=10.0)
    dA, dV = torch.from_numpy(A).to(DEV), torch.from_numpy(V).to(DEV)
    Yl = torch.empty_like(dV)
    P.expm_apply_dense(plans[16], dA, dV, Yl, t=0.5, shift_c=10.0)
    torch.cuda.synchronize()
    assert matrix.rel_err(Y, Yl.cpu().numpy()) <= 1e-12
    ref = matrix.eig_apply(Q, mu, V, lambda m: np.exp(10.0) * scalar.R_n(0.5 * m - 10.0, 16))
    assert matrix.rel_err(Y, ref) <= 1e-12


def test_reduced_with_mixed_tridiagonal_solves(plans):
    A, Q, mu, V = workloads.dense_symmetric(400, -50.0, 0.0, 8, workloads.rng(911), True)
    Y, info = _run(plans[16], A, V, prec=P.EXPM_MIXED_FP32, tol=1e-10, max_refine=2)
    assert info.status_worst == 0 and info.refine_iters_max >= 1
    ref = matrix.eig_apply(Q, mu, V, lambda m: scalar.R_n(m, 16))
    assert matrix.rel_err(Y, ref) <= 1e-8


def test_reduced_leaves_inputs_and_is_deterministic(plans):
    A, _, _, V = workloads.dense_symmetric(150, -10.0, 0.0, 2, workloads.rng(912), True)
    dA, dV = torch.from_numpy(A).to(DEV), torch.from_numpy(V).to(DEV)
    A0, V0 = dA.clone(), dV.clone()
    Y1, Y2 = torch.empty_like(dV), torch.empty_like(dV)
    P.expm_apply_dense_reduced(plans[12], dA, dV, Y1)
    P.expm_apply_dense_reduced(plans[12], dA, dV, Y2)
    torch.cuda.synchronize()
    assert torch.equal(dA, A0) and torch.equal(dV, V0)
    assert torch.equal(Y1, Y2)


def test_reduced_rejections(plans):
    A = np.eye(4)
    with pytest.raises(P.ExpmError) as ei:           # host buffers are not accepted
        P.expm_apply_dense_reduced(plans[12], A, np.ones((4, 1)), np.empty((4, 1)))
    assert ei.value.status == 1
