"""GPU parity of expm_apply_laplacian2d (separable 2D finite-difference Laplacian, Sec. 5):
DST-I along y as a product with S (binary64, or the binary64-accurate tensor-core slice
product in the mixed precisions), the pole-batched tridiagonal path on the
block-diagonal operator along x, DST-I back.  Against the oracle: per-pole dense solves on
the assembled matrix (small grids) and the 2D DST-I closed form (large grids).
Tolerances: 1e-12 (binary64 solves), 1e-8 (binary32 + refinement)."""

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
# 100 (1, -2, 1) along both axes: spectrum in (-800, 0)
AX, BX, AY, BY = 100.0, -200.0, 100.0, -200.0


@pytest.fixture(scope="module")
def plans():
    return {n: P.Plan(degree=n) for n in (12, 16)}


def _floor(V, n, unit=2.0 ** -53):
    th, a = coeffs.theta(n), coeffs.residues(n)
    return 64 * unit * float(np.sum(np.abs(a) / np.abs(th.imag))) * np.linalg.norm(V)


def _run(plan, dx, dy, V, **kw):
    dV = torch.from_numpy(np.ascontiguousarray(V)).to(DEV)
    dY = torch.empty_like(dV)
    info = P.expm_apply_laplacian2d(plan, dx, dy, AX, BX, AY, BY, dV, dY, **kw)
    torch.cuda.synchronize()
    return dY.cpu().numpy(), info


@pytest.mark.parametrize("dx,dy,r,complex_v", [(1, 1, 1, False), (7, 5, 2, False), (13, 9, 3, True), (40, 1, 2, False)])
def test_small_grids_match_dense_oracle(plans, dx, dy, r, complex_v):
    g = workloads.rng(950 + dx)
    V = g.standard_normal((dx * dy, r)) + (1j * g.standard_normal((dx * dy, r)) if complex_v else 0.0)
    Y, _ = _run(plans[12], dx, dy, V)
    A = matrix.laplacian2d_matrix(dx, dy, AX, BX, AY, BY)
    Yo, _ = matrix.apply_dense(A, V, coeffs.theta(12), coeffs.residues(12))
    assert np.linalg.norm(Y - Yo) <= 1e-12 * np.linalg.norm(Yo) + _floor(V, 12), matrix.rel_err(Y, Yo)


@pytest.mark.parametrize("dx,dy,r,complex_v", [(7, 5, 2, False), (13, 9, 3, True), (9, 7, 1, False), (1, 1, 2, False)])
def test_small_grids_tensor_core_transform(plans, dx, dy, r, complex_v):
    """The mixed precisions take the sine transforms through the binary64-accurate slice
    product on the tensor cores (an odd number of real columns falls back to the binary64
    product): float-float solves, against the dense oracle at 1e-11."""
    g = workloads.rng(970 + dx + dy)
    V = g.standard_normal((dx * dy, r)) + (1j * g.standard_normal((dx * dy, r)) if complex_v else 0.0)
    Y, _ = _run(plans[12], dx, dy, V, prec=P.EXPM_MIXED_F32X2)
    A = matrix.laplacian2d_matrix(dx, dy, AX, BX, AY, BY)
    Yo, _ = matrix.apply_dense(A, V, coeffs.theta(12), coeffs.residues(12))
    assert np.linalg.norm(Y - Yo) <= 1e-11 * np.linalg.norm(Yo) + _floor(V, 12, 2.0 ** -46), matrix.rel_err(Y, Yo)


@pytest.mark.parametrize("dx,dy,r", [(100, 200, 3), (257, 130, 2)])
def test_medium_grids_tensor_core_transform(plans, dx, dy, r):
    """Ragged tiles of the slice product (dy not a multiple of 128, dx r not of 96)."""
    g = workloads.rng(980 + dx)
    V = g.standard_normal((dx * dy, r))
    Y, _ = _run(plans[16], dx, dy, V, prec=P.EXPM_MIXED_F32X2)
    ref = matrix.laplacian2d_apply(dx, dy, AX, BX, AY, BY, V, lambda m: scalar.R_n(m, 16))
    assert np.linalg.norm(Y - ref) <= 1e-11 * np.linalg.norm(ref) + _floor(V, 16, 2.0 ** -46), matrix.rel_err(Y, ref)


@pytest.mark.parametrize("dx,dy", [(100, 80), (257, 130)])
def test_medium_grids_match_closed_form(plans, dx, dy):
    g = workloads.rng(960 + dx)
    V = g.standard_normal((dx * dy, 4))
    Y, _ = _run(plans[16], dx, dy, V)
    ref = matrix.laplacian2d_apply(dx, dy, AX, BX, AY, BY, V, lambda m: scalar.R_n(m, 16))
    assert np.linalg.norm(Y - ref) <= 1e-12 * np.linalg.norm(ref) + _floor(V, 16)


def test_time_and_shift(plans):
    """Remark 3.2: spectrum of A in (-760, 40), t = 0.5, c = 20 >= the largest eigenvalue of tA."""
    dx, dy = 60, 50
    g = workloads.rng(970)
    V = g.standard_normal((dx * dy, 2))
    dV = torch.from_numpy(V).to(DEV)
    dY = torch.empty_like(dV)
    P.expm_apply_laplacian2d(plans[16], dx, dy, AX, BX + 20.0, AY, BY + 20.0, dV, dY, t=0.5, shift_c=20.0)
    torch.cuda.synchronize()
    ref = matrix.laplacian2d_apply(dx, dy, AX, BX + 20.0, AY, BY + 20.0, V,
                                   lambda m: np.exp(20.0) * scalar.R_n(0.5 * m - 20.0, 16))
    assert matrix.rel_err(dY.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("prec,tol", [(P.EXPM_FP64, 1e-12), (P.EXPM_MIXED_FP32, 1e-8)])
def test_paper_size_grid(plans, prec, tol):
    """1024 x 1024 grid (N = 2^20 unknowns), one right-hand side, degree 16."""
    d = 1024
    g = workloads.rng(980)
    V = g.standard_normal((d * d, 1))
    kw = dict(tol=1e-10, max_refine=1) if prec == P.EXPM_MIXED_FP32 else {}
    Y, _ = _run(plans[16], d, d, V, prec=prec, **kw)
    ref = matrix.laplacian2d_apply(d, d, AX, BX, AY, BY, V, lambda m: scalar.R_n(m, 16))
    err = matrix.rel_err(Y, ref)
    print(f"2D 1024^2 prec={prec}: {err:.3e}")
    assert np.linalg.norm(Y - ref) <= tol * np.linalg.norm(ref) + _floor(V, 16, 2.0 ** -46)
