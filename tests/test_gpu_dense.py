"""GPU parity of the pole-batched dense path (expm_apply_dense) against the oracle,
through the C-ABI.

Tolerances: relative Frobenius error <= 1e-12 for the binary64 path; the mixed
path (binary32 LU + binary64 refinement) is held to 1e-10 (the dense mixed-path
tolerance) against both the oracle and the binary64 GPU path.
"""

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


def _oracle(A, V, n, t=1.0, c=0.0):
    Y, _ = matrix.apply_dense(A, V, coeffs.theta(n), coeffs.residues(n), t=t, c=c, workers=8)
    return Y


def _gpu(plan, A, V, prec, **kw):
    dA = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    dV = torch.from_numpy(np.ascontiguousarray(V)).to(DEV)
    out_dtype = torch.complex128 if (np.iscomplexobj(A) or np.iscomplexobj(V)) else torch.float64
    dY = torch.empty(V.shape, dtype=out_dtype, device=DEV)
    info = P.expm_apply_dense(plan, dA, dV, dY, prec=prec, **kw)
    torch.cuda.synchronize()
    return dY.cpu().numpy(), info


def test_dense_small_workload(plans):
    """64 x 64 real symmetric, spectrum U[-20, 0], one vector, degree 12 (FP64)."""
    w = workloads.dense_small()
    Y, info = _gpu(plans[12], w["A"], w["V"], P.EXPM_FP64)
    assert matrix.rel_err(Y, _oracle(w["A"], w["V"], 12)) <= 1e-12
    ref = matrix.eig_apply(w["Q"], w["mu"], w["V"], lambda m: scalar.R_n(m, 12))
    assert matrix.rel_err(Y, ref) <= 1e-12
    assert 0 < info.growth_max_seen < 1e3


@pytest.mark.parametrize("prec", [P.EXPM_FP64, P.EXPM_MIXED_FP32, P.EXPM_MIXED_TF32X3])
@pytest.mark.parametrize("n,k,deg", [(1, 1, 12), (5, 2, 16), (63, 3, 12), (64, 1, 16), (65, 5, 12),
                                     (130, 70, 16), (257, 4, 12), (333, 9, 16)])
def test_complex_hermitian(plans, prec, n, k, deg):
    """Ragged panel widths (n not a multiple of 64), several RHS tiles."""
    g = workloads.rng(300 + n + k)
    A, Q, mu, V = workloads.dense_symmetric(n, -30.0, 0.0, k, g, True)
    Y, info = _gpu(plans[deg], A, V, prec)
    Yo = _oracle(A, V, deg)
    tol = 1e-12 if prec == P.EXPM_FP64 else 1e-10
    assert _close(Y, Yo, V, deg, tol), matrix.rel_err(Y, Yo)
    if n >= 60:
        assert matrix.rel_err(Y, Yo) <= tol
    if prec != P.EXPM_FP64:
        assert info.refine_iters_max >= 1


@pytest.mark.parametrize("prec", [P.EXPM_FP64, P.EXPM_MIXED_FP32])
def test_real_symmetric_with_real_and_complex_rhs(plans, prec):
    g = workloads.rng(310)
    A, Q, mu, V = workloads.dense_symmetric(150, -25.0, 0.0, 3, g, False)
    Vc = V + 1j * g.standard_normal(V.shape)
    tol = 1e-12 if prec == P.EXPM_FP64 else 1e-10
    Y, _ = _gpu(plans[16], A, V, prec)
    assert Y.dtype == np.float64 and matrix.rel_err(Y, _oracle(A, V, 16)) <= tol
    Yc, _ = _gpu(plans[16], A, Vc, prec)
    assert Yc.dtype == np.complex128 and matrix.rel_err(Yc, _oracle(A, Vc, 16)) <= tol


def test_time_and_shift(plans):
    """e^c R_n(tA - cI)V with spectrum of tA in [0, 10] and c = 10 (Remark 3.2)."""
    g = workloads.rng(311)
    A, Q, mu, V = workloads.dense_symmetric(96, 0.0, 20.0, 2, g, True)
    Y, _ = _gpu(plans[16], A, V, P.EXPM_FP64, t=0.5, shift_c=10.0)
    assert matrix.rel_err(Y, _oracle(A, V, 16, t=0.5, c=10.0)) <= 1e-12


@pytest.mark.parametrize("prec", [P.EXPM_MIXED_FP32, P.EXPM_MIXED_TF32X3])
def test_mixed_matches_fp64_path(plans, prec):
    """Mid-size complex Hermitian: the refined mixed paths agree with the binary64 path."""
    g = workloads.rng(312)
    A, Q, mu, V = workloads.dense_symmetric(512, -50.0, 0.0, 32, g, True)
    Y64, _ = _gpu(plans[16], A, V, P.EXPM_FP64)
    Ymx, info = _gpu(plans[16], A, V, prec)
    assert matrix.rel_err(Ymx, Y64) <= 1e-10
    assert matrix.rel_err(Y64, _oracle(A, V, 16)) <= 1e-12
    assert info.resid_rel_max <= 1e-14


def test_host_buffers(plans):
    g = workloads.rng(313)
    A, Q, mu, V = workloads.dense_symmetric(70, -10.0, 0.0, 2, g, True)
    Yd, _ = _gpu(plans[12], A, V, P.EXPM_FP64)
    Yh = np.empty_like(V)
    P.expm_apply_dense(plans[12], A, V, Yh)
    np.testing.assert_array_equal(Yh, Yd)


def test_refinement_not_converged_is_reported(plans):
    """max_refine = 0 with a tight tolerance: EXPM_ENOCONV, injected from the host."""
    g = workloads.rng(314)
    A, Q, mu, V = workloads.dense_symmetric(80, -10.0, 0.0, 1, g, True)
    dA, dV = (torch.from_numpy(x).to(DEV) for x in (A, V))
    dY = torch.empty_like(dV)
    info = P.expm_apply_dense(plans[12], dA, dV, dY, prec=P.EXPM_MIXED_FP32, max_refine=0, tol=1e-15,
                              check=False)
    assert info.status_worst == 4                      # EXPM_ENOCONV


def test_growth_limit_is_reported(plans):
    """growth_max = 0.5 (below any real growth factor): EXPM_EGROWTH, Y still written."""
    g = workloads.rng(315)
    A, Q, mu, V = workloads.dense_symmetric(40, -10.0, 0.0, 1, g, True)
    dA, dV = (torch.from_numpy(x).to(DEV) for x in (A, V))
    dY = torch.zeros_like(dV)
    info = P.expm_apply_dense(plans[12], dA, dV, dY, growth_max=0.5, check=False)
    assert info.status_worst == 3 and info.growth_max_seen >= 0.5
    assert matrix.rel_err(dY.cpu().numpy(), _oracle(A, V, 12)) <= 1e-12


def test_tensor_core_gemm_against_torch():
    """The tcgen05 kind::tf32 kernel: C -= A B^T equals the product of the TF32-rounded
    operands (fp64 reference) to fp32 accumulation accuracy, on ragged tile edges."""
    import ctypes
    f = P.lib.expm_internal_tc_gemm_tf32
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_int]
    gen = torch.Generator(device="cpu").manual_seed(7)
    for M, N, K in [(128, 128, 32), (200, 72, 96), (1000, 520, 384), (129, 260, 36)]:
        A = torch.randn(M, K, generator=gen).to(DEV)
        B = torch.randn(N, K, generator=gen).to(DEV)
        C = torch.randn(M, N, generator=gen).to(DEV)
        C0 = C.clone()
        assert f(M, N, K, A.data_ptr(), K, B.data_ptr(), K, C.data_ptr(), N) == 0
        torch.cuda.synchronize()
        tf = lambda x: (x.view(torch.int32) & ~0x1FFF).view(torch.float32).double()
        ref = C0.double() - tf(A) @ tf(B).T
        err = (C.double() - ref).abs().max().item() / ref.abs().max().item()
        assert err < 1e-5, (M, N, K, err)
