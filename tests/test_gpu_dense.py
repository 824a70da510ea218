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


@pytest.mark.parametrize("prec", [P.EXPM_FP64, P.EXPM_MIXED_FP32, P.EXPM_MIXED_TF32X3, P.EXPM_MIXED_BF16X3])
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


@pytest.mark.parametrize("prec", [P.EXPM_FP64, P.EXPM_MIXED_FP32])
@pytest.mark.parametrize("n", [40, 256, 520])
def test_wide_solves_with_panel_inverses(plans, prec, n):
    """More than 8 columns: the triangular solves multiply by the inverses of the LU's
    128-row diagonal panels (one panel smaller than that, two full panels, four full panels
    and an 8-row one); real symmetric A (one solve per pair) with a real and a complex
    right-hand side, and the same columns solved narrow (4 at a time)."""
    g = workloads.rng(315 + n)
    A, Q, mu, V = workloads.dense_symmetric(n, -35.0, 0.0, 12, g, False)
    tol = 1e-12 if prec == P.EXPM_FP64 else 1e-10
    Y, info = _gpu(plans[16], A, V, prec)
    Yo = _oracle(A, V, 16)
    assert matrix.rel_err(Y, Yo) <= tol
    Yn = np.concatenate([_gpu(plans[16], A, V[:, c:c + 4], prec)[0] for c in range(0, 12, 4)], axis=1)
    assert matrix.rel_err(Yn, Yo) <= tol and matrix.rel_err(Y, Yn) <= 2 * tol
    Vc = V + 1j * g.standard_normal(V.shape)
    Yc, _ = _gpu(plans[12], A, Vc, prec)
    assert matrix.rel_err(Yc, _oracle(A, Vc, 12)) <= tol


def test_time_and_shift(plans):
    """e^c R_n(tA - cI)V with spectrum of tA in [0, 10] and c = 10 (Remark 3.2)."""
    g = workloads.rng(311)
    A, Q, mu, V = workloads.dense_symmetric(96, 0.0, 20.0, 2, g, True)
    Y, _ = _gpu(plans[16], A, V, P.EXPM_FP64, t=0.5, shift_c=10.0)
    assert matrix.rel_err(Y, _oracle(A, V, 16, t=0.5, c=10.0)) <= 1e-12


@pytest.mark.parametrize("prec", [P.EXPM_MIXED_FP32, P.EXPM_MIXED_TF32X3, P.EXPM_MIXED_BF16X3])
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


def test_bounded_wait_gives_up_and_reports(plans):
    """The bounded mbarrier wait the tensor-core kernels use, on a barrier that nothing
    completes (a flag nothing sets): it gives up after its poll limit and the host reads
    the time-out status; with the arrival made first it completes.  The context stays
    usable: a dense apply afterwards is still correct."""
    import ctypes
    f = P.lib.expm_internal_wait_probe
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    kclk = ctypes.c_int(-1)
    assert f(1 << 12, 1, ctypes.byref(kclk)) == 0
    assert f(1 << 12, 0, ctypes.byref(kclk)) == 2
    print(f"bounded wait: 4096 polls gave up after {kclk.value * 1024} SM clocks")
    assert kclk.value >= 0
    assert f(0, 0, None) == 1 and f((1 << 18) + 1, 0, None) == 1  # limits outside [1, 2^18]
    g = workloads.rng(318)
    A, Q, mu, V = workloads.dense_symmetric(96, -20.0, 0.0, 2, g, True)
    Y, info = _gpu(plans[12], A, V, P.EXPM_MIXED_FP32)
    assert info.status_worst == 0 and matrix.rel_err(Y, _oracle(A, V, 12)) <= 1e-10


def test_tensor_core_gemm_bf16_against_torch():
    """The tcgen05 kind::f16 kernel with bf16 operands: C -= A B^T equals the product of
    the bf16 operands (exact in binary32 per term; float64 reference) to fp32
    accumulation accuracy, on ragged tile edges."""
    import ctypes
    f = P.lib.expm_internal_tc_gemm_bf16
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_int]
    gen = torch.Generator(device="cpu").manual_seed(8)
    for M, N, K in [(128, 128, 64), (200, 72, 96), (1000, 520, 768), (129, 260, 40)]:
        A = torch.randn(M, K, generator=gen).to(torch.bfloat16).to(DEV)
        B = torch.randn(N, K, generator=gen).to(torch.bfloat16).to(DEV)
        C = torch.randn(M, N, generator=gen).to(DEV)
        C0 = C.clone()
        assert f(M, N, K, A.data_ptr(), K, B.data_ptr(), K, C.data_ptr(), N) == 0
        torch.cuda.synchronize()
        ref = C0.double() - A.double() @ B.double().T
        err = (C.double() - ref).abs().max().item() / ref.abs().max().item()
        assert err < 1e-5, (M, N, K, err)


def _oz_hook():
    import ctypes
    f = P.lib.expm_internal_oz_resid
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_void_p]
    return f


def _oz_run(A, X, R0, t, complex_a):
    """R_s - t A X_s on the GPU through the slice-product tensor-core kernel."""
    n, kc, nsys = A.shape[0], X.shape[2], X.shape[0]
    dA = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    dX = torch.from_numpy(np.ascontiguousarray(X)).to(DEV)
    dR = torch.from_numpy(np.ascontiguousarray(R0)).to(DEV)
    assert _oz_hook()(n, kc, nsys, int(complex_a), t, dA.data_ptr(), n, dX.data_ptr(), dR.data_ptr()) == 0
    torch.cuda.synchronize()
    return dR.cpu().numpy()


def _cgauss(g, shape):
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


@pytest.mark.parametrize("n,kc,nsys,complex_a", [(1, 1, 1, True), (100, 9, 2, True), (130, 70, 1, True),
                                                 (257, 33, 3, True), (300, 16, 3, False), (1030, 16, 8, True),
                                                 (200, 12, 5, False)])
def test_tensor_core_residual_product(n, kc, nsys, complex_a):
    """The binary64-accurate residual product R_s -= t A X_s on the bf16 tensor cores
    (six-slice splitting, 21 slice products): ragged tiles in M, N and K, real and
    complex A, against the float64 product on the host (whose own error, ~K 2^-53, is
    far below the bound)."""
    g = np.random.default_rng(4000 + n + kc)
    A = _cgauss(g, (n, n)) if complex_a else g.standard_normal((n, n))
    X = _cgauss(g, (nsys, n, kc))
    R0 = _cgauss(g, (nsys, n, kc))
    t = -0.75
    R = _oz_run(A, X, R0, t, complex_a)
    ref = R0 - t * np.einsum("il,slc->sic", A, X)
    prod = np.linalg.norm(t * np.einsum("il,slc->sic", A, X))
    assert np.linalg.norm(R - ref) <= 1e-13 * prod, np.linalg.norm(R - ref) / prod


def test_tensor_core_residual_scaling_and_special_values():
    """Per-row and per-column power-of-two scales: rows of A and columns of X spread
    over 2^-60 .. 2^60 keep the same relative accuracy; a zero row and a zero column
    leave R unchanged; a NaN in A poisons its row only, a NaN in X its column only."""
    g = np.random.default_rng(4100)
    n, kc, nsys = 260, 20, 2
    A = _cgauss(g, (n, n)) * np.exp2(g.integers(-60, 61, size=(n, 1)))
    X = _cgauss(g, (nsys, n, kc)) * np.exp2(g.integers(-60, 61, size=(nsys, 1, kc)))
    A[7, :] = 0.0
    X[1, :, 3] = 0.0
    R0 = _cgauss(g, (nsys, n, kc))
    R = _oz_run(A, X, R0, 1.0, True)
    ref = R0 - np.einsum("il,slc->sic", A, X)
    # error of each entry against max|A_i.| max|X_.j| sqrt(K) (scale-free), plus the final
    # rounding of R0 - t A X (one ulp of R, which decides where |A X| << |R0|)
    scale = np.abs(A).max(axis=1)[None, :, None] * np.abs(X).max(axis=1)[:, None, :] * np.sqrt(2 * n)
    err = np.abs(R - ref)
    assert (err <= 1e-13 * scale + 2.0 ** -52 * np.abs(ref)).all(), (err / np.where(scale > 0, scale, 1)).max()
    np.testing.assert_array_equal(R[:, 7, :], R0[:, 7, :])
    np.testing.assert_array_equal(R[1, :, 3], R0[1, :, 3])
    A2 = _cgauss(g, (n, n))
    A2[11, 5] = np.nan
    X2 = _cgauss(g, (nsys, n, kc))
    X2[0, 9, 4] = complex(np.nan, 0.0)
    R2 = _oz_run(A2, X2, R0, 1.0, True)
    bad = np.zeros(R2.shape, dtype=bool)
    bad[:, 11, :] = True
    bad[0, :, 4] = True
    assert np.isnan(R2[bad]).all()
    ref2 = R0 - np.einsum("il,slc->sic", np.nan_to_num(A2), np.nan_to_num(X2))
    assert np.abs(R2[~bad] - ref2[~bad]).max() <= 1e-12 * np.abs(ref2[~bad]).max()


@pytest.mark.parametrize("n,k", [(600, 20), (777, 64)])
def test_bf16x3_tensor_core_solves(plans, n, k):
    """EXPM_MIXED_BF16X3 with many columns: LU trailing updates and the triangular solves'
    panel updates on the tensor cores (several 256-row panels, a ragged last panel), both
    halves of the complex solve; against the oracle and the binary64 path."""
    g = workloads.rng(330 + n)
    A, Q, mu, V = workloads.dense_symmetric(n, -40.0, 0.0, k, g, True)
    Ybf, info = _gpu(plans[16], A, V, P.EXPM_MIXED_BF16X3)
    Y64, _ = _gpu(plans[16], A, V, P.EXPM_FP64)
    assert info.status_worst == 0 and 1 <= info.refine_iters_max <= 3
    assert matrix.rel_err(Ybf, Y64) <= 1e-10
    assert matrix.rel_err(Ybf, _oracle(A, V, 16)) <= 1e-10


@pytest.mark.parametrize("n,kc,nsys,complex_a", [(100, 9, 2, True), (300, 16, 3, False), (700, 20, 4, True)])
def test_tensor_core_residual_light(n, kc, nsys, complex_a):
    """The light residual update R_s -= t A D_s for a binary32 D (four slices of A and of
    D, the 10 slice products of order <= 3): about 2^-30 of the product, the accuracy a
    correction ~1e-6 of the solution needs."""
    import ctypes
    f = P.lib.expm_internal_oz_resid_light
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_void_p]
    g = np.random.default_rng(4200 + n)
    A = _cgauss(g, (n, n)) if complex_a else g.standard_normal((n, n))
    D = _cgauss(g, (nsys, n, kc)).astype(np.complex64)
    R0 = _cgauss(g, (nsys, n, kc))
    dA = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    dD = torch.from_numpy(np.ascontiguousarray(D)).to(DEV)
    dR = torch.from_numpy(np.ascontiguousarray(R0)).to(DEV)
    assert f(n, kc, nsys, int(complex_a), 0.5, dA.data_ptr(), n, dD.data_ptr(), dR.data_ptr()) == 0
    torch.cuda.synchronize()
    prod = 0.5 * np.einsum("il,slc->sic", A, D.astype(np.complex128))
    err = np.linalg.norm(dR.cpu().numpy() - (R0 - prod)) / np.linalg.norm(prod)
    assert err <= 1e-8, err
