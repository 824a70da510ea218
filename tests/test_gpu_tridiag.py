"""GPU parity of the pole-batched tridiagonal path (expm_apply_tridiag) against
the oracle, through the C-ABI.

Tolerances: relative Frobenius error <= 1e-12 for the binary64 path (the
configured FP64 tolerance) and <= 1e-8 for the float-float and the binary32 +
refinement paths (the mixed-path tolerance), each against the oracle's pivoted
banded solves on the same inputs.
"""

import numpy as np
import pytest

import workloads
from oracle import coeffs, matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2306_16778_gb300 as P  # noqa: E402

TOL = {P.EXPM_FP64: 1e-12, P.EXPM_MIXED_F32X2: 1e-8, P.EXPM_MIXED_FP32: 1e-8}
# rounding unit of the arithmetic that forms Y (binary64; float pairs for both mixed paths)
UNIT = {P.EXPM_FP64: 2.0 ** -53, P.EXPM_MIXED_F32X2: 2.0 ** -48, P.EXPM_MIXED_FP32: 2.0 ** -46}
ALL = [P.EXPM_FP64, P.EXPM_MIXED_F32X2, P.EXPM_MIXED_FP32]
DEV = torch.device("cuda:0")


def _close(Y, Yo, V, n, prec):
    """Relative error <= TOL, or below the rounding floor of the partial-fraction
    sum when R_n(T)V is tiny next to V (Sec. 4: each term a_k/(x + theta_k) is
    O(|a_k|/|Im theta_k|) and its rounding error does not cancel)."""
    th, a = coeffs.theta(n), coeffs.residues(n)
    floor = 64 * UNIT[prec] * float(np.sum(np.abs(a) / np.abs(th.imag))) * np.linalg.norm(V)
    err = np.linalg.norm(Y - Yo)
    return err <= TOL[prec] * np.linalg.norm(Yo) + floor, matrix.rel_err(Y, Yo)


def _oracle(d, e, V, n, t=1.0, c=0.0):
    Y, _ = matrix.apply_tridiag(d, e, V, coeffs.theta(n), coeffs.residues(n), t=t, c=c, workers=8)
    return Y


def _gpu(plan, d, e, V, prec, t=1.0, c=0.0, **kw):
    dd = torch.from_numpy(d).to(DEV)
    cplx_e = np.iscomplexobj(e)
    de = torch.from_numpy(e).to(DEV) if e.size else \
        torch.zeros(1, dtype=torch.complex128 if cplx_e else torch.float64, device=DEV)
    dv = torch.from_numpy(np.ascontiguousarray(V)).to(DEV)
    # Y is complex when V or e is complex
    dy = torch.empty(V.shape, dtype=torch.complex128 if cplx_e or np.iscomplexobj(V) else torch.float64, device=DEV)
    P.expm_apply_tridiag(plan, dd, de, dv, dy, prec=prec, t=t, shift_c=c, **kw)
    torch.cuda.synchronize()
    return dy.cpu().numpy()


def _random_tridiag(N, r, seed, complex_v=False):
    g = workloads.rng(seed)
    d = g.uniform(-12.0, -4.0, N)
    e = g.uniform(0.5, 2.0, max(N - 1, 0))      # Gershgorin: spectrum in (-16, 0)
    V = g.standard_normal((N, r))
    if complex_v:
        V = V + 1j * g.standard_normal((N, r))
    return d, e, V


@pytest.fixture(scope="module")
def plans():
    return {n: P.Plan(degree=n) for n in (12, 16)}


@pytest.mark.parametrize("prec", ALL)
@pytest.mark.parametrize("N,r,n", [(1, 1, 12), (2, 3, 16), (7, 2, 12), (100, 1, 16), (433, 8, 16),
                                   (4096 + 13, 5, 12), (50_000, 8, 16), (200_003, 3, 12)])
def test_random_tridiag_parity(plans, prec, N, r, n):
    """Several blocks, a ragged last block, single-row and tiny systems."""
    d, e, V = _random_tridiag(N, r, 200 + N + r)
    Y = _gpu(plans[n], d, e, V, prec)
    Yo = _oracle(d, e, V, n)
    ok, rel = _close(Y, Yo, V, n, prec)
    assert ok, rel
    if N >= 100:
        assert rel <= TOL[prec]


@pytest.mark.parametrize("prec", ALL)
def test_laplacian_mid_size(plans, prec):
    w = workloads.laplacian_1d(N=65_537, nrhs=8, offset=201)
    Y = _gpu(plans[16], w["d"], w["e"], w["V"], prec)
    Yo = _oracle(w["d"], w["e"], w["V"], 16)
    assert matrix.rel_err(Y, Yo) <= TOL[prec]


@pytest.fixture(scope="module")
def full_size():
    """The 1D Laplacian workload at full size: N = 2^20, 8 RHS, degree 16."""
    w = workloads.laplacian_1d()
    Yo = _oracle(w["d"], w["e"], w["V"], 16)
    return w, Yo


# the benchmark's settings for the binary32 + refinement path
BENCH_MIXED = dict(tol=1e-10, max_refine=1)


@pytest.mark.parametrize("prec", ALL)
def test_laplacian_full_size(plans, full_size, prec):
    """Full-size parity in the launch configuration the benchmark times."""
    w, Yo = full_size
    kw = BENCH_MIXED if prec == P.EXPM_MIXED_FP32 else {}
    Y = _gpu(plans[16], w["d"], w["e"], w["V"], prec, **kw)
    err = matrix.rel_err(Y, Yo)
    print(f"full-size rel err prec={prec}: {err:.3e}")
    assert err <= TOL[prec]


def test_host_buffers_match_device_buffers(plans):
    """Host (numpy) buffers are staged by the library; the result is bit-identical."""
    d, e, V = _random_tridiag(30_000, 4, 202)
    Yd = _gpu(plans[12], d, e, V, P.EXPM_FP64)
    Yh = np.empty_like(V)
    P.expm_apply_tridiag(plans[12], d, e, V, Yh)
    np.testing.assert_array_equal(Yh, Yd)


def test_complex_rhs_with_real_matrix(plans):
    """Complex V with real T: real and imaginary parts are independent columns."""
    d, e, V = _random_tridiag(5_000, 3, 203, complex_v=True)
    Y = _gpu(plans[16], d, e, V, P.EXPM_FP64)
    Yo = _oracle(d, e, V, 16)
    assert Y.dtype == np.complex128
    assert matrix.rel_err(Y, Yo) <= 1e-12


def test_time_and_shift(plans):
    """exp(tT)V ~ e^c R_n(tT - cI)V (Remark 3.2) with t != 1, c != 0."""
    d, e, V = _random_tridiag(10_000, 2, 204)
    d = d + 12.0                                       # spectrum now in (-4, 12)
    # c just above the largest eigenvalue of tT (< 6), as Remark 3.2 prescribes
    Y = _gpu(plans[16], d, e, V, P.EXPM_FP64, t=0.5, c=6.5)
    Yo = _oracle(d, e, V, 16, t=0.5, c=6.5)
    assert matrix.rel_err(Y, Yo) <= 1e-12


def test_nondefault_stream(plans):
    d, e, V = _random_tridiag(20_000, 2, 205)
    s = torch.cuda.Stream()
    dd, de, dv = (torch.from_numpy(x).to(DEV) for x in (d, e, V))
    dy = torch.empty_like(dv)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        P.expm_apply_tridiag(plans[12], dd, de, dv, dy)
    s.synchronize()
    assert matrix.rel_err(dy.cpu().numpy(), _oracle(d, e, V, 12)) <= 1e-12


def test_repeated_calls_are_deterministic(plans):
    d, e, V = _random_tridiag(40_000, 8, 206)
    a = _gpu(plans[16], d, e, V, P.EXPM_FP64)
    b = _gpu(plans[16], d, e, V, P.EXPM_FP64)
    np.testing.assert_array_equal(a, b)


def test_invalid_arguments(plans):
    d, e, V = _random_tridiag(100, 2, 207)
    dd, de, dv = (torch.from_numpy(x).to(DEV) for x in (d, e, V))
    dy = torch.empty_like(dv)
    with pytest.raises(P.ExpmError) as ei:             # r = 0
        P.expm_apply_tridiag(plans[12], dd, de, dv[:, :0], dy[:, :0])
    assert ei.value.status == 1                        # EXPM_EINVAL
    with pytest.raises(P.ExpmError) as ei:
        P.expm_apply_tridiag(plans[12], dd, de, dv, dy, prec=P.EXPM_MIXED_TF32X3)
    assert ei.value.status == 1                        # EXPM_EINVAL


# ------------------------------------------------------------------ binary32 + refinement

def _dev(d, e, V):
    dd, de, dv = (torch.from_numpy(np.ascontiguousarray(x)).to(DEV) for x in (d, e, V))
    return dd, de, dv, torch.empty_like(dv)


def test_mixed_refinement_info(plans):
    """The stopping test is met after at least one correction and reported in info."""
    d, e, V = _random_tridiag(60_000, 4, 208)
    dd, de, dv, dy = _dev(d, e, V)
    info = P.expm_apply_tridiag(plans[16], dd, de, dv, dy, prec=P.EXPM_MIXED_FP32, tol=1e-12, max_refine=4)
    assert info.status_worst == 0
    assert 1 <= info.refine_iters_max <= 4
    assert 0.0 <= info.resid_rel_max <= 1e-12
    assert matrix.rel_err(dy.cpu().numpy(), _oracle(d, e, V, 16)) <= 1e-10


def test_mixed_default_tolerance_is_tight(plans):
    """With the default tol (1e-14) the refined result is close to the binary64 floor."""
    w = workloads.laplacian_1d(N=30_011, nrhs=3, offset=209)
    Y = _gpu(plans[16], w["d"], w["e"], w["V"], P.EXPM_MIXED_FP32)
    assert matrix.rel_err(Y, _oracle(w["d"], w["e"], w["V"], 16)) <= 1e-11


def test_mixed_without_refinement_reports_enoconv(plans):
    """max_refine = 0 is the binary32 solve alone: its residual misses tol (EXPM_ENOCONV,
    left in info with check=False) and its error is binary32-sized."""
    d, e, V = _random_tridiag(20_000, 2, 210)
    dd, de, dv, dy = _dev(d, e, V)
    info = P.expm_apply_tridiag(plans[12], dd, de, dv, dy, prec=P.EXPM_MIXED_FP32, max_refine=0, check=False)
    assert info.status_worst == 4
    assert info.refine_iters_max == 0
    err = matrix.rel_err(dy.cpu().numpy(), _oracle(d, e, V, 12))
    assert 1e-9 < err < 1e-3
    with pytest.raises(P.ExpmError) as ei:
        P.expm_apply_tridiag(plans[12], dd, de, dv, dy, prec=P.EXPM_MIXED_FP32, max_refine=0)
    assert ei.value.status == 4


def test_mixed_early_stop(plans):
    """A loose tol is met by the binary32 solve: no correction pass runs."""
    d, e, V = _random_tridiag(20_000, 2, 211)
    dd, de, dv, dy = _dev(d, e, V)
    info = P.expm_apply_tridiag(plans[12], dd, de, dv, dy, prec=P.EXPM_MIXED_FP32, tol=1e-3, max_refine=3)
    assert info.status_worst == 0 and info.refine_iters_max == 0
    y0 = dy.clone()
    P.expm_apply_tridiag(plans[12], dd, de, dv, dy, prec=P.EXPM_MIXED_FP32, max_refine=0, check=False)
    assert torch.equal(dy, y0)


def test_mixed_async_and_skip_flag_give_identical_results(plans):
    """Without info the call stays asynchronous; skipping the final residual changes
    only the report.  All three runs produce bit-identical Y."""
    w = workloads.laplacian_1d(N=100_003, nrhs=8, offset=212)
    dd, de, dv, dy = _dev(w["d"], w["e"], w["V"])
    kw = dict(prec=P.EXPM_MIXED_FP32, tol=1e-10, max_refine=1)
    info = P.expm_apply_tridiag(plans[16], dd, de, dv, dy, **kw)
    ya = dy.clone()
    assert P.expm_apply_tridiag(plans[16], dd, de, dv, dy, want_info=False, **kw) is None
    torch.cuda.synchronize()
    yb = dy.clone()
    info2 = P.expm_apply_tridiag(plans[16], dd, de, dv, dy, flags=P.EXPM_FLAG_SKIP_FINAL_RESIDUAL, **kw)
    assert torch.equal(ya, yb) and torch.equal(ya, dy)
    assert info.refine_iters_max == 1 and info.resid_rel_max <= 1e-10
    assert info2.status_worst == 0 and info2.resid_rel_max > info.resid_rel_max   # residual before the last pass


def test_mixed_complex_rhs_time_shift(plans):
    """Complex V, t != 1 and c != 0 on the refined path."""
    d, e, V = _random_tridiag(12_000, 2, 213, complex_v=True)
    d = d + 12.0
    Y = _gpu(plans[16], d, e, V, P.EXPM_MIXED_FP32, t=0.5, c=6.5, tol=1e-12)
    assert matrix.rel_err(Y, _oracle(d, e, V, 16, t=0.5, c=6.5)) <= 1e-9


def test_mixed_invalid_options(plans):
    d, e, V = _random_tridiag(100, 2, 214)
    dd, de, dv, dy = _dev(d, e, V)
    for kw in (dict(max_refine=-1), dict(tol=-1.0), dict(flags=2)):
        with pytest.raises(P.ExpmError) as ei:
            P.expm_apply_tridiag(plans[12], dd, de, dv, dy, prec=P.EXPM_MIXED_FP32, **kw)
        assert ei.value.status == 1
    with pytest.raises(P.ExpmError) as ei:            # the flag belongs to the refined path only
        P.expm_apply_tridiag(plans[12], dd, de, dv, dy, flags=P.EXPM_FLAG_SKIP_FINAL_RESIDUAL)
    assert ei.value.status == 1


# ------------------------------------------------------------- complex Hermitian T

def _random_hermitian(N, r, seed, complex_v=False):
    """Complex off-diagonal e_i = |e_i| exp(i psi_i) with uniform phases (Gershgorin: the
    spectrum stays in (-16, 0) as for the real cases), a few exact zeros (T splits there),
    real negative and purely imaginary entries."""
    d, e_abs, V = _random_tridiag(N, r, seed, complex_v)
    g = workloads.rng(seed + 7)
    e = e_abs * np.exp(1j * g.uniform(0.0, 2 * np.pi, e_abs.shape))
    if N > 12:
        e[3] = 0.0
        e[5] = -e_abs[5]
        e[7] = 1j * e_abs[7]
        e[-1] = 0.0
    return d, e, V


@pytest.mark.parametrize("prec", ALL)
@pytest.mark.parametrize("N,r,n,cv", [(1, 1, 12, False), (2, 3, 16, True), (7, 2, 12, False), (433, 8, 16, True),
                                      (4096 + 13, 5, 12, False), (50_000, 8, 16, True), (200_003, 3, 12, False)])
def test_hermitian_tridiag_parity(plans, prec, N, r, n, cv):
    """Complex e: solved as the real symmetric D^H T D on D^H V (phases by a parallel prefix
    product over several scan blocks and a ragged tail), against the oracle's direct
    complex banded solves."""
    d, e, V = _random_hermitian(N, r, 230 + N + r, cv)
    Y = _gpu(plans[n], d, e, V, prec)     # N = 1: a complex-typed empty e, complex Y
    Yo = _oracle(d, e, V, n)
    assert Y.dtype == np.complex128
    ok, rel = _close(Y, Yo, V, n, prec)
    assert ok, rel
    if N >= 100:
        assert rel <= TOL[prec]


def test_hermitian_with_real_entries_is_the_real_path(plans):
    """A complex-typed e with real entries: every phase is exactly +-1, so the result is
    bit-identical to the real-off-diagonal path (positive e with the same data; negative
    e against |e| with the rows' signs flipped, rounding being sign-symmetric)."""
    d, e, V = _random_tridiag(30_001, 3, 240, complex_v=True)
    Yr = _gpu(plans[16], d, e, V, P.EXPM_FP64)
    Yc = _gpu(plans[16], d, e.astype(np.complex128), V, P.EXPM_FP64)
    np.testing.assert_array_equal(Yc, Yr)
    s = np.where(np.arange(30_001) % 2 == 0, 1.0, -1.0)   # D = diag(+-1): (D T D) has -e
    Yn = _gpu(plans[16], d, (-e).astype(np.complex128), V, P.EXPM_FP64)
    Yd = s[:, None] * _gpu(plans[16], d, e, s[:, None] * V, P.EXPM_FP64)
    np.testing.assert_array_equal(Yn, Yd)


@pytest.mark.parametrize("prec", ALL)
def test_hermitian_full_size_gauge_property(plans, full_size, prec):
    """The 1D Laplacian workload at full size (N = 2^20, 8 RHS, degree 16) under a random
    diagonal unitary gauge D0 = diag(exp(i psi)): T = D0 L D0^H has e_i = 100 exp(i(psi_i -
    psi_{i+1})) and exp(T)V = D0 exp(L) (D0^H V) exactly, so the complex-e result must
    equal D0 times the real path's result on D0^H V (the real path is checked against the
    oracle at this size by test_laplacian_full_size)."""
    w, _ = full_size
    g = workloads.rng(241)
    psi = g.uniform(0.0, 2 * np.pi, w["d"].shape[0])
    ph = np.exp(1j * psi)
    e = w["e"] * ph[:-1] * np.conj(ph[1:])
    V = w["V"] + 1j * g.standard_normal(w["V"].shape)
    Y = _gpu(plans[16], w["d"], e, V, prec)
    Yl = ph[:, None] * _gpu(plans[16], w["d"], w["e"], np.conj(ph)[:, None] * V, P.EXPM_FP64)
    assert matrix.rel_err(Y, Yl) <= TOL[prec]


def test_hermitian_host_buffers_time_shift_and_mixed_info(plans):
    """Host buffers (staged, complex e included), t and c, and the binary32 path's
    refinement report on a complex T."""
    d, e, V = _random_hermitian(40_000, 2, 242)
    d = d + 12.0
    Yd = _gpu(plans[16], d, e, V, P.EXPM_FP64, t=0.5, c=6.5)
    Yh = np.empty(V.shape, dtype=np.complex128)
    P.expm_apply_tridiag(plans[16], d, e, V, Yh, t=0.5, shift_c=6.5)
    np.testing.assert_array_equal(Yh, Yd)
    Yo = _oracle(d, e, V, 16, t=0.5, c=6.5)
    assert matrix.rel_err(Yd, Yo) <= 1e-12
    dd, de, dv = (torch.from_numpy(np.ascontiguousarray(x)).to(DEV) for x in (d, e, V))
    dy = torch.empty(V.shape, dtype=torch.complex128, device=DEV)
    info = P.expm_apply_tridiag(plans[16], dd, de, dv, dy, prec=P.EXPM_MIXED_FP32, t=0.5, shift_c=6.5)
    torch.cuda.synchronize()
    assert info.status_worst == 0 and info.refine_iters_max >= 1 and info.resid_rel_max <= 1e-12
    assert matrix.rel_err(dy.cpu().numpy(), Yo) <= 1e-8
