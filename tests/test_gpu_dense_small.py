"""The one-launch small dense path (n <= 64, at most 4 right-hand-side columns, at most
16 solved systems): one thread-block cluster, one CTA per solved system, the residue
sum reduced over the cluster's shared memory.  Checked against the oracle (pivoted
LAPACK solves per pole), the eigen closed form of R_n(A)V, and the blocked batched path
(different kernels) on the same inputs."""

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
TOL = {P.EXPM_FP64: 1e-12, P.EXPM_MIXED_FP32: 1e-10, P.EXPM_MIXED_BF16X3: 1e-10}


@pytest.fixture(scope="module")
def plans():
    return {n: P.Plan(degree=n) for n in (12, 16)}


def _floor(V, deg, unit=2.0 ** -53):
    """The partial-fraction rounding floor (Sec. 4) used by the dense tests."""
    th, a = coeffs.theta(deg), coeffs.residues(deg)
    return 64 * unit * float(np.sum(np.abs(a) / np.abs(th.imag))) * np.linalg.norm(V)


def _run(plan, A, V, prec, **kw):
    dA, dV = (torch.from_numpy(np.ascontiguousarray(x)).to(DEV) for x in (A, V))
    cplx = np.iscomplexobj(A) or np.iscomplexobj(V)
    dY = torch.empty(V.shape, dtype=torch.complex128 if cplx else torch.float64, device=DEV)
    info = P.expm_apply_dense(plan, dA, dV, dY, prec=prec, **kw)
    torch.cuda.synchronize()
    return dY.cpu().numpy(), info


@pytest.mark.parametrize("prec", [P.EXPM_FP64, P.EXPM_MIXED_FP32, P.EXPM_MIXED_BF16X3])
@pytest.mark.parametrize("n,k,deg,cplx", [(1, 1, 12, False), (2, 4, 16, True), (17, 3, 12, True),
                                          (32, 1, 16, False), (33, 2, 16, True), (64, 4, 16, True),
                                          (64, 1, 12, False), (48, 4, 12, False), (31, 2, 12, True),
                                          (63, 1, 16, False)])
def test_small_against_oracle_and_closed_form(plans, prec, n, k, deg, cplx):
    g = workloads.rng(1200 + n + 10 * k + deg)
    A, Q, mu, V = workloads.dense_symmetric(n, -30.0, 0.0, k, g, cplx)
    Y, info = _run(plans[deg], A, V, prec)
    Yo, _ = matrix.apply_dense(A, V, coeffs.theta(deg), coeffs.residues(deg))
    Ye = matrix.eig_apply(Q, mu, V, lambda m: scalar.R_n(m, deg))
    for ref in (Yo, Ye):
        assert np.linalg.norm(Y - ref) <= TOL[prec] * np.linalg.norm(ref) + _floor(V, deg), matrix.rel_err(Y, ref)
    assert 0.0 < info.growth_max_seen < 1e3
    if prec != P.EXPM_FP64:
        assert info.refine_iters_max >= 1 and info.resid_rel_max <= 1e-14


@pytest.mark.parametrize("prec", [P.EXPM_FP64, P.EXPM_MIXED_FP32])
def test_small_time_shift_and_complex_rhs_with_real_matrix(plans, prec):
    """t and c (Remark 3.2's shift) on a spectrum with positive eigenvalues, and a complex V
    with real symmetric A (its real and imaginary parts are separate real columns)."""
    g = workloads.rng(1250)
    A, Q, mu, V = workloads.dense_symmetric(40, -5.0, 8.0, 2, g, False)
    Vc = V + 1j * g.standard_normal(V.shape)
    t, c = 0.75, 6.0
    Y, _ = _run(plans[16], A, Vc, prec, t=t, shift_c=c)
    Yo, _ = matrix.apply_dense(A, Vc, coeffs.theta(16), coeffs.residues(16), t=t, c=c)
    assert Y.dtype == np.complex128
    assert matrix.rel_err(Y, Yo) <= TOL[prec]


@pytest.mark.parametrize("prec", [P.EXPM_FP64, P.EXPM_MIXED_FP32])
def test_small_matches_blocked_batched_path(plans, prec):
    """The same problem through expm_apply_batched (blocked kernels, one instance)."""
    g = workloads.rng(1260)
    A, Q, mu, V = workloads.dense_symmetric(61, -20.0, 0.0, 1, g, True)
    Y, _ = _run(plans[12], A, V, prec)
    dA, dV = (torch.from_numpy(x).to(DEV) for x in (A, V))
    dY = torch.empty_like(dV)
    P.expm_apply_batched(plans[12], [dA], [dV], [dY], prec=prec)
    torch.cuda.synchronize()
    assert matrix.rel_err(Y, dY.cpu().numpy()) <= TOL[prec]


def test_small_statuses(plans):
    g = workloads.rng(1270)
    A, Q, mu, V = workloads.dense_symmetric(24, -10.0, 0.0, 1, g, True)
    _, info = _run(plans[12], A, V, P.EXPM_MIXED_FP32, max_refine=0, tol=1e-15, check=False)
    assert info.status_worst == 4 and info.refine_iters_max == 0   # EXPM_ENOCONV
    Y, info = _run(plans[12], A, V, P.EXPM_FP64, growth_max=0.5, check=False)
    assert info.status_worst == 3 and info.growth_max_seen >= 0.5  # EXPM_EGROWTH, Y still written
    Yo, _ = matrix.apply_dense(A, V, coeffs.theta(12), coeffs.residues(12))
    assert matrix.rel_err(Y, Yo) <= 1e-12


@pytest.mark.parametrize("prec", [P.EXPM_FP64, P.EXPM_MIXED_FP32])
@pytest.mark.parametrize("n,k,cplx", [(64, 1, False), (37, 3, True)])
def test_small_captured_graph(plans, prec, n, k, cplx):
    """A batch graph of one small instance is the one-launch kernel on the caller's buffers:
    replays agree with the oracle, report the sweeps and growth, and follow new data in
    the same buffers."""
    g = workloads.rng(1280 + n)
    A, Q, mu, V = workloads.dense_symmetric(n, -20.0, 0.0, k, g, cplx)
    dA, dV = (torch.from_numpy(x).to(DEV) for x in (A, V))
    dY = torch.empty_like(dV)
    gr = P.BatchGraph(plans[12], [dA], [dV], [dY], prec=prec, scheme=-1)
    assert gr.info()["launch_groups"] == 1 and gr.buckets() == []
    for rep in range(2):
        infos = gr.replay(want_info=True)
        torch.cuda.synchronize()
        Yo, _ = matrix.apply_dense(A, V, coeffs.theta(12), coeffs.residues(12))
        assert matrix.rel_err(dY.cpu().numpy(), Yo) <= TOL[prec]
        assert infos[0].status_worst == 0 and 0.0 < infos[0].growth_max_seen < 1e3
        if prec != P.EXPM_FP64:
            assert infos[0].refine_iters_max >= 1 and infos[0].resid_rel_max <= 1e-14
        Vr = workloads.rng(1290 + rep).standard_normal(V.shape)
        V = Vr + 1j * workloads.rng(1295 + rep).standard_normal(V.shape) if cplx else Vr
        dV.copy_(torch.from_numpy(V))   # the graph reads the same buffer
    gr.close()


def test_small_captured_graph_growth_status(plans):
    g = workloads.rng(1300)
    A, Q, mu, V = workloads.dense_symmetric(16, -10.0, 0.0, 1, g, True)
    dA, dV = (torch.from_numpy(x).to(DEV) for x in (A, V))
    dY = torch.empty_like(dV)
    gr = P.BatchGraph(plans[12], [dA], [dV], [dY], prec=P.EXPM_FP64, scheme=0, growth_max=0.5)
    infos = gr.replay(want_info=True, check=False)
    assert infos[0].status_worst == 3        # EXPM_EGROWTH, Y still written
    Yo, _ = matrix.apply_dense(A, V, coeffs.theta(12), coeffs.residues(12))
    assert matrix.rel_err(dY.cpu().numpy(), Yo) <= 1e-12
    gr.close()
