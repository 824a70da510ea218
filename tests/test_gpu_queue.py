"""The device-fed work queue of small dense evaluations (expm_queue_*): a persistent
cluster kernel takes requests published in mapped host memory.  Each result must agree
with expm_apply_dense on the same inputs to rounding (the same evaluation as the one-launch
kernel, compiled into another kernel) and match the oracle; the bounded idle wait must end the kernel with
EXPM_ETIMEOUT and a later submit must start it again; the ring's capacity, ticket release
and the growth / convergence statuses behave as documented."""

import time

import numpy as np
import pytest

import workloads
from oracle import coeffs, matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2306_16778_gb300 as P  # noqa: E402

DEV = torch.device("cuda:0")
TOL = {P.EXPM_FP64: 1e-12, P.EXPM_MIXED_FP32: 1e-10}


def _wait(q, tickets, timeout=60.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for tk in tickets:
            if tk not in out:
                r = q.poll(tk)
                if r is not None:
                    out[tk] = r
        assert time.time() - t0 < timeout, "queue did not finish in time"
    return out


def _floor(V, deg, unit=2.0 ** -53):
    """The partial-fraction rounding floor (Sec. 4) of the dense tests: where R_n(tA - cI)V
    is tiny next to V (n = 1, a far negative eigenvalue) relative error means nothing."""
    th, a = coeffs.theta(deg), coeffs.residues(deg)
    return 64 * unit * float(np.sum(np.abs(a) / np.abs(th.imag))) * np.linalg.norm(V)


def _case(n, k, seed, complex_a, complex_v):
    g = workloads.rng(seed)
    A, Q, mu, V = workloads.dense_symmetric(n, -20.0, 0.0, k, g, complex_a)
    if complex_v and not complex_a:
        V = V + 1j * g.standard_normal(V.shape)
    return A, V


@pytest.mark.parametrize("prec", [P.EXPM_FP64, P.EXPM_MIXED_FP32])
@pytest.mark.parametrize("complex_a,complex_v,k,deg", [(False, False, 1, 12), (True, True, 2, 16),
                                                       (False, True, 2, 12), (True, True, 4, 8)])
def test_queue_equals_direct_call_and_oracle(prec, complex_a, complex_v, k, deg):
    """Requests of many orders (1..64, ragged), times and shifts, in flight together:
    equal to expm_apply_dense to rounding and within the tolerance of the oracle."""
    plan = P.Plan(degree=deg)
    q = P.Queue(plan, a_is_complex=complex_a, k=k, v_is_complex=complex_v, prec=prec, capacity=64)
    reqs = []
    for i, n in enumerate((64, 1, 37, 64, 2, 63, 17, 48, 64, 31, 5, 64)):
        A, V = _case(n, k, 1500 + 10 * i + deg, complex_a, complex_v)
        dA, dV = (torch.from_numpy(np.ascontiguousarray(x)).to(DEV) for x in (A, V))
        dY = torch.empty(V.shape, dtype=torch.complex128 if (complex_a or complex_v) else torch.float64, device=DEV)
        t, c = (1.0, 0.0) if i % 3 else (0.7, 1.5)
        reqs.append((A, V, dA, dV, dY, t, c))
    torch.cuda.current_stream().synchronize()
    tickets = [q.submit(dA, dV, dY, t=t, shift_c=c) for _, _, dA, dV, dY, t, c in reqs]
    res = _wait(q, tickets)
    th, a = coeffs.theta(deg), coeffs.residues(deg)
    for (A, V, dA, dV, dY, t, c), tk in zip(reqs, tickets):
        st, info = res[tk]
        assert st == 0 and 0.0 < info.growth_max_seen < 1e3
        if prec != P.EXPM_FP64:
            assert info.refine_iters_max >= 1 and info.resid_rel_max <= 1e-14
        alone = torch.empty_like(dY)
        P.expm_apply_dense(plan, dA, dV, alone, prec=prec, t=t, shift_c=c)
        torch.cuda.current_stream().synchronize()
        fl = np.exp(c) * _floor(V, deg)
        d = np.linalg.norm(dY.cpu().numpy() - alone.cpu().numpy())
        assert d <= 1e-13 * np.linalg.norm(alone.cpu().numpy()) + fl, matrix.rel_err(dY.cpu().numpy(), alone.cpu().numpy())
        Yo, _ = matrix.apply_dense(A, V, th, a, t=t, c=c)
        err = np.linalg.norm(dY.cpu().numpy() - Yo)
        assert err <= TOL[prec] * np.linalg.norm(Yo) + fl, matrix.rel_err(dY.cpu().numpy(), Yo)
    q.close()
    plan.close()


def test_queue_idle_timeout_and_restart():
    """No request for idle_ms: the bounded wait ends the kernel with EXPM_ETIMEOUT and the
    context stays usable; the next submit launches it again and the request completes."""
    plan = P.Plan(degree=12)
    q = P.Queue(plan, k=1, prec=P.EXPM_MIXED_FP32, idle_ms=20.0, max_clusters=2)
    A, V = _case(40, 1, 1600, False, False)
    dA, dV = (torch.from_numpy(x).to(DEV) for x in (A, V))
    Y1, Y2 = torch.empty_like(dV), torch.empty_like(dV)
    tk = q.submit(dA, dV, Y1)
    assert _wait(q, [tk])[tk][0] == 0
    t0 = time.time()
    while q.state()["running"]:
        assert time.time() - t0 < 10.0, "the idle wait did not end"
        time.sleep(0.005)
    s = q.state()
    assert s["last_exit"] == 5 and s["launches"] == 1 and s["clusters"] == 2   # EXPM_ETIMEOUT
    x = torch.ones(4, device=DEV) * 2                                          # context still usable
    assert float(x.sum()) == 8.0
    tk = q.submit(dA, dV, Y2)
    assert _wait(q, [tk])[tk][0] == 0
    assert q.state()["launches"] == 2
    assert torch.equal(Y1, Y2)
    q.close()


def test_queue_capacity_release_and_statuses():
    """capacity unpolled requests fill the ring (EXPM_EAGAIN); polling one frees a slot; a
    polled ticket is released (EXPM_ENOTFOUND); growth and convergence statuses."""
    plan = P.Plan(degree=12)
    A, V = _case(24, 1, 1700, True, True)
    dA, dV = (torch.from_numpy(x).to(DEV) for x in (A, V))
    q = P.Queue(plan, a_is_complex=True, k=1, v_is_complex=True, prec=P.EXPM_FP64, capacity=3)
    outs = [torch.empty_like(dV) for _ in range(4)]
    tks = [q.submit(dA, dV, outs[i]) for i in range(3)]
    assert all(t is not None for t in tks)
    assert q.submit(dA, dV, outs[3]) is None                       # ring full
    res = _wait(q, tks[:1])
    assert res[tks[0]][0] == 0
    with pytest.raises(P.ExpmError) as ei:
        q.poll(tks[0])
    assert ei.value.status == 8                                     # EXPM_ENOTFOUND: released
    t4 = q.submit(dA, dV, outs[3])
    assert t4 is not None
    _wait(q, tks[1:] + [t4])
    for y in outs[1:]:
        assert torch.equal(y, outs[0])
    q.close()
    qg = P.Queue(plan, a_is_complex=True, k=1, v_is_complex=True, prec=P.EXPM_FP64, growth_max=0.5)
    st, info = _wait(qg, [tk := qg.submit(dA, dV, outs[0])])[tk]
    assert st == 3 and info.growth_max_seen >= 0.5                  # EXPM_EGROWTH, Y written
    Yo, _ = matrix.apply_dense(A, V, coeffs.theta(12), coeffs.residues(12))
    assert matrix.rel_err(outs[0].cpu().numpy(), Yo) <= 1e-12
    qg.close()
    qc = P.Queue(plan, a_is_complex=True, k=1, v_is_complex=True, prec=P.EXPM_MIXED_FP32, max_refine=0, tol=1e-15)
    st, info = _wait(qc, [tk := qc.submit(dA, dV, outs[0])])[tk]
    assert st == 4 and info.refine_iters_max == 0                   # EXPM_ENOCONV
    qc.close()


def test_queue_rejections_and_destroy_with_pending_requests():
    plan = P.Plan(degree=12)
    with pytest.raises(P.ExpmError) as ei:
        P.Queue(plan, k=5)                                          # more than 4 columns
    assert ei.value.status == 1
    with pytest.raises(P.ExpmError) as ei:
        P.Queue(P.Plan(degree=40), k=1)                             # 20 systems > 16
    assert ei.value.status == 1
    q = P.Queue(plan, k=1, max_clusters=1, idle_ms=5000.0)
    A, V = _case(64, 1, 1800, False, False)
    dA, dV = (torch.from_numpy(x).to(DEV) for x in (A, V))
    with pytest.raises(P.ExpmError) as ei:                          # host buffers
        q.submit(A, V, np.empty_like(V))
    assert ei.value.status == 1
    big = torch.zeros(65, 65, dtype=torch.float64, device=DEV)
    with pytest.raises(P.ExpmError) as ei:                          # n > 64
        q.submit(big, torch.zeros(65, 1, dtype=torch.float64, device=DEV),
                 torch.zeros(65, 1, dtype=torch.float64, device=DEV))
    assert ei.value.status == 1
    outs = [torch.empty_like(dV) for _ in range(20)]
    for y in outs:
        assert q.submit(dA, dV, y) is not None
    t0 = time.time()
    q.close()                                                       # stop: returns without waiting for idle
    assert time.time() - t0 < 4.0
    x = torch.ones(4, device=DEV)
    assert float(x.sum()) == 4.0
