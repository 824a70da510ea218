"""The request server (expm_server_*): continuous batching of tridiagonal and dense
exp(tA)V requests.  Every result must equal the same computation done alone through
expm_apply_tridiag / expm_apply_dense (bit for bit: the kernels are deterministic and
nothing is reduced across requests) and match the oracle within the path's tolerance."""

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


def _wait(server, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for tk in tickets:
            if tk not in out:
                r = server.poll(tk)
                if r is not None:
                    out[tk] = r
        assert time.time() - t0 < timeout, "server did not finish in time"
        time.sleep(0.001)
    return out


def test_mixed_stream_same_alone_and_in_the_mix():
    g = workloads.rng(600)
    plans = {12: P.Plan(degree=12), 16: P.Plan(degree=16)}
    server = P.Server(hbm_budget_bytes=8 << 30, max_inflight=4)
    tri = []
    for N in (5000, 40_000, 120_001):
        w = workloads.laplacian_1d(N=N, nrhs=1, offset=600 + N)
        d, e = (torch.from_numpy(x).to(DEV) for x in (w["d"], w["e"]))
        tri.append((server.register_tridiag(d, e), d, e, w))
    den = []
    for n in (64, 200, 333):
        A, Q, mu, _ = workloads.dense_symmetric(n, -40.0, 0.0, 1, g, True)
        dA = torch.from_numpy(A).to(DEV)
        den.append((server.register_dense(dA), dA, A))
    reqs = []
    for i in range(24):
        deg = 12 if i % 2 else 16
        if i % 3 == 2:
            oid, dA, A = den[i % len(den)]
            V = torch.from_numpy(workloads.request_rhs(A.shape[0], 1 + i % 5, 700 + i, True)).to(DEV)
            prec = P.EXPM_MIXED_FP32 if i % 4 == 0 else P.EXPM_FP64
            reqs.append(("dense", oid, dA, None, V, deg, prec, A))
        else:
            oid, d, e, w = tri[i % len(tri)]
            V = torch.from_numpy(workloads.request_rhs(d.shape[0], 1 + i % 4, 700 + i, False)).to(DEV)
            prec = (P.EXPM_FP64, P.EXPM_MIXED_F32X2, P.EXPM_FP64, P.EXPM_MIXED_FP32)[i % 4]
            reqs.append(("tri", oid, d, e, V, deg, prec, w))
    outs = [torch.empty_like(r[4]) for r in reqs]
    torch.cuda.synchronize()
    tickets = [server.submit(r[1], plans[r[5]], r[4], y, prec=r[6]) for r, y in zip(reqs, outs)]
    results = _wait(server, tickets)
    for r, y, tk in zip(reqs, outs, tickets):
        st, info, ts = results[tk]
        assert st == 0, (st, r[0])
        assert ts[0] <= ts[1] <= ts[2] <= ts[3]
        alone = torch.empty_like(y)
        if r[0] == "tri":
            P.expm_apply_tridiag(plans[r[5]], r[2], r[3], r[4], alone, prec=r[6])
        else:
            P.expm_apply_dense(plans[r[5]], r[2], r[4], alone, prec=r[6])
        torch.cuda.synchronize()
        assert torch.equal(alone, y), r[0]
        th, a = coeffs.theta(r[5]), coeffs.residues(r[5])
        V = r[4].cpu().numpy()
        if r[0] == "tri":
            Yo, _ = matrix.apply_tridiag(r[7]["d"], r[7]["e"], V, th, a)
        else:
            Yo, _ = matrix.apply_dense(r[7], V, th, a)
        tol = 1e-12 if r[6] == P.EXPM_FP64 else 1e-8
        assert matrix.rel_err(y.cpu().numpy(), Yo) <= tol, (r[0], r[6])
    server.close()


def test_hermitian_tridiagonal_operator():
    """A tridiagonal operator with complex e (phases formed once at registration): each
    request equals the same call through expm_apply_tridiag bit for bit and matches the
    oracle's direct complex banded solves, for every tridiagonal precision and for real
    and complex V."""
    g = workloads.rng(610)
    N = 70_001
    d = g.uniform(-12.0, -4.0, N)
    e = g.uniform(0.5, 2.0, N - 1) * np.exp(1j * g.uniform(0.0, 2 * np.pi, N - 1))
    plan = P.Plan(degree=16)
    server = P.Server(hbm_budget_bytes=4 << 30, max_inflight=2)
    dd, de = (torch.from_numpy(x).to(DEV) for x in (d, e))
    oid = server.register_tridiag(dd, de)
    reqs = []
    for i, prec in enumerate((P.EXPM_FP64, P.EXPM_MIXED_F32X2, P.EXPM_MIXED_FP32, P.EXPM_FP64)):
        V = torch.from_numpy(workloads.request_rhs(N, 1 + i, 620 + i, i % 2 == 1)).to(DEV)
        Y = torch.empty(V.shape, dtype=torch.complex128, device=DEV)
        reqs.append((prec, V, Y))
    torch.cuda.synchronize()
    tickets = [server.submit(oid, plan, V, Y, prec=prec) for prec, V, Y in reqs]
    results = _wait(server, tickets)
    th, a = coeffs.theta(16), coeffs.residues(16)
    for (prec, V, Y), tk in zip(reqs, tickets):
        assert results[tk][0] == 0
        alone = torch.empty_like(Y)
        P.expm_apply_tridiag(plan, dd, de, V, alone, prec=prec)
        torch.cuda.synchronize()
        assert torch.equal(alone, Y), prec
        Yo, _ = matrix.apply_tridiag(d, e, V.cpu().numpy(), th, a)
        assert matrix.rel_err(Y.cpu().numpy(), Yo) <= (1e-12 if prec == P.EXPM_FP64 else 1e-8), prec
    server.close()


def test_narrow_and_wide_requests_on_one_dense_operator():
    """Requests of 3 and of 12 columns on one dense operator: the wide ones need the
    factor part with the diagonal-panel inverses, the narrow ones the plain one; each must
    equal the same computation done alone."""
    g = workloads.rng(640)
    plan = P.Plan(degree=16)
    server = P.Server(hbm_budget_bytes=8 << 30, max_inflight=2)
    A, Q, mu, _ = workloads.dense_symmetric(300, -40.0, 0.0, 1, g, True)
    dA = torch.from_numpy(A).to(DEV)
    oid = server.register_dense(dA)
    reqs = []
    for i, (k, prec) in enumerate([(3, P.EXPM_FP64), (12, P.EXPM_FP64), (12, P.EXPM_MIXED_FP32),
                                   (3, P.EXPM_MIXED_FP32), (12, P.EXPM_FP64), (3, P.EXPM_FP64)]):
        V = torch.from_numpy(workloads.request_rhs(300, k, 800 + i, True)).to(DEV)
        reqs.append((V, prec))
    outs = [torch.empty_like(V) for V, _ in reqs]
    torch.cuda.synchronize()
    tickets = [server.submit(oid, plan, V, y, prec=prec) for (V, prec), y in zip(reqs, outs)]
    results = _wait(server, tickets)
    th, a = coeffs.theta(16), coeffs.residues(16)
    for (V, prec), y, tk in zip(reqs, outs, tickets):
        assert results[tk][0] == 0
        alone = torch.empty_like(y)
        P.expm_apply_dense(plan, dA, V, alone, prec=prec)
        torch.cuda.synchronize()
        assert torch.equal(alone, y)
        Yo, _ = matrix.apply_dense(A, V.cpu().numpy(), th, a)
        assert matrix.rel_err(y.cpu().numpy(), Yo) <= (1e-12 if prec == P.EXPM_FP64 else 1e-8)
    server.close()


def test_server_rejections():
    server = P.Server(hbm_budget_bytes=1 << 20, max_inflight=1)
    plan = P.Plan(degree=16)
    w = workloads.laplacian_1d(N=100_000, nrhs=1, offset=650)
    d, e, V = (torch.from_numpy(x).to(DEV) for x in (w["d"], w["e"], w["V"]))
    oid = server.register_tridiag(d, e)
    with pytest.raises(P.ExpmError) as ei:           # needs far more than 1 MiB
        server.submit(oid, plan, V, torch.empty_like(V))
    assert ei.value.status == 2                       # EXPM_ENOMEM
    with pytest.raises(P.ExpmError) as ei:
        server.submit(oid + 99, plan, V, torch.empty_like(V))
    assert ei.value.status == 8                       # EXPM_ENOTFOUND
    st, _, _ = server.poll(12345)
    assert st == 8                                    # unknown ticket
    server.close()


def _tri_case(N, nrhs, offset):
    w = workloads.laplacian_1d(N=N, nrhs=nrhs, offset=offset)
    d, e, V = (torch.from_numpy(x).to(DEV) for x in (w["d"], w["e"], w["V"]))
    return w, d, e, V


def _oracle_tri(w, V, degree):
    Yo, _ = matrix.apply_tridiag(w["d"], w["e"], V.cpu().numpy(), coeffs.theta(degree), coeffs.residues(degree))
    return Yo


def test_plan_recreated_does_not_reuse_the_old_factorization():
    """A plan destroyed and one of another degree created (possibly at the same address):
    the cached factorization of the first must not serve the second (the cache is keyed
    by a plan id that is never reused)."""
    server = P.Server(hbm_budget_bytes=4 << 30, max_inflight=1)
    w, d, e, V = _tri_case(30_011, 2, 660)
    oid = server.register_tridiag(d, e)
    for prec in (P.EXPM_FP64, P.EXPM_MIXED_FP32):
        plan12 = P.Plan(degree=12)
        Y = torch.empty_like(V)
        st, _, _ = _wait(server, [tk := server.submit(oid, plan12, V, Y, prec=prec)])[tk]
        assert st == 0
        assert matrix.rel_err(Y.cpu().numpy(), _oracle_tri(w, V, 12)) <= 1e-8
        plan12.close()
        for _ in range(4):   # plans of another degree; allocations may land on the old address
            plan16 = P.Plan(degree=16)
            Y = torch.empty_like(V)
            st, _, _ = _wait(server, [tk := server.submit(oid, plan16, V, Y, prec=prec)])[tk]
            assert st == 0
            assert matrix.rel_err(Y.cpu().numpy(), _oracle_tri(w, V, 16)) <= 1e-8
            plan16.close()
    server.close()


def test_submit_rejects_host_buffers():
    server = P.Server(hbm_budget_bytes=1 << 30, max_inflight=1)
    plan = P.Plan(degree=12)
    w, d, e, V = _tri_case(1000, 1, 661)
    oid = server.register_tridiag(d, e)
    hV = V.cpu()
    for args in ((hV, torch.empty_like(V)), (V, torch.empty_like(hV))):
        with pytest.raises(P.ExpmError) as ei:
            server.submit(oid, plan, *args)
        assert ei.value.status == 1                   # EXPM_EINVAL
    server.close()


def test_full_queue_returns_eagain():
    """One worker busy with a long request and a queue limit of 1: a submit that finds the
    queue full returns EXPM_EAGAIN and queues nothing; accepted requests still complete,
    and the rejected one succeeds when retried."""
    server = P.Server(hbm_budget_bytes=8 << 30, max_inflight=1)
    server.set_queue_limit(1)
    with pytest.raises(P.ExpmError):
        server.set_queue_limit(0)
    plan = P.Plan(degree=16)
    g = workloads.rng(662)
    A, _, _, _ = workloads.dense_symmetric(1536, -40.0, 0.0, 1, g, True)
    dA = torch.from_numpy(A).to(DEV)
    big = server.register_dense(dA)
    Vb = torch.from_numpy(workloads.request_rhs(1536, 64, 663, True)).to(DEV)
    w, d, e, V = _tri_case(2000, 1, 664)
    small = server.register_tridiag(d, e)
    torch.cuda.synchronize()
    accepted, rejected = [], 0
    outs = []
    for i in range(6):   # the first keeps the worker busy for far longer than these submits take
        op, VV = (big, Vb) if i == 0 else (small, V)
        Y = torch.empty_like(VV)
        try:
            accepted.append(server.submit(op, plan, VV, Y))
            outs.append(Y)
        except P.ExpmError as ex:
            assert ex.status == 6                     # EXPM_EAGAIN
            rejected += 1
    assert rejected >= 1 and len(accepted) <= 3
    res = _wait(server, accepted)
    assert all(r[0] == 0 for r in res.values())
    Y = torch.empty_like(V)
    st, _, _ = _wait(server, [tk := server.submit(small, plan, V, Y)])[tk]
    assert st == 0 and matrix.rel_err(Y.cpu().numpy(), _oracle_tri(w, V, 16)) <= 1e-12
    server.close()


def test_failed_factor_build_is_dropped_and_rebuilt():
    """A factor build reported as failed (host-side fault injection) fails its request
    with EXPM_ECUDA; the entry is dropped once unused, so the next request on the same
    operator rebuilds it and succeeds."""
    server = P.Server(hbm_budget_bytes=4 << 30, max_inflight=2)
    plan = P.Plan(degree=16)
    w, d, e, V = _tri_case(20_000, 2, 665)
    oid = server.register_tridiag(d, e)
    for prec in (P.EXPM_FP64, P.EXPM_MIXED_FP32):
        assert P.lib.expm_internal_server_fail_next_factor(server._h) == 0
        Y = torch.empty_like(V)
        st, _, _ = _wait(server, [tk := server.submit(oid, plan, V, Y, prec=prec)])[tk]
        assert st == 7                                # EXPM_ECUDA
        for _ in range(2):
            Y = torch.empty_like(V)
            st, _, _ = _wait(server, [tk := server.submit(oid, plan, V, Y, prec=prec)])[tk]
            assert st == 0
            assert matrix.rel_err(Y.cpu().numpy(), _oracle_tri(w, V, 16)) <= 1e-8
    server.close()


def test_stopped_worker_is_restarted_and_queued_requests_complete():
    """Workers made to leave their loop between requests (host-side fault injection) are
    restarted by the next submit or poll; every queued request completes correctly."""
    server = P.Server(hbm_budget_bytes=4 << 30, max_inflight=2)
    plan = P.Plan(degree=12)
    w, d, e, V = _tri_case(50_000, 3, 666)
    oid = server.register_tridiag(d, e)
    for idx in (0, 1):
        assert P.lib.expm_internal_server_stop_worker(server._h, idx) == 0
    t0 = time.time()
    while P.lib.expm_internal_server_workers_alive(server._h) > 0:
        assert time.time() - t0 < 30
        time.sleep(0.01)
    outs = [torch.empty_like(V) for _ in range(6)]
    tickets = [server.submit(oid, plan, V, Y) for Y in outs]     # the first submit restarts them
    assert P.lib.expm_internal_server_workers_alive(server._h) == 2
    res = _wait(server, tickets)
    Yo = _oracle_tri(w, V, 12)
    for tk, Y in zip(tickets, outs):
        assert res[tk][0] == 0
        assert matrix.rel_err(Y.cpu().numpy(), Yo) <= 1e-12
    server.close()
