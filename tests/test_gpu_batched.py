"""GPU parity of expm_apply_batched (many dense Hermitian instances of uneven size)
against the oracle, through the C-ABI.  Tolerances: 1e-12 (binary64), 1e-8 for the
mixed path (the batched mixed-path tolerance)."""

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


def _close(Y, Yo, V, n, tol, unit=2.0 ** -53):
    th, a = coeffs.theta(n), coeffs.residues(n)
    floor = 64 * unit * float(np.sum(np.abs(a) / np.abs(th.imag))) * np.linalg.norm(V)
    return np.linalg.norm(Y - Yo) <= tol * np.linalg.norm(Yo) + floor


@pytest.mark.parametrize("prec,tol", [(P.EXPM_FP64, 1e-12), (P.EXPM_MIXED_FP32, 1e-8)])
def test_uneven_batch_parity(prec, tol):
    """Sizes log-uniform in [32, 300], several buckets, ragged sizes, k up to 3."""
    g = workloads.rng(500)
    sizes = list(workloads.batch_sizes(24, g, 5, 300)) + [1, 33, 64, 65]
    inst = []
    for i, n in enumerate(sizes):
        A, Q, mu, V = workloads.dense_symmetric(int(n), -30.0, 0.0, 1 + i % 3, g, True)
        inst.append((A, V))
    plan = P.Plan(degree=12)
    As = [torch.from_numpy(A).to(DEV) for A, _ in inst]
    Vs = [torch.from_numpy(V).to(DEV) for _, V in inst]
    Ys = [torch.empty_like(v) for v in Vs]
    infos = P.expm_apply_batched(plan, As, Vs, Ys, prec=prec, check=False)
    torch.cuda.synchronize()
    th, a = coeffs.theta(12), coeffs.residues(12)
    report = [(A.shape[0], V.shape[1], i.refine_iters_max, i.resid_rel_max, i.growth_max_seen, i.status_worst)
              for (A, V), i in zip(inst, infos)]
    for (A, V), Y, info in zip(inst, Ys, infos):
        Yo, _ = matrix.apply_dense(A, V, th, a)
        assert _close(Y.cpu().numpy(), Yo, V, 12, tol), (A.shape, matrix.rel_err(Y.cpu().numpy(), Yo), report)
    assert all(r[-1] == 0 for r in report), report


def test_batched_equals_single_calls():
    """Each instance of a batch matches expm_apply_dense on it alone (padding is exact)."""
    g = workloads.rng(501)
    plan = P.Plan(degree=16)
    inst = [workloads.dense_symmetric(n, -20.0, 0.0, 2, g, False)[::3] for n in (40, 70, 100)]
    As = [torch.from_numpy(A).to(DEV) for A, _ in inst]
    Vs = [torch.from_numpy(V).to(DEV) for _, V in inst]
    Ys = [torch.empty_like(v) for v in Vs]
    P.expm_apply_batched(plan, As, Vs, Ys)
    for A, V, Y in zip(As, Vs, Ys):
        Y1 = torch.empty_like(V)
        P.expm_apply_dense(plan, A, V, Y1)
        torch.cuda.synchronize()
        assert matrix.rel_err(Y.cpu().numpy(), Y1.cpu().numpy()) <= 1e-13


# ------------------------------------------------------------------ captured graph

def _batch(seed, count, lo, hi, complex_=True, kmax=3):
    g = workloads.rng(seed)
    sizes = list(workloads.batch_sizes(count, g, lo, hi)) + [1, 33]
    inst = [workloads.dense_symmetric(int(n), -30.0, 0.0, 1 + i % kmax, g, complex_) for i, n in enumerate(sizes)]
    As = [torch.from_numpy(A).to(DEV) for A, _, _, _ in inst]
    Vs = [torch.from_numpy(V).to(DEV) for _, _, _, V in inst]
    return inst, As, Vs


@pytest.mark.parametrize("prec", [P.EXPM_FP64, P.EXPM_MIXED_FP32])
def test_graph_replay_equals_batched_call(prec):
    """With the default bucket scheme the captured graph performs the same launches, the
    refinement decided on the device instead of the host: bit-identical results and the
    same per-instance reports (sweeps, growth, status; residual norms to rounding)."""
    inst, As, Vs = _batch(510, 30, 8, 400)
    plan = P.Plan(degree=12)
    Ya = [torch.empty_like(v) for v in Vs]
    ia = P.expm_apply_batched(plan, As, Vs, Ya, prec=prec)
    Yg = [torch.empty_like(v) for v in Vs]
    gr = P.BatchGraph(plan, As, Vs, Yg, prec=prec, scheme=0)
    for y in Yg:
        y.zero_()
    ig = gr.replay(want_info=True)
    torch.cuda.synchronize()
    for a, b in zip(Ya, Yg):
        assert torch.equal(a, b)
    for a, b in zip(ia, ig):
        # the residual norms are sums taken with atomics: equal up to their last bits
        assert (a.refine_iters_max, a.growth_max_seen, a.status_worst) == \
               (b.refine_iters_max, b.growth_max_seen, b.status_worst)
        assert abs(a.resid_rel_max - b.resid_rel_max) <= 1e-12 * max(a.resid_rel_max, 1e-300)
    gr.close()


def test_graph_replay_reads_new_data():
    """The graph reads the instance buffers at every launch: new V, new result."""
    inst, As, Vs = _batch(511, 20, 16, 300)
    plan = P.Plan(degree=12)
    Yg = [torch.empty_like(v) for v in Vs]
    gr = P.BatchGraph(plan, As, Vs, Yg, prec=P.EXPM_MIXED_FP32, scheme=1)
    g = workloads.rng(512)
    for v in Vs:
        v.copy_(torch.from_numpy(workloads.complex_normal(tuple(v.shape), g)))
    gr.replay()
    torch.cuda.synchronize()
    th, a = coeffs.theta(12), coeffs.residues(12)
    for (A, _, _, _), V, Y in zip(inst, Vs, Yg):
        Vh = V.cpu().numpy()
        Yo, _ = matrix.apply_dense(A, Vh, th, a)
        assert _close(Y.cpu().numpy(), Yo, Vh, 12, 1e-8)
    gr.close()


def test_graph_autotune():
    """scheme = -1 captures and times all three bucket schemes and keeps the fastest."""
    inst, As, Vs = _batch(513, 40, 16, 500, kmax=1)
    plan = P.Plan(degree=12)
    Yg = [torch.empty_like(v) for v in Vs]
    gr = P.BatchGraph(plan, As, Vs, Yg, prec=P.EXPM_MIXED_FP32, scheme=-1)
    info = gr.info()
    assert info["scheme"] in (0, 1, 2)
    assert all(ms > 0 for ms in info["ms_per_scheme"])
    assert info["ms_per_scheme"][info["scheme"]] == min(info["ms_per_scheme"])
    # every bucket (all factorised on the FP32 pipe here) timed both trailing-update tile
    # shapes and kept the faster; the groups cover every instance once
    bk = gr.buckets()
    assert len(bk) == info["launch_groups"] and sum(b["ninst"] for b in bk) == len(inst)
    sizes = sorted(A.shape[0] for A, _, _, _ in inst)
    assert max(b["order"] for b in bk) >= sizes[-1]
    for b in bk:
        m0, m1 = b["ms_tile"]
        assert m0 > 0 and m1 > 0 and b["tile"] == (1 if m1 < m0 else 0)
    infos = gr.replay(want_info=True)
    assert all(i.status_worst == 0 for i in infos)
    th, a = coeffs.theta(12), coeffs.residues(12)
    for (A, _, _, V), Y in zip(inst, Yg):
        Yo, _ = matrix.apply_dense(A, V, th, a)
        assert _close(Y.cpu().numpy(), Yo, V, 12, 1e-8)
    gr.close()


def test_graph_rejections():
    plan = P.Plan(degree=12)
    A = torch.eye(10, dtype=torch.complex128, device=DEV)
    V = torch.ones(10, 9, dtype=torch.complex128, device=DEV)
    with pytest.raises(P.ExpmError) as ei:                      # more than 8 columns
        P.BatchGraph(plan, [A], [V], [torch.empty_like(V)], scheme=0)
    assert ei.value.status == 1
    V = torch.ones(10, 1, dtype=torch.complex128, device=DEV)
    with pytest.raises(P.ExpmError) as ei:                      # unknown scheme
        P.BatchGraph(plan, [A], [V], [torch.empty_like(V)], scheme=3)
    assert ei.value.status == 1


@pytest.mark.parametrize("prec", [P.EXPM_MIXED_TF32X3, P.EXPM_MIXED_BF16X3])
def test_tensor_core_buckets(prec):
    """Buckets of padded order above 256 take the LU's trailing updates to the tensor cores
    (the smaller ones stay on the FP32 pipe), through the direct call and the captured
    graph: every instance within the mixed tolerance of the oracle, all statuses clean."""
    inst, As, Vs = _batch(520, 6, 200, 700, kmax=2)
    sizes = [A.shape[0] for A, _, _, _ in inst]
    assert any(n > 256 for n in sizes) and any(n <= 256 for n in sizes)
    plan = P.Plan(degree=12)
    th, a = coeffs.theta(12), coeffs.residues(12)
    Ya = [torch.empty_like(v) for v in Vs]
    ia = P.expm_apply_batched(plan, As, Vs, Ya, prec=prec)
    assert all(i.status_worst == 0 for i in ia)
    Yg = [torch.empty_like(v) for v in Vs]
    gr = P.BatchGraph(plan, As, Vs, Yg, prec=prec, scheme=0)
    # no tuning without autotuning: every group keeps the default shape, untimed
    assert all(b["tile"] == 0 and b["ms_tile"] == (-1.0, -1.0) for b in gr.buckets())
    ig = gr.replay(want_info=True)
    torch.cuda.synchronize()
    assert all(i.status_worst == 0 for i in ig)
    for (A, _, _, V), y1, y2 in zip(inst, Ya, Yg):
        Yo, _ = matrix.apply_dense(A, V, th, a)
        assert _close(y1.cpu().numpy(), Yo, V, 12, 1e-8)
        assert _close(y2.cpu().numpy(), Yo, V, 12, 1e-8)
    gr.close()
