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
