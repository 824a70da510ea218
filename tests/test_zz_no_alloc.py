"""The allocation-free tridiagonal entry point, expm_apply_tridiag_noalloc.

It exists for callers that must not let the library allocate device memory -- a
serving process whose memory is reserved up front by another framework, or a
latency-critical loop where cudaMalloc/cudaFree (which may synchronise the device)
is not acceptable.  It runs the same kernels as expm_apply_tridiag with their
scratch in a fixed array inside the library.  These tests call it through the
C interface and compare it with expm_apply_tridiag on two calls in a row (the
second on different data, so nothing left in the shared array from the first
call can leak into the second).

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes when run alone in a fresh process.
"""

import numpy as np
import pytest

import workloads
from oracle import matrix

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2306_16778_gb300 as P  # noqa: E402

DEV = torch.device("cuda:0")
TOL = {P.EXPM_FP64: 1e-12, P.EXPM_MIXED_F32X2: 1e-8}   # the tridiagonal tests' tolerances


def _inputs(N, r, seed):
    g = workloads.rng(seed)
    d = g.uniform(-12.0, -4.0, N)
    e = g.uniform(0.5, 2.0, N - 1)
    V = g.standard_normal((N, r))
    return tuple(torch.from_numpy(x).to(DEV) for x in (d, e, V))


@pytest.mark.parametrize("prec", [P.EXPM_FP64, P.EXPM_MIXED_F32X2])
def test_noalloc_matches_allocating_entry_point_twice(prec):
    plan = P.Plan(degree=16)
    for call, (N, r, seed) in enumerate([(16_001, 8, 400), (9_001, 3, 401)]):
        d, e, V = _inputs(N, r, seed)
        Y_ref = torch.empty_like(V)
        P.expm_apply_tridiag(plan, d, e, V, Y_ref, prec=prec)
        Y = torch.full_like(V, float("nan"))
        P.expm_apply_tridiag_noalloc(plan, d, e, V, Y, prec=prec)
        torch.cuda.synchronize()
        err = matrix.rel_err(Y.cpu().numpy(), Y_ref.cpu().numpy())
        assert np.isfinite(err) and err <= TOL[prec], (call, err)
    plan.close()


def test_noalloc_rejects_oversized_problems_and_host_buffers():
    plan = P.Plan(degree=16)
    d, e, V = _inputs(1 << 20, 8, 402)           # needs far more than the fixed scratch
    Y = torch.empty_like(V)
    with pytest.raises(P.ExpmError) as ei:
        P.expm_apply_tridiag_noalloc(plan, d, e, V, Y)
    assert ei.value.status == 1 and "EXPM_NOALLOC_SCRATCH_BYTES" in str(ei.value)
    hd, he, hV = (x[:100].cpu().numpy() for x in (d, e, V))
    with pytest.raises(P.ExpmError) as ei:
        P.expm_apply_tridiag_noalloc(plan, hd, he[:99], hV, np.empty_like(hV))
    assert ei.value.status == 1
    plan.close()
