"""The allocation-free tridiagonal entry point, expm_apply_tridiag_noalloc.

It exists for callers that must not let the library allocate device memory -- a
serving process whose memory is reserved up front by another framework, or a
latency-critical loop where cudaMalloc/cudaFree (which may synchronise the device)
is not acceptable.  It runs the same kernels as expm_apply_tridiag with their
scratch in a fixed array inside the library.  These tests call it through the
C interface and check it on two calls in a row (the second on different data, so
nothing left in the shared array from the first call can leak into the second):
against expm_apply_tridiag, against the oracle (independent of the GPU kernels), and
that no call after a warm-up changes the device's free memory.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes when run alone in a fresh process.
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

DEV = torch.device("cuda:0")
TOL = {P.EXPM_FP64: 1e-12, P.EXPM_MIXED_F32X2: 1e-8}   # the tridiagonal tests' tolerances
CASES = [(16_001, 8, 400), (9_001, 3, 401)]


def _inputs(N, r, seed):
    g = workloads.rng(seed)
    d = g.uniform(-12.0, -4.0, N)
    e = g.uniform(0.5, 2.0, N - 1)
    V = g.standard_normal((N, r))
    return (d, e, V), tuple(torch.from_numpy(x).to(DEV) for x in (d, e, V))


@pytest.mark.parametrize("prec", [P.EXPM_FP64, P.EXPM_MIXED_F32X2])
def test_noalloc_matches_allocating_entry_point_and_oracle_twice(prec):
    plan = P.Plan(degree=16)
    th, a = coeffs.theta(16), coeffs.residues(16)
    for call, (N, r, seed) in enumerate(CASES):
        (hd, he, hV), (d, e, V) = _inputs(N, r, seed)
        Y_ref = torch.empty_like(V)
        P.expm_apply_tridiag(plan, d, e, V, Y_ref, prec=prec)
        Y = torch.full_like(V, float("nan"))
        P.expm_apply_tridiag_noalloc(plan, d, e, V, Y, prec=prec)
        torch.cuda.synchronize()
        y = Y.cpu().numpy()
        err = matrix.rel_err(y, Y_ref.cpu().numpy())
        assert np.isfinite(err) and err <= TOL[prec], (call, err)
        Yo, _ = matrix.apply_tridiag(hd, he, hV, th, a)
        err_o = matrix.rel_err(y, Yo)
        assert np.isfinite(err_o) and err_o <= TOL[prec], (call, err_o)
    plan.close()


@pytest.mark.parametrize("prec", [P.EXPM_FP64, P.EXPM_MIXED_F32X2])
def test_noalloc_complex_hermitian(prec):
    """Complex e (the phases and D^H V in the fixed array too): equal to the allocating
    entry point and within the tolerance of the oracle."""
    plan = P.Plan(degree=16)
    N, r = 12_001, 2
    g = workloads.rng(403)
    hd = g.uniform(-12.0, -4.0, N)
    he = g.uniform(0.5, 2.0, N - 1) * np.exp(1j * g.uniform(0.0, 2 * np.pi, N - 1))
    hV = g.standard_normal((N, r))
    d, e, V = (torch.from_numpy(x).to(DEV) for x in (hd, he, hV))
    Y_ref = torch.empty((N, r), dtype=torch.complex128, device=DEV)
    P.expm_apply_tridiag(plan, d, e, V, Y_ref, prec=prec)
    Y = torch.full_like(Y_ref, float("nan"))
    P.expm_apply_tridiag_noalloc(plan, d, e, V, Y, prec=prec)
    torch.cuda.synchronize()
    assert torch.equal(Y, Y_ref)
    Yo, _ = matrix.apply_tridiag(hd, he, hV, coeffs.theta(16), coeffs.residues(16))
    assert matrix.rel_err(Y.cpu().numpy(), Yo) <= TOL[prec]
    plan.close()


def test_noalloc_calls_after_warm_up_allocate_nothing():
    """After one warm-up call (which may load the library's module and with it the fixed
    array), further calls leave the device's free memory unchanged."""
    plan = P.Plan(degree=16)
    ins = [_inputs(N, r, seed)[1] for N, r, seed in CASES]
    outs = [torch.empty_like(V) for _, _, V in ins]
    d, e, V = ins[0]
    P.expm_apply_tridiag_noalloc(plan, d, e, V, outs[0])   # warm-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for (d, e, V), Y in zip(ins, outs):
            P.expm_apply_tridiag_noalloc(plan, d, e, V, Y)
            P.expm_apply_tridiag_noalloc(plan, d, e, V, Y, prec=P.EXPM_MIXED_F32X2)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    plan.close()


def test_noalloc_rejects_oversized_problems_and_host_buffers():
    plan = P.Plan(degree=16)
    _, (d, e, V) = _inputs(1 << 20, 8, 402)      # needs far more than the fixed scratch
    Y = torch.empty_like(V)
    with pytest.raises(P.ExpmError) as ei:
        P.expm_apply_tridiag_noalloc(plan, d, e, V, Y)
    assert ei.value.status == 1 and "EXPM_NOALLOC_SCRATCH_BYTES" in str(ei.value)
    hd, he, hV = (x[:100].cpu().numpy() for x in (d, e, V))
    with pytest.raises(P.ExpmError) as ei:
        P.expm_apply_tridiag_noalloc(plan, hd, he[:99], hV, np.empty_like(hV))
    assert ei.value.status == 1
    plan.close()
