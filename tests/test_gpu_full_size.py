"""Full-size parity for the dense configurations, in the launch configuration the
benchmark's dense and batched modes time.

* Dense complex Hermitian 4096 x 4096, 256 RHS, degree 16: both paths against the
  exact closed form Q diag(R_n(mu)) Q^H V (Remark 3.1), FP64 <= 1e-12 and the mixed
  path <= 1e-10 (also against the FP64 GPU path).
* Uneven batch of 4096 instances (n in [32, 768], one RHS, degree 12): a sample of
  instances checked one by one against the oracle's per-pole solves, <= 1e-12 (FP64)
  and <= 1e-8 (mixed)."""

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


def test_dense_hermitian_4096():
    w = workloads.dense_hermitian()
    ref = matrix.eig_apply(w["Q"], w["mu"], w["V"], lambda m: scalar.R_n(m, 16))
    plan = P.Plan(degree=16)
    A, V = (torch.from_numpy(x).to(DEV) for x in (w["A"], w["V"]))
    Y64, Ymx, Ytc, Ybf = (torch.empty_like(V) for _ in range(4))
    P.expm_apply_dense(plan, A, V, Y64, prec=P.EXPM_FP64)
    info = P.expm_apply_dense(plan, A, V, Ymx, prec=P.EXPM_MIXED_FP32)
    itc = P.expm_apply_dense(plan, A, V, Ytc, prec=P.EXPM_MIXED_TF32X3)
    ibf = P.expm_apply_dense(plan, A, V, Ybf, prec=P.EXPM_MIXED_BF16X3)
    torch.cuda.synchronize()
    y64, ymx, ytc, ybf = Y64.cpu().numpy(), Ymx.cpu().numpy(), Ytc.cpu().numpy(), Ybf.cpu().numpy()
    e64, emx, etc = matrix.rel_err(y64, ref), matrix.rel_err(ymx, ref), matrix.rel_err(ytc, ref)
    d, dtc = matrix.rel_err(ymx, y64), matrix.rel_err(ytc, y64)
    assert matrix.rel_err(ybf, ref) <= 1e-10 and matrix.rel_err(ybf, y64) <= 1e-10
    assert ibf.status_worst == 0 and ibf.refine_iters_max >= 1
    print(f"dense 4096: fp64 {e64:.3e}, mixed {emx:.3e} ({info.refine_iters_max} sweeps), "
          f"tf32x3 {etc:.3e} ({itc.refine_iters_max} sweeps), vs fp64 {d:.3e} / {dtc:.3e}")
    assert e64 <= 1e-12 and emx <= 1e-10 and d <= 1e-10 and etc <= 1e-10 and dtc <= 1e-10


@pytest.mark.parametrize("prec,tol", [(P.EXPM_FP64, 1e-12), (P.EXPM_MIXED_FP32, 1e-8)])
def test_uneven_batch_4096(prec, tol):
    w = workloads.uneven_batch()
    plan = P.Plan(degree=12)
    As = [torch.from_numpy(i["A"]).to(DEV) for i in w["instances"]]
    Vs = [torch.from_numpy(i["V"]).to(DEV) for i in w["instances"]]
    Ys = [torch.empty_like(v) for v in Vs]
    infos = P.expm_apply_batched(plan, As, Vs, Ys, prec=prec)
    torch.cuda.synchronize()
    assert all(i.status_worst == 0 for i in infos)
    th, a = coeffs.theta(12), coeffs.residues(12)
    sample = list(range(0, len(As), len(As) // 40)) + [int(np.argmax(w["sizes"])), int(np.argmin(w["sizes"]))]
    worst = 0.0
    for i in sample:
        inst = w["instances"][i]
        Yo, _ = matrix.apply_dense(inst["A"], inst["V"], th, a)
        worst = max(worst, matrix.rel_err(Ys[i].cpu().numpy(), Yo))
    print(f"uneven batch prec={prec}: worst sampled rel err {worst:.3e}")
    assert worst <= tol
