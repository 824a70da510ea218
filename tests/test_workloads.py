"""The seeded input generators match the stated recipe of each workload (Sec. 5 shapes:
random Hermitian matrices with a fixed spectral range, the finite-difference Laplacian,
Gaussian right-hand sides), on sizes small enough for the CPU suite."""

import math

import numpy as np
import pytest

import workloads


def test_seeding_is_deterministic_and_per_offset():
    a = workloads.rng(7).standard_normal(5)
    b = workloads.rng(7).standard_normal(5)
    c = workloads.rng(8).standard_normal(5)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    assert workloads.BASE_SEED == 20230629


@pytest.mark.parametrize("complex_", [False, True])
def test_haar_factor_is_orthogonal_or_unitary(complex_):
    g = workloads.rng(900)
    Q = workloads.haar_unitary(40, g) if complex_ else workloads.haar_orthogonal(40, g)
    assert np.iscomplexobj(Q) == complex_
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(40), atol=1e-13)


def test_complex_normal_has_half_variance_parts():
    z = workloads.complex_normal((200_000,), workloads.rng(901))
    assert abs(np.var(z.real) - 0.5) < 0.01 and abs(np.var(z.imag) - 0.5) < 0.01
    assert abs(np.mean(z)) < 0.01


@pytest.mark.parametrize("complex_", [False, True])
def test_dense_symmetric_spectrum_and_symmetry(complex_):
    g = workloads.rng(902)
    A, Q, mu, V = workloads.dense_symmetric(60, -30.0, 0.0, 3, g, complex_)
    np.testing.assert_array_equal(A, A.conj().T)          # exactly Hermitian
    assert mu.min() >= -30.0 and mu.max() <= 0.0
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(A)), np.sort(mu), atol=1e-12)
    np.testing.assert_allclose(A, (Q * mu[None, :]) @ Q.conj().T, atol=1e-12)
    assert V.shape == (60, 3) and np.iscomplexobj(V) == complex_


def test_dense_small_and_dense_hermitian_recipes():
    w = workloads.dense_small()
    assert w["A"].shape == (64, 64) and not np.iscomplexobj(w["A"]) and w["degree"] == 12
    assert w["V"].shape == (64, 1) and -20.0 <= w["mu"].min() and w["mu"].max() <= 0.0
    h = workloads.dense_hermitian(n=48, nrhs=5)
    assert np.iscomplexobj(h["A"]) and h["V"].shape == (48, 5) and h["degree"] == 16
    assert -50.0 <= h["mu"].min() and h["mu"].max() <= 0.0


def test_laplacian_recipe_and_spectrum():
    N = 300
    w = workloads.laplacian_1d(N=N, nrhs=8)
    assert w["d"].shape == (N,) and w["e"].shape == (N - 1,) and w["V"].shape == (N, 8)
    assert np.all(w["d"] == -200.0) and np.all(w["e"] == 100.0) and w["degree"] == 16
    T = np.diag(w["d"]) + np.diag(w["e"], 1) + np.diag(w["e"], -1)
    ev = np.linalg.eigvalsh(T)
    # 100 (1, -2, 1) = dt/h^2 tridiag with dt = 100 h^2: eigenvalues -400 sin^2(j pi / (2 (N+1)))
    j = np.arange(1, N + 1)
    np.testing.assert_allclose(np.sort(ev), np.sort(-400.0 * np.sin(j * np.pi / (2 * (N + 1))) ** 2), atol=1e-9)
    assert ev.min() > -400.0 and ev.max() < 0.0


def test_uneven_batch_sizes_are_log_uniform_in_range():
    s = workloads.batch_sizes(20_000, workloads.rng(903))
    assert s.min() >= 32 and s.max() <= 768
    # log-uniform: mean of ln n near the midpoint of [ln 32, ln 768]
    assert abs(np.mean(np.log(s)) - 0.5 * (math.log(32) + math.log(768))) < 0.02
    b = workloads.uneven_batch(count=6, lo=32, hi=64)
    assert len(b["instances"]) == 6 and b["degree"] == 12
    for n, inst in zip(b["sizes"], b["instances"]):
        assert inst["A"].shape == (n, n) and inst["V"].shape == (n, 1)
        assert -30.0 <= inst["mu"].min() and inst["mu"].max() <= 0.0


def test_served_stream_mix():
    reqs = workloads.served_stream(4000, rate=500.0)
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0) and abs(np.mean(np.diff(t)) - 1 / 500.0) < 1e-4
    tri = [r for r in reqs if r["kind"] == "tridiag"]
    den = [r for r in reqs if r["kind"] == "dense"]
    assert abs(len(tri) / len(reqs) - 0.7) < 0.03
    assert all(1 <= r["nrhs"] <= 4 for r in tri) and all(1 <= r["nrhs"] <= 64 for r in den)
    assert {r["degree"] for r in reqs} == {12, 16}
    assert all(0 <= r["op"] < 64 for r in reqs)


def test_served_operators_sizes_in_range():
    for op in range(6):
        t = workloads.served_operator("tridiag", op)
        assert 2 ** 12 <= t["d"].shape[0] <= 2 ** 20
    for op in range(3):
        d = workloads.served_operator("dense", op)
        n = d["A"].shape[0]
        assert 64 <= n <= 2048 and -40.0 <= d["mu"].min() and d["mu"].max() <= 0.0
