"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 5).

This module holds input generation only -- no arithmetic of the method.  Both
the oracle-based tests and the GPU path draw their inputs from here, so the two
sides see identical host arrays.  Generators use numpy's PCG64 with base seed
20230629 plus a per-workload offset.

Workloads (sizes from the project's configuration list):

* ``dense_small``     real symmetric 64x64, A = Q diag(mu) Q^T with Q Haar
  orthogonal and mu ~ U[-20, 0]; one Gaussian vector; degree 12.
  (Sec. 5.2: random symmetric matrices with spectrum in a fixed range.)
* ``laplacian_1d``    T = c * tridiag(1, -2, 1) with c = dt/h^2; N = 2^20,
  h = 1/(N+1), dt = 100 h^2 (so c = 100 and the spectrum lies in (-400, 0));
  8 Gaussian right-hand sides; degree 16.  (Sec. 5: B = Delta^1_d.)
* ``dense_hermitian`` complex Hermitian 4096x4096, A = U diag(mu) U^H with U
  Haar unitary and mu ~ U[-50, 0]; V 4096x256 complex Gaussian; degree 16.
* ``uneven_batch``    4096 Hermitian instances with sizes round(exp(U[ln 32,
  ln 768])), mu ~ U[-30, 0], one complex Gaussian RHS each; degree 12.
* ``served_stream``   Poisson arrivals; 70 % tridiagonal Laplacian requests
  (N log-uniform in [2^12, 2^20], 1-4 RHS), 30 % dense Hermitian requests
  (n log-uniform in [64, 2048], 1-64 RHS, mu ~ U[-40, 0]); degree 12 or 16.

Haar sampling: QR of a real (complex) Ginibre matrix with the phases of R's
diagonal moved into Q (Mezzadri 2007).  Complex normals have independent real
and imaginary parts ~ N(0, 1/2).
"""

from __future__ import annotations

import math

import numpy as np

BASE_SEED = 20230629


def rng(offset: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + offset))


def haar_orthogonal(n: int, g: np.random.Generator) -> np.ndarray:
    Z = g.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))[None, :]


def haar_unitary(n: int, g: np.random.Generator) -> np.ndarray:
    Z = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / math.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    ph = np.diag(R) / np.abs(np.diag(R))
    return Q * ph[None, :]


def complex_normal(shape, g: np.random.Generator) -> np.ndarray:
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)) / math.sqrt(2.0)


def dense_symmetric(n: int, lo: float, hi: float, nrhs: int, g, complex_: bool):
    """A = Q diag(mu) Q^H (Hermitian), mu ~ U[lo, hi]; V Gaussian (n x nrhs)."""
    Q = haar_unitary(n, g) if complex_ else haar_orthogonal(n, g)
    mu = g.uniform(lo, hi, n)
    A = (Q * mu[None, :]) @ Q.conj().T
    A = 0.5 * (A + A.conj().T)          # exactly Hermitian in binary64
    V = complex_normal((n, nrhs), g) if complex_ else g.standard_normal((n, nrhs))
    return A, Q, mu, V


def dense_small(offset: int = 0, n: int = 64, nrhs: int = 1):
    """Real symmetric n x n, spectrum U[-20, 0], degree 12."""
    g = rng(offset)
    A, Q, mu, V = dense_symmetric(n, -20.0, 0.0, nrhs, g, complex_=False)
    return dict(A=A, Q=Q, mu=mu, V=V, degree=12)


def laplacian_1d(N: int = 1 << 20, nrhs: int = 8, offset: int = 1, c: float = 100.0,
                 degree: int = 16):
    """T = c tridiag(1, -2, 1) (c = dt/h^2 = 100 for dt = 100 h^2), V ~ N(0,1)^{N x nrhs}."""
    g = rng(offset)
    d = np.full(N, -2.0 * c)
    e = np.full(max(N - 1, 0), c)
    V = g.standard_normal((N, nrhs))
    return dict(d=d, e=e, V=V, d0=-2.0 * c, e0=c, degree=degree)


def dense_hermitian(n: int = 4096, nrhs: int = 256, offset: int = 2, lo: float = -50.0):
    """Complex Hermitian n x n, spectrum U[lo, 0], V complex Gaussian n x nrhs, degree 16."""
    g = rng(offset)
    A, Q, mu, V = dense_symmetric(n, lo, 0.0, nrhs, g, complex_=True)
    return dict(A=A, Q=Q, mu=mu, V=V, degree=16)


def batch_sizes(count: int, g, lo: int = 32, hi: int = 768) -> np.ndarray:
    return np.rint(np.exp(g.uniform(math.log(lo), math.log(hi), count))).astype(np.int64)


def _batch_instance(args):
    n, seed, mu_lo = args
    g = np.random.Generator(np.random.PCG64(seed))
    A, Q, mu, V = dense_symmetric(int(n), mu_lo, 0.0, 1, g, complex_=True)
    return dict(A=A, Q=Q, mu=mu, V=V)


def uneven_batch(count: int = 4096, offset: int = 3, lo: int = 32, hi: int = 768,
                 mu_lo: float = -30.0, workers: int = 1):
    """``count`` complex Hermitian instances, sizes log-uniform in [lo, hi], one RHS each.

    Instance i draws from its own generator (seed BASE_SEED + 1_000_000 * offset + i), so
    the batch is the same whether it is made sequentially or by ``workers`` threads (the
    QR factorizations and products release the interpreter lock)."""
    g = rng(offset)
    sizes = batch_sizes(count, g, lo, hi)
    args = [(int(n), BASE_SEED + 1_000_000 * offset + i, mu_lo) for i, n in enumerate(sizes)]
    if workers > 1 and count > 64:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(workers) as ex:
            inst = list(ex.map(_batch_instance, args))
    else:
        inst = [_batch_instance(x) for x in args]
    return dict(sizes=sizes, instances=inst, degree=12)


def served_stream(count: int, rate: float, offset: int = 4, pool: int = 64):
    """Request descriptors for a Poisson stream (arrival times in seconds).

    Each request names an operator id from a seeded pool (64 tridiagonal + 64
    dense ids) so that resident factorizations can be reused; the operators
    themselves are made by ``served_operator``.
    """
    g = rng(offset)
    gaps = g.exponential(1.0 / rate, count)
    arrival = np.cumsum(gaps)
    reqs = []
    for i in range(count):
        tri = g.uniform() < 0.7
        op = int(g.integers(0, pool))
        deg = 12 if g.uniform() < 0.5 else 16
        if tri:
            nrhs = int(g.integers(1, 5))
        else:
            nrhs = int(np.rint(math.exp(g.uniform(0.0, math.log(64.0)))))
        reqs.append(dict(t=float(arrival[i]), kind="tridiag" if tri else "dense",
                         op=op, degree=deg, nrhs=nrhs, seed=int(g.integers(0, 2**31))))
    return reqs


def served_operator(kind: str, op: int, offset: int = 4):
    """Operator ``op`` of the served-stream pool (deterministic per id)."""
    g = rng(1000 * (offset + 1) + op + (0 if kind == "tridiag" else 500))
    if kind == "tridiag":
        N = int(np.rint(math.exp(g.uniform(math.log(2.0**12), math.log(2.0**20)))))
        return laplacian_1d(N=N, nrhs=1, offset=10_000 + op)
    n = int(np.rint(math.exp(g.uniform(math.log(64.0), math.log(2048.0)))))
    A, Q, mu, _ = dense_symmetric(n, -40.0, 0.0, 1, g, complex_=True)
    return dict(A=A, Q=Q, mu=mu)


def request_rhs(n: int, nrhs: int, seed: int, complex_: bool):
    g = np.random.Generator(np.random.PCG64(seed))
    return complex_normal((n, nrhs), g) if complex_ else g.standard_normal((n, nrhs))
