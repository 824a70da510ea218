"""The C-ABI library: it loads, exports every symbol include/*.h declares, and its
host-only entry points behave as documented.  CPU only (no device compute)."""

import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(expm_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_2306_16778_gb300 as P
    return P


def test_every_declared_symbol_is_exported(P):
    names = _declared_functions()
    assert "expm_apply_tridiag" in names and "expm_coeffs" in names
    lib = ctypes.CDLL(P.library_path)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_every_public_export_is_declared(P):
    """The reverse: every exported expm_* entry point other than the expm_internal_* test
    hooks is declared (and documented) in include/*.h."""
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", P.library_path], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("nm not available")
    exported = {ln.split()[-1] for ln in out.stdout.splitlines() if ln.split() and ln.split()[-1].startswith("expm_")}
    public = {n for n in exported if not n.startswith("expm_internal_")}
    undeclared = sorted(public - set(_declared_functions()))
    assert not undeclared, f"exported but not declared: {undeclared}"


@pytest.mark.parametrize("n", [2, 4, 8, 12, 16, 20, 24, 32, 40, 48, 56])
def test_library_coefficients_equal_oracle(P, n):
    """The library's double-double Aberth-Ehrlich coefficients, rounded to
    binary64, equal the oracle's decimal Durand-Kerner ones bit for bit."""
    from oracle import coeffs
    p, r = P.expm_coeffs(n)
    po, ro = coeffs.abi_arrays(n)
    np.testing.assert_array_equal(p, po)
    np.testing.assert_array_equal(r, ro)


def test_library_coefficients_degree_64(P):
    from oracle import coeffs
    p, r = P.expm_coeffs(64)
    po, ro = coeffs.abi_arrays(64)
    np.testing.assert_allclose(p, po, rtol=0, atol=4e-16 * np.abs(po).max())
    np.testing.assert_allclose(r, ro, rtol=0, atol=4e-16 * np.abs(ro).max())


@pytest.mark.parametrize("n", [0, 1, 3, 66, -2])
def test_coefficients_reject_bad_degree(P, n):
    buf = (ctypes.c_double * 256)()
    assert P.lib.expm_coeffs(n, buf, buf) == 1          # EXPM_EINVAL
    assert P.lib.expm_coeffs(12, None, buf) == 1


def test_plan_create_validation(P):
    """Checks that run before any device call: pairing, R_n(0) = 1, degree."""
    p, r = P.expm_coeffs(12)
    bad = p.copy()
    bad[3] += 1e-3                      # partner no longer the conjugate
    with pytest.raises(P.ExpmError) as ei:
        P.Plan(bad, r, 12)
    assert ei.value.status == 1
    with pytest.raises(P.ExpmError) as ei:
        P.Plan(p, 2 * r, 12)            # R_n(0) = 2
    assert ei.value.status == 1
    with pytest.raises(P.ExpmError):
        P.Plan(p[:22], r[:22], 11)      # odd degree
    nan = p.copy()
    nan[0] = np.nan
    with pytest.raises(P.ExpmError):
        P.Plan(nan, r, 12)


def test_status_strings(P):
    assert P.lib.expm_status_string(0) == b"EXPM_OK"
    assert P.lib.expm_status_string(9) == b"EXPM_ENOTSUP"


def test_product_path_has_no_oracle_import():
    """The package never imports the oracle (the oracle is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_2306_16778_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(f).read()
        assert not re.search(r"^\s*(from|import)\s+oracle", src, flags=re.M), f
