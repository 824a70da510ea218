"""Oracle: a plain, slow, CPU-only restatement of what the partial-fraction
exp(A)V method computes (Hecht, Kaber, Perrin, Plagne, Salomon, "Parallel
approximation of the exponential of Hermitian matrices").

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it.  The
product path (the CUDA library and its Python binding) never imports, links or
calls anything here, and nothing here imports the product path.

Modules
-------
coeffs  roots theta_k of the truncated Taylor series exp_n (Sec. 2.1) and the
        residues a_k of Prop. 2.1 (eq. yoyo2), in high-precision decimal
        arithmetic, rounded once to binary64.
scalar  exp_n, R_n(x) = 1/exp_n(-x) (Sec. 2.2), the partial-fraction sum
        (eq. yoyo), and the error bounds M_1 (Prop. 2.2) and M_2 (Prop. 4.1).
matrix  R_n(A)V = sum_k a_k (A + theta_k I)^{-1} V (eqs. ExpoMatRat, expAx)
        by one direct pivoted solve per pole (LAPACK via numpy/scipy), plus the
        closed forms used to pin it: eigen-decomposition, DST-I for the 1D
        Laplacian, the product form n!/prod(z + theta_k), and exp itself.

Notation follows the paper: theta_k are the roots of exp_n, a_k the residues,
and R_n(A) = sum_k a_k (A + theta_k I)^{-1}.  The library's C interface carries
poles lambda_k = -theta_k and weights w_k = a_k; ``coeffs.abi_arrays`` converts.

Parity status of every function is stated in its docstring; every function
here is pinned by a test in ``tests/test_oracle_*.py`` against something other
than itself (closed forms, invariants the paper states, the paper's bounds,
brute force or an independent multiprecision library).
"""

from . import coeffs, scalar, matrix  # noqa: F401
