"""FP64 CPU oracle for the BCCB LASSO solvers (test infrastructure).

This package is test infrastructure, not part of the product.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import it.  It shares no code with the CUDA path and imports nothing from it.

It is the paper's "regular" implementation written out plainly: the sensing
matrix D_s = Psi (D2 kron D1) is formed explicitly in complex128 and every Gram
product is two dense matrix-vector products (Section II-B).  No FFT is used
anywhere in it; the FFT identity of Section III-B is what the CUDA path relies on
and what the tests check the two against.

``oracle.peaks`` holds the post-processing step of Section II-A: peak picking on
|c| and the map from harmonic pairs to the angles (phi, theta).
"""
from .lasso import (  # noqa: F401
    dictionary,
    dictionary_columns,
    adjoint_measurements_kron,
    harmonic_grid,
    element_positions,
    soft_threshold,
    step_size,
    adjoint_measurements,
    lambda_max,
    ista,
    fista,
    fista_momentum,
    admm,
    admm_c_update,
    admm_kron,
    fista_kron,
    KronDictionary,
    kkt_residual,
    objective,
    gram_first_column,
    gram_eigenvalues,
    unrolled_forward,
    unrolled_backward,
)
from . import peaks  # noqa: F401
