"""FP64 CPU oracle for the truncated SVD methods of Tomas, Quintana-Orti and Anzt,
"Fast Truncated SVD of Sparse and Dense Matrices on Graphics Processors".

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link or
execute this package: only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares no
code with the CUDA library (no kernels, headers, helpers, tables or constants) and
does not import it.

Every function follows the paper step by step in plain numpy/scipy FP64
arithmetic; library primitives (matrix product, sparse product, LAPACK SVD) serve
only as single steps.  Pins that tie it to something other than itself live in
``tests/test_oracle_*.py``.
"""

from .tsvd_oracle import (  # noqa: F401
    philox4x32_10,
    gaussian_block,
    cholesky_lower,
    cholqr2,
    cgs_cqr2,
    cgs_qr,
    small_svd,
    rsvd,
    blanczos,
    residuals,
    as_operator,
    OracleInfo,
)
from .tsvd_backward import svd_backward  # noqa: F401
