"""CPU oracle for the one-sided trigonometric / hyperbolic Jacobi method.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The product path (the CUDA
library and its binding in ``paper_1008_0201_gb300``) never imports this package.

The arithmetic lives in ``jacobi_oracle.c`` (plain C, IEEE double, wide-precision checks);
this module builds it with gcc and wraps it with ctypes + numpy.
"""
from .oracle import (  # noqa: F401
    build_oracle,
    load,
    hsvd,
    eigenpairs,
    rotation_params,
    pairs_modulus,
    pairs_round_robin,
    pairs_cycle_weight,
    block_offsets,
    check_offdiag,
    check_vjv,
    check_factor_residual,
    eig_backward,
    set_mutation,
    solve,
)
