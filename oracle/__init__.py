"""FP64 CPU oracle for the grid-side Hartree step (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does; the
two share no code.  See ``hartree_oracle.c`` for what each routine computes
and which passage of the paper it follows.
"""
from .oracle import (  # noqa: F401
    bisect,
    build,
    dft3d_brute,
    fft1d,
    fft3d,
    forces,
    get_threads,
    poisson,
    set_threads,
    splat,
    solve_system,
)
