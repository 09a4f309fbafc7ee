"""Communication volume of a distributed 3D FFT of N^3 points over P processes (Sec. 3.2.3).

This is the model behind the paper's comparison of its structure-B transposes with a one-dimensional
(slab) decomposition and with a two-dimensional (square pencil) decomposition. The paper gives the
volumes in closed form for P = N/4 .. 32 N. Counts are grid elements that leave their process over
one forward transform.

- Structure B ("ours"). Rows of the ab plane are dealt out first.
  - Up to N processes (P divides N), the abc -> cab transpose is the slab all-to-all:
    N^3 (1 - 1/P) elements.
  - Beyond that (P = m N), abc -> cab moves N^3 (1 - 1/N) elements and cab -> cba another
    N^3 (1 - 1/m). The total is (2 - 1/m) N^3 - N^2.
- Slab (one-dimensional): one all-to-all, N^3 (1 - 1/P), only for P <= N.
- Square pencils (two-dimensional): two all-to-alls within rows and columns of a sqrt(P) x sqrt(P)
  process grid, 2 N^3 (1 - 1/sqrt(P)).

The advantage the paper quotes is (2D - ours) / ours: 60.0% at P = 16 and 77.8% at P = 64 for N = 64,
falling to about 0 by P = 2048.
"""
from __future__ import annotations

import math


def ours(N: int, P: int) -> float:
    """Elements moved by the structure-B transposes abc -> cab -> cba for P processes."""
    if P < 1 or P > N * N:
        raise ValueError("P must be in [1, N^2]")
    if P <= N:
        return N ** 3 * (1.0 - 1.0 / P)
    m = P / N
    return (2.0 - 1.0 / m) * N ** 3 - N ** 2


def slab(N: int, P: int) -> float:
    """One-dimensional decomposition: one all-to-all (defined for P <= N only)."""
    if P < 1 or P > N:
        raise ValueError("the slab decomposition needs 1 <= P <= N")
    return N ** 3 * (1.0 - 1.0 / P)


def pencil(N: int, P: int) -> float:
    """Two-dimensional square decomposition: two all-to-alls on a sqrt(P) x sqrt(P) grid."""
    if P < 1 or P > N * N:
        raise ValueError("P must be in [1, N^2]")
    return 2.0 * N ** 3 * (1.0 - 1.0 / math.sqrt(P))


def advantage(N: int, P: int) -> float:
    """(pencil - ours) / ours, the paper's 'x% better'."""
    return (pencil(N, P) - ours(N, P)) / ours(N, P)
