"""The communication-volume model of the distributed 3D FFT (Sec. 3.2.3, N = 64).

The paper prints the advantage of its structure-B transposes over the square (two-dimensional)
decomposition: 60.0% at 16 processes, 77.8% at 64, about 0 at 2048 (the closed forms at
P = N/4 .. 32 N are the paper's).  The model also reproduces each closed form it lists.
"""
import pytest

from paper_1209_4506_gb300 import fft_comm_model as M

N = 64


def test_printed_advantages():
    assert round(100 * M.advantage(N, 16), 1) == 60.0
    assert round(100 * M.advantage(N, 64), 1) == 77.8
    assert 0.0 <= M.advantage(N, 2048) < 0.002


@pytest.mark.parametrize("k", [4, 2, 1])
def test_closed_forms_up_to_n_processes(k):
    P = N // k
    assert M.ours(N, P) == pytest.approx(N ** 3 - k * N ** 2, rel=1e-15)
    assert M.slab(N, P) == M.ours(N, P)


@pytest.mark.parametrize("m", [2, 4, 8, 16, 32])
def test_closed_forms_beyond_n_processes(m):
    P = m * N
    assert M.ours(N, P) == pytest.approx((2 - 1 / m) * N ** 3 - N ** 2, rel=1e-15)
    # the paper's form 2 N^3 - 2m N (N/m)^(3/2) of the square decomposition
    assert M.pencil(N, P) == pytest.approx(2 * N ** 3 - 2 * m * N * (N / m) ** 1.5, rel=1e-12)


def test_pencil_closed_forms_below_n_processes():
    # 2 N^3 - N/2 (4N)^(3/2) at N/4, 2 N^3 - N (2N)^(3/2) at N/2, 2 N^3 - 2 N^(5/2) at N
    assert M.pencil(N, N // 4) == pytest.approx(2 * N ** 3 - N / 2 * (4 * N) ** 1.5, rel=1e-12)
    assert M.pencil(N, N // 2) == pytest.approx(2 * N ** 3 - N * (2 * N) ** 1.5, rel=1e-12)
    assert M.pencil(N, N) == pytest.approx(2 * N ** 3 - 2 * N ** 2.5, rel=1e-12)


def test_slab_matches_structure_b_up_to_n_and_stops_there():
    for P in (1, 2, 8, 16, 64):
        assert M.slab(N, P) == M.ours(N, P)
    with pytest.raises(ValueError):
        M.slab(N, 128)


def test_structure_b_never_moves_more_than_the_square_decomposition():
    for P in range(2, N * N + 1):
        assert M.ours(N, P) <= M.pencil(N, P) * (1 + 1e-12)
