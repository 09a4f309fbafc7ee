"""The atom decomposition (Sec. 3.1: modified recursive bisection with the inertia-tensor principal
axis) on the device, hartree_atoms_reorder_device, against the host reorder and the oracle's
bisection (which the host tests pin to the paper's worked example).

The device sums the centre of mass and the moment matrix in a different order than the host, so
the two agree exactly wherever no two projections of one node are tied to within the last bits;
the jittered diamond systems used here have no such ties.  Cases: the paper's experiment of
Sec. 5.2.1 (16,384 atoms over 19 processes), the bench's 4,096 atoms over 256 leaves, weights
(Sec. 3.1.4), more leaves than atoms (empty leaves), one leaf, no atoms, and 65,536 atoms whose
first levels exceed the shared-memory sort and go through the global scratch.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1209_4506_gb300 import capi, synth
from paper_1209_4506_gb300.hartree import HartreePlan, atoms_reorder

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def device_reorder(plan, pos, n_leaves, w=None, stream=None):
    n = pos.shape[0]
    P = torch.tensor(pos, device="cuda")
    W = torch.tensor(w, device="cuda") if w is not None else None
    perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    ls = torch.empty(n_leaves + 1, dtype=torch.int32, device="cuda")
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    capi.check(capi.hartree_atoms_reorder_device(plan.handle, P.data_ptr() if n else None,
                                                 W.data_ptr() if W is not None else None, n, n_leaves,
                                                 perm.data_ptr(), ls.data_ptr(), s))
    torch.cuda.synchronize()
    return perm.cpu().numpy()[:n], ls.cpu().numpy()


def diamond(reps, seed):
    rng = np.random.default_rng(seed)
    cell = tuple(r * synth.DIAMOND_A for r in reps)
    return synth.jitter(rng, synth.diamond_supercell(reps), 0.1, cell), cell


@pytest.fixture(scope="module")
def plan():
    P = HartreePlan((32, 32, 32), (10.0, 10.0, 10.0), 0.5, "fp32", max_atoms=65536)
    yield P
    P.close()


@pytest.mark.parametrize("reps,n_leaves,seed", [((16, 16, 8), 19, 5), ((8, 8, 8), 256, 3), ((4, 4, 4), 7, 11),
                                                ((2, 2, 2), 100, 2), ((1, 1, 1), 1, 4)])
def test_device_bisection_equals_host_and_oracle(plan, reps, n_leaves, seed):
    pos, _ = diamond(reps, seed)
    perm_d, ls_d = device_reorder(plan, pos, n_leaves)
    perm_h, ls_h = atoms_reorder(pos, n_leaves)
    perm_o, ls_o = O.bisect(pos, n_leaves)
    assert np.array_equal(ls_d, ls_h) and np.array_equal(perm_d, perm_h)
    assert np.array_equal(ls_d, ls_o) and np.array_equal(perm_d, perm_o)
    assert np.array_equal(np.sort(perm_d), np.arange(pos.shape[0]))


def test_device_bisection_with_weights(plan):
    """Sec. 3.1.4: w_i = Etime_i / Mtime; the cut balances weight, not atom counts."""
    pos, _ = diamond((4, 4, 4), 21)
    w = np.random.default_rng(8).uniform(0.2, 3.0, size=pos.shape[0])
    perm_d, ls_d = device_reorder(plan, pos, 13, w)
    perm_h, ls_h = atoms_reorder(pos, 13, w)
    perm_o, ls_o = O.bisect(pos, 13, w)
    assert np.array_equal(ls_d, ls_h) and np.array_equal(perm_d, perm_h)
    assert np.array_equal(ls_d, ls_o) and np.array_equal(perm_d, perm_o)


def test_device_bisection_edge_cases(plan):
    perm, ls = device_reorder(plan, np.zeros((0, 3)), 4)  # no atoms: every leaf empty
    assert perm.size == 0 and ls.tolist() == [0, 0, 0, 0, 0]
    one = np.array([[1.0, 2.0, 3.0]])
    perm, ls = device_reorder(plan, one, 3)  # one atom, three leaves
    perm_h, ls_h = atoms_reorder(one, 3)
    assert perm.tolist() == perm_h.tolist() == [0] and ls.tolist() == ls_h.tolist()
    with pytest.raises(capi.HartreeError):
        device_reorder(plan, one, 0)


def test_device_bisection_65536_atoms_global_sort(plan):
    """The paper's 65,536-atom system over 4,096 leaves: the root's range exceeds the shared-memory
    sort (2^14 entries) and is sorted in the plan's global scratch."""
    pos, _ = diamond((32, 16, 16), 9)
    perm_d, ls_d = device_reorder(plan, pos, 4096)
    perm_h, ls_h = atoms_reorder(pos, 4096)
    assert np.array_equal(ls_d, ls_h) and np.array_equal(perm_d, perm_h)
    sizes = np.diff(ls_d)
    assert sizes.min() == 16 and sizes.max() == 16


def test_device_bisection_replays_from_a_cuda_graph(plan):
    """The reorder reads nothing back to the host: it is captured once and replayed."""
    pos, _ = diamond((8, 8, 8), 3)
    P = torch.tensor(pos, device="cuda")
    perm = torch.empty(pos.shape[0], dtype=torch.int32, device="cuda")
    ls = torch.empty(257, dtype=torch.int32, device="cuda")

    def run():
        capi.check(capi.hartree_atoms_reorder_device(plan.handle, P.data_ptr(), None, pos.shape[0], 256,
                                                     perm.data_ptr(), ls.data_ptr(),
                                                     torch.cuda.current_stream().cuda_stream))

    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        run()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run()
    perm.zero_()
    g.replay()
    torch.cuda.synchronize()
    perm_h, ls_h = atoms_reorder(pos, 256)
    assert np.array_equal(perm.cpu().numpy(), perm_h) and np.array_equal(ls.cpu().numpy(), ls_h)
