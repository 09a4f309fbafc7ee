"""Host-side checks of the C-ABI library that need no GPU.

* the shared library loads and exports every function include/hartree.h declares;
* plan validation rejects bad descriptors before touching the device;
* the library's host bisection (hartree_atoms_reorder) reproduces the oracle's
  modified recursive bisection exactly on inputs with a well-separated
  principal axis, and is a valid decomposition otherwise.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1209_4506_gb300 import capi, synth
from paper_1209_4506_gb300.hartree import atoms_reorder

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names.update(re.findall(r"\b(hartree_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    lib = capi.lib()
    declared = declared_functions()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} is declared but not exported"
    assert declared == set(capi.EXPORTED)


def test_status_strings():
    lib = capi.lib()
    for st in range(7):
        assert lib.hartree_status_string(st)
    assert lib.hartree_status_string(99) == b"unknown status"


def _desc(n=(32, 32, 32), cell=(6.0, 6.0, 6.0), sigma=0.5, prec=capi.HARTREE_FP32, cutoff=0.0):
    d = capi.hartree_desc()
    for i in range(3):
        d.n[i] = n[i]
        d.cell[i] = cell[i]
    d.sigma = sigma
    d.cutoff_sigmas = cutoff
    d.precision = prec
    d.atoms_per_leaf = 0
    d.max_atoms = 0
    d.flags = 0
    return d


@pytest.mark.parametrize(
    "kw,status",
    [
        (dict(n=(32, 32, 33)), capi.HARTREE_ERR_UNSUPPORTED_SIZE),  # odd N3
        (dict(n=(32, 11, 32)), capi.HARTREE_ERR_UNSUPPORTED_SIZE),  # prime 11 (radices are 2, 3, 5, 7)
        (dict(n=(1, 32, 32)), capi.HARTREE_ERR_UNSUPPORTED_SIZE),
        (dict(n=(32, 32, 2)), capi.HARTREE_ERR_UNSUPPORTED_SIZE),
        (dict(n=(8192, 32, 32)), capi.HARTREE_ERR_UNSUPPORTED_SIZE),
        (dict(cell=(6.0, -1.0, 6.0)), capi.HARTREE_ERR_INVALID),
        (dict(cell=(6.0, float("nan"), 6.0)), capi.HARTREE_ERR_INVALID),
        (dict(sigma=0.0), capi.HARTREE_ERR_INVALID),
        (dict(cutoff=17.0), capi.HARTREE_ERR_INVALID),
        (dict(prec=7), capi.HARTREE_ERR_INVALID),
        (dict(n=(32, 32, 32), cell=(600.0, 6.0, 6.0), sigma=20.0, cutoff=16.0), capi.HARTREE_ERR_UNSUPPORTED_SIZE),
    ],
)
def test_plan_validation_rejects_before_any_device_work(kw, status):
    h = ctypes.c_void_p()
    st = capi.hartree_plan_create(ctypes.byref(_desc(**kw)), ctypes.byref(h))
    assert st == status
    assert not h.value
    assert capi.hartree_last_error()


def test_null_arguments_are_rejected():
    assert capi.hartree_plan_create(None, None) == capi.HARTREE_ERR_INVALID
    assert capi.hartree_solve(None, None, None, 0, None, None, None, None) == capi.HARTREE_ERR_INVALID
    assert capi.hartree_forces(None, None, None, 0, None, None, None, None) == capi.HARTREE_ERR_INVALID
    assert capi.hartree_splat(None, None, None, 0, None, None) == capi.HARTREE_ERR_INVALID
    assert capi.hartree_solve_density(None, None, None, None, None) == capi.HARTREE_ERR_INVALID
    assert capi.hartree_step_host(None, None, None, 0, None, None, None) == capi.HARTREE_ERR_INVALID
    capi.hartree_plan_destroy(None)


# ------------------------------------------------------------------ bisection parity
def _top_gap(pos):
    C = pos.mean(axis=0)
    X = pos - C
    lam = np.linalg.eigvalsh(X.T @ X)
    return (lam[2] - lam[1]) / lam[2]


CASES = {
    "cfg1-8atoms-4leaves": (lambda: synth.config1().pos, 4),
    "cfg2-64atoms-4leaves": (lambda: synth.config2().pos, 4),
    "cfg2-64atoms-64leaves": (lambda: synth.config2().pos, 64),
    "cfg3a-4096atoms-256leaves": (lambda: synth.config3a().pos, 256),
    "cfg3b-ortho-108leaves": (lambda: synth.config3b().pos, 108),
    "cfg5-512atoms-32leaves": (lambda: synth.config5().pos, 32),
    "random-1000-19": (lambda: np.random.default_rng(3).uniform(0, [20, 30, 40], (1000, 3)), 19),
    "diamond16384-19": (lambda: synth.jitter(np.random.default_rng(5), synth.diamond_supercell((16, 16, 8)), 0.1,
                                             (16 * 6.74, 16 * 6.74, 8 * 6.74)), 19),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_library_bisection_matches_oracle(case):
    make, nl = CASES[case]
    pos = make()
    perm_o, ls_o = O.bisect(pos, nl)
    perm_l, ls_l = atoms_reorder(pos, nl)
    assert ls_l.tolist() == ls_o.tolist()
    assert perm_l.tolist() == perm_o.tolist()


def test_library_bisection_weighted_matches_oracle():
    rng = np.random.default_rng(12)
    pos = rng.uniform(0, 15, (700, 3)) * np.array([1.0, 0.6, 0.3])
    w = rng.uniform(0.1, 1.0, 700)
    perm_o, ls_o = O.bisect(pos, 13, w)
    perm_l, ls_l = atoms_reorder(pos, 13, w)
    assert ls_l.tolist() == ls_o.tolist()
    assert perm_l.tolist() == perm_o.tolist()


def test_library_bisection_degenerate_input_is_valid():
    """Unjittered cubic diamond has a degenerate inertia tensor: any principal
    axis in the degenerate plane is correct, so only validity is checked."""
    pos = synth.diamond_supercell((4, 4, 4))
    perm, ls = atoms_reorder(pos, 8)
    assert sorted(perm.tolist()) == list(range(len(pos)))
    sizes = np.diff(ls)
    assert sizes.max() - sizes.min() <= 1 and sizes.sum() == len(pos)


@pytest.mark.parametrize("n,nl", [(0, 1), (0, 5), (1, 1), (1, 3), (5, 8), (3, 3)])
def test_library_bisection_edge_counts(n, nl):
    pos = np.random.default_rng(n * 10 + nl).uniform(0, 5, (n, 3))
    perm_o, ls_o = O.bisect(pos, nl)
    perm_l, ls_l = atoms_reorder(pos, nl)
    assert ls_l.tolist() == ls_o.tolist()
    assert perm_l.tolist() == perm_o.tolist()


def test_library_bisection_rejects_bad_input():
    pos = np.zeros((4, 3))
    pos[2, 1] = np.nan
    with pytest.raises(capi.HartreeError):
        atoms_reorder(pos, 2)
    with pytest.raises(capi.HartreeError):
        atoms_reorder(np.zeros((4, 3)), 0)


def _fp32_desc(prec=None):
    d = capi.hartree_desc()
    for i in range(3):
        d.n[i] = 48
        d.cell[i] = 8.0
    d.sigma = 0.6
    d.precision = capi.HARTREE_FP32 if prec is None else prec
    return d


def test_batch_create_rejects_before_any_device_work():
    h = ctypes.c_void_p()
    descs = (capi.hartree_desc * 3)(_fp32_desc(), _fp32_desc(), _fp32_desc(capi.HARTREE_FP64))
    counts = np.array([4, 0, 7], dtype=np.int32)
    # the third cell is FP64: rejected before the first cell's workspace is created
    assert capi.hartree_batch_create(descs, counts.ctypes.data, 3, ctypes.byref(h)) == capi.HARTREE_ERR_INVALID
    assert h.value is None
    descs[2] = _fp32_desc()
    bad = np.array([4, -1, 7], dtype=np.int32)
    assert capi.hartree_batch_create(descs, bad.ctypes.data, 3, ctypes.byref(h)) == capi.HARTREE_ERR_INVALID
    assert capi.hartree_batch_create(descs, counts.ctypes.data, 0, ctypes.byref(h)) == capi.HARTREE_ERR_INVALID
    assert capi.hartree_batch_create(None, None, 1, None) == capi.HARTREE_ERR_INVALID
    assert capi.hartree_solve_batched(None, None, None, None, None, None) == capi.HARTREE_ERR_INVALID
    assert capi.hartree_batch_offsets(None, None, None) == capi.HARTREE_ERR_INVALID
    assert capi.hartree_batch_device_status(None) == capi.HARTREE_ERR_INVALID
    capi.hartree_batch_destroy(None)


def test_split_precision_requires_n2_256():
    d = _fp32_desc(capi.HARTREE_FP32_TC_SPLIT)  # 48^3
    h = ctypes.c_void_p()
    assert capi.hartree_plan_create(ctypes.byref(d), ctypes.byref(h)) == capi.HARTREE_ERR_UNSUPPORTED_SIZE
    assert b"N2 = 256" in capi.hartree_last_error()


def test_paper_decomposition_experiment_16384_atoms_19_processes():
    """The experiment of Sec. 5.2.1: 16,384 diamond atoms split over 19 processes by the modified
    recursive bisection.  Every leaf holds 862 or 863 atoms (w = 1), and the leaves are compact:
    their mean radius of gyration is within 25% of a cube of the same volume and less than half
    that of a random 19-way split."""
    rng = np.random.default_rng(5)
    cell = (16 * 6.74, 16 * 6.74, 8 * 6.74)
    pos = synth.jitter(rng, synth.diamond_supercell((16, 16, 8)), 0.1, cell)
    perm, ls = atoms_reorder(pos, 19)
    sizes = np.diff(ls)
    assert sizes.sum() == 16384 and sizes.min() == 862 and sizes.max() == 863

    def rg(p):
        return np.sqrt(((p - p.mean(0)) ** 2).sum(1).mean())

    r_bis = np.mean([rg(pos[perm[ls[i]:ls[i + 1]]]) for i in range(19)])
    rnd = np.random.default_rng(0).permutation(len(pos))
    r_rand = np.mean([rg(pos[rnd[ls[i]:ls[i + 1]]]) for i in range(19)])
    r_cube = (np.prod(cell) / 19) ** (1 / 3) * np.sqrt(3 / 12)
    assert r_bis <= 1.25 * r_cube
    assert r_bis <= 0.5 * r_rand
