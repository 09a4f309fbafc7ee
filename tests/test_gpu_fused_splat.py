"""The splat fused into the r2c pass (FP32 plans with HARTREE_FLAG_FUSED_SPLAT).

With the flag, hartree_step / hartree_solve with rho = NULL compute each tile's density inside
the first transform pass, so the density never reaches device memory.  Checked here through the
C ABI:
  * element-wise parity with the FP64 oracle: V_H (relative L2 <= 2e-6 and max abs), E_H
    (relative <= 1e-7), forces and dE_H/dq (<= 1e-5 Ha/Bohr) at the 64-atom diamond cell on
    120^3 (c half length M = 60, 16-line tiles that stop short at N2 = 120);
  * the fused path ran: one launch fewer than the same step with a density grid;
  * agreement with the separate splat (the default) on every compiled line length, to FP32
    rounding of the different summation order;
  * edge cases: no atoms, boxes wider than the cell (several images per point), more leaves
    than one CTA scans at once and more atoms per tile than one staging batch holds;
  * bitwise repeatability.
The full-size grids (512^3, 360 x 384 x 400, 420 x 420 x 210, 420^3) are compared with the
oracle in test_gpu_full_size.py, fused and separate.
"""
FUSED = 2  # HARTREE_FLAG_FUSED_SPLAT
import functools
import os

import numpy as np
import pytest

import oracle as O
from paper_1209_4506_gb300 import capi, synth
from paper_1209_4506_gb300.hartree import HartreePlan, atoms_reorder

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = dict(v=2e-6, e=1e-7, f=1e-5)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), device="cuda")


@functools.lru_cache(maxsize=None)
def oracle_system(name):
    O.set_threads(os.cpu_count() or 1)
    S = {"cfg2": synth.config2}[name]()
    return S, O.solve_system(S)


def fused_step(S, order=None, **plan_kw):
    """(vh, eh, forces, phi, launches) of one hartree_step with no density grid."""
    pos, q = (S.pos, S.q) if order is None else (S.pos[order], S.q[order])
    plan = HartreePlan(S.n, S.cell, S.sigma, "fp32", max_atoms=max(len(q), 1), flags=FUSED, **plan_kw)
    assert plan.fused_splat
    P, Q = dev(pos), dev(q)
    n0 = plan.launch_count
    vh, eh, f, phi = plan.step(P, Q, want_phi=True)
    torch.cuda.synchronize()
    plan.device_status()
    launches = plan.launch_count - n0
    out = dict(vh=vh.double().cpu().numpy(), eh=float(eh.item()), f=f.cpu().numpy(), phi=phi.cpu().numpy(),
               launches=launches)
    if order is not None:
        inv = np.empty_like(order)
        inv[order] = np.arange(len(order))
        out["f"], out["phi"] = out["f"][inv], out["phi"][inv]
    plan.close()
    return out


def check_oracle(g, ref):
    assert rel_l2(g["vh"], ref["vh"]) <= TOL["v"]
    assert np.max(np.abs(g["vh"] - ref["vh"])) <= TOL["v"] * np.max(np.abs(ref["vh"])) * 4
    assert abs(g["eh"] - ref["eh"]) <= TOL["e"] * abs(ref["eh"])
    assert np.max(np.abs(g["f"] - ref["forces"])) <= TOL["f"]
    assert np.max(np.abs(g["phi"] - ref["phi"])) <= TOL["f"]


@pytest.mark.parametrize("apl", [16, 1])
def test_fused_step_matches_oracle_cfg2(apl):
    """apl = 1: 64 leaves of one atom each (every atom selected through its own leaf box)."""
    S, ref = oracle_system("cfg2")
    perm, _ = atoms_reorder(S.pos, (S.n_atoms + apl - 1) // apl)
    g = fused_step(S, order=perm, atoms_per_leaf=apl)
    check_oracle(g, ref)


def test_fused_path_is_taken_and_saves_a_launch():
    assert capi.HARTREE_FLAG_FUSED_SPLAT == FUSED
    S = synth.config2()
    plan = HartreePlan(S.n, S.cell, S.sigma, "fp32", flags=FUSED)
    P, Q = dev(S.pos), dev(S.q)
    rho = torch.empty(S.n, dtype=torch.float32, device="cuda")
    n0 = plan.launch_count
    plan.step(P, Q, rho=rho)
    n1 = plan.launch_count
    plan.step(P, Q)
    n2 = plan.launch_count
    torch.cuda.synchronize()
    assert (n2 - n1) == (n1 - n0) - 1
    sep = HartreePlan(S.n, S.cell, S.sigma, "fp32")
    assert not sep.fused_splat
    m0 = sep.launch_count
    sep.step(P, Q)
    assert sep.launch_count - m0 == n1 - n0
    plan.close()
    sep.close()


# one grid per compiled line length of the fused kernel (M = N3 / 2), N2 not always a multiple of 16
FUSED_GRIDS = [
    ((40, 36, 120), (9.0, 8.0, 26.0)),   # M = 60
    ((32, 40, 128), (7.0, 8.5, 27.0)),   # M = 64
    ((24, 20, 210), (5.0, 4.5, 45.0)),   # M = 105
    ((36, 48, 256), (8.0, 10.0, 54.0)),  # M = 128
    ((20, 24, 400), (4.5, 5.0, 84.0)),   # M = 200
    ((16, 18, 420), (3.5, 4.0, 90.0)),   # M = 210
    ((12, 32, 512), (2.5, 7.0, 108.0)),  # M = 256
]


@pytest.mark.parametrize("n,cell", FUSED_GRIDS)
def test_fused_equals_separate_splat(n, cell):
    S = synth.random_system(n, cell, 40, 0.45, seed=sum(n), precision="fp32")
    perm, _ = atoms_reorder(S.pos, 5)
    P, Q = dev(S.pos[perm]), dev(S.q[perm])
    outs = []
    for flags in (FUSED, 0):
        plan = HartreePlan(n, cell, S.sigma, "fp32", atoms_per_leaf=8, max_atoms=40, flags=flags)
        vh, eh, f = plan.step(P, Q)
        torch.cuda.synchronize()
        plan.device_status()
        outs.append((vh.double().cpu().numpy(), eh.item(), f.cpu().numpy()))
        plan.close()
    (v1, e1, f1), (v2, e2, f2) = outs
    assert rel_l2(v1, v2) <= 1e-6
    assert abs(e1 - e2) <= 1e-7 * abs(e2)
    assert np.max(np.abs(f1 - f2)) <= 1e-5


@pytest.mark.parametrize("n,cell", [FUSED_GRIDS[0], FUSED_GRIDS[3]])
def test_fused_wide_cutoff_many_images_matches_oracle(n, cell):
    """Boxes wider than the cell along a and b (several images per grid point), and along c for
    the 26 Bohr cell: the image sums of the staged factors."""
    S = synth.random_system(n, (2.5, 3.0, cell[2] / 10.0), 6, 0.6, seed=91, precision="fp32")
    ref = O.solve_system(S, rc_sigmas=8.0)
    g = fused_step(S, cutoff_sigmas=8.0)
    check_oracle(g, ref)


@pytest.mark.parametrize("n_atoms", [300, 1100])
def test_fused_dense_tiles_span_several_batches_and_leaf_rounds(n_atoms):
    """Atoms in a small cell on a 120-point c axis, one atom per leaf, every box covering the whole
    a and b range: 300 or 1100 leaf boxes (two or five rounds of 256), every tile takes more
    atoms than one staging batch holds, and with 1100 atoms a unit of tiles selects more atoms
    than its records hold, so its tiles select theirs in rounds."""
    S = synth.random_system((24, 20, 120), (4.0, 3.5, 20.0), n_atoms, 0.5, seed=5, precision="fp32")
    ref = O.solve_system(S)
    perm, _ = atoms_reorder(S.pos, n_atoms)
    g = fused_step(S, order=perm, atoms_per_leaf=1)
    check_oracle(g, ref)


def test_fused_pass_needs_the_flag():
    """hartree_splat_pass refuses plans that do not use the fused kernel: no flag, or FP64."""
    S = synth.config2()
    P, Q = dev(S.pos), dev(S.q)
    for precision, flags in (("fp32", 0), ("fp64", FUSED)):
        plan = HartreePlan(S.n, S.cell, S.sigma, precision, flags=flags)
        assert not plan.fused_splat
        with pytest.raises(capi.HartreeError) as ei:
            plan.splat_pass(P, Q)
        assert ei.value.status == capi.HARTREE_ERR_UNSUPPORTED_SIZE
        plan.close()


def test_fused_no_atoms():
    S = synth.config2()
    plan = HartreePlan(S.n, S.cell, S.sigma, "fp32", flags=FUSED)
    P = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    Q = torch.empty((0,), dtype=torch.float64, device="cuda")
    vh, eh = plan.solve(P, Q)
    torch.cuda.synchronize()
    assert float(vh.abs().max()) == 0.0 and eh.item() == 0.0
    plan.close()


def test_fused_repeat_runs_are_bitwise_deterministic():
    S = synth.config2()
    a = fused_step(S)
    b = fused_step(S)
    assert np.array_equal(a["vh"], b["vh"]) and a["eh"] == b["eh"] and np.array_equal(a["f"], b["f"])
