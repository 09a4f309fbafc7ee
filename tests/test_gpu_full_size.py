"""Parity at the full workload sizes, in the launch configuration bench.py times.

The 8x8x8 diamond supercell on 512^3 (4,096 Gaussian charges, sigma 0.5 Bohr),
the orthorhombic 37.9 x 40.4 x 42.1 Bohr cell on 360 x 384 x 400 (1,728
atoms) and the 16x16x8 supercell on the paper's 420 x 420 x 210 grid (16,384
atoms, sigma 0.8 Bohr, radix 7): atoms in the order of the modified recursive bisection with 16 atoms
per leaf, kernel variants picked by the autotuner, and the whole step
(splat, Poisson solve, E_H, forces) in one hartree_step call, against the
FP64 oracle on the host cores with the same per-axis cutoff of 5 sigma.

Bars (FP32 path): V_H and rho relative L2 <= 2e-6, E_H relative <= 1e-7,
forces and dE_H/dq <= 1e-5 absolute.  Also checked: charge neutrality of the
grid density and Newton's third law on the forces.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1209_4506_gb300 import synth
from paper_1209_4506_gb300.hartree import HartreePlan, atoms_reorder

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RC_SIGMAS = 5.0  # the FP32 plans' default per-axis cutoff; the oracle truncates at the same radius


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("name", ["cfg3a", "cfg3b", "paper420"])
def test_full_size_step_matches_oracle(name):
    S = {"cfg3a": synth.config3a, "cfg3b": synth.config3b, "paper420": synth.config_paper420}[name]()
    O.set_threads(os.cpu_count() or 1)
    rho_o = O.splat(S.n, S.cell, S.sigma, S.pos, S.q, RC_SIGMAS)
    vh_o, eh_o, eh_spec, _ = O.poisson(S.cell, rho_o)
    f_o, phi_o = O.forces(S.n, S.cell, S.sigma, S.pos, S.q, vh_o, RC_SIGMAS)

    apl = 16
    perm, _ = atoms_reorder(S.pos, (S.n_atoms + apl - 1) // apl)
    plan = HartreePlan(S.n, S.cell, S.sigma, "fp32", atoms_per_leaf=apl, max_atoms=S.n_atoms)
    plan.autotune()
    pos = torch.tensor(S.pos[perm], device="cuda")
    q = torch.tensor(S.q[perm], device="cuda")
    rho = torch.empty(S.n, dtype=torch.float32, device="cuda")
    vh, eh, f, phi = plan.step(pos, q, rho=rho, want_phi=True)
    torch.cuda.synchronize()
    plan.device_status()
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    f_g = f.cpu().numpy()[inv]
    phi_g = phi.cpu().numpy()[inv]
    rho_g = rho.double().cpu().numpy()
    vh_g = vh.double().cpu().numpy()
    dV = float(np.prod(S.cell)) / S.n_tot

    assert rel_l2(rho_g, rho_o) <= 2e-6
    assert abs(rho_g.sum() * dV - S.q.sum()) <= 1e-6 * np.abs(S.q).sum()
    assert rel_l2(vh_g, vh_o) <= 2e-6
    assert abs(eh.item() - eh_o) <= 1e-7 * abs(eh_o)
    # the oracle's two E_H forms agree to its own FP64 summation error over ~1e8 terms
    assert abs(eh_o - eh_spec) <= 1e-10 * abs(eh_o)
    assert np.max(np.abs(f_g - f_o)) <= 1e-5
    assert np.max(np.abs(phi_g - phi_o)) <= 1e-5
    # Newton's third law: sum F = 0 up to the FP32 error of the 4 N_atoms terms (relative to sum |F|)
    assert np.max(np.abs(f_g.sum(axis=0))) <= 1e-7 * np.abs(f_o).sum()
    plan.close()
