"""Adjoint (autograd) forms of the Hartree energy, checked against the oracle and gradcheck.

dE_H/drho = V_H dV (the discrete gradient of the functional derivative V_H),
dE_H/dR = -F, dE_H/dq = phi; the backward passes recompute V_H.
"""
import numpy as np
import pytest

import oracle as O
from paper_1209_4506_gb300 import synth
from paper_1209_4506_gb300.autograd import hartree_energy, hartree_energy_atoms
from paper_1209_4506_gb300.hartree import HartreePlan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_density_gradient_is_potential_times_dV():
    n, cell = (24, 30, 36), (5.0, 6.2, 7.4)
    rng = np.random.default_rng(3)
    r = rng.standard_normal(n)
    plan = HartreePlan(n, cell, 0.5, "fp64")
    rho = torch.tensor(r, device="cuda", requires_grad=True)
    e = hartree_energy(rho, plan)
    e.backward()
    v_ref, e_ref, _, _ = O.poisson(cell, r)
    dV = np.prod(cell) / np.prod(n)
    assert abs(e.item() - e_ref) <= 1e-12 * abs(e_ref)
    g = rho.grad.cpu().numpy()
    assert np.linalg.norm(g - v_ref * dV) <= 1e-12 * np.linalg.norm(v_ref * dV)


def test_density_gradcheck_tiny_grid():
    plan = HartreePlan((6, 4, 8), (2.0, 1.7, 2.4), 0.5, "fp64")
    rho = torch.randn((6, 4, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: hartree_energy(x, plan), (rho,), eps=1e-6, atol=1e-8, rtol=1e-6)


@pytest.mark.parametrize("store", [False, True])
def test_atom_gradients_match_oracle_forces_fp64(store):
    S = synth.config1()
    ref = O.solve_system(S)
    plan = HartreePlan(S.n, S.cell, S.sigma, "fp64")
    pos = torch.tensor(S.pos, device="cuda", requires_grad=True)
    q = torch.tensor(S.q, device="cuda", requires_grad=True)
    e = hartree_energy_atoms(pos, q, plan, store_potential=store)
    e.backward()
    assert abs(e.item() - ref["eh"]) <= 1e-12 * abs(ref["eh"])
    assert np.max(np.abs(pos.grad.cpu().numpy() + ref["forces"])) <= 1e-10
    assert np.max(np.abs(q.grad.cpu().numpy() - ref["phi"])) <= 1e-10


def test_atom_gradcheck_fp64():
    S = synth.random_system((20, 24, 30), (4.0, 4.5, 5.0), 3, 0.6, seed=4, precision="fp64")
    plan = HartreePlan(S.n, S.cell, S.sigma, "fp64")
    pos = torch.tensor(S.pos, device="cuda", requires_grad=True)
    q = torch.tensor(S.q, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda p, c: hartree_energy_atoms(p, c, plan), (pos, q), eps=1e-5, atol=1e-6,
                                    rtol=1e-5)


def test_atom_gradients_fp32_within_force_tolerance():
    S = synth.config2()
    ref = O.solve_system(S)
    plan = HartreePlan(S.n, S.cell, S.sigma, "fp32")
    pos = torch.tensor(S.pos, device="cuda", requires_grad=True)
    q = torch.tensor(S.q, device="cuda")
    e = hartree_energy_atoms(pos, q, plan)
    (2.0 * e).backward()
    assert np.max(np.abs(pos.grad.cpu().numpy() + 2.0 * ref["forces"])) <= 2e-5
    assert q.grad is None
