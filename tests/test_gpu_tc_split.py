"""HARTREE_FP32_TC_SPLIT: the b passes as two radix-16 stages on the tensor cores.

Each 16-point DFT is a 16-bit matrix product with split operands and FP32
accumulation.  FP16 parts (the default, rows scaled by a power of two):
x_h M_h + x_h M_l + x_l M_h, dropped terms about 2^-22 relative per product.
BF16 parts (HARTREE_FLAG_TC_BF16): three parts per value, the six products of
order <= 2, dropped terms about 2^-24.  Both meet the split-path bars against
the FP64 oracle: V_H 1e-5 relative L2, E_H 1e-5 relative, forces 1e-5 Ha/Bohr.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1209_4506_gb300 import capi, synth
from paper_1209_4506_gb300.autograd import hartree_energy_atoms
from paper_1209_4506_gb300.hartree import HartreePlan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_V, TOL_E, TOL_F = 1e-5, 1e-5, 1e-5


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


FLAGS = {"fp16": 0, "bf16": capi.HARTREE_FLAG_TC_BF16}


@pytest.mark.parametrize("parts", ["fp16", "bf16"])
@pytest.mark.parametrize("n,cell", [((8, 256, 32), (2.0, 30.0, 4.0)), ((16, 256, 24), (3.0, 27.0, 3.5)),
                                    ((5, 256, 6), (1.0, 20.0, 1.5))])
def test_split_poisson_of_white_noise(n, cell, parts):
    rng = np.random.default_rng(sum(n))
    rho = rng.standard_normal(n)
    v_ref, e_ref, _, _ = O.poisson(cell, rho)
    plan = HartreePlan(n, cell, 0.5, "bf16split", flags=FLAGS[parts])
    vh, eh = plan.solve_density(torch.tensor(rho, dtype=torch.float32, device="cuda"))
    plan.device_status()
    assert rel_l2(vh.double().cpu().numpy(), v_ref) <= TOL_V
    # white noise: E_H is dominated by the few smallest |G|, each carrying the split error of one coefficient
    assert abs(eh.item() - e_ref) <= 2 * TOL_E * abs(e_ref)


def test_split_matches_fp32_path_closely():
    # the same density through the FP32 and the split plans: only the b passes differ
    n, cell = (32, 256, 40), (5.0, 30.0, 6.0)
    S = synth.random_system(n, cell, 40, 0.6, seed=8, precision="fp32")
    P32 = HartreePlan(n, cell, 0.6, "fp32")
    PTC = HartreePlan(n, cell, 0.6, "bf16split")
    pos, q = torch.tensor(S.pos, device="cuda"), torch.tensor(S.q, device="cuda")
    v1, e1 = P32.solve(pos, q)
    v2, e2 = PTC.solve(pos, q)
    assert rel_l2(v2.double().cpu().numpy(), v1.double().cpu().numpy()) <= TOL_V
    assert abs(e2.item() - e1.item()) <= TOL_E * abs(e1.item())


@pytest.fixture(scope="module")
def cfg5():
    O.set_threads(os.cpu_count() or 1)
    S = synth.config5()
    return S, O.solve_system(S, rc_sigmas=8.0)


@pytest.mark.parametrize("parts", ["fp16", "bf16"])
def test_config5_step_matches_oracle(cfg5, parts):
    S, ref = cfg5
    plan = HartreePlan(S.n, S.cell, S.sigma, "bf16split", flags=FLAGS[parts])
    pos, q = torch.tensor(S.pos, device="cuda"), torch.tensor(S.q, device="cuda")
    vh, eh, f = plan.step(pos, q)
    plan.device_status()
    assert rel_l2(vh.double().cpu().numpy(), ref["vh"]) <= TOL_V
    assert abs(eh.item() - ref["eh"]) <= TOL_E * abs(ref["eh"])
    assert np.max(np.abs(f.cpu().numpy() - ref["forces"])) <= TOL_F


def test_config5_autograd_forward_backward(cfg5):
    S, ref = cfg5
    plan = HartreePlan(S.n, S.cell, S.sigma, "bf16split")
    pos = torch.tensor(S.pos, device="cuda", requires_grad=True)
    q = torch.tensor(S.q, device="cuda", requires_grad=True)
    e = hartree_energy_atoms(pos, q, plan)  # backward recomputes V_H; nothing of the spectrum is kept
    e.backward()
    assert abs(e.item() - ref["eh"]) <= TOL_E * abs(ref["eh"])
    assert np.max(np.abs(-pos.grad.cpu().numpy() - ref["forces"])) <= TOL_F
    assert np.max(np.abs(q.grad.cpu().numpy() - ref["phi"])) <= 1e-4 * np.max(np.abs(ref["phi"]))


def test_bf16_three_part_split_is_near_fp32():
    """BF16 with three parts carries 24 significant bits per value: the split path's V_H differs from
    the FP32 path's by FP32 rounding (radix 16 x 16 on the tensor cores against the FP32 path's own
    radix order), within the FP32 path's own bar of 2e-6, five times inside the split bar."""
    n, cell = (8, 256, 32), (2.0, 30.0, 4.0)
    rho = torch.tensor(np.random.default_rng(sum(n)).standard_normal(n), dtype=torch.float32, device="cuda")
    v32, _ = HartreePlan(n, cell, 0.5, "fp32").solve_density(rho)
    plan = HartreePlan(n, cell, 0.5, "bf16split", flags=capi.HARTREE_FLAG_TC_BF16)
    vh, _ = plan.solve_density(rho)
    plan.device_status()
    assert rel_l2(vh.double().cpu().numpy(), v32.double().cpu().numpy()) <= 2e-6
