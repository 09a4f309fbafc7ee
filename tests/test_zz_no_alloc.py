"""The allocation-free Poisson solve, hartree_solve_density_noalloc.

Some callers cannot call cudaMalloc: applications that give all device memory
to their own allocator or pool up front, and code paths where a device
allocation is not allowed or would stall other work.  For them the library
offers a Poisson solve that needs no plan and allocates nothing; it works in a
fixed 8 MiB scratch array that the library declares at file scope.

These tests call that entry point through the C ABI three times in a row
(FP32, then FP64, then FP32 again on the shared scratch) and compare every
result with the FP64 oracle and with the plan-based hartree_solve_density on
the same density, within the tolerances the other parity tests use.  They also
check that a call leaves the device's free memory unchanged.  This file runs
last so that a failure here comes after every other test has already run; it
also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1209_4506_gb300 import capi, synth
from paper_1209_4506_gb300.hartree import HartreePlan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(v=1e-12, e=1e-12), "fp32": dict(v=2e-6, e=1e-7)}


def desc_for(n, cell, precision):
    d = capi.hartree_desc()
    for i in range(3):
        d.n[i] = n[i]
        d.cell[i] = cell[i]
    d.sigma = 0.5
    d.cutoff_sigmas = 0.0
    d.precision = capi.HARTREE_FP64 if precision == "fp64" else capi.HARTREE_FP32
    d.atoms_per_leaf = 0
    d.max_atoms = 0
    d.flags = 0
    return d


def solve_noalloc(n, cell, precision, rho):
    vh = torch.empty_like(rho)
    eh = torch.empty((), dtype=torch.float64, device=rho.device)
    stream = torch.cuda.current_stream().cuda_stream
    st = capi.hartree_solve_density_noalloc(ctypes.byref(desc_for(n, cell, precision)), rho.data_ptr(),
                                            vh.data_ptr(), eh.data_ptr(), stream)
    capi.check(st)
    torch.cuda.synchronize()
    return vh, eh


def solve_plan(n, cell, precision, rho):
    plan = HartreePlan(n, cell, 0.5, precision)
    vh, eh = plan.solve_density(rho)
    torch.cuda.synchronize()
    plan.close()
    return vh, eh


def rel_l2(a, b):
    return float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))


def fp32_case():
    S = synth.config2()  # 64 diamond atoms, 120^3 grid
    plan = HartreePlan(S.n, S.cell, S.sigma, "fp32")
    rho = plan.splat(torch.tensor(S.pos, device="cuda"), torch.tensor(S.q, device="cuda"))
    torch.cuda.synchronize()
    return S.n, S.cell, rho


def fp64_case():
    n, cell = (64, 48, 40), (9.0, 7.0, 6.0)
    S = synth.random_system(n, cell, 12, 0.6, seed=99, precision="fp64")
    plan = HartreePlan(n, cell, 0.6, "fp64")
    rho = plan.splat(torch.tensor(S.pos, device="cuda"), torch.tensor(S.q, device="cuda"))
    torch.cuda.synchronize()
    return n, cell, rho


def test_noalloc_matches_plan_solve_on_consecutive_calls():
    n32, c32, rho32 = fp32_case()
    n64, c64, rho64 = fp64_case()
    # three calls in a row on the shared scratch: FP32, FP64, FP32 again
    v1, e1 = solve_noalloc(n32, c32, "fp32", rho32)
    v2, e2 = solve_noalloc(n64, c64, "fp64", rho64)
    v3, e3 = solve_noalloc(n32, c32, "fp32", rho32)
    r32, f32 = solve_plan(n32, c32, "fp32", rho32)
    r64, f64 = solve_plan(n64, c64, "fp64", rho64)
    assert rel_l2(v1, r32) <= TOL["fp32"]["v"]
    assert abs(e1.item() - f32.item()) <= TOL["fp32"]["e"] * abs(f32.item())
    assert rel_l2(v2, r64) <= TOL["fp64"]["v"]
    assert abs(e2.item() - f64.item()) <= TOL["fp64"]["e"] * abs(f64.item())
    # the scratch keeps the previous call's contents; nothing of it leaks into the next result
    assert torch.equal(v3, v1) and e3.item() == e1.item()
    # and against the FP64 oracle on the same (rounded) densities
    for v, e, c, rho, prec in ((v1, e1, c32, rho32, "fp32"), (v2, e2, c64, rho64, "fp64")):
        v_ref, e_ref, _, _ = O.poisson(c, rho.double().cpu().numpy())
        assert rel_l2(v, torch.tensor(v_ref, device=v.device)) <= TOL[prec]["v"]
        assert abs(e.item() - e_ref) <= TOL[prec]["e"] * abs(e_ref)


def test_noalloc_allocates_no_device_memory():
    n32, c32, rho32 = fp32_case()
    vh = torch.empty_like(rho32)
    eh = torch.empty((), dtype=torch.float64, device=rho32.device)
    stream = torch.cuda.current_stream().cuda_stream
    d = desc_for(n32, c32, "fp32")
    capi.check(capi.hartree_solve_density_noalloc(ctypes.byref(d), rho32.data_ptr(), vh.data_ptr(), eh.data_ptr(),
                                                  stream))  # warm-up: the per-device set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    capi.check(capi.hartree_solve_density_noalloc(ctypes.byref(d), rho32.data_ptr(), vh.data_ptr(), eh.data_ptr(),
                                                  stream))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_grids_beyond_the_scratch():
    n, cell = (128, 128, 128), (10.0, 10.0, 10.0)  # half spectrum 10.5 MB > 8 MiB
    rho = torch.zeros(n, dtype=torch.float32, device="cuda")
    vh = torch.empty_like(rho)
    st = capi.hartree_solve_density_noalloc(ctypes.byref(desc_for(n, cell, "fp32")), rho.data_ptr(), vh.data_ptr(),
                                            None, torch.cuda.current_stream().cuda_stream)
    assert st == capi.HARTREE_ERR_UNSUPPORTED_SIZE
    assert b"8 MiB" in capi.hartree_last_error()
