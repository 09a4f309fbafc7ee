"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (stated per result):
  FP64 path: V_H relative L2 <= 1e-12, E_H relative <= 1e-12, forces <= 1e-10 Ha/Bohr
  FP32 path: V_H relative L2 <= 2e-6,  E_H relative <= 1e-7,  forces <= 1e-5 Ha/Bohr
"""
import functools
import os

import numpy as np
import pytest

import oracle as O
from paper_1209_4506_gb300 import synth
from paper_1209_4506_gb300.hartree import HartreePlan, atoms_reorder

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {
    "fp64": dict(v=1e-12, e=1e-12, f=1e-10),
    "fp32": dict(v=2e-6, e=1e-7, f=1e-5),
}
# White-noise densities are not the physical workload: their E_H = sum_k g_k |rho~_k|^2
# is dominated by the few smallest |G| (g = 4 pi / G^2 with |rho~_k| flat), so it
# averages nothing and inherits the FP32 transform error of single coefficients,
# 2 eps sqrt(log2 N) ~ 2 * 6e-8 * 4.6 ~ 5.5e-7 for N <= 2^21.  Bar: 1e-6.
WHITE_NOISE_E_TOL = {"fp64": 1e-12, "fp32": 1e-6}


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), device="cuda")


@functools.lru_cache(maxsize=None)
def oracle_cfg(name):
    O.set_threads(os.cpu_count() or 1)
    S = {"cfg1": synth.config1, "cfg2": synth.config2, "cfg5": synth.config5}[name]()
    return S, O.solve_system(S)


def gpu_step(S, precision, pos=None, q=None, order=None, **plan_kw):
    pos = S.pos if pos is None else pos
    q = S.q if q is None else q
    plan = HartreePlan(S.n, S.cell, S.sigma, precision, **plan_kw)
    if order is not None:
        pos, q = pos[order], q[order]
    P, Q = dev(pos), dev(q)
    vh, eh, rho = plan.solve(P, Q, want_rho=True)
    f, phi = plan.forces(P, Q, vh)
    torch.cuda.synchronize()
    out = dict(vh=vh.cpu().numpy().astype(np.float64), rho=rho.cpu().numpy().astype(np.float64), eh=float(eh.item()),
               forces=f.cpu().numpy(), phi=phi.cpu().numpy())
    if order is not None:
        inv = np.empty_like(order)
        inv[order] = np.arange(len(order))
        out["forces"] = out["forces"][inv]
        out["phi"] = out["phi"][inv]
    plan.close()
    return out


# ------------------------------------------------------------------ Poisson solve of a given density
POISSON_SHAPES = [
    ((24, 30, 36), (5.0, 6.2, 7.4)),
    ((48, 40, 60), (9.1, 7.7, 11.3)),
    ((45, 27, 20), (8.0, 5.0, 4.0)),  # odd N1, N2 (radix 3, 5 only)
    ((16, 16, 16), (4.0, 4.0, 4.0)),
    ((2, 2, 4), (1.0, 1.5, 2.0)),  # smallest grid: single-stage transforms on every axis
    ((128, 96, 80), (20.0, 15.0, 12.5)),
    ((64, 64, 512), (8.0, 8.0, 60.0)),  # long c lines
    ((512, 8, 8), (60.0, 2.0, 2.0)),  # long a lines
    ((4096, 4, 4), (400.0, 1.0, 1.0)),  # largest axis, a
    ((4, 4096, 4), (1.0, 400.0, 1.0)),  # largest axis, b
    ((4, 4, 4096), (1.0, 1.0, 400.0)),  # largest axis, c
    ((120, 120, 120), (13.48, 13.48, 13.48)),
    ((14, 21, 28), (3.0, 4.5, 6.0)),  # radix 7 on every axis
    ((70, 42, 84), (15.0, 9.0, 18.0)),  # 7 with 2, 3, 5 (c: M = 42)
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,cell", POISSON_SHAPES)
def test_poisson_matches_oracle(shape, cell, precision):
    rng = np.random.default_rng(sum(shape))
    rho = rng.standard_normal(shape)
    v_ref, e_ref, e_spec, _ = O.poisson(cell, rho)
    plan = HartreePlan(shape, cell, 0.5, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    r = torch.tensor(rho, dtype=dt, device="cuda")
    vh, eh = plan.solve_density(r)
    torch.cuda.synchronize()
    v = vh.double().cpu().numpy()
    # the FP32 input is itself rounded: compare against the oracle on the same rounded input
    if precision == "fp32":
        v_ref, e_ref, _, _ = O.poisson(cell, rho.astype(np.float32).astype(np.float64))
    assert rel_l2(v, v_ref) <= TOL[precision]["v"]
    assert abs(eh.item() - e_ref) <= WHITE_NOISE_E_TOL[precision] * abs(e_ref)
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_poisson_aliasing_rho_and_vh(precision):
    shape, cell = (24, 30, 36), (5.0, 6.2, 7.4)
    rng = np.random.default_rng(1)
    rho = rng.standard_normal(shape)
    dt = torch.float64 if precision == "fp64" else torch.float32
    rho_in = rho if precision == "fp64" else rho.astype(np.float32).astype(np.float64)
    v_ref = O.poisson(cell, rho_in)[0]
    plan = HartreePlan(shape, cell, 0.5, precision)
    buf = torch.tensor(rho, dtype=dt, device="cuda")
    plan.solve_density(buf, vh=buf)
    torch.cuda.synchronize()
    assert rel_l2(buf.double().cpu().numpy(), v_ref) <= TOL[precision]["v"]


# ------------------------------------------------------------------ full step: splat + solve + forces
@pytest.mark.parametrize("name,precision", [("cfg1", "fp64"), ("cfg2", "fp32"), ("cfg2", "fp64"), ("cfg1", "fp32")])
def test_full_step_matches_oracle(name, precision):
    S, ref = oracle_cfg(name)
    g = gpu_step(S, precision)
    tol = TOL[precision]
    assert rel_l2(g["rho"], ref["rho"]) <= tol["v"]
    assert rel_l2(g["vh"], ref["vh"]) <= tol["v"]
    assert abs(g["eh"] - ref["eh"]) <= tol["e"] * abs(ref["eh"])
    assert np.max(np.abs(g["forces"] - ref["forces"])) <= tol["f"]
    assert np.max(np.abs(g["phi"] - ref["phi"])) <= tol["f"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_leaf_larger_than_the_setup_block(precision):
    """All 64 atoms of config 2 in one leaf: the setup kernel's (atom, axis) tasks (192) and its
    per-atom binning warps take several rounds of its 128 threads."""
    S, ref = oracle_cfg("cfg2")
    g = gpu_step(S, precision, atoms_per_leaf=64, max_atoms=64)
    tol = TOL[precision]
    assert rel_l2(g["rho"], ref["rho"]) <= tol["v"]
    assert rel_l2(g["vh"], ref["vh"]) <= tol["v"]
    assert abs(g["eh"] - ref["eh"]) <= tol["e"] * abs(ref["eh"])
    assert np.max(np.abs(g["forces"] - ref["forces"])) <= tol["f"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_bisection_order_changes_nothing(precision):
    S, ref = oracle_cfg("cfg2")
    perm, _ = atoms_reorder(S.pos, 4)
    a = gpu_step(S, precision)
    b = gpu_step(S, precision, order=perm)
    rnd = np.random.default_rng(0).permutation(S.n_atoms)
    c = gpu_step(S, precision, order=rnd)
    tol = TOL[precision]
    for other in (b, c):
        assert rel_l2(other["vh"], a["vh"]) <= tol["v"]
        assert np.max(np.abs(other["forces"] - a["forces"])) <= tol["f"]
    assert rel_l2(b["vh"], ref["vh"]) <= tol["v"]


def test_forces_central_differences_fp64_gpu():
    """F = -dE/dR on the GPU FP64 path itself, all 64 atoms of the 2x2x2 cell, h = 1e-4."""
    S = synth.config2()
    plan = HartreePlan(S.n, S.cell, S.sigma, "fp64")
    P, Q = dev(S.pos), dev(S.q)
    vh, eh = plan.solve(P, Q)
    f, _ = plan.forces(P, Q, vh)
    F = f.cpu().numpy()
    h = 1e-4
    # all 6 displaced copies of every atom, energies only
    E = np.empty((S.n_atoms, 3, 2))
    for i in range(S.n_atoms):
        for d in range(3):
            for s, sign in enumerate((+1.0, -1.0)):
                p = S.pos.copy()
                p[i, d] += sign * h
                _, e = plan.solve(dev(p), Q, vh=vh)
                E[i, d, s] = e.item()
    fd = -(E[:, :, 0] - E[:, :, 1]) / (2 * h)
    assert np.max(np.abs(fd - F)) <= 1e-7
    plan.close()


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_edge_no_atoms(precision):
    S = synth.config1()
    plan = HartreePlan(S.n, S.cell, S.sigma, precision)
    P = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    Q = torch.empty((0,), dtype=torch.float64, device="cuda")
    vh, eh, rho = plan.solve(P, Q, want_rho=True)
    f, phi = plan.forces(P, Q, vh)
    torch.cuda.synchronize()
    assert float(rho.abs().max()) == 0.0 and float(vh.abs().max()) == 0.0 and eh.item() == 0.0
    assert f.numel() == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_edge_single_charged_atom_unwrapped_positions(precision):
    """A net charge (G = 0 dropped) and positions far outside [0, L)."""
    cell = (7.0, 8.0, 9.0)
    n = (36, 40, 48)
    pos = np.array([[-13.3, 25.1, 4.4], [3.0, -0.2, 100.7]])
    q = np.array([0.8, 0.0])
    S = synth.System("edge", n, cell, 0.7, pos, q, precision)
    ref = O.solve_system(S)
    g = gpu_step(S, precision)
    tol = TOL[precision]
    assert rel_l2(g["vh"], ref["vh"]) <= tol["v"]
    assert abs(g["eh"] - ref["eh"]) <= tol["e"] * abs(ref["eh"])
    assert np.max(np.abs(g["forces"] - ref["forces"])) <= tol["f"]


@pytest.mark.parametrize("n3", [30, 32])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_edge_wide_cutoff_many_images(precision, n3):
    """Cutoff box wider than the cell: one grid point receives several images (N3 = 32: the
    FP32 gather on 16-byte vectors, N3 = 30: on 8-byte vectors)."""
    S = synth.random_system((20, 24, n3), (3.0, 3.5, 4.0), 5, 0.6, seed=77, precision=precision)
    ref = O.solve_system(S)
    g = gpu_step(S, precision, cutoff_sigmas=8.0)
    tol = TOL[precision]
    assert rel_l2(g["vh"], ref["vh"]) <= tol["v"]
    assert np.max(np.abs(g["forces"] - ref["forces"])) <= tol["f"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_force_gathers_agree(precision):
    """The force gather on 16-byte vectors (V_H 16-byte aligned; FP32: 128-thread CTAs) and on
    8-byte vectors (V_H at an 8-byte offset) give the same forces up to summation order, and
    both match the oracle."""
    S, ref = oracle_cfg("cfg2")
    plan = HartreePlan(S.n, S.cell, S.sigma, precision)
    P, Q = dev(S.pos), dev(S.q)
    vh, _ = plan.solve(P, Q)
    off = 8 // vh.element_size()
    buf = torch.empty(vh.numel() + off, dtype=vh.dtype, device="cuda")
    vh8 = buf[off:].view(vh.shape)
    vh8.copy_(vh)
    assert vh.data_ptr() % 16 == 0 and vh8.data_ptr() % 16 == 8
    f, phi = plan.forces(P, Q, vh)
    f8, phi8 = plan.forces(P, Q, vh8)
    torch.cuda.synchronize()
    plan.device_status()
    f, f8 = f.cpu().numpy(), f8.cpu().numpy()
    scale = np.abs(ref["forces"]).max()
    rel = {"fp64": 1e-13, "fp32": 1e-6}[precision]
    assert np.max(np.abs(f - f8)) <= rel * scale
    assert np.max(np.abs(phi.cpu().numpy() - phi8.cpu().numpy())) <= rel * np.abs(ref["phi"]).max()
    for g in (f, f8):
        assert np.max(np.abs(g - ref["forces"])) <= TOL[precision]["f"]
    plan.close()


@pytest.mark.parametrize("n", [(24, 18, 30), (20, 21, 30), (16, 20, 42)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_force_gather_row_residues(precision, n):
    """Rows of V that start off the 16-byte grid (N3 = 2 mod 4): the gather reads aligned
    groups that reach into the neighbouring rows with zero weight.  Atoms sit at the cell's
    corners and faces, so their boxes wrap past N2 and N3."""
    cell = (4.0, 4.5, 5.0)
    rng = np.random.default_rng(sum(n))
    L = np.asarray(cell)
    corners = np.array([[0.02, 0.03, 0.01], [0.98, 0.97, 0.99], [0.5, 0.01, 0.99], [0.01, 0.99, 0.5]]) * L
    pos = np.vstack([corners, rng.uniform(0.0, 1.0, size=(6, 3)) * L])
    q = rng.uniform(-1.0, 1.0, size=pos.shape[0])
    q -= q.mean()
    S = synth.System("residues", n, cell, 0.45, pos, q, precision)
    # the oracle truncates spherically, the library per axis: at 8 sigma (FP64) the difference
    # is e^-64, at 5 sigma (FP32) e^-25, each below its bar
    rc = 8.0 if precision == "fp64" else 5.0
    ref = O.solve_system(S, rc_sigmas=rc)
    g = gpu_step(S, precision, cutoff_sigmas=rc)
    tol = TOL[precision]
    assert np.max(np.abs(g["forces"] - ref["forces"])) <= tol["f"]
    assert np.max(np.abs(g["phi"] - ref["phi"])) <= tol["f"]


def test_fp32_factor_runs_longer_than_one_recurrence():
    """FP32 boxes of more than 64 points per axis: the 1D factors are built in several runs of
    the ratio recurrence (each restarted from exponentials); rho, V_H and the forces still
    match the oracle.  Cell 6 x 6.25 x 7 Bohr on 96 x 100 x 112 (h = 0.0625 Bohr), sigma 0.6 Bohr,
    5 sigma cutoff: 97 points per axis."""
    S = synth.random_system((96, 100, 112), (6.0, 6.25, 7.0), 6, 0.6, seed=4242, precision="fp32")
    ref = O.solve_system(S, rc_sigmas=5.0)
    g = gpu_step(S, "fp32", cutoff_sigmas=5.0)
    tol = TOL["fp32"]
    assert rel_l2(g["rho"], ref["rho"]) <= tol["v"]
    assert rel_l2(g["vh"], ref["vh"]) <= tol["v"]
    assert abs(g["eh"] - ref["eh"]) <= tol["e"] * abs(ref["eh"])
    assert np.max(np.abs(g["forces"] - ref["forces"])) <= tol["f"]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("n,cell,sigma", [
    ((48, 40, 56), (9.0, 8.5, 10.0), 0.7),     # 37-39 box points per axis: one FP32 run
    ((112, 112, 120), (7.0, 7.0, 7.5), 0.6),   # 96-97 box points per axis: two FP32 runs
])
def test_single_atom_density_is_a_few_roundings_from_the_gaussian(n, cell, sigma, precision):
    """One atom: inside its cutoff sphere rho = q n fa fb fc, each 1D factor the working-precision
    rounding of exp(-d^2/s^2).  Against the oracle's FP64 Gaussian the FP32 error is then at most
    7 roundings (three factors, q n times the c factor, two products), bar 8 u = 2^-21; a factor
    recurrence that drifted by one rounding per box point would miss it by far.  Box points
    outside the sphere (the oracle's cutoff is spherical) stay below e^-25 q n."""
    rc = 5.0
    rng = np.random.default_rng(sum(n))
    pos = (rng.random((1, 3)) * np.array(cell))
    q = np.array([1.3])
    ref = O.splat(n, cell, sigma, pos, q, rc_sigmas=rc)
    plan = HartreePlan(n, cell, sigma, precision, cutoff_sigmas=rc)
    rho = plan.splat(dev(pos), dev(q))
    torch.cuda.synchronize()
    plan.device_status()
    g = rho.double().cpu().numpy()
    plan.close()
    inside = ref != 0.0
    bar = 2.0 ** -21 if precision == "fp32" else 1e-13
    assert inside.sum() > 1000
    assert np.max(np.abs(g[inside] - ref[inside]) / ref[inside]) <= bar
    qn = q[0] * (np.pi * sigma * sigma) ** -1.5
    assert np.max(np.abs(g[~inside])) <= np.exp(-rc * rc) * qn * (1 + 1e-5)


def test_forces_recompute_when_vh_is_null():
    S, ref = oracle_cfg("cfg2")
    plan = HartreePlan(S.n, S.cell, S.sigma, "fp32")
    f, phi = plan.forces(dev(S.pos), dev(S.q), vh=None)
    torch.cuda.synchronize()
    assert np.max(np.abs(f.cpu().numpy() - ref["forces"])) <= TOL["fp32"]["f"]


def test_step_host_end_to_end():
    S, ref = oracle_cfg("cfg2")
    plan = HartreePlan(S.n, S.cell, S.sigma, "fp32")
    eh, f = plan.step_host(S.pos, S.q)
    assert abs(eh - ref["eh"]) <= TOL["fp32"]["e"] * abs(ref["eh"])
    assert np.max(np.abs(f - ref["forces"])) <= TOL["fp32"]["f"]
    # the same into caller-owned (here pinned) output arrays
    eh_out = torch.empty(1, dtype=torch.float64).pin_memory().numpy()
    f_out = torch.empty((S.n_atoms, 3), dtype=torch.float64).pin_memory().numpy()
    eh2, f2 = plan.step_host(S.pos, S.q, eh_out=eh_out, f_out=f_out)
    assert f2 is f_out and eh2 == eh and np.array_equal(f2, f)
    with pytest.raises(ValueError):
        plan.step_host(S.pos, S.q, f_out=np.empty((S.n_atoms, 2)))


def test_step_host_graph_follows_counts_variants_and_forces():
    """hartree_step_host replays a captured graph: a new atom count, new variant picks or a call
    without forces must capture again, and every replay must match the device step."""
    S = synth.config2()
    plan = HartreePlan(S.n, S.cell, S.sigma, "fp32", max_atoms=S.n_atoms)
    pos, q = S.pos[:40], S.q[:40] - S.q[:40].mean()
    for _ in range(2):
        eh_a, f_a = plan.step_host(S.pos, S.q)
        eh_b, f_b = plan.step_host(pos, q)
    _, eh_d, f_d = plan.step(dev(pos), dev(q))
    torch.cuda.synchronize()
    assert eh_b == eh_d.item() and np.array_equal(f_b, f_d.cpu().numpy())
    n0 = plan.launch_count
    plan.step_host(pos, q)
    per_call = plan.launch_count - n0
    assert per_call > 1  # the replay counts the graph's kernels
    eh_c, f_c = plan.step_host(pos, q, forces=False)
    assert f_c is None and eh_c == eh_b
    plan.set_variants([0, 0, 0])
    eh_e, f_e = plan.step_host(pos, q)
    assert abs(eh_e - eh_b) <= 1e-6 * abs(eh_b) and np.max(np.abs(f_e - f_b)) <= 1e-5
    plan.close()


def test_too_many_atoms_is_rejected():
    from paper_1209_4506_gb300 import capi

    S = synth.config1()
    plan = HartreePlan(S.n, S.cell, S.sigma, "fp64", max_atoms=4)
    with pytest.raises(capi.HartreeError) as ei:
        plan.solve(dev(S.pos), dev(S.q))
    assert ei.value.status == capi.HARTREE_ERR_INVALID


def test_repeat_runs_are_bitwise_deterministic():
    S = synth.config2()
    a = gpu_step(S, "fp32")
    b = gpu_step(S, "fp32")
    assert np.array_equal(a["vh"], b["vh"]) and a["eh"] == b["eh"] and np.array_equal(a["forces"], b["forces"])


def test_step_entry_point_matches_separate_calls():
    S, ref = oracle_cfg("cfg2")
    plan = HartreePlan(S.n, S.cell, S.sigma, "fp32")
    P, Q = dev(S.pos), dev(S.q)
    vh, eh, f, phi = plan.step(P, Q, want_phi=True)
    vh2, eh2 = plan.solve(P, Q)
    f2, phi2 = plan.forces(P, Q, vh2)
    torch.cuda.synchronize()
    assert torch.equal(vh, vh2) and eh.item() == eh2.item()
    assert torch.equal(f, f2) and torch.equal(phi, phi2)
    assert np.max(np.abs(f.cpu().numpy() - ref["forces"])) <= TOL["fp32"]["f"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_single_passes_reproduce_solve_density(precision):
    shape, cell = (48, 40, 60), (9.1, 7.7, 11.3)
    rng = np.random.default_rng(5)
    dt = torch.float64 if precision == "fp64" else torch.float32
    rho = torch.tensor(rng.standard_normal(shape), dtype=dt, device="cuda")
    plan = HartreePlan(shape, cell, 0.5, precision)
    vh_ref, _ = plan.solve_density(rho)
    vh = torch.empty_like(rho)
    n0 = plan.launch_count
    for p in range(5):
        plan.solve_pass(p, rho=rho, vh=vh)
    torch.cuda.synchronize()
    assert plan.launch_count - n0 == 5
    assert torch.equal(vh, vh_ref)


@pytest.mark.parametrize(
    "shape,precision",
    [((512, 256, 512), "fp32"), ((256, 512, 256), "fp32"), ((256, 512, 256), "fp64"), ((360, 384, 400), "fp32"),
     ((420, 420, 210), "fp32"), ((840, 24, 420), "fp32"), ((840, 24, 420), "fp64"),
     # odd line counts (315 lines, M = 200 and 210): the paired c passes' last pair has one line
     ((15, 21, 400), "fp32"), ((15, 21, 420), "fp32")],
)
def test_kernel_variants_agree(shape, precision):
    """Every compiled variant of every pass kind (tile shapes, thread counts, radix orders,
    TMA / bulk-copy streams, CTAs per SM) computes V_H and E_H within tolerance of the oracle.

    Variants are switched one pass kind at a time.  Variants with the radix order of the
    plain kernels differ only in which thread does a butterfly; others (radix-32 stages,
    the streamed inverse c pass) round differently: all agree with variant 0 to FP32
    rounding."""
    from paper_1209_4506_gb300 import capi

    cell = (20.0, 12.0, 21.0)
    rng = np.random.default_rng(17)
    dt = torch.float64 if precision == "fp64" else torch.float32
    rho = torch.tensor(rng.standard_normal(shape), dtype=dt, device="cuda")
    v_ref_np, e_ref, _, _ = O.poisson(cell, rho.double().cpu().numpy())
    v_ref = torch.tensor(v_ref_np, device="cuda")
    ref_norm = torch.linalg.vector_norm(v_ref).item()
    plan = HartreePlan(shape, cell, 0.5, precision)
    plan.set_variants([0, 0, 0])
    v0, e0 = plan.solve_density(rho)
    v0 = v0.double()
    n_checked = 0
    for kind in range(3):
        for var in range(64):
            choice = [0, 0, 0]
            choice[kind] = var
            try:
                plan.set_variants(choice)
            except capi.HartreeError:
                break
            vh, eh = plan.solve_density(rho)
            torch.cuda.synchronize()
            vd = vh.double()
            assert torch.linalg.vector_norm(vd - v_ref).item() <= TOL[precision]["v"] * ref_norm, choice
            assert torch.linalg.vector_norm(vd - v0).item() <= 1e-6 * ref_norm, choice
            assert abs(eh.item() - e_ref) <= WHITE_NOISE_E_TOL[precision] * abs(e_ref), choice
            n_checked += 1
    plan.device_status()
    assert n_checked >= 3  # at least one variant of each pass kind
    picks = plan.autotune()
    plan.device_status()
    vh, eh = plan.solve_density(rho)
    torch.cuda.synchronize()
    assert torch.linalg.vector_norm(vh.double() - v_ref).item() <= TOL[precision]["v"] * ref_norm, picks
    with pytest.raises(capi.HartreeError):
        plan.set_variants([0, 0, 99])


@pytest.mark.parametrize(
    "shape,cell",
    [((5, 9, 256), (1.0, 1.3, 30.0)),  # M = 128: 45 lines, tiles of 32 (ragged last tile of 13)
     ((3, 10, 512), (0.8, 2.0, 60.0)),  # M = 256: 30 lines, tiles of 16 (last tile 14 lines)
     ((3, 5, 1024), (0.7, 1.0, 110.0)),  # M = 512: 15 lines, tiles of 8
     ((3, 10, 400), (0.8, 2.0, 42.0)),  # M = 200 (radices 8, 5, 5): 30 lines, tiles of 16
     ((3, 16, 210), (0.8, 3.0, 27.0)),  # M = 105 (odd; radices 3, 5, 7): 48 lines, whole tiles only
     ((512, 64, 512), (60.0, 8.0, 60.0))],  # 2,048 tiles: every ring slot reused many times
)
def test_streamed_c_passes_equal_plain_kernels(shape, cell):
    """The bulk-streamed c passes (variant 2 of pass kind 0) match the plain kernels.

    The forward pass does the same arithmetic in the same order, so E_H (formed
    from its output) is bit-identical; the inverse pass may contract its products
    into FMAs differently, so V_H agrees to FP32 rounding.  A grid pointer that
    is not 16-byte aligned cannot be bulk-copied: the call then takes the plain
    kernel, with the same V_H bit for bit."""
    rng = np.random.default_rng(sum(shape) + 7)
    rho32 = rng.standard_normal(shape).astype(np.float32)
    v_ref, e_ref, _, _ = O.poisson(cell, rho32.astype(np.float64))
    plan = HartreePlan(shape, cell, 0.5, "fp32")
    rho = torch.tensor(rho32, device="cuda")
    plan.set_variants([0, 0, 0])
    v0, e0 = plan.solve_density(rho)
    plan.set_variants([1 if shape[2] in (400, 210) else 2, 0, 0])  # the streamed c passes
    v2, e2 = plan.solve_density(rho)
    torch.cuda.synchronize()
    plan.device_status()
    assert rel_l2(v2.double().cpu().numpy(), v0.double().cpu().numpy()) <= 1e-6
    assert e0.item() == e2.item()
    assert rel_l2(v2.double().cpu().numpy(), v_ref) <= TOL["fp32"]["v"]
    assert abs(e2.item() - e_ref) <= WHITE_NOISE_E_TOL["fp32"] * abs(e_ref)
    # grids 8- but not 16-byte aligned (offset by two floats): the plain kernels run instead
    buf_in = torch.empty(rho.numel() + 2, dtype=torch.float32, device="cuda")
    buf_out = torch.empty(rho.numel() + 2, dtype=torch.float32, device="cuda")
    r_mis = buf_in[2:].view(shape)
    r_mis.copy_(rho)
    v_mis = buf_out[2:].view(shape)
    plan.solve_density(r_mis, vh=v_mis)
    torch.cuda.synchronize()
    plan.device_status()
    assert torch.equal(v_mis, v0)
    plan.close()


def test_grids_off_the_pair_alignment_are_rejected():
    """Grid lines move as (re, im) pairs: a grid not aligned to twice the element size is
    refused on the host (HARTREE_ERR_INVALID) before any kernel is launched."""
    from paper_1209_4506_gb300 import capi

    shape, cell = (8, 8, 16), (2.0, 2.0, 4.0)
    for precision, dt, off in (("fp32", torch.float32, 1), ("fp64", torch.float64, 1)):
        plan = HartreePlan(shape, cell, 0.5, precision)
        buf = torch.zeros(int(np.prod(shape)) + off, dtype=dt, device="cuda")
        good = torch.zeros(shape, dtype=dt, device="cuda")
        bad = buf[off:].view(shape)
        with pytest.raises(capi.HartreeError) as ei:
            plan.solve_density(bad, vh=good)
        assert ei.value.status == capi.HARTREE_ERR_INVALID
        with pytest.raises(capi.HartreeError):
            plan.solve_density(good, vh=bad)
        with pytest.raises(capi.HartreeError):
            plan.solve_pass(0, rho=bad, vh=good)
        plan.close()


def test_autotune_cache_roundtrip(tmp_path):
    from paper_1209_4506_gb300 import autotune

    plan = HartreePlan((256, 256, 256), (20.0, 20.0, 20.0), 0.5, "fp32")
    path = str(tmp_path / "cache.json")
    first = autotune.tuned(plan, path)
    again = autotune.tuned(plan, path)
    assert first == again
    import json
    assert len(json.load(open(path))) == 1


def test_dense_tile_beyond_the_bin_sort_capacity():
    # 1100 atoms in a cell of one splat tile: the tile's list is longer than the
    # binned splat sorts in shared memory, so that tile takes the leaf-selecting path
    S = synth.random_system((16, 8, 32), (3.0, 2.0, 5.0), 1100, 0.6, seed=21, precision="fp32")
    ref = O.solve_system(S)
    g = gpu_step(S, "fp32")
    assert rel_l2(g["rho"], ref["rho"]) <= 2e-6
    assert rel_l2(g["vh"], ref["vh"]) <= TOL["fp32"]["v"]
    assert abs(g["eh"] - ref["eh"]) <= TOL["fp32"]["e"] * abs(ref["eh"])
    assert np.max(np.abs(g["forces"] - ref["forces"])) <= TOL["fp32"]["f"]
