"""Plant plausible mistakes in a copy of the oracle and check the pins reject each one.

Each mutant is the oracle source with one textual change (a dropped term, a
wrong sign, a transposed index or operand), compiled to a temporary library.
The pins used are the same independent facts as in test_oracle_pins.py.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from oracle import oracle as OO
from paper_1209_4506_gb300 import synth
from test_oracle_pins import SMALL_ORTHO, _mode_case, lattice_sum_energy_forces, small_ortho_system

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "hartree_oracle.c")

MUTANTS = {
    "green-transposed-L": ("TWO_PI * fold(k2, n[1]) / L[1]", "TWO_PI * fold(k2, n[1]) / L[0]"),
    "no-frequency-fold": ("return (2 * k <= n) ? k : k - n;", "return k;"),
    "splat-norm-exponent": ("double norm = pow(PI * sigma * sigma, -1.5);\n    double inv_s2 = 1.0 / (sigma * sigma);\n    long N",
                            "double norm = pow(PI * sigma * sigma, -1.0);\n    double inv_s2 = 1.0 / (sigma * sigma);\n    long N"),
    "force-sign": ("f[3 * a + 0] = -dV * q[a] * fx;", "f[3 * a + 0] = dV * q[a] * fx;"),
    "force-dropped-factor-2": ("fy += gv * 2.0 * dy * inv_s2;", "fy += gv * dy * inv_s2;"),
    "twiddle-index": ("long e = ((long)r * idx) % n;", "long e = ((long)r * k) % n;"),
    "energy-half-dropped": ("espec *= omega / (2.0 * (double)N * (double)N);", "espec *= omega / ((double)N * (double)N);"),
    "inverse-scale-axis": ("double re = s[i].re / (double)N, im", "double re = s[i].re / (double)n[0], im"),
    "inertia-offdiag-sign": ("T[1] -= w * X * Y;", "T[1] += w * X * Y;"),
    "splat-offset-axis": ("double dy = (double)j * h[1] - R[1];\n                for (long k = lo[2]; k <= hi[2]; ++k) {\n                    double dz = (double)k * h[2] - R[2];\n                    double d2 = dx * dx + dy * dy + dz * dz;\n                    if (d2 >= rc * rc) continue;\n                    long idx = (wrap_index(i, n[0]) * n[1] + wrap_index(j, n[1])) * n[2] + wrap_index(k, n[2]);\n                    rho",
                          "double dy = (double)j * h[0] - R[1];\n                for (long k = lo[2]; k <= hi[2]; ++k) {\n                    double dz = (double)k * h[2] - R[2];\n                    double d2 = dx * dx + dy * dy + dz * dz;\n                    if (d2 >= rc * rc) continue;\n                    long idx = (wrap_index(i, n[0]) * n[1] + wrap_index(j, n[1])) * n[2] + wrap_index(k, n[2]);\n                    rho"),
}


def _pins_hold():
    """A fast subset of the pins; True when all hold."""
    checks = []
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 6, 10)) + 1j * rng.standard_normal((4, 6, 10))
    checks.append(np.max(np.abs(O.fft3d(x) - O.dft3d_brute(x))) <= 1e-13 * np.max(np.abs(x)) * 240)
    n, cell = SMALL_ORTHO["n"], SMALL_ORTHO["cell"]
    for m, kind in [((2, -3, 1), "sin"), ((-1, 4, -5), "cos"), ((0, 0, 18), "cos")]:
        rho, v_exact, G2 = _mode_case(n, cell, m, kind)
        vh, e_real, e_spec, _ = O.poisson(cell, rho)
        e_exact = 0.5 * 4 * np.pi / G2 * float(np.sum(rho * rho)) * np.prod(cell) / np.prod(n)
        checks.append(np.max(np.abs(vh - v_exact)) <= 1e-13 * np.max(np.abs(v_exact)))
        checks.append(abs(e_spec - e_exact) <= 2e-12 * abs(e_exact))
    S = small_ortho_system()
    r = O.solve_system(S)
    E_ls, F_ls = lattice_sum_energy_forces(S.cell, S.sigma, S.pos, S.q)
    checks.append(abs(r["eh"] - E_ls) <= 1e-12 * abs(E_ls))
    checks.append(np.max(np.abs(r["forces"] - F_ls)) <= 1e-10)
    checks.append(abs(r["rho"].sum() * np.prod(S.cell) / S.n_tot - S.q.sum()) <= 1e-12)
    # bisection: a cloud stretched along an oblique direction must be cut across that direction
    u = np.array([1.0, 1.0, 0.3]) / np.linalg.norm([1.0, 1.0, 0.3])
    pos = rng.standard_normal((60, 3)) * 0.5 + rng.standard_normal((60, 1)) * 4.0 * u[None, :]
    perm, ls = O.bisect(pos, 2)
    t = pos @ u
    checks.append(ls.tolist() == [0, 30, 60] and t[perm[:30]].max() < t[perm[30:]].min())
    perm, ls = O.bisect(synth.diamond_supercell((2, 2, 2))[:13], 2)
    checks.append(np.diff(ls).tolist() == [7, 6])
    return all(bool(c) for c in checks)


def test_unmutated_oracle_passes_the_fast_pins():
    assert _pins_hold()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_rejected(name, tmp_path):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = src.replace(old, new, 1)
    cpath = tmp_path / "mutant.c"
    cpath.write_text(mutated)
    lib = str(tmp_path / "libmutant.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", lib, str(cpath), "-lm"], check=True)
    with OO.use_library(lib):
        assert not _pins_hold(), f"mutant {name} slipped through the pins"
