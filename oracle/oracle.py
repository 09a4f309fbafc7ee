"""ctypes front end of the FP64 C oracle (test infrastructure only).

Builds ``_lib/libhartree_oracle.so`` from ``hartree_oracle.c`` with the system
C compiler when it is missing or older than the source.  Every function takes
and returns float64 numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hartree_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libhartree_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no fast-math)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_fft1d.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int]
            lib.oracle_fft3d.argtypes = [_ip, _dp, ctypes.c_int]
            lib.oracle_dft3d_brute.argtypes = [_ip, _dp, _dp, ctypes.c_int]
            lib.oracle_splat.argtypes = [_ip, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]
            lib.oracle_poisson.argtypes = [_ip, _dp, _dp, _dp, _dp]
            lib.oracle_poisson.restype = ctypes.c_int
            lib.oracle_forces.argtypes = [
                _ip, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp, _dp, _dp,
            ]
            lib.oracle_bisect.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, _ip, _ip]
            lib.oracle_bisect.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_get_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


class use_library:
    """Context manager: route every call through another build of the oracle.

    Used by the mutation tests, which compile a deliberately broken copy of the
    source and check that the pins reject it.
    """

    def __init__(self, path: str):
        self.path = path
        self.saved = None

    def __enter__(self):
        global _lib
        _load()
        with _lock:
            self.saved = _lib
            _lib = None
        real_build = globals()["build"]
        globals()["build"] = lambda force=False: self.path
        try:
            _load()
        finally:
            globals()["build"] = real_build
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _i(a: np.ndarray):
    return a.ctypes.data_as(_ip)


def _n3(n) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(n, dtype=np.int32).reshape(3))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def set_threads(n: int) -> None:
    """Number of POSIX threads the 3D transforms split their lines over."""
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def fft1d(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised 1D DFT, exp(sign 2 pi i j k / n)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
    out = np.empty_like(x)
    _load().oracle_fft1d(x.size, x.ctypes.data_as(_dp), out.ctypes.data_as(_dp), int(sign))
    return out


def fft3d(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised 3D DFT of a C-order complex array (axes c, b, a forward)."""
    out = np.array(x, dtype=np.complex128, order="C", copy=True)
    _load().oracle_fft3d(_i(_n3(out.shape)), out.ctypes.data_as(_dp), int(sign))
    return out


def dft3d_brute(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """O(N^2) 3D DFT from the definition (tiny grids only)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
    out = np.empty_like(x)
    _load().oracle_dft3d_brute(_i(_n3(x.shape)), x.ctypes.data_as(_dp), out.ctypes.data_as(_dp), int(sign))
    return out


def splat(n, cell, sigma: float, pos, q, rc_sigmas: float = 8.0) -> np.ndarray:
    """Gaussian charges on the grid, all periodic images within rc = rc_sigmas * sigma."""
    n3 = _n3(n)
    pos = _f64(pos).reshape(-1, 3)
    q = _f64(q).reshape(-1)
    rho = np.empty(tuple(int(v) for v in n3), dtype=np.float64)
    _load().oracle_splat(
        _i(n3), _d(_f64(cell)), float(sigma), float(rc_sigmas * sigma), int(q.size), _d(pos), _d(q), _d(rho)
    )
    return rho


def poisson(cell, rho: np.ndarray) -> Tuple[np.ndarray, float, float, float]:
    """(V_H, E_H real-space, E_H spectral, max|Im V|/max|Re V|) for a density on the grid."""
    rho = _f64(rho)
    vh = np.empty_like(rho)
    out3 = np.zeros(3, dtype=np.float64)
    rc = _load().oracle_poisson(_i(_n3(rho.shape)), _d(_f64(cell)), _d(rho), _d(vh), _d(out3))
    if rc != 0:
        raise MemoryError("oracle_poisson: allocation failed")
    return vh, float(out3[0]), float(out3[1]), float(out3[2])


def forces(n, cell, sigma: float, pos, q, vh: np.ndarray, rc_sigmas: float = 8.0) -> Tuple[np.ndarray, np.ndarray]:
    """(F[n_atoms, 3] = -dE_H/dR, phi[n_atoms] = dE_H/dq) by the real-space gather."""
    pos = _f64(pos).reshape(-1, 3)
    q = _f64(q).reshape(-1)
    f = np.empty((q.size, 3), dtype=np.float64)
    phi = np.empty(q.size, dtype=np.float64)
    _load().oracle_forces(
        _i(_n3(n)), _d(_f64(cell)), float(sigma), float(rc_sigmas * sigma), int(q.size), _d(pos), _d(q),
        _d(_f64(vh)), _d(f), _d(phi),
    )
    return f, phi


def bisect(pos, n_leaves: int, w: Optional[np.ndarray] = None) -> Tuple[np.ndarray, np.ndarray]:
    """(perm[n_atoms], leaf_start[n_leaves + 1]) from the modified recursive bisection."""
    pos = _f64(pos).reshape(-1, 3)
    nat = pos.shape[0]
    perm = np.empty(max(nat, 1), dtype=np.int32)
    ls = np.empty(n_leaves + 1, dtype=np.int32)
    wp = _d(_f64(w)) if w is not None else None
    rc = _load().oracle_bisect(int(nat), _d(pos), wp, int(n_leaves), _i(perm), _i(ls))
    if rc != 0:
        raise ValueError("oracle_bisect: bad arguments")
    return perm[:nat].copy(), ls


def solve_system(system, rc_sigmas: float = 8.0, with_forces: bool = True) -> dict:
    """Whole Hartree step for a synth.System: rho, V_H, E_H (both forms), forces, phi."""
    rho = splat(system.n, system.cell, system.sigma, system.pos, system.q, rc_sigmas)
    vh, e_real, e_spec, imag = poisson(system.cell, rho)
    out = {"rho": rho, "vh": vh, "eh": e_real, "eh_spectral": e_spec, "imag_rel": imag}
    if with_forces:
        f, phi = forces(system.n, system.cell, system.sigma, system.pos, system.q, vh, rc_sigmas)
        out["forces"] = f
        out["phi"] = phi
    return out
