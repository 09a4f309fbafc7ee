"""Thin PyTorch-facing wrapper over the C ABI: device memory and streams only.

Every computation happens in libhartree_gb300.so; this module allocates
output tensors, checks dtypes/devices/shapes and passes raw pointers and the
current CUDA stream to the library.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence, Tuple

import numpy as np

from . import capi

_PREC = {"fp64": capi.HARTREE_FP64, "fp32": capi.HARTREE_FP32, "bf16split": capi.HARTREE_FP32_TC_SPLIT}


def _torch():
    import torch

    return torch


def _stream_handle(device) -> int:
    torch = _torch()
    return int(torch.cuda.current_stream(device).cuda_stream)


def atoms_reorder(pos: np.ndarray, n_leaves: int, w: Optional[np.ndarray] = None) -> Tuple[np.ndarray, np.ndarray]:
    """Modified recursive bisection (host, FP64): (perm[n], leaf_start[n_leaves + 1])."""
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
    n = pos.shape[0]
    perm = np.empty(max(n, 1), dtype=np.int32)
    ls = np.empty(int(n_leaves) + 1, dtype=np.int32)
    wp = None
    if w is not None:
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(-1))
        wp = w.ctypes.data
    capi.check(capi.hartree_atoms_reorder(pos.ctypes.data, wp, n, int(n_leaves), perm.ctypes.data, ls.ctypes.data))
    return perm[:n].copy(), ls


class HartreePlan:
    """One grid / cell / width / precision; owns the library plan and its workspace."""

    def __init__(
        self,
        n: Sequence[int],
        cell: Sequence[float],
        sigma: float,
        precision: str = "fp32",
        cutoff_sigmas: float = 0.0,
        atoms_per_leaf: int = 0,
        max_atoms: int = 0,
        device=None,
        flags: int = 0,
    ):
        torch = _torch()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index)
        self.n = tuple(int(v) for v in n)
        self.cell = tuple(float(v) for v in cell)
        self.sigma = float(sigma)
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        d = capi.hartree_desc()
        for i in range(3):
            d.n[i] = self.n[i]
            d.cell[i] = self.cell[i]
        d.sigma = self.sigma
        d.cutoff_sigmas = float(cutoff_sigmas)
        d.precision = _PREC[precision]
        d.atoms_per_leaf = int(atoms_per_leaf)
        d.max_atoms = int(max_atoms)
        d.flags = int(flags)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            capi.check(capi.hartree_plan_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h

    # ------------------------------------------------------------ helpers
    @property
    def handle(self) -> int:
        if self._h is None:
            raise RuntimeError("plan is closed")
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            capi.hartree_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def workspace_bytes(self) -> int:
        return int(capi.hartree_plan_workspace_bytes(self.handle))

    def _grid(self, t, name):
        torch = _torch()
        if t is None:
            return torch.empty(self.n, dtype=self.dtype, device=self.device)
        if t.dtype != self.dtype or t.device != self.device or tuple(t.shape) != self.n or not t.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous {self.dtype} tensor of shape {self.n} on {self.device}")
        return t

    def _atoms(self, pos, q):
        torch = _torch()
        if pos.dtype != torch.float64 or q.dtype != torch.float64:
            raise ValueError("pos and q must be float64")
        if pos.device != self.device or q.device != self.device:
            raise ValueError("pos and q must live on the plan's device")
        pos = pos.contiguous().reshape(-1, 3)
        q = q.contiguous().reshape(-1)
        if pos.shape[0] != q.shape[0]:
            raise ValueError("pos and q disagree on the atom count")
        return pos, q, int(q.shape[0])

    # ------------------------------------------------------------ entry points
    def splat(self, pos, q, rho=None):
        pos, q, n = self._atoms(pos, q)
        rho = self._grid(rho, "rho")
        capi.check(capi.hartree_splat(self.handle, pos.data_ptr(), q.data_ptr(), n, rho.data_ptr(),
                                      _stream_handle(self.device)))
        return rho

    def solve_density(self, rho, vh=None, eh=None):
        torch = _torch()
        rho = self._grid(rho, "rho")
        vh = self._grid(vh, "vh")
        if eh is None:
            eh = torch.empty((), dtype=torch.float64, device=self.device)
        capi.check(capi.hartree_solve_density(self.handle, rho.data_ptr(), vh.data_ptr(), eh.data_ptr(),
                                              _stream_handle(self.device)))
        return vh, eh

    def solve(self, pos, q, vh=None, rho=None, eh=None, want_rho: bool = False):
        torch = _torch()
        pos, q, n = self._atoms(pos, q)
        vh = self._grid(vh, "vh")
        if want_rho and rho is None:
            rho = self._grid(None, "rho")
        elif rho is not None:
            rho = self._grid(rho, "rho")
        if eh is None:
            eh = torch.empty((), dtype=torch.float64, device=self.device)
        capi.check(capi.hartree_solve(self.handle, pos.data_ptr(), q.data_ptr(), n,
                                      rho.data_ptr() if rho is not None else None, vh.data_ptr(), eh.data_ptr(),
                                      _stream_handle(self.device)))
        return (vh, eh, rho) if want_rho else (vh, eh)

    def forces(self, pos, q, vh=None, f=None, phi=None, want_phi: bool = True):
        torch = _torch()
        pos, q, n = self._atoms(pos, q)
        if vh is not None:
            vh = self._grid(vh, "vh")
        if f is None:
            f = torch.empty((n, 3), dtype=torch.float64, device=self.device)
        if want_phi and phi is None:
            phi = torch.empty((n,), dtype=torch.float64, device=self.device)
        capi.check(capi.hartree_forces(self.handle, pos.data_ptr(), q.data_ptr(), n,
                                       vh.data_ptr() if vh is not None else None, f.data_ptr(),
                                       phi.data_ptr() if want_phi else None, _stream_handle(self.device)))
        return (f, phi) if want_phi else f

    def step(self, pos, q, vh=None, eh=None, f=None, phi=None, rho=None, want_phi: bool = False):
        """Splat + solve + E_H + forces in one call: (vh, eh, f[, phi])."""
        torch = _torch()
        pos, q, n = self._atoms(pos, q)
        vh = self._grid(vh, "vh")
        if rho is not None:
            rho = self._grid(rho, "rho")
        if eh is None:
            eh = torch.empty((), dtype=torch.float64, device=self.device)
        if f is None:
            f = torch.empty((n, 3), dtype=torch.float64, device=self.device)
        if want_phi and phi is None:
            phi = torch.empty((n,), dtype=torch.float64, device=self.device)
        capi.check(capi.hartree_step(self.handle, pos.data_ptr(), q.data_ptr(), n,
                                     rho.data_ptr() if rho is not None else None, vh.data_ptr(), eh.data_ptr(),
                                     f.data_ptr(), phi.data_ptr() if phi is not None else None,
                                     _stream_handle(self.device)))
        return (vh, eh, f, phi) if want_phi else (vh, eh, f)

    def splat_pass(self, pos, q):
        """Launch the splat fused into pass 0 alone (atoms -> half spectrum); for timing and profiling."""
        pos, q, n = self._atoms(pos, q)
        capi.check(capi.hartree_splat_pass(self.handle, pos.data_ptr(), q.data_ptr(), n, _stream_handle(self.device)))

    @property
    def fused_splat(self) -> bool:
        """True if steps with no density grid compute the density inside pass 0."""
        return bool(capi.hartree_plan_fused_splat(self.handle))

    def solve_pass(self, pass_id: int, rho=None, vh=None):
        """Launch one Poisson pass alone (0: c r2c .. 4: c c2r); for timing and profiling."""
        if rho is not None:
            rho = self._grid(rho, "rho")
        if vh is not None:
            vh = self._grid(vh, "vh")
        capi.check(capi.hartree_solve_pass(self.handle, int(pass_id), rho.data_ptr() if rho is not None else None,
                                           vh.data_ptr() if vh is not None else None, _stream_handle(self.device)))

    def autotune(self):
        """Time every kernel variant on this plan's workspace and keep the fastest; returns the picks."""
        choice = (ctypes.c_int * 3)()
        capi.check(capi.hartree_plan_autotune(self.handle, _stream_handle(self.device), choice))
        return [int(v) for v in choice]

    def set_variants(self, choice):
        arr = (ctypes.c_int * 3)(*[int(v) for v in choice])
        capi.check(capi.hartree_plan_set_variants(self.handle, arr))

    def device_status(self):
        """Raise HartreeError(TIMEOUT) if a bounded device wait gave up since the last check."""
        capi.check(capi.hartree_plan_device_status(self.handle))

    @property
    def launch_count(self) -> int:
        return int(capi.hartree_plan_launch_count(self.handle))

    def step_host(self, pos: np.ndarray, q: np.ndarray, forces: bool = True, eh_out=None, f_out=None):
        """Host arrays in, (E_H, F or None) out; copies and waits inside the library.  eh_out ([1]) and
        f_out ([n][3]), float64 and C-contiguous, receive the results if given (pinned arrays make
        the read-back a direct copy)."""
        pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
        q = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(-1))
        n = q.size
        for name, arr, shape in (("eh_out", eh_out, (1,)), ("f_out", f_out, (n, 3))):
            if arr is not None and (arr.dtype != np.float64 or arr.shape != shape or not arr.flags.c_contiguous):
                raise ValueError(f"{name} must be a C-contiguous float64 array of shape {shape}")
        eh = eh_out if eh_out is not None else np.zeros(1, dtype=np.float64)
        f = (f_out if f_out is not None else np.empty((n, 3), dtype=np.float64)) if forces else None
        capi.check(capi.hartree_step_host(self.handle, pos.ctypes.data, q.ctypes.data, n, eh.ctypes.data,
                                          f.ctypes.data if forces else None, _stream_handle(self.device)))
        return float(eh[0]), f


class HartreeBatch:
    """Many FP32 cells (each its own grid, cell, width and atom count) solved in one persistent launch.

    cells: sequence of (n, cell, sigma, n_atoms).  Positions and charges of all
    cells are concatenated in cell order; V_H of all cells is one flat float32
    buffer, cell c occupying grid_off[c]:grid_off[c + 1] in C order.
    """

    def __init__(self, cells, cutoff_sigmas: float = 0.0, atoms_per_leaf: int = 0, device=None):
        torch = _torch()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index)
        cells = list(cells)
        self.n_cells = len(cells)
        descs = (capi.hartree_desc * max(self.n_cells, 1))()
        counts = np.zeros(max(self.n_cells, 1), dtype=np.int32)
        self.shapes = []
        for c, (n, cell, sigma, nat) in enumerate(cells):
            d = descs[c]
            for i in range(3):
                d.n[i] = int(n[i])
                d.cell[i] = float(cell[i])
            d.sigma = float(sigma)
            d.cutoff_sigmas = float(cutoff_sigmas)
            d.precision = capi.HARTREE_FP32
            d.atoms_per_leaf = int(atoms_per_leaf)
            d.max_atoms = 0
            d.flags = 0
            counts[c] = int(nat)
            self.shapes.append(tuple(int(v) for v in n))
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            capi.check(capi.hartree_batch_create(descs, counts.ctypes.data, self.n_cells, ctypes.byref(h)))
        self._h = h
        go = np.zeros(self.n_cells + 1, dtype=np.int64)
        ao = np.zeros(self.n_cells + 1, dtype=np.int32)
        capi.check(capi.hartree_batch_offsets(self.handle, go.ctypes.data, ao.ctypes.data))
        self.grid_off = go
        self.atom_off = ao

    @property
    def handle(self) -> int:
        if self._h is None:
            raise RuntimeError("batch is closed")
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            capi.hartree_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, pos, q, vh=None, eh=None):
        """V_H (flat float32 [grid_off[-1]]) and E_H (float64 [n_cells]) of every cell."""
        torch = _torch()
        n_at = int(self.atom_off[-1])
        if pos.dtype != torch.float64 or q.dtype != torch.float64 or pos.device != self.device or q.device != self.device:
            raise ValueError("pos and q must be float64 tensors on the batch's device")
        pos = pos.contiguous().reshape(-1, 3)
        q = q.contiguous().reshape(-1)
        if pos.shape[0] != n_at or q.shape[0] != n_at:
            raise ValueError(f"expected {n_at} atoms in total")
        total = int(self.grid_off[-1])
        if vh is None:
            vh = torch.empty(total, dtype=torch.float32, device=self.device)
        elif vh.dtype != torch.float32 or vh.numel() != total or not vh.is_contiguous() or vh.device != self.device:
            raise ValueError(f"vh: expected a contiguous float32 tensor of {total} elements")
        if eh is None:
            eh = torch.empty(self.n_cells, dtype=torch.float64, device=self.device)
        elif eh.dtype != torch.float64 or eh.numel() != self.n_cells or eh.device != self.device:
            raise ValueError(f"eh: expected a float64 tensor of {self.n_cells} elements")
        capi.check(capi.hartree_solve_batched(self.handle, pos.data_ptr(), q.data_ptr(), vh.data_ptr(), eh.data_ptr(),
                                              _stream_handle(self.device)))
        return vh, eh

    def cell_view(self, vh, c):
        """The grid of cell c inside the flat buffer, shaped [N1][N2][N3]."""
        return vh[int(self.grid_off[c]):int(self.grid_off[c + 1])].view(self.shapes[c])

    def device_status(self):
        capi.check(capi.hartree_batch_device_status(self.handle))

    def fault_inject(self, skip_stage: int = -1, skip_cell: int = 0, spin_limit: int = 0):
        """Test hook: item 0 of (skip_stage, skip_cell) never reports done, and dependency waits give up
        after spin_limit probes (0: the default).  skip_stage = -1 switches it off."""
        capi.check(capi.hartree_batch_fault_inject(self.handle, int(skip_stage), int(skip_cell), int(spin_limit)))
