"""GB300 particle-in-cell cycle with the pair-potential force of Mitchell, Schumacher & Chowdhury,
"Modeling crater formation in femtosecond-pulse laser damage from basic principles"
(arXiv:1502.07722).

This module is a thin ctypes binding of the C ABI in include/pic.h (libgbpic.so, built for
sm_103a by `_build.build()`). Every step of the cycle runs in the library's CUDA kernels; the
binding only marshals arguments. PyTorch provides the device workspace and the stream.
There is no CPU fallback: if the library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes

import numpy as np
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libgbpic.so")

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA, PIC_ENAN, PIC_EMOVE, PIC_ESTATE = 0, -1, -2, -3, -4, -5, -6
PIC_EOVERFLOW = -7
PIC_MODE_FULL, PIC_MODE_TRANSPORT = 0, 1
PIC_LASER_NONE, PIC_LASER_PLANE, PIC_LASER_GAUSSIAN = 0, 1, 2
PIC_TEMP_UNIFORM, PIC_TEMP_SPOT = 0, 1
PIC_LATTICE_CUBIC, PIC_LATTICE_HCP = 0, 1
FIELDS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")


class pic_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("nz", ctypes.c_int32), ("slab_k", ctypes.c_int32), ("mode", ctypes.c_int32),
        ("ppc_ion", ctypes.c_int32), ("ppc_electron", ctypes.c_int32), ("pot_mode", ctypes.c_int32),
        ("laser_profile", ctypes.c_int32), ("tile", ctypes.c_int32), ("sort_every", ctypes.c_int32),
        ("max_particles", ctypes.c_int64),
        ("dx", ctypes.c_double), ("cfl", ctypes.c_double), ("dt_override", ctypes.c_double),
        ("n_atoms", ctypes.c_double), ("T_ion_K", ctypes.c_double), ("T_electron_eV", ctypes.c_double),
        ("ion_charge", ctypes.c_double), ("ion_mass_amu", ctypes.c_double), ("D_eV", ctypes.c_double),
        ("r0", ctypes.c_double), ("c_att", ctypes.c_double), ("s_rep", ctypes.c_double),
        ("lambda_", ctypes.c_double), ("I0", ctypes.c_double), ("tau_fwhm", ctypes.c_double),
        ("w0", ctypes.c_double), ("t_peak", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("ny", ctypes.c_int32), ("dims", ctypes.c_int32),
        ("temp_profile", ctypes.c_int32), ("lattice", ctypes.c_int32),
        ("T_spot_K", ctypes.c_double), ("spot_w", ctypes.c_double), ("spot_depth", ctypes.c_double),
        ("morse_a", ctypes.c_double),
        ("eam_ec", ctypes.c_double), ("eam_phi", ctypes.c_double), ("eam_alpha", ctypes.c_double),
        ("eam_beta", ctypes.c_double), ("eam_gamma", ctypes.c_double),
    ]


class pic_info(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("weight", ctypes.c_double), ("rho_scale", ctypes.c_double),
                ("r0", ctypes.c_double), ("time", ctypes.c_double), ("step", ctypes.c_int64),
                ("num_particles", ctypes.c_int64 * 2), ("nspecies", ctypes.c_int32), ("ntiles", ctypes.c_int32)]


class pic_energy_t(ctypes.Structure):
    _fields_ = [("kinetic_ion", ctypes.c_double), ("kinetic_electron", ctypes.c_double),
                ("field_E", ctypes.c_double), ("field_B", ctypes.c_double), ("pair", ctypes.c_double),
                ("step", ctypes.c_int64), ("injected", ctypes.c_double)]


class pic_state_view(ctypes.Structure):
    _P = ctypes.c_void_p
    _fields_ = [("n", ctypes.c_int64 * 2), ("cell", _P * 2), ("fx", _P * 2), ("fz", _P * 2), ("ux", _P * 2),
                ("uy", _P * 2), ("uz", _P * 2), ("F", _P * 6), ("rho", _P)]


class pic_adjoint_buffers(ctypes.Structure):
    _P = ctypes.c_void_p
    _fields_ = [("lam_pos", _P * 2), ("lam_u", _P * 2), ("lam_nodes", _P), ("lam_F", _P), ("lam_j", _P),
                ("grads", _P)]


# name -> (restype, argtypes) of every exported C entry point
_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_SIGNATURES = {
    "pic_config_bytes": (ctypes.c_size_t, []),
    "pic_workspace_size": (ctypes.c_int, [ctypes.POINTER(pic_config), ctypes.POINTER(ctypes.c_size_t)]),
    "pic_init": (ctypes.c_int, [ctypes.POINTER(pic_config), _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
    "pic_free": (None, [_VP]),
    "pic_step": (ctypes.c_int, [_VP, _I32]),
    "pic_deposit_density": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_double)]),
    "pic_pair_force": (ctypes.c_int, [_VP, _VP]),
    "pic_crater_profile": (ctypes.c_int, [_VP, _VP, _VP]),
    "pic_cell_temperature": (ctypes.c_int, [_VP, _I32, _VP, _VP]),
    "pic_set_temperature": (ctypes.c_int, [_VP, _I32, _VP, ctypes.c_double]),
    "pic_regrid_cells": (ctypes.c_int, [_I32, _VP, _I32, _I32, _I32, ctypes.c_double, _I32, _VP, _I32, _I32, _I32,
                                        ctypes.c_double, _I32, ctypes.c_double, _VP]),
    "pic_pair_force_at": (ctypes.c_int, [_VP, ctypes.c_int64, _VP, _VP, _VP, _I32, ctypes.c_double, ctypes.c_double, _VP]),
    "pic_energy": (ctypes.c_int, [_VP, ctypes.POINTER(pic_energy_t)]),
    "pic_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(pic_info)]),
    "pic_get_particles": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _I32]),
    "pic_set_particles": (ctypes.c_int, [_VP, _I32, ctypes.c_int64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _I32]),
    "pic_get_field": (ctypes.c_int, [_VP, _I32, _VP, _I32]),
    "pic_set_field": (ctypes.c_int, [_VP, _I32, _VP, _I32]),
    "pic_get_current": (ctypes.c_int, [_VP, _VP, _I32]),
    "pic_get_density": (ctypes.c_int, [_VP, _VP, _I32]),
    "pic_sort": (ctypes.c_int, [_VP]),
    "pic_set_timing": (ctypes.c_int, [_VP, _I32]),
    "pic_get_timing": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    "pic_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "pic_energy_noalloc": (ctypes.c_int, [ctypes.POINTER(pic_config), ctypes.POINTER(pic_state_view), _VP, _VP]),
    "pic_batch_workspace_size": (ctypes.c_int, [ctypes.POINTER(pic_config), _I32, ctypes.POINTER(ctypes.c_size_t)]),
    "pic_batch_init": (ctypes.c_int, [ctypes.POINTER(pic_config), _I32, _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
    "pic_batch_step": (ctypes.c_int, [_VP, _I32]),
    "pic_batch_slab": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_VP)]),
    "pic_batch_set_timing": (ctypes.c_int, [_VP, _I32]),
    "pic_batch_get_timing": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    "pic_batch_free": (None, [_VP]),
    "pic_checkpoint_size": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_size_t)]),
    "pic_checkpoint_save": (ctypes.c_int, [_VP, _VP, _I32]),
    "pic_checkpoint_restore": (ctypes.c_int, [_VP, _VP, _I32]),
    "pic_node_functional": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_double)]),
    "pic_adjoint_seed": (ctypes.c_int, [_VP, ctypes.c_double, _VP, ctypes.POINTER(pic_adjoint_buffers),
                                        ctypes.POINTER(ctypes.c_double)]),
    "pic_adjoint_step": (ctypes.c_int, [_VP, ctypes.POINTER(pic_adjoint_buffers)]),
}

_lib = None


def load_library():
    """Load libgbpic.so; raise if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError(f"{LIBPATH} is missing: build it with paper_1502_07722_gb300._build.build()")
        L = ctypes.CDLL(LIBPATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        if L.pic_config_bytes() != ctypes.sizeof(pic_config):
            raise RuntimeError(f"{LIBPATH} was built with another pic_config layout: rebuild it")
        _lib = L
    return _lib


class PicError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = load_library().pic_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})")


def _check(code, where):
    if code != PIC_OK:
        raise PicError(code, where)
    return code


def make_config(phys: dict, **over) -> pic_config:
    """pic_config from a dict of physical inputs (see workloads.py)."""
    d = dict(phys)
    d.update(over)
    c = pic_config()
    for name, _ in pic_config._fields_:
        key = "lambda" if name == "lambda_" else name
        if key in d:
            setattr(c, name, d[key])
    return c


# ---- C-ABI names, argument marshalling only -------------------------------------------------

def pic_workspace_size(cfg: pic_config) -> int:
    n = ctypes.c_size_t()
    _check(load_library().pic_workspace_size(ctypes.byref(cfg), ctypes.byref(n)), "pic_workspace_size")
    return n.value


def pic_init(cfg: pic_config, workspace_ptr: int, workspace_bytes: int, stream_ptr: int):
    h = _VP()
    _check(load_library().pic_init(ctypes.byref(cfg), workspace_ptr, workspace_bytes, stream_ptr, ctypes.byref(h)),
           "pic_init")
    return h


def pic_free(h):
    load_library().pic_free(h)


def pic_step(h, nsteps: int) -> int:
    return _check(load_library().pic_step(h, int(nsteps)), "pic_step")


def pic_deposit_density(h, dev_out_ptr: int) -> float:
    s = ctypes.c_double()
    _check(load_library().pic_deposit_density(h, dev_out_ptr, ctypes.byref(s)), "pic_deposit_density")
    return s.value


def pic_pair_force(h, dev_out_ptr: int):
    _check(load_library().pic_pair_force(h, dev_out_ptr), "pic_pair_force")


def pic_crater_profile(h, dev_rho0_ptr: int, dev_out_ptr: int):
    _check(load_library().pic_crater_profile(h, dev_rho0_ptr, dev_out_ptr), "pic_crater_profile")


def pic_pair_force_at(h, n: int, cell_ptr: int, fx_ptr: int, fz_ptr: int, pot_mode: int, c_att: float, s_rep: float,
                      out_ptr: int):
    _check(load_library().pic_pair_force_at(h, int(n), cell_ptr, fx_ptr, fz_ptr, int(pot_mode), float(c_att),
                                            float(s_rep), out_ptr), "pic_pair_force_at")


def pic_cell_temperature(h, species: int, dev_work_ptr: int, dev_T_ptr: int):
    _check(load_library().pic_cell_temperature(h, int(species), dev_work_ptr, dev_T_ptr), "pic_cell_temperature")


def pic_set_temperature(h, species: int, dev_T_ptr: int, T_from: float):
    _check(load_library().pic_set_temperature(h, int(species), dev_T_ptr, float(T_from)), "pic_set_temperature")


def pic_regrid_cells(dims: int, src_ptr: int, src_grid: tuple, dst_ptr: int, dst_grid: tuple, fill: float,
                     stream_ptr: int = 0):
    """src_grid / dst_grid: (nx, ny, nz, dx, surface) of each grid (ny ignored in 2D)."""
    snx, sny, snz, sdx, ssf = src_grid
    dnx, dny, dnz, ddx, dsf = dst_grid
    _check(load_library().pic_regrid_cells(int(dims), src_ptr, int(snx), int(sny), int(snz), float(sdx), int(ssf),
                                           dst_ptr, int(dnx), int(dny), int(dnz), float(ddx), int(dsf), float(fill),
                                           stream_ptr or None), "pic_regrid_cells")


def regrid_cells(src, src_grid: tuple, dst_grid: tuple, fill: float, dims: int = 2):
    """Conservative remap of a cell map (a CUDA float64 tensor of shape (nz, nx) or (nz, ny, nx))
    from src_grid onto dst_grid, both (nx, ny, nz, dx, surface); returns a new tensor on the
    current stream (see pic_regrid_cells)."""
    import torch
    src = torch.as_tensor(src, dtype=torch.float64).cuda().contiguous()
    dnx, dny, dnz = dst_grid[0], dst_grid[1], dst_grid[2]
    out = torch.empty((dnz, dny, dnx) if dims == 3 else (dnz, dnx), dtype=torch.float64, device="cuda")
    pic_regrid_cells(dims, src.data_ptr(), src_grid, out.data_ptr(), dst_grid, fill,
                     torch.cuda.current_stream().cuda_stream)
    return out


def pic_energy(h) -> dict:
    e = pic_energy_t()
    _check(load_library().pic_energy(h, ctypes.byref(e)), "pic_energy")
    return {k: getattr(e, k) for k, _ in pic_energy_t._fields_}


def pic_get_info(h) -> dict:
    i = pic_info()
    _check(load_library().pic_get_info(h, ctypes.byref(i)), "pic_get_info")
    return dict(dt=i.dt, weight=i.weight, rho_scale=i.rho_scale, r0=i.r0, time=i.time, step=i.step,
                num_particles=(i.num_particles[0], i.num_particles[1]), nspecies=i.nspecies, ntiles=i.ntiles)


def pic_get_particles(h, species, ptrs, on_host):
    _check(load_library().pic_get_particles(h, species, *ptrs, 1 if on_host else 0), "pic_get_particles")


def pic_set_particles(h, species, n, ptrs, on_host):
    _check(load_library().pic_set_particles(h, species, int(n), *ptrs, 1 if on_host else 0), "pic_set_particles")


def pic_get_field(h, which, ptr, on_host):
    _check(load_library().pic_get_field(h, which, ptr, 1 if on_host else 0), "pic_get_field")


def pic_set_field(h, which, ptr, on_host):
    _check(load_library().pic_set_field(h, which, ptr, 1 if on_host else 0), "pic_set_field")


def pic_get_current(h, ptr, on_host):
    _check(load_library().pic_get_current(h, ptr, 1 if on_host else 0), "pic_get_current")


def pic_get_density(h, ptr, on_host):
    _check(load_library().pic_get_density(h, ptr, 1 if on_host else 0), "pic_get_density")


def pic_sort(h):
    _check(load_library().pic_sort(h), "pic_sort")


def pic_set_timing(h, enable):
    _check(load_library().pic_set_timing(h, 1 if enable else 0), "pic_set_timing")


def pic_get_timing(h):
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_int64 * 4)()
    _check(load_library().pic_get_timing(h, ms, n), "pic_get_timing")
    return list(ms), list(n)


def pic_energy_noalloc(cfg, view, dev_out_ptr, stream_ptr):
    _check(load_library().pic_energy_noalloc(ctypes.byref(cfg), ctypes.byref(view), dev_out_ptr, stream_ptr),
           "pic_energy_noalloc")


def pic_batch_workspace_size(cfgs) -> int:
    arr = (pic_config * len(cfgs))(*cfgs)
    n = ctypes.c_size_t()
    _check(load_library().pic_batch_workspace_size(arr, len(cfgs), ctypes.byref(n)), "pic_batch_workspace_size")
    return n.value


def pic_batch_init(cfgs, workspace_ptr, workspace_bytes, stream_ptr):
    arr = (pic_config * len(cfgs))(*cfgs)
    h = _VP()
    _check(load_library().pic_batch_init(arr, len(cfgs), workspace_ptr, workspace_bytes, stream_ptr, ctypes.byref(h)),
           "pic_batch_init")
    return h


def pic_batch_step(b, nsteps):
    return _check(load_library().pic_batch_step(b, int(nsteps)), "pic_batch_step")


def pic_batch_slab(b, i):
    h = _VP()
    _check(load_library().pic_batch_slab(b, int(i), ctypes.byref(h)), "pic_batch_slab")
    return h


def pic_batch_set_timing(b, enable):
    _check(load_library().pic_batch_set_timing(b, 1 if enable else 0), "pic_batch_set_timing")


def pic_batch_get_timing(b):
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_int64 * 4)()
    _check(load_library().pic_batch_get_timing(b, ms, n), "pic_batch_get_timing")
    return list(ms), list(n)


def pic_batch_free(b):
    load_library().pic_batch_free(b)


def pic_checkpoint_size(h) -> int:
    n = ctypes.c_size_t()
    _check(load_library().pic_checkpoint_size(h, ctypes.byref(n)), "pic_checkpoint_size")
    return n.value


def pic_checkpoint_save(h, ptr, on_host=False):
    _check(load_library().pic_checkpoint_save(h, ptr, 1 if on_host else 0), "pic_checkpoint_save")


def pic_checkpoint_restore(h, ptr, on_host=False):
    _check(load_library().pic_checkpoint_restore(h, ptr, 1 if on_host else 0), "pic_checkpoint_restore")


def pic_node_functional(h, dev_weights_ptr) -> float:
    v = ctypes.c_double()
    _check(load_library().pic_node_functional(h, dev_weights_ptr, ctypes.byref(v)), "pic_node_functional")
    return v.value


def pic_adjoint_seed(h, kin, dev_weights_ptr, bufs) -> float:
    v = ctypes.c_double()
    _check(load_library().pic_adjoint_seed(h, float(kin), dev_weights_ptr, ctypes.byref(bufs), ctypes.byref(v)),
           "pic_adjoint_seed")
    return v.value


def pic_adjoint_step(h, bufs):
    _check(load_library().pic_adjoint_step(h, ctypes.byref(bufs)), "pic_adjoint_step")


# ---- convenience wrapper: torch owns the workspace and the stream -----------------------------

class Simulation:
    """One simulation on the current CUDA device; device memory comes from torch."""

    def __init__(self, phys: dict, stream=None, **over):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.torch = torch
        self.cfg = make_config(phys, **over)
        nbytes = pic_workspace_size(self.cfg)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = pic_init(self.cfg, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)
        info = self.info()
        self.nx, self.nz = self.cfg.nx, self.cfg.nz
        self.dims = 3 if self.cfg.dims == 3 else 2
        self.ny = self.cfg.ny if self.dims == 3 else 1
        self.nspecies = info["nspecies"]

    def close(self):
        if getattr(self, "h", None):
            pic_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return pic_get_info(self.h)

    def step(self, n=1):
        return pic_step(self.h, n)

    def energy(self):
        return pic_energy(self.h)

    def sort(self):
        pic_sort(self.h)

    def checkpoint(self, out=None, on_host=False):
        """Save the whole state into a buffer (allocated when not given: a device tensor, or a
        pinned host tensor with on_host) and return it."""
        if out is None:
            n = pic_checkpoint_size(self.h)
            out = (self.torch.empty(n, dtype=self.torch.uint8).pin_memory() if on_host
                   else self.torch.empty(n, dtype=self.torch.uint8, device="cuda"))
        pic_checkpoint_save(self.h, out.data_ptr(), out.device.type == "cpu")
        return out

    def restore(self, buf):
        pic_checkpoint_restore(self.h, buf.data_ptr(), buf.device.type == "cpu")

    def _shape(self):
        return (self.nz + 1, self.ny, self.nx) if self.dims == 3 else (self.nz + 1, self.nx)

    def _grid(self, dtype):
        return self.torch.empty(self._shape(), dtype=dtype, device="cuda")

    def deposit_density(self):
        out = self._grid(self.torch.int64)
        scale = pic_deposit_density(self.h, out.data_ptr())
        return out, scale

    def _cells(self):
        return (self.nz, self.ny, self.nx) if self.dims == 3 else (self.nz, self.nx)

    def cell_grid(self):
        """(nx, ny, nz, dx, surface) of the context's cells (surface: the first row above the slab),
        the grid description regrid_cells takes."""
        return (self.nx, self.ny, self.nz, self.cfg.dx, self.cfg.slab_k)

    def cell_temperature(self, species):
        """Lattice temperature (K) of a species per cell, about each cell's mean flow."""
        t = self.torch
        shape = self._cells()
        work = t.empty(5 * int(np.prod(shape)), dtype=t.float64, device="cuda")
        out = t.empty(shape, dtype=t.float64, device="cuda")
        pic_cell_temperature(self.h, species, work.data_ptr(), out.data_ptr())
        self.stream.synchronize()
        return out

    def set_temperature(self, species, T, T_from):
        """Scale a species' momenta (drawn at T_from) to the per-cell temperatures T (K)."""
        t = self.torch
        T = t.as_tensor(T, dtype=t.float64).cuda().contiguous()
        assert tuple(T.shape) == self._cells()
        self.stream.synchronize()
        pic_set_temperature(self.h, species, T.data_ptr(), T_from)
        self.stream.synchronize()

    def crater_profile(self, rho0):
        """Material missing from each column of the original slab (m of solid-density material)
        against the node sums rho0 of an earlier state (from deposit_density)."""
        out = self.torch.empty((self.ny, self.nx) if self.dims == 3 else (self.nx,), dtype=self.torch.float64,
                               device="cuda")
        pic_crater_profile(self.h, rho0.data_ptr(), out.data_ptr())
        return out

    def pair_force_at(self, cell, fx, fz, pot_mode=None, c_att=None, s_rep=None):
        """Pair force (N) at probe positions (cell index, offsets) from the current node density;
        the probes add nothing to it. pot_mode / c_att / s_rep default to the configuration's."""
        t = self.torch
        cell = t.as_tensor(cell, dtype=t.int32).cuda().contiguous()
        fx = t.as_tensor(fx, dtype=t.float32).cuda().contiguous()
        fz = t.as_tensor(fz, dtype=t.float32).cuda().contiguous()
        out = t.empty((cell.numel(), 3), dtype=t.float32, device="cuda")
        self.stream.synchronize()
        pic_pair_force_at(self.h, cell.numel(), cell.data_ptr(), fx.data_ptr(), fz.data_ptr(),
                          self.cfg.pot_mode if pot_mode is None else pot_mode,
                          self.cfg.c_att if c_att is None else c_att, self.cfg.s_rep if s_rep is None else s_rep,
                          out.data_ptr())
        self.stream.synchronize()
        return out

    def pair_force(self):
        n = self.info()["num_particles"][0]
        out = self.torch.empty((n, 3), dtype=self.torch.float32, device="cuda")
        pic_pair_force(self.h, out.data_ptr())
        return out

    def get_particles(self, species):
        n = self.info()["num_particles"][species]
        t = self.torch
        names = ("cell", "fx", "fy", "fz", "ux", "uy", "uz")
        arrs = [t.empty(n, dtype=t.int32, device="cuda")] + [t.empty(n, dtype=t.float32, device="cuda") for _ in range(6)]
        if n:
            ptrs = [a.data_ptr() for a in arrs]
            if self.dims == 2:
                ptrs[2] = None
            pic_get_particles(self.h, species, ptrs, False)
        self.stream.synchronize()
        out = dict(zip(names, arrs))
        if self.dims == 2:
            del out["fy"]
        return out

    def set_particles(self, species, cell, fx, fz, ux, uy, uz, fy=None):
        t = self.torch
        arrs = [t.as_tensor(cell, dtype=t.int32).cuda().contiguous()] + \
               [t.as_tensor(a, dtype=t.float32).cuda().contiguous() for a in (fx, fz, ux, uy, uz)]
        fyt = t.as_tensor(fy, dtype=t.float32).cuda().contiguous() if fy is not None else None
        self.stream.synchronize()
        ptrs = [a.data_ptr() for a in arrs]
        ptrs.insert(2, fyt.data_ptr() if fyt is not None else None)
        pic_set_particles(self.h, species, arrs[0].numel(), ptrs, False)

    def get_field(self, which):
        out = self._grid(self.torch.float32)
        pic_get_field(self.h, which, out.data_ptr(), False)
        self.stream.synchronize()
        return out

    def set_field(self, which, values):
        v = self.torch.as_tensor(values, dtype=self.torch.float32).cuda().contiguous()
        assert v.numel() == (self.nz + 1) * self.ny * self.nx
        self.stream.synchronize()
        pic_set_field(self.h, which, v.data_ptr(), False)

    def get_current(self):
        out = self.torch.empty((3,) + self._shape(), dtype=self.torch.int64, device="cuda")
        pic_get_current(self.h, out.data_ptr(), False)
        self.stream.synchronize()
        return out

    def get_density(self):
        out = self._grid(self.torch.int64)
        pic_get_density(self.h, out.data_ptr(), False)
        self.stream.synchronize()
        return out


class SlabView(Simulation):
    """A slab of a Batch, accessed with the Simulation methods (state, energies, forces)."""

    def __init__(self, batch, i, cfg):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.stream = batch.stream
        self.h = pic_batch_slab(batch.b, i)
        self.nx, self.nz = cfg.nx, cfg.nz
        self.dims, self.ny = 2, 1
        self.nspecies = self.info()["nspecies"]
        self._owner = batch

    def close(self):
        self.h = None           # owned by the batch

    def step(self, n=1):
        raise RuntimeError("a slab of a batch is stepped through its Batch")


class Batch:
    """Several independent slabs advanced together (one persistent launch per step, CUDA graph)."""

    def __init__(self, phys_list, **over):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.torch = torch
        self.cfgs = [make_config(p, **over) for p in phys_list]
        nbytes = pic_batch_workspace_size(self.cfgs)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = torch.cuda.Stream()
        torch.cuda.synchronize()
        self.b = pic_batch_init(self.cfgs, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)
        self.slabs = [SlabView(self, i, c) for i, c in enumerate(self.cfgs)]

    def step(self, n=1):
        return pic_batch_step(self.b, n)

    def close(self):
        if getattr(self, "b", None):
            pic_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
