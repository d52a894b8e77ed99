"""FP64 CPU oracle of the PIC cycle with the pair-potential force (arXiv:1502.07722).

TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import this package. The product library never imports it and shares no code
with it; the C source (pic_oracle.c) holds the arithmetic, this module only marshals arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile pic_oracle.c into liboracle.so (plain gcc, contraction off)."""
    import platform
    stamp = _LIB + ".arch"
    if not os.path.exists(stamp) or open(stamp).read().strip() != platform.machine():
        force = True
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
        with open(stamp, "w") as f:
            f.write(platform.machine() + "\n")
    return _LIB


class OracleConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("nz", ctypes.c_int32), ("slab_k", ctypes.c_int32),
        ("mode", ctypes.c_int32), ("ppc_ion", ctypes.c_int32), ("ppc_electron", ctypes.c_int32),
        ("pot_mode", ctypes.c_int32), ("laser_profile", ctypes.c_int32),
        ("dx", ctypes.c_double), ("cfl", ctypes.c_double), ("dt_override", ctypes.c_double),
        ("n_atoms", ctypes.c_double), ("T_ion_K", ctypes.c_double), ("T_electron_eV", ctypes.c_double),
        ("ion_charge", ctypes.c_double), ("ion_mass_amu", ctypes.c_double),
        ("D_eV", ctypes.c_double), ("r0", ctypes.c_double), ("c_att", ctypes.c_double),
        ("s_rep", ctypes.c_double), ("lambda_", ctypes.c_double), ("I0", ctypes.c_double),
        ("tau_fwhm", ctypes.c_double), ("w0", ctypes.c_double), ("t_peak", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("temp_profile", ctypes.c_int32), ("lattice", ctypes.c_int32),
        ("T_spot_K", ctypes.c_double), ("spot_w", ctypes.c_double), ("spot_depth", ctypes.c_double),
        ("morse_a", ctypes.c_double),
        ("eam_ec", ctypes.c_double), ("eam_phi", ctypes.c_double), ("eam_alpha", ctypes.c_double),
        ("eam_beta", ctypes.c_double), ("eam_gamma", ctypes.c_double),
    ]


class OracleConfig3(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("slab_k", ctypes.c_int32),
        ("mode", ctypes.c_int32), ("ppc_ion", ctypes.c_int32), ("ppc_electron", ctypes.c_int32),
        ("pot_mode", ctypes.c_int32), ("laser_profile", ctypes.c_int32),
        ("dx", ctypes.c_double), ("cfl", ctypes.c_double), ("dt_override", ctypes.c_double),
        ("n_atoms", ctypes.c_double), ("T_ion_K", ctypes.c_double), ("T_electron_eV", ctypes.c_double),
        ("ion_charge", ctypes.c_double), ("ion_mass_amu", ctypes.c_double),
        ("D_eV", ctypes.c_double), ("r0", ctypes.c_double), ("c_att", ctypes.c_double),
        ("s_rep", ctypes.c_double), ("lambda_", ctypes.c_double), ("I0", ctypes.c_double),
        ("tau_fwhm", ctypes.c_double), ("w0", ctypes.c_double), ("t_peak", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("temp_profile", ctypes.c_int32), ("lattice", ctypes.c_int32),
        ("T_spot_K", ctypes.c_double), ("spot_w", ctypes.c_double), ("spot_depth", ctypes.c_double),
        ("morse_a", ctypes.c_double),
        ("eam_ec", ctypes.c_double), ("eam_phi", ctypes.c_double), ("eam_alpha", ctypes.c_double),
        ("eam_beta", ctypes.c_double), ("eam_gamma", ctypes.c_double),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I64 = ctypes.POINTER(ctypes.c_int64)
_lib_handle = None


def lib():
    global _lib_handle
    if _lib_handle is None:
        L = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        sig = {
            "oracle_create": (vp, [ctypes.POINTER(OracleConfig), ctypes.c_int32]),
            "oracle_free": (None, [vp]),
            "oracle_num_particles": (ctypes.c_int64, [vp, ctypes.c_int32]),
            "oracle_dt": (ctypes.c_double, [vp]),
            "oracle_weight": (ctypes.c_double, [vp]),
            "oracle_rho_scale": (ctypes.c_double, [vp]),
            "oracle_step_count": (ctypes.c_int64, [vp]),
            "oracle_get_particles": (None, [vp, ctypes.c_int32, _D, _D, _D, _D, _D]),
            "oracle_set_particles": (None, [vp, ctypes.c_int32, ctypes.c_int64, _D, _D, _D, _D, _D]),
            "oracle_get_field": (None, [vp, ctypes.c_int32, _D]),
            "oracle_set_field": (None, [vp, ctypes.c_int32, _D]),
            "oracle_get_rho": (None, [vp, _I64]),
            "oracle_set_rho": (None, [vp, _I64]),
            "oracle_get_current": (None, [vp, _I64]),
            "oracle_set_current": (None, [vp, _I64]),
            "oracle_set_step": (None, [vp, ctypes.c_int64]),
            "oracle_pair_force": (None, [vp, _D]),
            "oracle_gather_density": (None, [vp, ctypes.c_double, ctypes.c_double, _D]),
            "oracle_gather_fields": (None, [vp, ctypes.c_double, ctypes.c_double, _D]),
            "oracle_step": (None, [vp, ctypes.c_int32]),
            "oracle_maxwell": (None, [vp]),
            "oracle_energy": (None, [vp, _D]),
            "oracle_laser_field": (ctypes.c_double, [vp, ctypes.c_double, ctypes.c_double]),
            "oracle_lj_U": (ctypes.c_double, [ctypes.c_double]),
            "oracle_lj_dU": (ctypes.c_double, [ctypes.c_double]),
            "oracle_morse_U": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
            "oracle_morse_dU": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
            "oracle_neighbor_distances": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, _D]),
            "oracle_boris": (None, [ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, _D, _D, _D]),
            "oracle_jy_code": (ctypes.c_int64, [ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int32]),
            "oracle_jy_bits": (ctypes.c_int32, [ctypes.c_int64]),
            "oracle_eam_atom2": (None, [ctypes.c_double] * 10 + [_D]),
            "oracle_deposit_density": (None, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _D, _D, _I64]),
            "oracle_deposit_current": (None, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                              _D, _D, _D, _D, _F, _F, _F, ctypes.c_int32, _I64, _I64, _I64]),
        }
        sig.update({
            "oracle_transport_grad": (None, [vp, ctypes.c_int32, _D, ctypes.c_double, _D]),
            "oracle_transport_loss": (ctypes.c_double, [vp, ctypes.c_int32, _D, ctypes.c_double, ctypes.c_double,
                                                        ctypes.c_double]),
            "oracle_D": (ctypes.c_double, [vp]),
            "oracle_E0": (ctypes.c_double, [vp]),
            "oracle_injected": (ctypes.c_double, [vp]),
            "oracle_init_particle": (None, [vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _D]),
            "oracle_push_one": (None, [vp, ctypes.c_int32, _D]),
            "oracle3_init_particle": (None, [vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int64, _D]),
            "oracle3_push_one": (None, [vp, ctypes.c_int32, _D]),
            "oracle3_injected": (ctypes.c_double, [vp]),
            "oracle_full_grad": (None, [vp, ctypes.c_int32, _D, ctypes.c_double, _D]),
            "oracle_full_loss": (ctypes.c_double, [vp, ctypes.c_int32, _D, ctypes.c_double, ctypes.c_double,
                                                   ctypes.c_double, ctypes.c_double]),
            "oracle_maxwell_cont": (None, [vp, _D, _D, ctypes.c_double, ctypes.c_int64]),
            "oracle_maxwell_cont_T": (None, [vp, _D, _D, ctypes.c_int64, _D]),
            "oracle_r0": (ctypes.c_double, [vp]),
            "oracle_crater_profile": (None, [vp, _I64, _I64, _D]),
            "oracle_cell_temperature": (None, [vp, ctypes.c_int32, _D]),
            "oracle_set_temperature": (None, [vp, ctypes.c_int32, _D, ctypes.c_double]),
            "oracle_regrid_cells": (None, [ctypes.c_int32, _D, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_double, ctypes.c_int32, _D, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_double]),
            "oracle3_create": (vp, [ctypes.POINTER(OracleConfig3), ctypes.c_int32]),
            "oracle3_free": (None, [vp]),
            "oracle3_num_particles": (ctypes.c_int64, [vp, ctypes.c_int32]),
            "oracle3_dt": (ctypes.c_double, [vp]),
            "oracle3_weight": (ctypes.c_double, [vp]),
            "oracle3_rho_scale": (ctypes.c_double, [vp]),
            "oracle3_set_step": (None, [vp, ctypes.c_int64]),
            "oracle3_get_particles": (None, [vp, ctypes.c_int32, _D, _D, _D, _D, _D, _D]),
            "oracle3_set_particles": (None, [vp, ctypes.c_int32, ctypes.c_int64, _D, _D, _D, _D, _D, _D]),
            "oracle3_get_field": (None, [vp, ctypes.c_int32, _D]),
            "oracle3_set_field": (None, [vp, ctypes.c_int32, _D]),
            "oracle3_get_rho": (None, [vp, _I64]),
            "oracle3_crater_profile": (None, [vp, _I64, _I64, _D]),
            "oracle3_set_rho": (None, [vp, _I64]),
            "oracle3_get_current": (None, [vp, _I64]),
            "oracle3_set_current": (None, [vp, _I64]),
            "oracle3_pair_force": (None, [vp, _D]),
            "oracle3_gather_fields": (None, [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]),
            "oracle3_maxwell": (None, [vp]),
            "oracle3_step": (None, [vp, ctypes.c_int32]),
            "oracle3_energy": (None, [vp, _D]),
            "oracle3_deposit_density": (None, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                               _D, _D, _D, _I64]),
            "oracle3_deposit_current": (None, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                               ctypes.c_int32, _D, _D, _D, _D, _D, _D, _I64, _I64, _I64]),
        })
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib_handle = L
    return _lib_handle


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


FIELD_NAMES = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")


def make_config(phys: dict) -> OracleConfig:
    """Fill the oracle's own configuration from a dict of physical inputs."""
    c = OracleConfig()
    for name, _ in OracleConfig._fields_:
        key = "lambda" if name == "lambda_" else name
        if key in phys:
            setattr(c, name, phys[key])
    return c


class Oracle:
    """One FP64 simulation state (2D3V). Positions are global cell coordinates."""

    def __init__(self, phys: dict, with_particles: bool = True):
        self.phys = dict(phys)
        self.cfg = make_config(phys)
        self._s = lib().oracle_create(ctypes.byref(self.cfg), 1 if with_particles else 0)
        self.nx, self.nz = self.cfg.nx, self.cfg.nz
        self.nspecies = 2 if self.cfg.mode == 0 else 1

    def __del__(self):
        if getattr(self, "_s", None):
            lib().oracle_free(self._s)
            self._s = None

    # scalars
    @property
    def dt(self):
        return lib().oracle_dt(self._s)

    @property
    def weight(self):
        return lib().oracle_weight(self._s)

    @property
    def rho_scale(self):
        return lib().oracle_rho_scale(self._s)

    @property
    def step_count(self):
        return lib().oracle_step_count(self._s)

    def set_step(self, n):
        lib().oracle_set_step(self._s, int(n))

    # particles
    def num_particles(self, sp):
        return lib().oracle_num_particles(self._s, sp)

    def get_particles(self, sp):
        n = self.num_particles(sp)
        arrs = [np.empty(n, np.float64) for _ in range(5)]
        lib().oracle_get_particles(self._s, sp, *[_p(a, ctypes.c_double) for a in arrs])
        return dict(zip(("x", "z", "ux", "uy", "uz"), arrs))

    def set_particles(self, sp, x, z, ux, uy, uz):
        arrs = [_f64(a) for a in (x, z, ux, uy, uz)]
        lib().oracle_set_particles(self._s, sp, len(arrs[0]), *[_p(a, ctypes.c_double) for a in arrs])

    # grids
    def _nn(self):
        return self.nx * (self.nz + 1)

    def get_field(self, f):
        out = np.empty(self._nn(), np.float64)
        lib().oracle_get_field(self._s, f, _p(out, ctypes.c_double))
        return out.reshape(self.nz + 1, self.nx)

    def set_field(self, f, a):
        a = _f64(a).reshape(-1)
        assert a.size == self._nn()
        lib().oracle_set_field(self._s, f, _p(a, ctypes.c_double))

    def get_rho(self):
        out = np.empty(self._nn(), np.int64)
        lib().oracle_get_rho(self._s, _p(out, ctypes.c_int64))
        return out.reshape(self.nz + 1, self.nx)

    def set_rho(self, a):
        a = np.ascontiguousarray(a, np.int64).reshape(-1)
        lib().oracle_set_rho(self._s, _p(a, ctypes.c_int64))

    def cell_temperature(self, sp):
        """Kinetic temperature (K) of species sp per cell about the cell's mean flow, (nz, nx)."""
        out = np.empty(self.nx * self.nz, np.float64)
        lib().oracle_cell_temperature(self._s, sp, _p(out, ctypes.c_double))
        return out.reshape(self.nz, self.nx)

    def set_temperature(self, sp, T, T_from):
        """Scale species sp's momenta by sqrt(T_cell / T_from), T a (nz, nx) map."""
        t = np.ascontiguousarray(T, np.float64).reshape(-1)
        assert t.size == self.nx * self.nz
        lib().oracle_set_temperature(self._s, sp, _p(t, ctypes.c_double), float(T_from))

    def crater_profile(self, rho0, rho=None):
        """Material missing from each node column of the original slab (m of solid-density
        material) between node sums rho0 and rho (default: the state's own)."""
        r0 = np.ascontiguousarray(rho0, np.int64).reshape(-1)
        assert r0.size == self._nn()
        r = None if rho is None else np.ascontiguousarray(rho, np.int64).reshape(-1)
        out = np.empty(self.nx, np.float64)
        lib().oracle_crater_profile(self._s, _p(r0, ctypes.c_int64),
                                    None if r is None else _p(r, ctypes.c_int64), _p(out, ctypes.c_double))
        return out

    def get_current(self):
        out = np.empty(3 * self._nn(), np.int64)
        lib().oracle_get_current(self._s, _p(out, ctypes.c_int64))
        return out.reshape(3, self.nz + 1, self.nx)

    def set_current(self, a):
        a = np.ascontiguousarray(a, np.int64).reshape(-1)
        lib().oracle_set_current(self._s, _p(a, ctypes.c_int64))

    # physics
    def step(self, n=1):
        lib().oracle_step(self._s, int(n))

    def maxwell(self):
        lib().oracle_maxwell(self._s)

    def pair_force(self):
        n = self.num_particles(0)
        out = np.empty(3 * n, np.float64)
        lib().oracle_pair_force(self._s, _p(out, ctypes.c_double))
        return out.reshape(n, 3)

    def gather_density(self, x, z):
        out = np.empty(3, np.float64)
        lib().oracle_gather_density(self._s, float(x), float(z), _p(out, ctypes.c_double))
        return out

    def gather_fields(self, x, z):
        """(Ex, Ey, Ez, Bx, By, Bz) interpolated to the point (x, z) in cells, as the push sees them."""
        out = np.zeros(6)
        lib().oracle_gather_fields(self._s, float(x), float(z), _p(out, ctypes.c_double))
        return out

    def energy(self):
        out = np.empty(5, np.float64)
        lib().oracle_energy(self._s, _p(out, ctypes.c_double))
        d = dict(zip(("kinetic_ion", "kinetic_electron", "field_E", "field_B", "pair"), out))
        d["injected"] = lib().oracle_injected(self._s)
        return d

    def transport_grad(self, nsteps, cw, kin):
        """Continuous-deposition transport run of nsteps with the loss sum(cw * n^) + kin * KE and
        its gradient: returns (L, dL/dD, dL/dr0). Advances the state."""
        cw = _f64(cw).reshape(-1)
        out = np.empty(3, np.float64)
        lib().oracle_transport_grad(self._s, int(nsteps), _p(cw, ctypes.c_double), float(kin), _p(out, ctypes.c_double))
        return tuple(out)

    def transport_loss(self, nsteps, cw, kin, D, r0):
        cw = _f64(cw).reshape(-1)
        return lib().oracle_transport_loss(self._s, int(nsteps), _p(cw, ctypes.c_double), float(kin), float(D), float(r0))

    def full_grad(self, nsteps, cw, kin):
        """Continuous-deposition full cycle (ions, electrons, fields, laser) of nsteps from the
        current state with the loss sum(cw * n^) + kin * (kinetic energy of all species) and its
        gradient: returns (L, dL/dD, dL/dr0, dL/dI0). The state is left unchanged."""
        cw = _f64(cw).reshape(-1)
        out = np.empty(4, np.float64)
        lib().oracle_full_grad(self._s, int(nsteps), _p(cw, ctypes.c_double), float(kin), _p(out, ctypes.c_double))
        return tuple(out)

    def full_loss(self, nsteps, cw, kin, D, r0, I0):
        cw = _f64(cw).reshape(-1)
        return lib().oracle_full_loss(self._s, int(nsteps), _p(cw, ctypes.c_double), float(kin), float(D), float(r0),
                                      float(I0))

    def maxwell_cont(self, F, j, E0, step):
        """One Maxwell update of the continuous cycle: F (6, nz+1, nx) fields, j (3, nz+1, nx) the
        scaled current dt J / eps0; returns the new fields."""
        F = _f64(F).copy()
        j = _f64(j)
        lib().oracle_maxwell_cont(self._s, _p(F, ctypes.c_double), _p(j, ctypes.c_double), float(E0), int(step))
        return F

    def maxwell_cont_T(self, lF, step):
        """Transpose of maxwell_cont: returns (adjoint of the old fields, adjoint of j, dL/dE0)."""
        lF = _f64(lF).copy()
        lj = np.zeros((3,) + lF.shape[1:], np.float64)
        g = np.zeros(1, np.float64)
        lib().oracle_maxwell_cont_T(self._s, _p(lF, ctypes.c_double), _p(lj, ctypes.c_double), int(step),
                                    _p(g, ctypes.c_double))
        return lF, lj, g[0]

    @property
    def E0(self):
        return lib().oracle_E0(self._s)

    @property
    def D(self):
        return lib().oracle_D(self._s)

    @property
    def r0(self):
        return lib().oracle_r0(self._s)

    def init_particle(self, sp, i, k, j):
        """Initial (x, z, ux, uy, uz) of the particle in slot j of cell (i, k)."""
        v = np.empty(5, np.float64)
        lib().oracle_init_particle(self._s, int(sp), int(i), int(k), int(j), _p(v, ctypes.c_double))
        return v

    def push_one(self, sp, v):
        """One particle's step (gather, pair force, Boris, move) from the current fields and node
        density: (x, z, ux, uy, uz) -> new values."""
        v = _f64(v).copy()
        lib().oracle_push_one(self._s, int(sp), _p(v, ctypes.c_double))
        return v

    def laser_field(self, x_cells, t):
        return lib().oracle_laser_field(self._s, float(x_cells), float(t))


# standalone helpers --------------------------------------------------------------------

def lj_U(r):
    return lib().oracle_lj_U(float(r))


def lj_dU(r):
    return lib().oracle_lj_dU(float(r))


def morse_U(a, r):
    """Morse potential (units D, r in units of r0, minimum -1 at r = 1), stiffness a = alpha r0."""
    return lib().oracle_morse_U(float(a), float(r))


def morse_dU(a, r):
    return lib().oracle_morse_dU(float(a), float(r))


def neighbor_distances(n, dn, r0_dx):
    a = ctypes.c_double()
    b = ctypes.c_double()
    rbar = lib().oracle_neighbor_distances(float(n), float(dn), float(r0_dx), ctypes.byref(a), ctypes.byref(b))
    return rbar, a.value, b.value


def boris(q, m, dt, E, B, F, u):
    E, B, F = (np.ascontiguousarray(v, np.float64) for v in (E, B, F))
    u = np.array(u, np.float64)
    lib().oracle_boris(q, m, dt, _p(E, ctypes.c_double), _p(B, ctypes.c_double), _p(F, ctypes.c_double),
                       _p(u, ctypes.c_double))
    return u


def jy_code(ux, uy, uz, bits=18):
    """J_y code V = rint(beta_y 2^bits) of one particle, taken in FP32 as the kernel takes it."""
    return lib().oracle_jy_code(float(np.float32(ux)), float(np.float32(uy)), float(np.float32(uz)), int(bits))


def eam_atom2(phys, n, dnx, dnz, r0_dx):
    """Embedded-atom force along x and z (units D / r0) and energy (units D) of one atom at density
    n (units n0) with gradient (dnx, dnz) per cell; r0_dx = r0 / dx."""
    out = np.zeros(3)
    lib().oracle_eam_atom2(phys["D_eV"], phys["eam_ec"], phys["eam_phi"], phys["eam_alpha"], phys["eam_beta"],
                           phys["eam_gamma"], float(n), float(dnx), float(dnz), float(r0_dx),
                           _p(out, ctypes.c_double))
    return out


def jy_bits(per_cell):
    """Resolution of the J_y code for a 2D slab with per_cell macroparticles per cell (both species)."""
    return lib().oracle_jy_bits(int(per_cell))


def regrid_cells(src, src_grid, dst_grid, fill, dims=2):
    """Conservative remap of a cell map between grids (nx, ny, nz, dx, surface) placed on each other
    by the slab surface and the laser axis; src of shape (nz, nx) or (nz, ny, nx)."""
    snx, sny, snz, sdx, ssf = src_grid
    dnx, dny, dnz, ddx, dsf = dst_grid
    if dims == 2:
        sny = dny = 1
    a = np.ascontiguousarray(src, dtype=np.float64).reshape(-1)
    assert a.size == snx * sny * snz
    out = np.empty(dnx * dny * dnz, np.float64)
    lib().oracle_regrid_cells(dims, _p(a, ctypes.c_double), snx, sny, snz, float(sdx), ssf, _p(out, ctypes.c_double),
                              dnx, dny, dnz, float(ddx), dsf, float(fill))
    return out.reshape((dnz, dny, dnx) if dims == 3 else (dnz, dnx))


def deposit_density(nx, nz, x, z):
    x, z = _f64(x), _f64(z)
    out = np.zeros(nx * (nz + 1), np.int64)
    lib().oracle_deposit_density(nx, nz, len(x), _p(x, ctypes.c_double), _p(z, ctypes.c_double),
                                 _p(out, ctypes.c_int64))
    return out.reshape(nz + 1, nx)


def deposit_current(nx, nz, sign, x0, z0, x1, z1, ux, uy, uz, out=None, bits=18):
    x0, z0, x1, z1 = (_f64(a) for a in (x0, z0, x1, z1))
    ux, uy, uz = (np.ascontiguousarray(a, np.float32) for a in (ux, uy, uz))
    if out is None:
        out = np.zeros((3, nz + 1, nx), np.int64)
    lib().oracle_deposit_current(nx, nz, len(x0), sign, _p(x0, ctypes.c_double), _p(z0, ctypes.c_double),
                                 _p(x1, ctypes.c_double), _p(z1, ctypes.c_double), _p(ux, ctypes.c_float),
                                 _p(uy, ctypes.c_float), _p(uz, ctypes.c_float), int(bits),
                                 _p(out[0], ctypes.c_int64), _p(out[1], ctypes.c_int64), _p(out[2], ctypes.c_int64))
    return out


class Oracle3D:
    """One FP64 simulation state in 3D (x, y periodic; walls in z). Positions in cells."""

    def __init__(self, phys: dict, with_particles: bool = True):
        self.phys = dict(phys)
        c = OracleConfig3()
        for name, _ in OracleConfig3._fields_:
            key = "lambda" if name == "lambda_" else name
            if key in phys:
                setattr(c, name, phys[key])
        self.cfg = c
        self._s = lib().oracle3_create(ctypes.byref(c), 1 if with_particles else 0)
        self.nx, self.ny, self.nz = c.nx, c.ny, c.nz
        self.nspecies = 2 if c.mode == 0 else 1

    def __del__(self):
        if getattr(self, "_s", None):
            lib().oracle3_free(self._s)
            self._s = None

    @property
    def dt(self):
        return lib().oracle3_dt(self._s)

    @property
    def weight(self):
        return lib().oracle3_weight(self._s)

    @property
    def rho_scale(self):
        return lib().oracle3_rho_scale(self._s)

    def set_step(self, n):
        lib().oracle3_set_step(self._s, int(n))

    def _shape(self):
        return (self.nz + 1, self.ny, self.nx)

    def _nn(self):
        return (self.nz + 1) * self.ny * self.nx

    def num_particles(self, sp):
        return lib().oracle3_num_particles(self._s, sp)

    def get_particles(self, sp):
        n = self.num_particles(sp)
        arrs = [np.empty(n, np.float64) for _ in range(6)]
        lib().oracle3_get_particles(self._s, sp, *[_p(a, ctypes.c_double) for a in arrs])
        return dict(zip(("x", "y", "z", "ux", "uy", "uz"), arrs))

    def set_particles(self, sp, x, y, z, ux, uy, uz):
        arrs = [_f64(a) for a in (x, y, z, ux, uy, uz)]
        lib().oracle3_set_particles(self._s, sp, len(arrs[0]), *[_p(a, ctypes.c_double) for a in arrs])

    def get_field(self, f):
        out = np.empty(self._nn(), np.float64)
        lib().oracle3_get_field(self._s, f, _p(out, ctypes.c_double))
        return out.reshape(self._shape())

    def set_field(self, f, a):
        a = _f64(a).reshape(-1)
        assert a.size == self._nn()
        lib().oracle3_set_field(self._s, f, _p(a, ctypes.c_double))

    def get_rho(self):
        out = np.empty(self._nn(), np.int64)
        lib().oracle3_get_rho(self._s, _p(out, ctypes.c_int64))
        return out.reshape(self._shape())

    def crater_profile(self, rho0, rho=None):
        """Material missing from each node column (j, i) of the original slab (m of solid-density
        material) between node sums rho0 and rho (default: the state's own); shape (ny, nx)."""
        r0 = np.ascontiguousarray(rho0, np.int64).reshape(-1)
        assert r0.size == self.nx * self.ny * (self.nz + 1)
        r = None if rho is None else np.ascontiguousarray(rho, np.int64).reshape(-1)
        out = np.empty((self.ny, self.nx), np.float64)
        lib().oracle3_crater_profile(self._s, _p(r0, ctypes.c_int64),
                                     None if r is None else _p(r, ctypes.c_int64), _p(out, ctypes.c_double))
        return out

    def set_rho(self, a):
        a = np.ascontiguousarray(a, np.int64).reshape(-1)
        lib().oracle3_set_rho(self._s, _p(a, ctypes.c_int64))

    def get_current(self):
        out = np.empty(3 * self._nn(), np.int64)
        lib().oracle3_get_current(self._s, _p(out, ctypes.c_int64))
        return out.reshape((3,) + self._shape())

    def set_current(self, a):
        a = np.ascontiguousarray(a, np.int64).reshape(-1)
        lib().oracle3_set_current(self._s, _p(a, ctypes.c_int64))

    def pair_force(self):
        n = self.num_particles(0)
        out = np.empty(3 * n, np.float64)
        lib().oracle3_pair_force(self._s, _p(out, ctypes.c_double))
        return out.reshape(n, 3)

    def gather_fields(self, x, y, z):
        """(Ex, Ey, Ez, Bx, By, Bz) interpolated to the point (x, y, z) in cells, as the push sees them."""
        out = np.zeros(6)
        lib().oracle3_gather_fields(self._s, float(x), float(y), float(z), _p(out, ctypes.c_double))
        return out

    def maxwell(self):
        lib().oracle3_maxwell(self._s)

    def step(self, n=1):
        lib().oracle3_step(self._s, int(n))

    def init_particle(self, sp, i, j, k, q):
        """Initial (x, y, z, ux, uy, uz) of the particle in slot q of cell (i, j, k)."""
        v = np.empty(6, np.float64)
        lib().oracle3_init_particle(self._s, int(sp), int(i), int(j), int(k), int(q), _p(v, ctypes.c_double))
        return v

    def push_one(self, sp, v):
        """One particle's step from the current fields and node density: (x, y, z, ux, uy, uz)."""
        v = _f64(v).copy()
        lib().oracle3_push_one(self._s, int(sp), _p(v, ctypes.c_double))
        return v

    def energy(self):
        out = np.empty(5, np.float64)
        lib().oracle3_energy(self._s, _p(out, ctypes.c_double))
        d = dict(zip(("kinetic_ion", "kinetic_electron", "field_E", "field_B", "pair"), out))
        d["injected"] = lib().oracle3_injected(self._s)
        return d


def deposit_density3(nx, ny, nz, x, y, z):
    x, y, z = _f64(x), _f64(y), _f64(z)
    out = np.zeros(nx * ny * (nz + 1), np.int64)
    lib().oracle3_deposit_density(nx, ny, nz, len(x), _p(x, ctypes.c_double), _p(y, ctypes.c_double),
                                  _p(z, ctypes.c_double), _p(out, ctypes.c_int64))
    return out.reshape(nz + 1, ny, nx)


def deposit_current3(nx, ny, nz, sign, x0, y0, z0, x1, y1, z1, out=None):
    a = [_f64(v) for v in (x0, y0, z0, x1, y1, z1)]
    if out is None:
        out = np.zeros((3, nz + 1, ny, nx), np.int64)
    lib().oracle3_deposit_current(nx, ny, nz, len(a[0]), sign, *[_p(v, ctypes.c_double) for v in a],
                                  _p(out[0], ctypes.c_int64), _p(out[1], ctypes.c_int64), _p(out[2], ctypes.c_int64))
    return out


def far_field(profile):
    """Median of the profile over the columns at least a quarter of the period away from the
    deepest column (the half of the columns farthest from it). A 3D profile (ny, nx): the distance
    is the periodic one in the x-y plane, compared squared in whole cells; columns at equal
    distance stay in row-major order."""
    d = np.asarray(profile, np.float64)
    if d.ndim == 2:
        ny, nx = d.shape
        flat = d.ravel()
        c = int(np.argmax(flat))
        cj, ci = c // nx, c % nx
        away = []
        for j in range(ny):
            for i in range(nx):
                ddx = min((i - ci) % nx, (ci - i) % nx)
                ddy = min((j - cj) % ny, (cj - j) % ny)
                away.append((ddx * ddx + ddy * ddy, j * nx + i))
        away.sort(key=lambda t: t[0])
        keep = [q for _, q in away[flat.size - flat.size // 2:]]
        return float(np.median(flat[keep])) if keep else 0.0
    n = d.size
    c = int(np.argmax(d))
    away = [(min((i - c) % n, (c - i) % n), i) for i in range(n)]
    away.sort(key=lambda t: t[0])
    keep = [i for _, i in away[n - n // 2:]]
    return float(np.median(d[keep])) if keep else 0.0


def crater_width(profile, dx, threshold=None):
    """Width of the crater around its deepest column: the columns above the threshold that join
    the deepest one form the crater; each edge is placed where the straight line between the last
    column inside and the first outside meets the threshold. x periodic. Returns (depth, width) in
    metres."""
    d = np.asarray(profile, np.float64)
    th = 0.5 * dx if threshold is None else threshold
    n = d.size
    c = int(np.argmax(d))
    if d[c] <= th:
        return float(d[c]), 0.0
    if np.all(d > th):
        return float(d[c]), float(n * dx)
    # walk the periodic line from the deepest column to the first column at or below the
    # threshold on each side (one exists: not every column is above it)
    hi = c
    while d[(hi + 1) % n] > th:
        hi += 1
    lo = c
    while d[(lo - 1) % n] > th:
        lo -= 1
    def edge(j_in, j_out):
        t = (d[j_in % n] - th) / (d[j_in % n] - d[j_out % n])
        return j_in + t * (j_out - j_in)
    return float(d[c]), float((edge(hi, hi + 1) - edge(lo, lo - 1)) * dx)


def crater_width_3d(profile, dx, threshold=None):
    """3D crater (profile (ny, nx), both axes periodic): depth at the deepest column and the widths
    of the crater along the row and along the column through it, each measured as crater_width
    does on that line. Returns (depth, width_x, width_y) in metres."""
    d = np.asarray(profile, np.float64)
    ny, nx = d.shape
    c = int(np.argmax(d.ravel()))
    cj, ci = c // nx, c % nx
    depth, wx = crater_width(d[cj, :], dx, threshold)
    _, wy = crater_width(d[:, ci], dx, threshold)
    return depth, wx, wy


def calibrate_c_att(phys, rho, k_from, k_to, points=8, halvings=20):
    """Attractive correction factor from the work the attractive branch of the pair force does on
    one probe atom pulled out of the slab whose node sums are rho (paper: the factor is found by
    integrating the force on a single atom leaving the target out to infinity). Probes on every
    column x = i + 1/2 cross the cell rows k_from .. k_to - 1. Each row is cut at 1/2, 1/4, ...,
    2^-halvings from both of its edges and each piece gets a `points`-point Gauss-Legendre rule:
    where the density tail meets the vacuum, Eq. 2 brings the lower neighbour arbitrarily close,
    which gives the attraction a narrow spike next to the edge (and makes the repulsion diverge,
    so the repulsive branch is left out). Removing one atom of the cubic lattice along the normal
    costs one bond, D, so c_att = -D / W_att. Returns (c_att, W_att)."""
    t, wt = np.polynomial.legendre.leggauss(points)
    cuts = [0.0, 1.0]
    for j in range(1, halvings + 1):
        cuts += [0.5 ** j, 1.0 - 0.5 ** j]
    cuts = sorted(set(cuts))
    nx = phys["nx"]
    zs, ws = [], []
    for k in range(k_from, k_to):
        for a, b in zip(cuts[:-1], cuts[1:]):
            for ti, wi in zip(t, wt):
                zs.append(k + a + 0.5 * (b - a) * (ti + 1.0))
                ws.append(0.5 * (b - a) * wi)
    zs, ws = np.array(zs), np.array(ws)
    px = np.tile(np.arange(nx) + 0.5, zs.size)
    pz = np.repeat(zs, nx)
    zero = np.zeros(px.size)
    o = Oracle(dict(phys, pot_mode=1, c_att=1.0, s_rep=0.0), with_particles=False)
    o.set_particles(0, px, pz, zero, zero, zero)
    o.set_rho(rho)
    fz = o.pair_force()[:, 2].reshape(zs.size, nx).mean(axis=1)
    w_att = float(np.dot(fz, ws) * phys["dx"])
    D = phys["D_eV"] * 1.602176634e-19
    return -D / w_att, w_att
