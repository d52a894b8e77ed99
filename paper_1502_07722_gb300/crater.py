"""Crater depth, width and threshold fluence from a column profile (paper: once the crater has
solidified its width and depth are measured from the density map; Eq. 5 turns the crater width
into a damage threshold fluence).

The profile comes from `Simulation.crater_profile` (material missing from each column of the
original slab, metres of solid-density material; column i sits at x = i dx). The width is the
distance between the two threshold crossings that bound the deepest column, located by linear
interpolation between columns (x periodic).
"""
import math

import numpy as np


def _periodic_offsets(n: int, i0: int) -> np.ndarray:
    """Signed distance (cells) of each index from i0 on a period of n, in [-n/2, n/2)."""
    return (np.arange(n) - i0 + n // 2) % n - n // 2


def far_field_level(profile) -> float:
    """Surface level far from the crater: the median of the profile over the half of the columns
    farthest (periodic distance) from the deepest column. The whole slab of the model relaxes (its
    density settles slightly below the start density, so material leaves the original rows
    everywhere); the crater is the loss beyond that level. A 3D profile (ny, nx) takes the squared
    distance in the x-y plane; columns at equal distance keep their row-major order."""
    d = np.asarray(profile, dtype=np.float64)
    if d.ndim == 2:
        j0, i0 = np.unravel_index(int(np.argmax(d)), d.shape)
        dy, dxc = _periodic_offsets(d.shape[0], j0), _periodic_offsets(d.shape[1], i0)
        dist = (dy[:, None] ** 2 + dxc[None, :] ** 2).ravel()
        d = d.ravel()
    else:
        d = d.ravel()
        dist = np.abs(_periodic_offsets(d.size, int(np.argmax(d))))
    n = d.size
    far = np.argsort(dist, kind="stable")[n - n // 2:]
    return float(np.median(d[far])) if far.size else 0.0


def _width_1d(d: np.ndarray, i0: int, th: float, dx: float):
    """Width and crossings of the run of columns above th that holds column i0 (periodic)."""
    n = len(d)
    if (d > th).all():                       # no edge: the whole line is below the threshold
        return n * dx, None, None
    r = i0
    while r - i0 < n - 1 and d[(r + 1) % n] > th:
        r += 1
    a, b = d[r % n], d[(r + 1) % n]
    right = r + (a - th) / (a - b)
    left_i = i0
    while i0 - left_i < n - 1 and d[(left_i - 1) % n] > th:
        left_i -= 1
    a, b = d[left_i % n], d[(left_i - 1) % n]
    left = left_i - (a - th) / (a - b)
    return (right - left) * dx, left * dx, right * dx


def crater_metrics(profile, dx: float, threshold: float = None, far_field: bool = False) -> dict:
    """depth (m, the deepest column), width (m), left / right crossings (m). threshold: missing
    material that counts as crater (default half a cell). far_field: measure from the far-field
    surface level (`far_field_level`, returned as "level") instead of the original surface.

    A 3D profile (ny, nx) is measured along the row and the column through the deepest column:
    width_x and width_y, and width = their mean, the diameter Eq. (5) takes; left / right are the
    crossings along x."""
    d = np.asarray(profile, dtype=np.float64)
    level = far_field_level(d) if far_field else 0.0
    d = d - level
    th = 0.5 * dx if threshold is None else float(threshold)
    if d.ndim == 2:
        j0, i0 = np.unravel_index(int(np.argmax(d)), d.shape)
        depth = float(d[j0, i0])
        if depth <= th:
            return {"depth": depth, "width": 0.0, "width_x": 0.0, "width_y": 0.0, "left": None,
                    "right": None, "level": level}
        wx, left, right = _width_1d(d[j0, :], int(i0), th, dx)
        wy, _, _ = _width_1d(d[:, i0], int(j0), th, dx)
        return {"depth": depth, "width": 0.5 * (wx + wy), "width_x": wx, "width_y": wy, "left": left,
                "right": right, "level": level}
    d = d.ravel()
    i0 = int(np.argmax(d))
    depth = float(d[i0])
    if depth <= th:
        return {"depth": depth, "width": 0.0, "left": None, "right": None, "level": level}
    width, left, right = _width_1d(d, i0, th, dx)
    return {"depth": depth, "width": width, "left": left, "right": right, "level": level}


def threshold_fluence(fluence: float, width: float, beam_diameter: float) -> float:
    """Eq. (5): F_th = F exp(-(Gamma / a)^2), Gamma the crater diameter, a the beam diameter."""
    return fluence * math.exp(-(width / beam_diameter) ** 2)


def run_crater(phys: dict, steps: int, every: int, fluence: float = None, beam_diameter: float = None):
    """Atomic-transport run from a lattice-temperature start: the crater's depth and width below
    the far-field surface level every `every` steps (and the Eq. 5 threshold when a fluence and
    beam diameter are given). Yields one dict per report; the simulation runs on the GPU."""
    from . import Simulation
    sim = Simulation(phys)
    try:
        rho0, _ = sim.deposit_density()
        done = 0
        while done < steps:
            n = min(every, steps - done)
            sim.step(n)
            done += n
            m = crater_metrics(sim.crater_profile(rho0).cpu().numpy(), phys["dx"], far_field=True)
            m["step"] = done
            m["time_s"] = sim.info()["time"]
            if fluence is not None and beam_diameter:
                m["F_th"] = threshold_fluence(fluence, m["width"], beam_diameter)
            yield m
    finally:
        sim.close()


if __name__ == "__main__":
    import argparse
    import json

    from .workloads import workload
    ap = argparse.ArgumentParser(description="crater run of the atomic-transport stage")
    ap.add_argument("--workload", default="crater")
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--every", type=int, default=10000)
    ap.add_argument("--fluence", type=float, default=None, help="J/cm^2 the start stands for (Eq. 5)")
    ap.add_argument("--beam-diameter", type=float, default=None, help="m (Eq. 5)")
    ap.add_argument("--calibrate", action="store_true",
                    help="run the altered potential with c_att calibrated on the initial slab")
    a = ap.parse_args()
    w = workload(a.workload)
    if a.calibrate:
        from . import Simulation
        probe = Simulation(w)
        cal = calibrate_c_att(probe)
        probe.close()
        print(json.dumps({"calibration": cal}), flush=True)
        w = dict(w, pot_mode=1, c_att=cal["c_att"], s_rep=1.0)
    for m in run_crater(w, a.steps or w["steps"], a.every, a.fluence, a.beam_diameter):
        print(json.dumps(m), flush=True)


def _cell_rule(order: int, levels: int):
    """Quadrature nodes and weights on [0, 1]: `order`-point Gauss-Legendre on subintervals that
    halve towards both ends (breakpoints 2^-j and 1 - 2^-j, j = 1..levels), so that features
    next to a cell edge are resolved."""
    t, wt = np.polynomial.legendre.leggauss(order)
    b = sorted({0.0, 1.0, *[2.0 ** -j for j in range(1, levels + 1)], *[1.0 - 2.0 ** -j for j in range(1, levels + 1)]})
    nodes, weights = [], []
    for a, c in zip(b[:-1], b[1:]):
        nodes.append(a + 0.5 * (c - a) * (t + 1.0))
        weights.append(0.5 * (c - a) * wt)
    return np.concatenate(nodes), np.concatenate(weights)


def calibrate_c_att(sim, z_from: int = None, z_to: int = None, order: int = 8, levels: int = 20) -> dict:
    """Attractive correction factor of the altered potential (paper: a multiplicative factor on the
    attractive force, found by integrating the force on a single atom that leaves the target and
    travels out to infinity). Probes cross the surface of the context's current slab along z on
    every column (x = i + 1/2), cell row by cell row from z_from to z_to (default slab_k - 1 to
    slab_k + 2, where the density has fallen to zero); the lateral mean of the z force of the
    attractive branch alone (c_att = 1, no repulsion) is integrated over each cell with
    `_cell_rule`. Where the density tail meets the vacuum, Eq. 2 puts the lower neighbour at
    rbar / (1 + g/2) -> 0: the attraction has a narrow spike there (resolved by the halving
    subintervals) and the repulsion diverges (not integrable, so it takes no part). Taking one atom
    out of the model's cubic lattice along the normal costs one bond, D (the first-order force of
    Eq. 2 integrates to exactly -D across a smooth surface), so c_att = -D / W_att."""
    nx, slab_k, dx = sim.nx, sim.cfg.slab_k, sim.cfg.dx
    k0 = max(slab_k - 1, 0) if z_from is None else int(z_from)
    k1 = min(slab_k + 2, sim.nz) if z_to is None else int(z_to)
    if not 0 <= k0 < k1 <= sim.nz:
        raise ValueError("probe rows must lie inside the grid")
    f_in, w_in = _cell_rule(order, levels)
    rows = np.arange(k0, k1)
    K, J, I = np.meshgrid(rows, np.arange(f_in.size), np.arange(nx), indexing="ij")
    cell = (K * nx + I).astype(np.int32).ravel()
    fx = np.full(cell.size, 0.5, np.float32)
    fz = f_in[J].astype(np.float32).ravel()
    f = sim.pair_force_at(cell, fx, fz, pot_mode=1, c_att=1.0, s_rep=0.0)[:, 2].cpu().numpy()
    fm = f.astype(np.float64).reshape(rows.size, f_in.size, nx).mean(axis=2)
    w_att = float((fm * w_in).sum() * dx)
    D = sim.cfg.D_eV * 1.602176634e-19
    return {"c_att": -D / w_att, "W_att": w_att, "D": D}


def transport_from_laser(laser, transport_phys: dict):
    """Second stage of the two-stage run (paper: the atomic-transport run starts from the lattice
    temperature the laser-interaction run leaves): a transport context whose atoms, drawn at the
    transport start temperature T_ion_K, are re-tempered to the ion temperature of `laser` cell by
    cell (cells the laser stage leaves colder or without ions keep T_ion_K). The transport grid may
    differ from the laser stage's (the paper's laser stage uses much finer cells): the temperature
    map is then remapped conservatively onto it, the grids placed on each other by the slab surface
    and the laser axis, with T_ion_K where the laser stage has no cells (regrid_cells)."""
    import torch

    from . import Simulation, regrid_cells
    dims = 3 if transport_phys.get("dims") == 3 else 2
    assert laser.dims == dims
    T_from = float(transport_phys["T_ion_K"])
    T = torch.clamp(laser.cell_temperature(0), min=T_from)
    tr = Simulation(transport_phys)
    if laser.cell_grid() != tr.cell_grid():
        T = regrid_cells(T, laser.cell_grid(), tr.cell_grid(), T_from, dims=dims)
        torch.cuda.current_stream().synchronize()
    tr.set_temperature(0, T, T_from)
    return tr


def laser_from_transport(transport, laser_phys: dict):
    """The next shot of a few-shot study (paper: the target structure a transport run leaves, as a
    density and temperature profile, initialises another laser-interaction run): a laser-stage
    context on the same grid whose ions are the transport stage's atoms (positions and lattice
    momenta) and whose electrons sit on the same positions (a neutral start) with the thermal
    momenta the new context drew for its own electrons. The two stages need the same particle
    count per species (same slab and ppc)."""
    import torch

    from . import Simulation
    las = Simulation(laser_phys)
    atoms = transport.get_particles(0)
    n = atoms["cell"].numel()
    if las.info()["num_particles"][1] != n:
        las.close()
        raise ValueError("the laser stage needs as many electrons as the transport stage has atoms")
    electrons = las.get_particles(1)
    fy = atoms.get("fy")
    las.set_particles(0, atoms["cell"], atoms["fx"], atoms["fz"], atoms["ux"], atoms["uy"], atoms["uz"], fy=fy)
    las.set_particles(1, atoms["cell"], atoms["fx"], atoms["fz"], electrons["ux"], electrons["uy"], electrons["uz"],
                      fy=fy)
    torch.cuda.synchronize()
    return las
