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


def far_field_level(profile) -> float:
    """Surface level far from the crater: the median of the profile over the half of the columns
    farthest (periodic distance) from the deepest column. The whole slab of the model relaxes (its
    density settles slightly below the start density, so material leaves the original rows
    everywhere); the crater is the loss beyond that level."""
    d = np.asarray(profile, dtype=np.float64).ravel()
    n = d.size
    dist = np.abs((np.arange(n) - int(np.argmax(d)) + n // 2) % n - n // 2)
    far = np.argsort(dist, kind="stable")[n - n // 2:]
    return float(np.median(d[far])) if far.size else 0.0


def crater_metrics(profile, dx: float, threshold: float = None, far_field: bool = False) -> dict:
    """depth (m, the deepest column), width (m), left / right crossings (m). threshold: missing
    material that counts as crater (default half a cell). far_field: measure from the far-field
    surface level (`far_field_level`, returned as "level") instead of the original surface."""
    d = np.asarray(profile, dtype=np.float64).ravel()
    level = far_field_level(d) if far_field else 0.0
    d = d - level
    th = 0.5 * dx if threshold is None else float(threshold)
    n = len(d)
    i0 = int(np.argmax(d))
    depth = float(d[i0])
    if depth <= th:
        return {"depth": depth, "width": 0.0, "left": None, "right": None, "level": level}
    if (d > th).all():                       # no edge: the whole surface is below the threshold
        return {"depth": depth, "width": n * dx, "left": None, "right": None, "level": level}
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
    return {"depth": depth, "width": (right - left) * dx, "left": left * dx, "right": right * dx, "level": level}


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
    a = ap.parse_args()
    w = workload(a.workload)
    for m in run_crater(w, a.steps or w["steps"], a.every, a.fluence, a.beam_diameter):
        print(json.dumps(m), flush=True)
