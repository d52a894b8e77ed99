"""Seeded synthetic inputs shared by the oracle and the CUDA path in the tests.

This module only draws numbers (positions, momenta, grids); it holds none of the method's
arithmetic. Positions are global cell coordinates, representable in FP32 as an integer cell
plus an FP32 offset so that both sides see bit-identical inputs.
"""
from __future__ import annotations

import numpy as np


def f32_offsets(rng, n):
    """Offsets in [0, 1) with 24 random bits (exact in FP32)."""
    return (rng.integers(0, 1 << 24, size=n) / float(1 << 24)).astype(np.float64)


def slab_particles(seed, nx, nz, slab_k, ppc, u_spread, clump=0.0):
    """ppc particles per cell in rows k < slab_k, uniform offsets, Gaussian momenta.

    clump > 0 moves that fraction of the particles of every cell towards the cell's lower-left
    corner (a density perturbation, for non-zero pair forces)."""
    rng = np.random.default_rng(seed)
    ncell = nx * slab_k
    n = ncell * ppc
    cell = np.repeat(np.arange(ncell), ppc)
    i = cell % nx
    k = cell // nx
    fx = f32_offsets(rng, n)
    fz = f32_offsets(rng, n)
    if clump > 0:
        sel = rng.random(n) < clump
        fx[sel] = np.floor(fx[sel] * 0.3 * (1 << 24)) / (1 << 24)
        fz[sel] = np.floor(fz[sel] * 0.3 * (1 << 24)) / (1 << 24)
    x = i + fx
    z = k + fz
    u = rng.normal(0.0, u_spread, size=(3, n))
    return dict(x=x, z=z, ux=u[0].astype(np.float32).astype(np.float64),
                uy=u[1].astype(np.float32).astype(np.float64), uz=u[2].astype(np.float32).astype(np.float64))


def edge_particles(seed, nx, nz, n, u_spread):
    """Particles on and next to the special places: the periodic seam (x near 0 and nx),
    the walls (z near 0 and nz), exact nodes and exact cell centres."""
    rng = np.random.default_rng(seed)
    eps = 1.0 / (1 << 20)
    xs = np.concatenate([
        rng.uniform(0, eps * 8, n // 8), nx - rng.uniform(eps, eps * 8, n // 8),
        rng.integers(0, nx, n // 8).astype(np.float64),
        rng.integers(0, nx, n // 8) + 0.5,
        rng.uniform(0, nx, n - 4 * (n // 8)),
    ])
    zs = np.concatenate([
        rng.uniform(0, eps * 8, n // 8), nz - rng.uniform(eps, eps * 8, n // 8),
        rng.integers(0, nz, n // 8).astype(np.float64),
        rng.integers(0, nz, n // 8) + 0.5,
        rng.uniform(0, nz, n - 4 * (n // 8)),
    ])
    rng.shuffle(zs)
    # snap to the FP32 cell + offset grid
    xs = np.floor(xs) + np.floor((xs - np.floor(xs)) * (1 << 24)) / (1 << 24)
    zs = np.floor(zs) + np.floor((zs - np.floor(zs)) * (1 << 24)) / (1 << 24)
    xs = np.mod(xs, nx)
    zs = np.clip(zs, 0, nz - 1.0 / (1 << 24))
    u = rng.normal(0.0, u_spread, size=(3, n)).astype(np.float32).astype(np.float64)
    return dict(x=xs, z=zs, ux=u[0], uy=u[1], uz=u[2])


def random_fields(seed, nx, nz, scale_E, scale_B):
    rng = np.random.default_rng(seed)
    E = [rng.normal(0, scale_E, (nz + 1, nx)).astype(np.float32).astype(np.float64) for _ in range(3)]
    B = [rng.normal(0, scale_B, (nz + 1, nx)).astype(np.float32).astype(np.float64) for _ in range(3)]
    return E + B
