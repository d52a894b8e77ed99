"""Pins of the 3D section of the FP64 oracle (CPU only): exact integer invariants of the
deposition, closed forms of the Yee scheme, Gauss's law, and consistency with the 2D cycle."""
import math

import numpy as np
import pytest

import oracle
from paper_1502_07722_gb300.workloads import workload

C = 299792458.0
QE = 1.602176634e-19
EPS0 = 8.8541878128e-12
Q3 = 2 ** 14


def cfg3(**kw):
    w = workload("tiny", laser_profile=0)
    w.update(dict(ny=kw.pop("ny", 8)))
    w.update(kw)
    return w


def _moves(seed, nx, ny, nz, n):
    rng = np.random.default_rng(seed)
    g = lambda a: np.floor(a * Q3) / Q3
    x0 = g(rng.uniform(0, nx, n)); y0 = g(rng.uniform(0, ny, n)); z0 = g(rng.uniform(0, nz - 1e-6, n))
    d = rng.uniform(-0.95, 0.95, (3, n))
    d[:, : n // 5] = 0.0
    x1 = np.mod(g(x0 + d[0]), nx); y1 = np.mod(g(y0 + d[1]), ny)
    z1 = z0 + d[2]
    z1 = np.where(z1 < 0, -z1, z1)
    z1 = np.where(z1 >= nz, 2 * nz - z1 - 1e-6, z1)
    return x0, y0, z0, x1, y1, g(z1)


def test_density3_weight_and_moments():
    nx, ny, nz = 10, 7, 9
    rng = np.random.default_rng(1)
    n = 3000
    x = np.floor(rng.uniform(0, nx, n) * Q3) / Q3
    y = np.floor(rng.uniform(0, ny, n) * Q3) / Q3
    z = np.floor(rng.uniform(0, nz, n) * Q3) / Q3
    rho = oracle.deposit_density3(nx, ny, nz, x, y, z)
    assert rho.sum() == n * 2 ** 42
    k = np.arange(nz + 1, dtype=np.int64)[:, None, None]
    assert int((rho * k).sum()) == int(np.rint(z * Q3).astype(np.int64).sum()) * 2 ** 28
    # one particle at a cell centre: 1/8 of its weight on each corner
    r1 = oracle.deposit_density3(nx, ny, nz, [3.5], [2.5], [4.5])
    assert (r1[4:6, 2:4, 3:5] == 2 ** 39).all() and r1.sum() == 2 ** 42


def test_current3_continuity_and_dipole():
    """6 (rho1 - rho0) + div(J6) = 0 exactly at every node (across seams and walls), and
    sum J6x = 6 Q^2 dX for each particle."""
    nx, ny, nz = 8, 6, 7
    x0, y0, z0, x1, y1, z1 = _moves(3, nx, ny, nz, 1500)
    J = oracle.deposit_current3(nx, ny, nz, 1, x0, y0, z0, x1, y1, z1)
    r0 = oracle.deposit_density3(nx, ny, nz, x0, y0, z0)
    r1 = oracle.deposit_density3(nx, ny, nz, x1, y1, z1)
    div = (J[0] - np.roll(J[0], 1, axis=2)) + (J[1] - np.roll(J[1], 1, axis=1))
    div[0:nz] += J[2][0:nz]
    div[1:nz + 1] -= J[2][0:nz]
    assert np.array_equal(6 * (r1 - r0) + div, np.zeros_like(div))
    for p in range(0, 1500, 97):
        Jp = oracle.deposit_current3(nx, ny, nz, 1, x0[p:p + 1], y0[p:p + 1], z0[p:p + 1], x1[p:p + 1],
                                     y1[p:p + 1], z1[p:p + 1])
        P = nx * Q3
        dX = (round(x1[p] * Q3) - round(x0[p] * Q3) + P // 2) % P - P // 2
        dZ = round(z1[p] * Q3) - round(z0[p] * Q3)
        assert int(Jp[0].sum()) == 6 * Q3 * Q3 * dX
        assert int(Jp[2].sum()) == 6 * Q3 * Q3 * dZ


@pytest.mark.parametrize("pot", [{}, {"pot_mode": 2, "morse_a": 4.0}, {"lattice": 1}], ids=["lj", "morse", "hcp"])
def test_uniform_lattice3_zero_force_and_energy(pot):
    """Identical offsets in every cell of a full-height slab: uniform node density, zero force,
    and -3 D per atom at the equilibrium density (six neighbours at r0; both potentials have their
    minimum -D there)."""
    nx, ny, nz = 6, 5, 6
    w = cfg3(nx=nx, ny=ny, nz=nz, slab_k=nz, ppc_ion=2, ppc_electron=2, **pot)
    o = oracle.Oracle3D(w, with_particles=False)
    cells = np.arange(nx * ny * nz)
    i, j, k = cells % nx, (cells // nx) % ny, cells // (nx * ny)
    x = np.concatenate([i + 0.25, i + 0.75])
    y = np.concatenate([j + 0.5, j + 0.5])
    z = np.concatenate([k + 0.5, k + 0.5])
    n = len(x)
    o.set_particles(0, x, y, z, np.zeros(n), np.zeros(n), np.zeros(n))
    F = o.pair_force()
    assert (not F.any()) if not pot.get("lattice") else np.abs(F).max() < 1e-25   # HCP: directions' rounding
    D = 0.41 * QE
    bonds = 12 if pot.get("lattice") == 1 else 6
    assert o.energy()["pair"] == pytest.approx(-bonds / 2 * D * n * o.weight, rel=1e-12)


@pytest.mark.parametrize("pot", [{}, {"pot_mode": 2, "morse_a": 4.0}, {"lattice": 1}, {"pot_mode": 3}],
                         ids=["lj", "morse", "hcp", "eam"])
def test_pair_force_3d_equals_2d_on_y_uniform_state(pot):
    """The 2D method is the 3D method on a state that does not vary along y: same x and z forces
    (the y force vanishes), for either pair potential, the HCP geometry and the embedded-atom form
    (whose 2D form puts the +-y neighbours at rbar with their own density n)."""
    nx, nz, ny = 12, 10, 4
    rng = np.random.default_rng(5)
    ncell = nx * 5
    cells = np.repeat(np.arange(ncell), 4)
    xs = cells % nx + np.floor(rng.random(len(cells)) * Q3) / Q3
    zs = cells // nx + np.floor(rng.random(len(cells)) * 0.8 * Q3) / Q3
    w2 = workload("tiny", nx=nx, nz=nz, slab_k=5, ppc_ion=4, ppc_electron=4, laser_profile=0, **pot)
    o2 = oracle.Oracle(w2, with_particles=False)
    n = len(xs)
    o2.set_particles(0, xs, zs, np.zeros(n), np.zeros(n), np.zeros(n))
    F2 = o2.pair_force()
    w3 = cfg3(nx=nx, ny=ny, nz=nz, slab_k=5, ppc_ion=4, ppc_electron=4, **pot)
    o3 = oracle.Oracle3D(w3, with_particles=False)
    X = np.tile(xs, ny)
    Y = np.repeat(np.arange(ny) + 0.5, n)
    Z = np.tile(zs, ny)
    o3.set_particles(0, X, Y, Z, np.zeros(n * ny), np.zeros(n * ny), np.zeros(n * ny))
    F3 = o3.pair_force()[:n]
    np.testing.assert_allclose(F3[:, 0], F2[:, 0], rtol=1e-12, atol=1e-12 * np.abs(F2).max())
    np.testing.assert_allclose(F3[:, 2], F2[:, 2], rtol=1e-12, atol=1e-12 * np.abs(F2).max())
    assert np.abs(F3[:, 1]).max() <= 1e-12 * np.abs(F2).max()


@pytest.mark.parametrize("axis", ["x", "y"])
def test_yee3_dispersion(axis):
    """A Fourier mode obeys E^(n+1) + E^(n-1) = 2 cos(w dt) E^n with
    sin(w dt/2) = (c dt/dx) sin(k dx/2) (3D time step)."""
    nx, ny, nz = 12, 12, 8
    w = cfg3(nx=nx, ny=ny, nz=nz, slab_k=0)
    o = oracle.Oracle3D(w, with_particles=False)
    kk = 2 * math.pi * 2 / 12
    a = C * o.dt / w["dx"]
    two_cos = 2 - 4 * a * a * math.sin(kk / 2) ** 2
    shape = (nz + 1, ny, nx)
    zz, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx), indexing="ij")
    if axis == "x":
        o.set_field(2, np.cos(kk * ii))                      # Ez(i, j, k+1/2)
        o.set_field(4, 0.2 / C * np.sin(kk * (ii + 0.5)))    # By(i+1/2, j, k+1/2)
    else:
        o.set_field(2, np.cos(kk * jj))                      # Ez
        o.set_field(3, -0.2 / C * np.sin(kk * (jj + 0.5)))   # Bx(i, j+1/2, k+1/2)
    e0 = o.get_field(2)
    o.step(1)
    e1 = o.get_field(2)
    o.step(1)
    e2 = o.get_field(2)
    np.testing.assert_allclose((e2 + e0)[:nz], (two_cos * e1)[:nz], atol=1e-12)
    assert e0.shape == shape


def test_gauss3_preserved():
    w = cfg3(nx=8, ny=6, nz=12, slab_k=6, ppc_ion=2, ppc_electron=2, T_electron_eV=50.0, laser_profile=1,
             I0=1e19, t_peak=10 * 1.8e-17)
    o = oracle.Oracle3D(w)
    o.step(25)
    ions, els = o.get_particles(0), o.get_particles(1)
    nx, ny, nz, dx = 8, 6, 12, w["dx"]
    rq = (oracle.deposit_density3(nx, ny, nz, ions["x"], ions["y"], ions["z"]) -
          oracle.deposit_density3(nx, ny, nz, els["x"], els["y"], els["z"]))
    rho = rq * QE * o.weight / (2 ** 42 * dx ** 3)
    Ex, Ey, Ez = o.get_field(0), o.get_field(1), o.get_field(2)
    div = (Ex - np.roll(Ex, 1, axis=2)) / dx + (Ey - np.roll(Ey, 1, axis=1)) / dx
    div[1:nz] += (Ez[1:nz] - Ez[0:nz - 1]) / dx
    scale = np.abs(rho[1:nz] / EPS0).max()
    assert scale > 0
    np.testing.assert_allclose(div[1:nz], rho[1:nz] / EPS0, atol=1e-9 * scale)


def test_init3_statistics():
    w = cfg3(nx=6, ny=5, nz=8, slab_k=4, ppc_ion=8, ppc_electron=8)
    o = oracle.Oracle3D(w)
    ions, els = o.get_particles(0), o.get_particles(1)
    assert len(ions["x"]) == 6 * 5 * 4 * 8
    for key in ("x", "y", "z"):
        assert np.array_equal(ions[key], els[key])
    cell = (np.floor(ions["z"]) * 5 + np.floor(ions["y"])) * 6 + np.floor(ions["x"])
    assert np.array_equal(np.bincount(cell.astype(int), minlength=120), np.full(120, 8))
    assert o.get_rho().sum() == len(ions["x"]) * 2 ** 42


# Yee positions of the 3D field components (offsets along x, y, z) and whether they live on the nz
# half planes (True) or on the nz + 1 node planes
STAGGER_3D = [(0.5, 0.0, 0.0, False), (0.0, 0.5, 0.0, False), (0.0, 0.0, 0.5, True),   # Ex Ey Ez
              (0.0, 0.5, 0.5, True), (0.5, 0.0, 0.5, True), (0.5, 0.5, 0.0, False)]    # Bx By Bz


def test_field_gather3_reproduces_linear_fields():
    """3D fields seen by the push: each Yee component set to its own linear function
    a + b x + c y + d z at its staggered positions is returned exactly at interior points (a wrong
    half-cell offset along any axis is off by half a slope); near a wall a half-plane component
    returns its edge plane's value (z clamped to [1/2, nz - 1/2])."""
    nx, ny, nz = 12, 10, 9
    o = oracle.Oracle3D(cfg3(nx=nx, ny=ny, nz=nz, slab_k=nz, dims=3), with_particles=False)
    k, j, i = np.mgrid[0:nz + 1, 0:ny, 0:nx]
    rng = np.random.default_rng(6)
    coef = rng.uniform(1.0, 3.0, (6, 4)) * np.array([1.0, 0.1, 0.15, 0.2])
    for f, (sx, sy, sz, half) in enumerate(STAGGER_3D):
        a, b, c, d = coef[f]
        grid = a + b * (i + sx) + c * (j + sy) + d * (k + sz)
        if half:
            grid[nz] = 0.0
        o.set_field(f, grid)
    pts = [(rng.uniform(1.0, nx - 2.0), rng.uniform(1.0, ny - 2.0), rng.uniform(0.0, nz)) for _ in range(60)]
    pts += [(rng.uniform(1.0, nx - 2.0), rng.uniform(1.0, ny - 2.0), z) for z in (0.0, 0.3, 0.5, nz - 0.5, nz - 0.2)]
    for x, y, z in pts:
        got = o.gather_fields(x, y, z)
        for f, (sx, sy, sz, half) in enumerate(STAGGER_3D):
            a, b, c, d = coef[f]
            zc = min(max(z, 0.5), nz - 0.5) if half else z
            assert got[f] == pytest.approx(a + b * x + c * y + d * zc, rel=1e-13, abs=1e-13), (f, x, y, z)
