"""Parity of the 3D CUDA path with the 3D FP64 oracle (through the C ABI)."""
import numpy as np
import pytest

import oracle
from paper_1502_07722_gb300.workloads import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
Q3 = 2 ** 14


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1502_07722_gb300 import _build
    _build.build()
    oracle.build()
    import paper_1502_07722_gb300 as m
    return m


def w3(**kw):
    base = dict(workload("tiny"), dims=3, ny=12, nx=14, nz=16, slab_k=8, ppc_ion=4, ppc_electron=4, tile=4,
                laser_profile=1, I0=1e19, t_peak=5 * 1.83e-17)
    base.update(kw)
    return base


def to_global3(p, nx, ny):
    cell = p["cell"].cpu().numpy().astype(np.int64)
    i, j, k = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    f = lambda key: p[key].cpu().numpy().astype(np.float64)
    return i + f("fx"), j + f("fy"), k + f("fz"), [f("ux"), f("uy"), f("uz")]


def set_both3(sim, orc, sp, x, y, z, u):
    i, j, k = np.floor(x).astype(np.int64), np.floor(y).astype(np.int64), np.floor(z).astype(np.int64)
    cell = ((k * sim.ny + j) * sim.nx + i).astype(np.int32)
    sim.set_particles(sp, cell, (x - i).astype(np.float32), (z - k).astype(np.float32), *u,
                      fy=(y - j).astype(np.float32))
    g = sim.get_particles(sp)
    X, Y, Z, U = to_global3(g, sim.nx, sim.ny)
    orc.set_particles(sp, X, Y, Z, *U)
    return g


def random_state(seed, nx, ny, nz, slab, n, spread):
    rng = np.random.default_rng(seed)
    g = lambda a: np.floor(a * (1 << 24)) / (1 << 24)
    x = g(rng.uniform(0, nx, n)) % nx
    y = g(rng.uniform(0, ny, n)) % ny
    z = g(rng.uniform(0, slab, n))
    sel = rng.random(n) < 0.3
    x[sel] = np.floor(x[sel]) + g(rng.random(sel.sum()) * 0.3)
    u = [rng.normal(0, spread, n).astype(np.float32).astype(np.float64) for _ in range(3)]
    return x, y, z, u


def test_init3_matches_oracle(gb):
    w = w3()
    sim = gb.Simulation(w)
    orc = oracle.Oracle3D(w)
    for sp in (0, 1):
        X, Y, Z, U = to_global3(sim.get_particles(sp), w["nx"], w["ny"])
        o = orc.get_particles(sp)
        kg, ko = np.lexsort((Z, Y, X)), np.lexsort((o["z"], o["y"], o["x"]))
        assert np.array_equal(X[kg], o["x"][ko]) and np.array_equal(Y[kg], o["y"][ko])
        assert np.array_equal(Z[kg], o["z"][ko])
        np.testing.assert_allclose(U[0][kg], o["ux"][ko], rtol=1e-6, atol=1e-7 * np.abs(o["ux"]).max())
    assert np.array_equal(sim.get_density().cpu().numpy(), orc.get_rho())


@pytest.mark.parametrize("pot", [{}, dict(pot_mode=2, morse_a=4.0), dict(lattice=1), dict(pot_mode=3)],
                         ids=["lj", "morse", "hcp", "eam"])
def test_density3_and_pair_force(gb, pot):
    w = w3(max_particles=6000, **pot)
    sim = gb.Simulation(w)
    orc = oracle.Oracle3D(w, with_particles=False)
    x, y, z, u = random_state(1, 14, 12, 16, 8, 3000, 1e-4)
    set_both3(sim, orc, 0, x, y, z, u)
    out, _ = sim.deposit_density()
    assert np.array_equal(out.cpu().numpy(), orc.get_rho())
    assert out.sum().item() == 3000 * 2 ** 42
    Fg = sim.pair_force().cpu().numpy().astype(np.float64)
    Fo = orc.pair_force()
    scale = np.abs(Fo).max()
    assert scale > 0
    assert (np.abs(Fg - Fo) <= 1e-5 * np.abs(Fo) + 1e-5 * scale).all()


@pytest.mark.parametrize("seed,tile,pot", [(3, 4, {}), (4, 4, {}), (5, 10, {}), (6, 16, {}),
                                           (7, 10, dict(pot_mode=2, morse_a=4.0)), (8, 10, dict(lattice=1)),
                                           (9, 10, dict(pot_mode=3))],
                         ids=["t4a", "t4b", "t10", "t16", "t10-morse", "t10-hcp", "t10-eam"])
def test_one_step3_full(gb, seed, tile, pot):
    """One 3D cycle: particles to 1e-5, current and node density bit-exact against the oracle's
    deposition of the GPU's own move, fields against the oracle's Maxwell update. Tile 4: several
    tiles with staged windows; tile 10: ragged tiles (14 x 12 x 16 cells) and the kernel instances
    with the window edge compiled in, for every potential and lattice variant; tile 16: the window
    is too large to stage, every gather and deposit takes the global path."""
    nx, ny, nz = 14, 12, 16
    w = w3(max_particles=6000, sort_every=0, tile=tile, **pot)
    sim = gb.Simulation(w)
    orc = oracle.Oracle3D(w, with_particles=False)
    g0 = []
    for sp, spread in ((0, 2e-4), (1, 3e-3)):
        x, y, z, u = random_state(seed * 10 + sp, nx, ny, nz, 8, 4000, spread)
        g0.append(set_both3(sim, orc, sp, x, y, z, u))
    rng = np.random.default_rng(seed)
    fields = [rng.normal(0, 3e9 if f < 3 else 10.0, (nz + 1, ny, nx)).astype(np.float32).astype(np.float64)
              for f in range(6)]
    for f in range(6):
        sim.set_field(f, fields[f])
        orc.set_field(f, fields[f])
    sim.step(1)
    orc.step(1)
    J = np.zeros((3, nz + 1, ny, nx), np.int64)
    for sp, sign in ((0, 1), (1, -1)):
        g1 = sim.get_particles(sp)
        X1, Y1, Z1, U1 = to_global3(g1, nx, ny)
        X0, Y0, Z0, _ = to_global3(g0[sp], nx, ny)
        o = orc.get_particles(sp)
        for a, b, a0 in ((X1, o["x"], X0), (Y1, o["y"], Y0)):
            d = np.abs(np.mod(a - b + nx / 2, nx) - nx / 2)
            disp = np.abs(np.mod(b - a0 + nx / 2, nx) - nx / 2)
            assert (d <= 1e-5 * disp + 2.0 ** -22).all()
        assert (np.abs(Z1 - o["z"]) <= 1e-5 * np.abs(o["z"] - Z0) + 2.0 ** -22).all()
        for c, key in enumerate(("ux", "uy", "uz")):
            np.testing.assert_allclose(U1[c], o[key], rtol=1e-5, atol=1e-6 * np.abs(o[key]).max())
        oracle.deposit_current3(nx, ny, nz, sign, X0, Y0, Z0, X1, Y1, Z1, out=J)
    assert np.array_equal(sim.get_current().cpu().numpy(), J)
    X1, Y1, Z1, _ = to_global3(sim.get_particles(0), nx, ny)
    assert np.array_equal(sim.get_density().cpu().numpy(), oracle.deposit_density3(nx, ny, nz, X1, Y1, Z1))
    fo = oracle.Oracle3D(w, with_particles=False)
    for f in range(6):
        fo.set_field(f, fields[f])
    fo.set_current(J)
    fo.maxwell()
    for f in range(6):
        a = sim.get_field(f).cpu().numpy().astype(np.float64)
        b = fo.get_field(f)
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())


@pytest.mark.parametrize("pot", [dict(pot_mode=2, morse_a=4.0), dict(lattice=1), dict(pot_mode=3)],
                         ids=["morse", "hcp", "eam"])
def test_one_step3_transport_variants_compiled_window(gb, pot):
    """One 3D transport step of each potential and lattice variant with 10-cell tiles, the kernel
    instances that have the 13-node window edge compiled in (ragged tiles: 14 x 12 x 16 cells):
    atoms to 1e-5 of the oracle and the node density bit-exact against the oracle's deposit of the
    GPU's own move."""
    nx, ny, nz = 14, 12, 16
    w = w3(max_particles=6000, sort_every=0, tile=10, mode=1, ion_charge=0.0, ppc_electron=0, laser_profile=0,
           dt_override=12e-15, T_ion_K=3000.0, **pot)
    sim = gb.Simulation(w)
    orc = oracle.Oracle3D(w, with_particles=False)
    # the workload's own start (lattice slab at 3000 K), handed to the oracle as it stands
    x, y, z, u = to_global3(sim.get_particles(0), nx, ny)
    g0 = set_both3(sim, orc, 0, x, y, z, u)
    sim.step(1)
    orc.step(1)
    X1, Y1, Z1, U1 = to_global3(sim.get_particles(0), nx, ny)
    X0, Y0, Z0, _ = to_global3(g0, nx, ny)
    o = orc.get_particles(0)
    for a, b, a0 in ((X1, o["x"], X0), (Y1, o["y"], Y0)):
        d = np.abs(np.mod(a - b + nx / 2, nx) - nx / 2)
        disp = np.abs(np.mod(b - a0 + nx / 2, nx) - nx / 2)
        assert (d <= 1e-5 * disp + 2.0 ** -22).all()
    assert (np.abs(Z1 - o["z"]) <= 1e-5 * np.abs(o["z"] - Z0) + 2.0 ** -22).all()
    for c, key in enumerate(("ux", "uy", "uz")):
        np.testing.assert_allclose(U1[c], o[key], rtol=1e-5, atol=1e-5 * np.abs(o[key]).max())
    assert np.array_equal(sim.get_density().cpu().numpy(), oracle.deposit_density3(nx, ny, nz, X1, Y1, Z1))


def test_energy3_matches_oracle(gb):
    w = w3()
    sim = gb.Simulation(w)
    orc = oracle.Oracle3D(w)
    sim.step(3)
    orc.step(3)
    eg, eo = sim.energy(), orc.energy()
    stored = ("kinetic_ion", "kinetic_electron", "field_E", "field_B", "pair")
    tg = sum(eg[k] for k in stored)
    to = sum(eo[k] for k in stored)
    assert tg == pytest.approx(to, rel=1e-3)
    assert eg["injected"] == pytest.approx(eo["injected"], rel=1e-4, abs=1e-6 * abs(eo["field_E"]))
    assert eg["pair"] == pytest.approx(eo["pair"], rel=1e-3)
    assert eg["kinetic_electron"] == pytest.approx(eo["kinetic_electron"], rel=1e-3)


@pytest.mark.parametrize("pot", [{}, dict(pot_mode=2, morse_a=4.0), dict(lattice=1), dict(pot_mode=3)],
                         ids=["lj", "morse", "hcp", "eam"])
def test_transport3_steps(gb, pot):
    w = w3(mode=1, ion_charge=0.0, ppc_electron=0, laser_profile=0, dt_override=12e-15, T_ion_K=3000.0, **pot)
    sim = gb.Simulation(w)
    orc = oracle.Oracle3D(w)
    sim.step(20)
    orc.step(20)
    pg = sim.get_density().cpu().numpy().sum(axis=(1, 2)).astype(np.float64)
    po = orc.get_rho().sum(axis=(1, 2)).astype(np.float64)
    assert np.linalg.norm(pg - po) / np.linalg.norm(po) < 1e-3
    eg, eo = sim.energy(), orc.energy()
    assert eg["kinetic_ion"] + eg["pair"] == pytest.approx(eo["kinetic_ion"] + eo["pair"], rel=1e-3)


@pytest.mark.parametrize("profile", [1, 2])
def test_vacuum3_antenna_matches_oracle(gb, profile):
    """No particles; the 3D antenna (plane wave, or the round focused Gaussian beam: width,
    wavefront curvature, amplitude w0/w and the full Gouy phase at the antenna, focus at row
    slab_k) drives the 3D Yee scheme. Fields after one step and after 150 steps agree with the
    oracle to 1e-5 of the largest E (for E components) or B (for B components) component."""
    w = w3(nx=24, ny=20, nz=40, slab_k=10, ppc_ion=0, ppc_electron=0, laser_profile=profile, w0=0.06e-6,
           I0=1e17, tau_fwhm=2e-15, t_peak=3e-15, tile=8, **{"lambda": 200e-9})
    sim = gb.Simulation(w)
    assert sum(sim.info()["num_particles"]) == 0
    orc = oracle.Oracle3D(w, with_particles=False)
    for nsteps in (1, 149):
        sim.step(nsteps)
        orc.step(nsteps)
        o = [orc.get_field(f) for f in range(6)]
        for f in range(6):
            g = sim.get_field(f).cpu().numpy().reshape(o[f].shape)
            # a component that symmetry keeps at zero (Bx of an x-polarised round beam) carries the
            # FP32 rounding of the others: the scale is the largest E (or B) component
            scale = max(np.abs(o[q]).max() for q in (range(3) if f < 3 else range(3, 6)))
            assert np.abs(g - o[f]).max() <= 1e-5 * scale, (nsteps, f)
    sim.close()


def test_electric_gather3_reproduces_linear_fields(gb):
    """The 3D E gather against a closed form: Ex, Ey, Ez set to their own linear functions at
    their own Yee positions, B = 0, electrons at rest stepped once with dt = 1e-21 s. Then
    u = q dt E / (m c) at the particle, E the linear function there (a half-cell offset along any
    axis is off by half a slope); the half-plane Ez takes its edge plane next to the walls."""
    C, QE, ME = 299792458.0, 1.602176634e-19, 9.1093837015e-31
    nx, ny, nz = 24, 20, 16
    w = w3(nx=nx, ny=ny, nz=nz, slab_k=nz, ppc_ion=1, ppc_electron=1, tile=6, dt_override=1e-21, laser_profile=0,
           max_particles=8000)
    sim = gb.Simulation(w, sort_every=0)
    rng = np.random.default_rng(12)
    n = 3000
    g = lambda a: np.floor(a * 2 ** 20) / 2 ** 20
    x = g(rng.uniform(1.0, nx - 2.0, n))
    y = g(rng.uniform(1.0, ny - 2.0, n))
    z = np.minimum(g(np.concatenate([rng.uniform(0.0, nz, n - 200), rng.uniform(0.0, 0.5, 100),
                                    rng.uniform(nz - 0.5, nz, 100)])), nz - 2 ** -20)
    i0, j0, k0 = np.floor(x).astype(np.int64), np.floor(y).astype(np.int64), np.floor(z).astype(np.int64)
    cell = ((k0 * ny + j0) * nx + i0).astype(np.int32)
    zero = np.zeros(n, np.float32)
    sim.set_particles(1, cell, (x - i0).astype(np.float32), (z - k0).astype(np.float32), zero, zero, zero,
                      fy=(y - j0).astype(np.float32))
    sim.set_particles(0, cell[:0], zero[:0], zero[:0], zero[:0], zero[:0], zero[:0], fy=zero[:0])
    k, j, i = np.mgrid[0:nz + 1, 0:ny, 0:nx]
    coef = {0: (3e5, 1e5, -2e5), 1: (-2e5, 4e5, 1e5), 2: (1e5, -1e5, 3e5)}        # slopes along x, y, z
    stag = {0: (0.5, 0.0, 0.0, False), 1: (0.0, 0.5, 0.0, False), 2: (0.0, 0.0, 0.5, True)}
    for f in range(6):
        grid = np.zeros((nz + 1, ny, nx))
        if f in coef:
            (b, c, d), (sx, sy, sz, half) = coef[f], stag[f]
            grid = b * (i + sx) + c * (j + sy) + d * (k + sz)
            if half:
                grid[nz] = 0.0
        sim.set_field(f, grid.astype(np.float32))
    X, Y, Z, _ = to_global3(sim.get_particles(1), nx, ny)
    sim.step(1)
    p1 = sim.get_particles(1)
    scale = QE * w["dt_override"] / (ME * C)
    for f in range(3):
        (b, c, d), (sx, sy, sz, half) = coef[f], stag[f]
        zc = np.clip(Z, 0.5, nz - 0.5) if half else Z
        expect = -(b * X + c * Y + d * zc)
        got = p1[("ux", "uy", "uz")[f]].cpu().numpy().astype(np.float64) / scale
        np.testing.assert_allclose(got, expect, rtol=1e-5, atol=1e-5 * np.abs(expect).max())
    sim.close()
