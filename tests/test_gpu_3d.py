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


@pytest.mark.parametrize("pot", [{}, dict(pot_mode=2, morse_a=4.0), dict(lattice=1)], ids=["lj", "morse", "hcp"])
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


@pytest.mark.parametrize("seed,tile", [(3, 4), (4, 4), (5, 10), (6, 16)])
def test_one_step3_full(gb, seed, tile):
    """One 3D cycle: particles to 1e-5, current and node density bit-exact against the oracle's
    deposition of the GPU's own move, fields against the oracle's Maxwell update. Tile 4: several
    tiles with staged windows; tile 10: ragged tiles (14 x 12 x 16 cells); tile 16: the window is
    too large to stage, every gather and deposit takes the global path."""
    nx, ny, nz = 14, 12, 16
    w = w3(max_particles=6000, sort_every=0, tile=tile)
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


@pytest.mark.parametrize("pot", [{}, dict(pot_mode=2, morse_a=4.0), dict(lattice=1)], ids=["lj", "morse", "hcp"])
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
