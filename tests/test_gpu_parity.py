"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Node density and current are compared bit for bit (exact integer sums of the same fixed-point
inputs). Floating-point state is compared within the tolerances of the FP32 arithmetic:
1e-5 relative for single-step particle and field state, with an absolute floor where a value is
a difference of nearly equal terms (stated per test).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1502_07722_gb300.workloads import workload
from tests import inputs
from tests.sort_layout import cell_key, undo_layout

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

C = 299792458.0
QE = 1.602176634e-19
ME = 9.1093837015e-31


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1502_07722_gb300 import _build
    _build.build()
    oracle.build()


def gb():
    import paper_1502_07722_gb300 as m
    return m


def to_global(p, nx):
    cell = p["cell"].cpu().numpy().astype(np.int64)
    x = (cell % nx) + p["fx"].cpu().numpy().astype(np.float64)
    z = (cell // nx) + p["fz"].cpu().numpy().astype(np.float64)
    u = [p[k].cpu().numpy().astype(np.float64) for k in ("ux", "uy", "uz")]
    return x, z, u


def from_global(x, z, nx):
    i = np.floor(x).astype(np.int64)
    k = np.floor(z).astype(np.int64)
    fx = (x - i).astype(np.float32)
    fz = (z - k).astype(np.float32)
    return (k * nx + i).astype(np.int32), fx, fz


def set_both(sim, orc, sp, d):
    cell, fx, fz = from_global(d["x"], d["z"], sim.nx)
    sim.set_particles(sp, cell, fx, fz, d["ux"], d["uy"], d["uz"])
    g = sim.get_particles(sp)                     # the context's (sorted) order
    x, z, u = to_global(g, sim.nx)
    orc.set_particles(sp, x, z, *u)
    return g


# ---------------------------------------------------------------------------------------------

def test_initial_state_matches_oracle():
    """Same seed: the same slab (positions bit-exact, momenta to FP32 rounding) and the same
    node density."""
    w = workload("tiny", nx=40, nz=36, slab_k=18)
    sim = gb().Simulation(w)
    orc = oracle.Oracle(w)
    for sp in (0, 1):
        g = sim.get_particles(sp)
        x, z, u = to_global(g, w["nx"])
        o = orc.get_particles(sp)
        kg = np.lexsort((z, x))
        ko = np.lexsort((o["z"], o["x"]))
        assert np.array_equal(x[kg], o["x"][ko]) and np.array_equal(z[kg], o["z"][ko])
        for c, comp in enumerate(("ux", "uy", "uz")):
            np.testing.assert_allclose(u[c][kg], o[comp][ko], rtol=1e-6, atol=1e-7 * np.abs(o[comp]).max())
    assert np.array_equal(sim.get_density().cpu().numpy(), orc.get_rho())


@pytest.mark.parametrize("shape", [(70, 52, 16), (33, 20, 8), (64, 64, 32)])
def test_deposit_density_bit_exact(shape):
    """Node density of random and edge-placed particles (seam, walls, exact nodes), on grids
    with ragged tiles: identical int64 sums."""
    nx, nz, T = shape
    w = workload("tiny", nx=nx, nz=nz, slab_k=nz // 2, tile=T, max_particles=60000)
    sim = gb().Simulation(w)
    orc = oracle.Oracle(w, with_particles=False)
    a = inputs.slab_particles(11, nx, nz, nz // 2, 8, 1e-3, clump=0.3)
    b = inputs.edge_particles(12, nx, nz, 4000, 1e-3)
    d = {k: np.concatenate([a[k], b[k]]) for k in a}
    set_both(sim, orc, 0, d)
    out, scale = sim.deposit_density()
    assert np.array_equal(out.cpu().numpy(), orc.get_rho())
    assert np.array_equal(sim.get_density().cpu().numpy(), orc.get_rho())
    assert out.sum().item() == len(d["x"]) * 2 ** 32
    assert scale == pytest.approx(orc.weight / (2 ** 32 * w["dx"] ** 2), rel=1e-15)


@pytest.mark.parametrize("pot", [{}, dict(pot_mode=2, morse_a=4.0), dict(lattice=1), dict(lattice=1, pot_mode=2, morse_a=4.0),
                                 dict(pot_mode=3)], ids=["lj", "morse", "hcp", "hcp-morse", "eam"])
def test_pair_force_matches_oracle(pot):
    """Eqs. (1)-(3) on a perturbed slab with a free surface, with Eq. (3) and with the Morse form.
    Tolerance: 1e-5 relative, plus an absolute floor of 1e-5 of the largest force for atoms whose
    force is a near-cancellation (FP32 rounding of the node densities, ~6e-8 relative, limits
    those)."""
    nx, nz = 48, 40
    w = workload("tiny", nx=nx, nz=nz, slab_k=20, max_particles=20000, **pot)
    sim = gb().Simulation(w)
    orc = oracle.Oracle(w, with_particles=False)
    d = inputs.slab_particles(21, nx, nz, 20, 8, 1e-4, clump=0.25)
    set_both(sim, orc, 0, d)
    Fg = sim.pair_force().cpu().numpy().astype(np.float64)
    Fo = orc.pair_force()
    scale = np.abs(Fo).max()
    assert scale > 0
    err = np.abs(Fg - Fo)
    assert (err <= 1e-5 * np.abs(Fo) + 1e-5 * scale).all(), err.max() / scale
    assert not Fg[:, 1].any()


def test_eam_force_in_vapour_above_the_surface_matches_oracle():
    """The embedded-atom form with vapour above a dense slab (128 atoms per cell): clusters of 12
    atoms, each with a lone atom at the edge of the cluster's support. The lone atom's -x neighbour
    sits where the interpolated density has nearly vanished, so its embedding density is held at its
    bond's f(r) (the floor branch of the kernel; the floor moves these forces by ~0.6 %). All atoms
    at the pair-force tolerance, the lone atoms' x force at 1e-4 of its own size."""
    nx, nz, ppc, sk = 32, 40, 128, 6
    w = workload("tiny", nx=nx, nz=nz, slab_k=sk, ppc_ion=ppc, ppc_electron=ppc, max_particles=40000, pot_mode=3)
    sim = gb().Simulation(w)
    orc = oracle.Oracle(w, with_particles=False)
    d = inputs.slab_particles(23, nx, nz, sk, ppc, 1e-4, clump=0.25)
    rng = np.random.default_rng(24)
    ns = 12
    ci, ck = rng.integers(0, nx - 3, ns), rng.integers(10, 36, ns)
    cx = np.repeat(ci, 12) + 1.5 + rng.uniform(-0.05, 0.05, 12 * ns)
    cz = np.repeat(ck, 12) + 0.5 + rng.uniform(-0.05, 0.05, 12 * ns)
    lx, lz = ci + rng.uniform(0.01, 0.05, ns), ck + rng.uniform(0.4, 0.6, ns)
    nv = 13 * ns
    vx = np.concatenate([cx, lx]).astype(np.float32).astype(np.float64)
    vz = np.concatenate([cz, lz]).astype(np.float32).astype(np.float64)
    d = {k: np.concatenate([d[k], v]) for k, v in
         dict(x=vx, z=vz, ux=np.zeros(nv), uy=np.zeros(nv), uz=np.zeros(nv)).items()}
    g = set_both(sim, orc, 0, d)
    Fg = sim.pair_force().cpu().numpy().astype(np.float64)
    Fo = orc.pair_force()
    assert np.isfinite(Fo).all()
    scale = np.abs(Fo).max()
    err = np.abs(Fg - Fo)
    assert (err <= 1e-5 * np.abs(Fo) + 1e-5 * scale).all(), err.max() / scale
    # the lone atoms, found in the context's order by their positions
    x, z, _ = to_global(g, nx)
    lone = np.zeros(len(x), bool)
    for a, b in zip(lx, lz):
        lone |= (np.abs(x - np.float32(a)) < 1e-6) & (np.abs(z - np.float32(b)) < 1e-6)
    assert lone.sum() == ns
    assert (err[lone, 0] <= 1e-4 * np.abs(Fo[lone, 0])).all(), (err[lone, 0] / np.abs(Fo[lone, 0])).max()
    sim.close()


def test_uniform_lattice_zero_force_on_gpu():
    nx, nz = 32, 16
    w = workload("tiny", nx=nx, nz=nz, slab_k=nz, ppc_ion=4, ppc_electron=4, max_particles=4096)
    sim = gb().Simulation(w)
    n = nx * nz * 4
    cell = np.repeat(np.arange(nx * nz), 4).astype(np.int32)
    fx = np.tile(np.array([0.1, 0.35, 0.6, 0.85], np.float32), nx * nz)
    fz = np.full(n, 0.5, np.float32)
    z = np.zeros(n, np.float32)
    sim.set_particles(0, cell, fx, fz, z, z, z)
    assert not sim.pair_force().any().item()


def _random_state(nx, nz, slab_k, seed, w):
    ions = inputs.slab_particles(seed, nx, nz, slab_k, 8, 2e-4, clump=0.2)
    els = inputs.slab_particles(seed + 1, nx, nz, slab_k, 8, 3e-3)
    fields = inputs.random_fields(seed + 2, nx, nz, 3e9, 10.0)
    return ions, els, fields


def _compare_particles(g, o_after, g_before, nx, rtol=1e-5):
    x, z, u = to_global(g, nx)
    ox, oz = o_after["x"], o_after["z"]
    xb, zb, _ = to_global(g_before, nx)
    dx = np.mod(ox - xb + nx / 2, nx) - nx / 2
    ex = np.abs(np.mod(x - ox + nx / 2, nx) - nx / 2)
    ez = np.abs(z - oz)
    # displacement to 1e-5 relative plus the FP32 rounding of the offset (2^-23 cells)
    assert (ex <= rtol * np.abs(dx) + 2.0 ** -22).all(), ex.max()
    assert (ez <= rtol * np.abs(oz - zb) + 2.0 ** -22).all(), ez.max()
    for c, comp in enumerate(("ux", "uy", "uz")):
        ref = o_after[comp]
        scale = np.abs(ref).max()
        np.testing.assert_allclose(u[c], ref, rtol=rtol, atol=1e-6 * scale)


@pytest.mark.parametrize("seed,ppc", [(31, 8), (32, 8), (33, 40)])
def test_one_step_full_mode(seed, ppc):
    """One full cycle from identical state (random fields, perturbed slab): particles and
    fields to 1e-5; the current and the new node density bit-exact against the oracle's
    deposition of the GPU's own new positions. A slab configured with 40 + 40 particles per cell
    takes the J_y code at 2^17 (its int64 node sums would not be proven exact at 2^18)."""
    nx, nz, sk = 56, 44, 22
    w = workload("tiny", nx=nx, nz=nz, slab_k=sk, max_particles=nx * sk * max(ppc, 8), I0=1e19, ppc_ion=ppc,
                 ppc_electron=ppc)
    bits = oracle.jy_bits(2 * ppc)
    assert bits == (18 if ppc == 8 else 17)
    sim = gb().Simulation(w, sort_every=0)
    orc = oracle.Oracle(w, with_particles=False)
    ions, els, fields = _random_state(nx, nz, sk, seed, w)
    g0 = [set_both(sim, orc, 0, ions), set_both(sim, orc, 1, els)]
    for f, a in enumerate(fields):
        sim.set_field(f, a)
        orc.set_field(f, a)
    assert np.array_equal(sim.get_density().cpu().numpy(), orc.get_rho())
    sim.step(1)
    orc.step(1)
    g1 = [sim.get_particles(0), sim.get_particles(1)]
    for sp in (0, 1):
        _compare_particles(g1[sp], orc.get_particles(sp), g0[sp], nx)
    # deposition of the GPU's own move, bit-exact
    J = np.zeros((3, nz + 1, nx), np.int64)
    for sp, sign in ((0, 1), (1, -1)):
        x0, z0, _ = to_global(g0[sp], nx)
        x1, z1, u1 = to_global(g1[sp], nx)
        oracle.deposit_current(nx, nz, sign, x0, z0, x1, z1, *[v.astype(np.float32) for v in u1], out=J, bits=bits)
    assert np.array_equal(sim.get_current().cpu().numpy(), J)
    x1, z1, _ = to_global(g1[0], nx)
    assert np.array_equal(sim.get_density().cpu().numpy(), oracle.deposit_density(nx, nz, x1, z1))
    # fields: the oracle's Maxwell update from the same start and the same (bit-exact) current
    fo = oracle.Oracle(w, with_particles=False)
    for f, a in enumerate(fields):
        fo.set_field(f, a)
    fo.set_current(J)
    fo.maxwell()
    for f in range(6):
        a = sim.get_field(f).cpu().numpy().astype(np.float64)
        b = fo.get_field(f)
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())


def test_electric_gather_reproduces_linear_fields():
    """The E gather of the particle kernel against a closed form, not against the oracle: Ex, Ey,
    Ez are each set to their own linear function a + b x + c z at their own Yee positions, B = 0,
    and electrons at rest take one step of a tiny dt (1e-21 s: they move ~1e-12 cells). With
    B = 0 the two half kicks give u = 2 (q dt / 2 m c) E at the particle, so u / (q dt / m c) must
    be the linear function at the particle's position (a wrong half-cell offset is off by half a
    slope: more than 1e-3 here). Positions span several tiles, the tiles' edges and the rows next
    to both walls (where the half-row Ez takes its edge row)."""
    nx, nz = 40, 24
    w = workload("tiny", nx=nx, nz=nz, slab_k=nz, ppc_ion=1, ppc_electron=1, tile=8, dt_override=1e-21,
                 laser_profile=0, max_particles=5000)
    sim = gb().Simulation(w, sort_every=0)
    rng = np.random.default_rng(11)
    n = 4000
    x = np.concatenate([rng.uniform(1.0, nx - 2.0, n), rng.uniform(1.0, nx - 2.0, 200)])
    z = np.concatenate([rng.uniform(0.0, nz, n), rng.uniform(0.0, 0.5, 100), rng.uniform(nz - 0.5, nz, 100)])
    x = np.floor(x * 2 ** 20) / 2 ** 20
    z = np.minimum(np.floor(z * 2 ** 20) / 2 ** 20, nz - 2 ** -20)
    cell, fx, fz = from_global(x, z, nx)
    zero = np.zeros(len(x), np.float32)
    sim.set_particles(1, cell, fx, fz, zero, zero, zero)
    sim.set_particles(0, cell[:0], fx[:0], fz[:0], zero[:0], zero[:0], zero[:0])
    k, i = np.mgrid[0:nz + 1, 0:nx]
    coef = {0: (0.0, 3e5, 1e5), 1: (0.0, -2e5, 4e5), 2: (0.0, 1e5, -3e5)}     # V/m per cell
    stag = {0: (0.5, 0.0, False), 1: (0.0, 0.0, False), 2: (0.0, 0.5, True)}
    for f in range(6):
        grid = np.zeros((nz + 1, nx))
        if f in coef:
            a, b, c = coef[f]
            sx, sz, half = stag[f]
            grid = a + b * (i + sx) + c * (k + sz)
            if half:
                grid[nz] = 0.0
        sim.set_field(f, grid.astype(np.float32))
    g0 = sim.get_particles(1)
    x0, z0, _ = to_global(g0, nx)
    sim.step(1)
    g1 = sim.get_particles(1)
    scale = QE * w["dt_override"] / (ME * C)          # u per V/m after the two half kicks
    for f in range(3):
        a, b, c = coef[f]
        sx, sz, half = stag[f]
        zc = np.clip(z0, 0.5, nz - 0.5) if half else z0
        expect = -(a + b * x0 + c * zc)                 # electrons: q = -e
        got = g1[("ux", "uy", "uz")[f]].cpu().numpy().astype(np.float64) / scale
        np.testing.assert_allclose(got, expect, rtol=1e-5, atol=1e-5 * np.abs(expect).max())
    sim.close()


@pytest.mark.parametrize("pot", [{}, dict(pot_mode=1, c_att=0.65, s_rep=2.5), dict(pot_mode=2, morse_a=4.0),
                                 dict(lattice=1), dict(pot_mode=3)], ids=["lj", "altered", "morse", "hcp", "eam"])
def test_one_step_transport_mode(pot):
    """One transport step (pair force only) against the oracle, with Eq. (3) as printed, with
    the altered potential (attractive and repulsive branches scaled) and with the Morse form. The
    altered force changes its factor at a neighbour distance of r0: a distance within FP32
    rounding of r0 can fall on the other branch than in FP64. So with the altered potential all
    momenta but those few are held to 1e-5 (at most 0.2 % of the atoms may exceed it; measured: a
    handful of the 9600), and those few to 2e-4 (measured up to ~1e-4)."""
    nx, nz, sk = 40, 30, 15
    w = workload("transport", nx=nx, nz=nz, slab_k=sk, max_particles=nx * sk * 16, **pot)
    sim = gb().Simulation(w, sort_every=0)
    orc = oracle.Oracle(w, with_particles=False)
    d = inputs.slab_particles(41, nx, nz, sk, 16, 3e-7, clump=0.3)
    g0 = set_both(sim, orc, 0, d)
    sim.step(1)
    orc.step(1)
    altered = pot.get("pot_mode") == 1
    g1, o1 = sim.get_particles(0), orc.get_particles(0)
    _compare_particles(g1, o1, g0, nx, rtol=2e-4 if altered else 1e-5)
    if altered:
        _, _, u = to_global(g1, nx)
        off_branch = np.zeros(len(u[0]), bool)
        for c, comp in enumerate(("ux", "uy", "uz")):
            ref = o1[comp]
            off_branch |= np.abs(u[c] - ref) > 1e-5 * np.abs(ref) + 1e-6 * np.abs(ref).max()
        assert off_branch.sum() <= max(2, len(off_branch) // 500), off_branch.sum()
    x1, z1, _ = to_global(sim.get_particles(0), nx)
    assert np.array_equal(sim.get_density().cpu().numpy(), oracle.deposit_density(nx, nz, x1, z1))


@pytest.mark.parametrize("pot", [{}, dict(pot_mode=2, morse_a=4.0), dict(lattice=1), dict(pot_mode=3)],
                         ids=["lj", "morse", "hcp", "eam"])
def test_energy_matches_oracle(pot):
    nx, nz, sk = 48, 40, 20
    w = workload("tiny", nx=nx, nz=nz, slab_k=sk, max_particles=nx * sk * 8, **pot)
    sim = gb().Simulation(w)
    orc = oracle.Oracle(w, with_particles=False)
    ions, els, fields = _random_state(nx, nz, sk, 51, w)
    set_both(sim, orc, 0, ions)
    set_both(sim, orc, 1, els)
    for f, a in enumerate(fields):
        sim.set_field(f, a)
        orc.set_field(f, a)
    eg, eo = sim.energy(), orc.energy()
    for key in ("kinetic_ion", "kinetic_electron", "field_E", "field_B"):
        assert eg[key] == pytest.approx(eo[key], rel=1e-6), key
    assert eg["pair"] == pytest.approx(eo["pair"], rel=1e-5)


def test_sort_is_a_permutation_into_tiles():
    w = workload("tiny", nx=70, nz=52, slab_k=30, tile=16)
    sim = gb().Simulation(w, sort_every=0)
    sim.step(5)
    before = [sim.get_particles(s) for s in (0, 1)]
    sim.sort()
    after = [sim.get_particles(s) for s in (0, 1)]
    T, nx = 16, 70
    for b, a in zip(before, after):
        kb = np.lexsort([b[k].cpu().numpy() for k in ("uz", "uy", "ux", "fz", "fx", "cell")])
        ka = np.lexsort([a[k].cpu().numpy() for k in ("uz", "uy", "ux", "fz", "fx", "cell")])
        for k in b:
            assert np.array_equal(b[k].cpu().numpy()[kb], a[k].cpu().numpy()[ka])
        # tile-major; inside a tile the cell order, stored by blocks of 1024 as 32-row matrices
        key = cell_key(a["cell"].cpu().numpy().astype(np.int64), nx, 1, T, 2)
        ordered, _ = undo_layout(key, T * T, 1024)
        assert (np.diff(ordered) >= 0).all()


def test_deterministic_grids():
    """Integer deposition makes density and current independent of the order of the atomics
    and of the particle order inside a cell."""
    w = workload("tiny", nx=64, nz=48, slab_k=24, sort_every=3)
    res = []
    for _ in range(2):
        sim = gb().Simulation(w)
        sim.step(7)
        res.append((sim.get_density().cpu().numpy(), sim.get_current().cpu().numpy(),
                    [sim.get_field(f).cpu().numpy() for f in range(6)]))
        sim.close()
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
    for a, b in zip(res[0][2], res[1][2]):
        assert np.array_equal(a, b)


def test_empty_slab_and_vacuum():
    w = workload("tiny", nx=32, nz=32, slab_k=0)
    sim = gb().Simulation(w)
    assert sim.info()["num_particles"] == (0, 0)
    sim.step(3)
    out, _ = sim.deposit_density()
    assert not out.any().item()
    assert sim.energy()["kinetic_ion"] == 0.0


@pytest.mark.slow
def test_tiny_workload_200_steps_aggregates():
    """The tiny copper-slab workload (64 x 64, 8 + 8 ppc, 200 steps): total energy and the
    depth profile of the node density agree with the FP64 oracle within 1e-3."""
    w = workload("tiny")
    sim = gb().Simulation(w)
    orc = oracle.Oracle(w)
    sim.step(200)
    orc.step(200)
    eg, eo = sim.energy(), orc.energy()
    stored = ("kinetic_ion", "kinetic_electron", "field_E", "field_B", "pair")
    tg = sum(eg[k] for k in stored)
    to = sum(eo[k] for k in stored)
    assert tg == pytest.approx(to, rel=1e-3)
    assert eg["kinetic_electron"] == pytest.approx(eo["kinetic_electron"], rel=1e-3)
    # the laser energy sent towards the slab: the net flux through the row below the antenna
    # includes the part the overdense slab reflects back within the 200 steps, which carries the
    # same plasma noise as the field energies; the bar is the totals' 1e-3 (measured 1.1e-4)
    assert eo["injected"] > 0
    assert eg["injected"] == pytest.approx(eo["injected"], rel=1e-3)
    # The field energy here is the electrostatic noise of the unresolved plasma (10 nm cells);
    # it is chaotic in the particle trajectories: rounding the oracle's own state to FP32 after
    # every step moves it by 1.2e-3 (field_E) and 1.3e-4 (field_B) after 200 steps. Per component
    # the bar is therefore 5e-3; the totals above carry the 1e-3 requirement.
    for key in ("field_E", "field_B"):
        assert eg[key] == pytest.approx(eo[key], rel=5e-3), key
    pg = sim.get_density().cpu().numpy().sum(axis=1).astype(np.float64)
    po = orc.get_rho().sum(axis=1).astype(np.float64)
    assert np.linalg.norm(pg - po) / np.linalg.norm(po) < 1e-3


STORED = ("kinetic_ion", "kinetic_electron", "field_E", "field_B", "pair")


@pytest.mark.slow
def test_full_cycle_1000_steps_resolved_plasma():
    """The full cycle (Cu+ ions with the pair force, electrons, fields) over 1000 steps on the tiny
    slab's geometry (64 x 64 cells, 8 + 8 ppc) at a density whose Debye length the 10 nm cells
    resolve (n = 1e26 m^-3, 100 eV electrons: lambda_D = 0.74 cells, w_pe dt = 0.013). Here the
    cycle is not chaotic at the scale of the bars: rounding the oracle's initial momenta to FP32
    moves its 1000-step energies by 5e-8. With the laser on (1e13 W/cm^2, peak at the surface at
    step 500) the stored energy, the injected energy and the depth profile of the node density
    agree with the oracle within 1e-3; with the laser off the stored energy drifts (by +1.1 % in
    the oracle: mild numerical heating at lambda_D ~ dx) and the GPU's drift equals the oracle's
    within 1e-4."""
    base = dict(n_atoms=1e26, T_electron_eV=100.0, t_peak=500 * 2.24072e-17)
    for I0 in (1e17, 0.0):
        w = workload("tiny", I0=I0, **base)
        sim = gb().Simulation(w)
        orc = oracle.Oracle(w)
        e0g, e0o = sim.energy(), orc.energy()
        t0g, t0o = sum(e0g[k] for k in STORED), sum(e0o[k] for k in STORED)
        assert t0g == pytest.approx(t0o, rel=1e-6)
        sim.step(1000)
        orc.step(1000)
        eg, eo = sim.energy(), orc.energy()
        tg, to = sum(eg[k] for k in STORED), sum(eo[k] for k in STORED)
        if I0 > 0:
            assert eo["injected"] > 0.5 * to
            assert tg == pytest.approx(to, rel=1e-3)
            assert eg["injected"] == pytest.approx(eo["injected"], rel=1e-3)
            pg = sim.get_density().cpu().numpy().sum(axis=1).astype(np.float64)
            po = orc.get_rho().sum(axis=1).astype(np.float64)
            assert np.linalg.norm(pg - po) / np.linalg.norm(po) < 1e-3
        else:
            dg, do = (tg - t0g) / abs(t0g), (to - t0o) / abs(t0o)
            assert abs(do) > 1e-3                       # the oracle's drift is measurable
            assert abs(dg - do) <= 1e-4, (dg, do)
        sim.close()


@pytest.mark.slow
def test_tiny_workload_1000_steps_full_cycle():
    """The tiny workload itself (solid density, 1 eV electrons, laser on) over 1000 steps. Its
    10 nm cells are 400 Debye lengths: the explicit cycle heats the electrons by the finite-grid
    instability (their kinetic energy grows 1000-fold in the oracle) and amplifies rounding, so the
    1000-step energies are not reproducible below a few per cent by any implementation: the oracle
    against itself with its initial momenta rounded to FP32, with one momentum component scaled by
    1 + 1e-7, or with its state rounded to FP32 after one step differs by +2.3 %, -0.9 % and +5.1 %
    in the stored energy. The bar on the energies is therefore that ensemble's spread (3 sigma,
    10 %); the depth profile of the node density (the ions barely move in 1000 steps) keeps the
    1e-3 bar (the ensemble: 2.5e-5)."""
    w = workload("tiny", t_peak=500 * 2.24072e-17)
    sim = gb().Simulation(w)
    orc = oracle.Oracle(w)
    sim.step(1000)
    orc.step(1000)
    eg, eo = sim.energy(), orc.energy()
    tg, to = sum(eg[k] for k in STORED), sum(eo[k] for k in STORED)
    assert tg == pytest.approx(to, rel=0.1)
    assert eg["kinetic_electron"] == pytest.approx(eo["kinetic_electron"], rel=0.1)
    pg = sim.get_density().cpu().numpy().sum(axis=1).astype(np.float64)
    po = orc.get_rho().sum(axis=1).astype(np.float64)
    assert np.linalg.norm(pg - po) / np.linalg.norm(po) < 1e-3
    sim.close()


@pytest.mark.slow
def test_transport_1000_steps_energy_drift_and_profile():
    """Transport mode (neutral atoms, pair force only), 1000 steps of 12 fs: the GPU's energy
    drift stays within 1e-4 of the oracle's and the depth profile of the node density agrees
    within 1e-3."""
    w = workload("transport", nx=32, nz=48, slab_k=24)
    sim = gb().Simulation(w)
    orc = oracle.Oracle(w)
    e0g, e0o = sim.energy(), orc.energy()
    t0g = e0g["kinetic_ion"] + e0g["pair"]
    t0o = e0o["kinetic_ion"] + e0o["pair"]
    sim.step(1000)
    orc.step(1000)
    eg, eo = sim.energy(), orc.energy()
    dg = (eg["kinetic_ion"] + eg["pair"] - t0g) / abs(t0g)
    do = (eo["kinetic_ion"] + eo["pair"] - t0o) / abs(t0o)
    assert abs(dg - do) <= 1e-4, (dg, do)
    pg = sim.get_density().cpu().numpy().sum(axis=1).astype(np.float64)
    po = orc.get_rho().sum(axis=1).astype(np.float64)
    assert np.linalg.norm(pg - po) / np.linalg.norm(po) < 1e-3


@pytest.mark.parametrize("pot,curv", [({}, 72.0), (dict(pot_mode=2, morse_a=4.0), 32.0), (dict(lattice=1), 144.0),
                                      (dict(pot_mode=3), 5.09 ** 2 * (3.54 / 0.41) / 3.0)],
                         ids=["lj", "morse", "hcp", "eam"])
def test_transport_acoustic_wave_period(pot, curv):
    """The GPU transport stage carries a small standing acoustic wave (64-cell wavelength, strain
    1e-3) with the period of the linearised Eqs. (1)-(3), lambda / sqrt(U''(r0) r0^2 / (3 m)),
    over 2.5 periods (8300 steps for Eq. 3, U''(r0) r0^2 = 72 D; 12 450 for the Morse form with
    a = 4, 2 a^2 D = 32 D), like the oracle."""
    import math
    nx, nz = 64, 4
    dt = 50e-15
    w = workload("transport", nx=nx, nz=nz, slab_k=nz, ppc_ion=4, T_ion_K=0.0, dt_override=dt,
                 max_particles=nx * nz * 4, **pot)
    sim = gb().Simulation(w, sort_every=0)
    cells = np.arange(nx * nz)
    i, k = cells % nx, cells // nx
    offs = [(0.25, 0.25), (0.75, 0.25), (0.25, 0.75), (0.75, 0.75)]
    x0 = np.concatenate([i + a for a, b in offs]).astype(np.float64)
    z0 = np.concatenate([k + b for a, b in offs]).astype(np.float64)
    kk = 2 * math.pi / nx
    eps = 1e-2
    cell, fx, fz = from_global(x0 + eps * np.sin(kk * x0), z0, nx)
    zeros = np.zeros(len(x0), np.float32)
    sim.set_particles(0, cell, fx, fz, zeros, zeros, zeros)
    g = sim.get_particles(0)                    # the context's order
    xg, _, _ = to_global(g, nx)
    xeq = np.round((xg - 0.25) * 2) / 2 + 0.25  # nearest lattice site (0.25 + multiples of 0.5)
    m = 63.546 * 1.66053906660e-27
    period = (nx * w["dx"]) / math.sqrt(curv * 0.41 * 1.602176634e-19 / (3 * m))
    amps = []
    chunk = 20
    for s in range(0, int(2.5 * period / dt), chunk):
        sim.step(chunk)
        x, _, _ = to_global(sim.get_particles(0), nx)
        d = (x - xeq + nx / 2) % nx - nx / 2
        amps.append((s + chunk, (d * np.sin(kk * xeq)).sum() / (np.sin(kk * xeq) ** 2).sum()))
    a = np.array(amps)
    crossings = [a[j - 1, 0] + (a[j, 0] - a[j - 1, 0]) * a[j - 1, 1] / (a[j - 1, 1] - a[j, 1])
                 for j in range(1, len(a)) if (a[j - 1, 1] > 0) != (a[j, 1] > 0)]
    assert len(crossings) >= 4
    assert 2 * np.diff(crossings).mean() * dt == pytest.approx(period, rel=1e-2)
    assert np.abs(a[:, 1]).max() == pytest.approx(eps, rel=2e-2)
    sim.close()


@pytest.mark.parametrize("profile,slab_k", [(1, 0), (2, 0), (2, 10)])
def test_vacuum_without_particles_matches_oracle(profile, slab_k):
    """Degenerate input: no particles (slab_k = 0, or a slab row without macroparticles, ppc 0).
    The context initialises, the laser propagates, and fields and injected energy follow the oracle
    after one step and after 150 steps: the plane wave (profile 1) and the focused Gaussian beam
    (profile 2: width, wavefront curvature and half Gouy phase at the antenna, focus at row
    slab_k)."""
    over = dict(ppc_ion=0, ppc_electron=0) if slab_k else {}
    w = workload("tiny", nx=128, nz=80, slab_k=slab_k, laser_profile=profile, w0=0.4e-6, I0=1e17,
                 tau_fwhm=5e-15, t_peak=8e-15, **over)
    sim = gb().Simulation(w)
    assert sum(sim.info()["num_particles"]) == 0
    orc = oracle.Oracle(w, with_particles=False)
    for nsteps in (1, 149):
        sim.step(nsteps)
        orc.step(nsteps)
        for f in range(6):
            g, o = sim.get_field(f).cpu().numpy(), orc.get_field(f)
            scale = np.abs(o).max()
            assert scale == 0 or np.abs(g - o).max() <= 1e-5 * scale, (nsteps, f)

    eg, eo = sim.energy(), orc.energy()
    assert eo["injected"] > 0
    assert eg["injected"] == pytest.approx(eo["injected"], rel=1e-5)
    assert eg["kinetic_ion"] == 0.0 and eg["kinetic_electron"] == 0.0 and eg["pair"] == 0.0
    assert not sim.get_density().any() and not sim.get_current().any()
    sim.close()
