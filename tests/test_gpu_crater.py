"""The atomic-transport stage beyond the cycle itself, through the C ABI against the oracle: the
lattice-temperature start of a laser spot (a synthetic stand-in for the paper's Fig. 2) and the
crater measurement (column profile of missing material, width, Eq. 5).

The crater profile is an exact integer column sum times one FP64 factor, so the GPU's profile of
its own density maps equals the oracle's profile of the same maps to the last bits of that factor
(relative 1e-14)."""
import math

import numpy as np
import pytest

import oracle
from paper_1502_07722_gb300.workloads import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1502_07722_gb300 import _build
    _build.build()
    oracle.build()
    import paper_1502_07722_gb300 as m
    return m


def spot(**kw):
    w = dict(workload("transport"), nx=72, nz=48, slab_k=30, ppc_ion=16, temp_profile=1, T_ion_K=300.0,
             T_spot_K=20000.0, spot_w=150e-9, spot_depth=60e-9, sort_every=10)
    w.update(kw)
    return w


def test_spot_start_matches_oracle(gb):
    """Same seed: positions bit-exact, momenta at the local spot temperature to FP32 rounding."""
    w = spot()
    sim = gb.Simulation(w)
    orc = oracle.Oracle(w)
    g = sim.get_particles(0)
    cell = g["cell"].cpu().numpy().astype(np.int64)
    x = cell % w["nx"] + g["fx"].cpu().numpy().astype(np.float64)
    z = cell // w["nx"] + g["fz"].cpu().numpy().astype(np.float64)
    o = orc.get_particles(0)
    kg, ko = np.lexsort((z, x)), np.lexsort((o["z"], o["x"]))
    assert np.array_equal(x[kg], o["x"][ko]) and np.array_equal(z[kg], o["z"][ko])
    for comp in ("ux", "uy", "uz"):
        u = g[comp].cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(u[kg], o[comp][ko], rtol=1e-6, atol=1e-7 * np.abs(o[comp]).max())
    # hotter on the axis than at the edges
    ax = np.abs(x - w["nx"] / 2) < 4
    u2 = sum(g[c].cpu().numpy().astype(np.float64) ** 2 for c in ("ux", "uy", "uz"))
    assert u2[ax].mean() > 10 * u2[np.abs(x - w["nx"] / 2) > 30].mean()
    sim.close()


def test_spot_start_rejected_without_a_spot(gb):
    with pytest.raises(gb.PicError) as e:
        gb.Simulation(dict(spot(), spot_w=0.0))
    assert e.value.code == gb.PIC_EINVAL
    with pytest.raises(gb.PicError) as e:
        gb.Simulation(dict(spot(), dims=3, ny=8, spot_depth=-1.0))
    assert e.value.code == gb.PIC_EINVAL


@pytest.mark.parametrize("tile", [4, 10])
def test_spot_start_3d_matches_oracle(gb, tile):
    """3D lattice-temperature start (radial Gaussian about the axis through the middle of the x-y
    plane): positions bit-exact, momenta to FP32 rounding, on a grid whose sides are not
    multiples of the tile."""
    w = spot(dims=3, nx=26, ny=22, nz=18, slab_k=11, ppc_ion=6, tile=tile, spot_w=60e-9, spot_depth=40e-9)
    sim = gb.Simulation(w)
    orc = oracle.Oracle3D(w)
    g = {k: v.cpu().numpy() for k, v in sim.get_particles(0).items()}
    cell = g["cell"].astype(np.int64)
    x = cell % w["nx"] + g["fx"].astype(np.float64)
    y = (cell // w["nx"]) % w["ny"] + g["fy"].astype(np.float64)
    z = cell // (w["nx"] * w["ny"]) + g["fz"].astype(np.float64)
    o = orc.get_particles(0)
    kg, ko = np.lexsort((z, y, x)), np.lexsort((o["z"], o["y"], o["x"]))
    for a, b in ((x, "x"), (y, "y"), (z, "z")):
        assert np.array_equal(a[kg], o[b][ko])
    for comp in ("ux", "uy", "uz"):
        u = g[comp].astype(np.float64)
        np.testing.assert_allclose(u[kg], o[comp][ko], rtol=1e-6, atol=1e-7 * np.abs(o[comp]).max())
    r2 = (x - w["nx"] / 2) ** 2 + (y - w["ny"] / 2) ** 2
    u2 = sum(g[c].astype(np.float64) ** 2 for c in ("ux", "uy", "uz"))
    top = z > w["slab_k"] - 2
    assert u2[(r2 < 4) & top].mean() > 10 * u2[(r2 > 100) & top].mean()
    sim.close()


def test_crater_profile_matches_oracle(gb):
    """A hot spot expands and evaporates for 2000 steps (24 ps): the GPU's profile of its own maps
    equals the oracle's profile of the same maps; width and depth agree between the two
    measurements."""
    from paper_1502_07722_gb300 import crater
    w = spot()
    sim = gb.Simulation(w)
    rho0, _ = sim.deposit_density()
    assert float(sim.crater_profile(rho0).abs().max()) == 0.0
    sim.step(2000)
    prof = sim.crater_profile(rho0).cpu().numpy()
    orc = oracle.Oracle(w, with_particles=False)
    expect = orc.crater_profile(rho0.cpu().numpy(), sim.get_density().cpu().numpy())
    np.testing.assert_allclose(prof, expect, rtol=1e-14, atol=0)
    assert prof.max() > 0.5 * w["dx"]                          # material has left the hot spot
    m = crater.crater_metrics(prof, w["dx"])
    depth, width = oracle.crater_width(expect, w["dx"])
    assert m["depth"] == pytest.approx(depth, rel=1e-14)
    assert m["width"] == pytest.approx(width, rel=1e-9)
    assert 0 < m["width"] < w["nx"] * w["dx"]
    mf = crater.crater_metrics(prof, w["dx"], far_field=True)
    assert mf["level"] == pytest.approx(oracle.far_field(expect), rel=1e-12)
    assert mf["width"] == pytest.approx(oracle.crater_width(expect - oracle.far_field(expect), w["dx"])[1], rel=1e-9)
    f_th = crater.threshold_fluence(2.0, m["width"], 2 * w["spot_w"])
    assert f_th == pytest.approx(2.0 * math.exp(-(width / (2 * w["spot_w"])) ** 2), rel=1e-9)
    sim.close()


def test_crater_profile_3d_counts_removed_material(gb):
    """3D: removing the atoms of the top h cell rows of an m_x x m_y block of columns leaves
    h m_x m_y cells of solid material missing; the (ny, nx) profile sums to h m_x m_y dx."""
    w = dict(workload("tiny"), dims=3, nx=16, ny=12, nz=14, slab_k=8, ppc_ion=4, ppc_electron=4, mode=1,
             ion_charge=0.0, laser_profile=0, tile=4)
    sim = gb.Simulation(w)
    rho0, _ = sim.deposit_density()
    g = {k: v.cpu().numpy() for k, v in sim.get_particles(0).items()}
    cell = g["cell"].astype(np.int64)
    i, j, k = cell % 16, (cell // 16) % 12, cell // (16 * 12)
    h, gone = 2, (i >= 5) & (i < 9) & (j >= 3) & (j < 6) & (k >= w["slab_k"] - 2)
    keep = ~gone
    sim.set_particles(0, cell[keep].astype(np.int32), g["fx"][keep], g["fz"][keep], g["ux"][keep], g["uy"][keep],
                      g["uz"][keep], fy=g["fy"][keep])
    prof = sim.crater_profile(rho0).cpu().numpy()
    assert prof.shape == (12, 16)
    assert prof.sum() == pytest.approx(h * 4 * 3 * w["dx"], rel=1e-12)
    assert (prof[:, :5] == 0).all() and (prof[:, 10:] == 0).all() and (prof[:3] == 0).all() and (prof[7:] == 0).all()
    sim.close()


def test_crater_3d_matches_oracle(gb):
    """3D spot run (800 steps, 9.6 ps): the GPU's (ny, nx) profile of its own maps equals the
    oracle's profile of the same maps; depth and the widths along x and y agree between the two
    measurements."""
    from paper_1502_07722_gb300 import crater
    w = spot(dims=3, nx=28, ny=24, nz=20, slab_k=12, ppc_ion=8, tile=10, spot_w=80e-9, spot_depth=40e-9)
    sim = gb.Simulation(w)
    rho0, _ = sim.deposit_density()
    assert float(sim.crater_profile(rho0).abs().max()) == 0.0
    sim.step(800)
    prof = sim.crater_profile(rho0).cpu().numpy()
    assert prof.shape == (24, 28)
    orc = oracle.Oracle3D(w, with_particles=False)
    expect = orc.crater_profile(rho0.cpu().numpy(), sim.get_density().cpu().numpy())
    np.testing.assert_allclose(prof, expect, rtol=1e-14, atol=0)
    th = 0.25 * w["dx"]
    m = crater.crater_metrics(prof, w["dx"], threshold=th)
    depth, wx, wy = oracle.crater_width_3d(expect, w["dx"], th)
    assert m["depth"] == pytest.approx(depth, rel=1e-14)
    assert (m["width_x"], m["width_y"]) == pytest.approx((wx, wy), rel=1e-9)
    assert prof.max() > th                                 # material has left the hot spot
    sim.close()


def test_c_att_calibration_matches_oracle(gb):
    """The attractive-factor calibration on the GPU's initial slab (probe forces through the C ABI)
    against the oracle's calibration on the same node sums, with the same rule per cell (8-point
    Gauss-Legendre on 41 pieces that halve towards both cell edges): the work to FP32 force
    accuracy, and the factor. The rule is converged: 16 points per piece change the work by less
    than 0.5 % (0.24 % measured on the oracle)."""
    from paper_1502_07722_gb300 import crater
    w = dict(workload("transport"), nx=48, nz=40, slab_k=24, ppc_ion=16)
    sim = gb.Simulation(w)
    got = crater.calibrate_c_att(sim)
    rho = sim.get_density().cpu().numpy()
    c_att, w_att = oracle.calibrate_c_att(w, rho, w["slab_k"] - 1, w["slab_k"] + 2)
    assert got["W_att"] == pytest.approx(w_att, rel=2e-4)
    assert got["c_att"] == pytest.approx(c_att, rel=2e-4)
    assert w_att < 0 < c_att
    assert crater.calibrate_c_att(sim, order=16)["W_att"] == pytest.approx(got["W_att"], rel=5e-3)
    # probes outside the grid read nothing
    f = sim.pair_force_at([-1, 0], [0.5, 1.5], [0.5, 0.5]).cpu().numpy()
    assert np.isnan(f).all()
    sim.close()


@pytest.mark.parametrize("pot", [dict(pot_mode=2, morse_a=4.0), dict(pot_mode=2, morse_a=4.0, lattice=1)],
                         ids=["morse", "morse-hcp"])
def test_morse_probe_forces_match_oracle(gb, pot):
    """Probe forces of the Morse form (pot_mode 2, a = 4; on the cubic and the HCP lattice) around
    the surface of a transport slab against the oracle's force on atoms at the same positions over
    the same node sums, and the context's own stiffness used when the configuration is L-J;
    tolerance as for the pair force."""
    w = dict(workload("transport"), nx=32, nz=30, slab_k=16, ppc_ion=8, **pot)
    sim = gb.Simulation(w)
    rho = sim.get_density().cpu().numpy()
    rng = np.random.default_rng(3)
    n = 600
    x = rng.uniform(0, 32, n)
    z = rng.uniform(8, 19.999, n)
    i, k = np.floor(x).astype(np.int64), np.floor(z).astype(np.int64)
    fx, fz = (x - i).astype(np.float32), (z - k).astype(np.float32)
    cell = (k * 32 + i).astype(np.int32)
    Fg = sim.pair_force_at(cell, fx, fz).cpu().numpy().astype(np.float64)
    orc = oracle.Oracle(w, with_particles=False)
    zeros = np.zeros(n)
    orc.set_particles(0, i + fx.astype(np.float64), k + fz.astype(np.float64), zeros, zeros, zeros)
    orc.set_rho(rho)
    Fo = orc.pair_force()
    scale = np.abs(Fo).max()
    assert scale > 0
    assert (np.abs(Fg - Fo) <= 1e-5 * np.abs(Fo) + 1e-5 * scale).all(), np.abs(Fg - Fo).max() / scale
    assert not Fg[:, 1].any()
    sim.close()
    # an L-J context has no Morse stiffness to lend
    lj = gb.Simulation(dict(w, pot_mode=0, morse_a=0.0))
    with pytest.raises(gb.PicError) as e:
        lj.pair_force_at(cell[:4], fx[:4], fz[:4], pot_mode=2)
    assert e.value.code == gb.PIC_EINVAL
    lj.close()


def _laser_stage(gb, steps=120):
    w = dict(workload("tiny"), nx=48, nz=40, slab_k=20, ppc_ion=12, ppc_electron=12, I0=3e19,
             t_peak=30 * 2.24072e-17, sort_every=20)
    sim = gb.Simulation(w)
    sim.step(steps)
    return w, sim


def _oracle_from(w, parts):
    """An oracle state holding given particle arrays (one dict per species, in the GPU's layout:
    cell index and offsets), positions turned into global coordinates."""
    orc = oracle.Oracle(w, with_particles=False)
    for sp, g in enumerate(parts):
        cell = np.asarray(g["cell"], np.int64)
        x = cell % w["nx"] + np.asarray(g["fx"], np.float64)
        z = cell // w["nx"] + np.asarray(g["fz"], np.float64)
        orc.set_particles(sp, x, z, *(np.asarray(g[k], np.float64) for k in ("ux", "uy", "uz")))
    return orc


def _host(sim, sp):
    return {k: v.cpu().numpy() for k, v in sim.get_particles(sp).items()}


def test_cell_temperature_matches_oracle(gb):
    """Ion and electron temperature maps after 120 laser steps against the oracle's maps of the
    same particles (FP64 sums on both sides; only their order differs)."""
    w, sim = _laser_stage(gb)
    orc = _oracle_from(w, [_host(sim, 0), _host(sim, 1)])
    for sp in (0, 1):
        got = sim.cell_temperature(sp).cpu().numpy()
        exp = orc.cell_temperature(sp)
        np.testing.assert_allclose(got, exp, rtol=1e-9, atol=1e-12 * exp.max())
        assert (got[w["slab_k"] + 2:] == 0).all() and (got[:w["slab_k"] - 1] > 0).all()
    with pytest.raises(gb.PicError) as e:
        sim.cell_temperature(2)
    assert e.value.code == gb.PIC_EINVAL
    sim.close()


def test_two_stage_start_matches_oracle(gb):
    """The transport context takes the laser stage's ion temperature map: the re-tempered momenta
    equal the oracle's re-tempering of the same draws to the last bit (one FP64 multiply, rounded
    to FP32), and each cell's temperature scales by its map value over the start temperature."""
    from paper_1502_07722_gb300 import crater
    w, las = _laser_stage(gb)
    tw = dict(workload("transport"), nx=w["nx"], nz=w["nz"], slab_k=w["slab_k"], ppc_ion=12, T_ion_K=300.0)
    cold = gb.Simulation(tw)
    before = _host(cold, 0)
    T_before = cold.cell_temperature(0).cpu().numpy()
    cold.close()
    tr = crater.transport_from_laser(las, tw)
    Tmap = np.maximum(las.cell_temperature(0).cpu().numpy(), 300.0)
    after = _host(tr, 0)
    # two contexts order a cell's particles differently (atomic cursors of the sort): match them by
    # position, which is unique
    ka = np.lexsort((after["fz"], after["fx"], after["cell"]))
    kb = np.lexsort((before["fz"], before["fx"], before["cell"]))
    for k in ("cell", "fx", "fz"):
        assert np.array_equal(after[k][ka], before[k][kb])
    orc = _oracle_from(tw, [before])
    orc.set_temperature(0, Tmap, 300.0)
    o = orc.get_particles(0)
    for k in ("ux", "uy", "uz"):
        assert np.array_equal(after[k][ka], o[k].astype(np.float32)[kb])
    T_after = tr.cell_temperature(0).cpu().numpy()
    slab = T_before > 0
    np.testing.assert_allclose(T_after[slab], T_before[slab] * Tmap[slab] / 300.0, rtol=2e-6)
    with pytest.raises(gb.PicError) as e:
        tr.set_temperature(0, Tmap, 0.0)
    assert e.value.code == gb.PIC_EINVAL
    tr.close()
    las.close()


def test_few_shot_hand_back(gb):
    """Transport stage -> next laser stage: the laser context's ions are the transport atoms (same
    positions and momenta, hence the same node density bit for bit), its electrons sit on the same
    positions (neutral start), and it steps."""
    from paper_1502_07722_gb300 import crater
    tw = dict(workload("transport"), nx=40, nz=36, slab_k=18, ppc_ion=8, T_ion_K=3000.0)
    tr = gb.Simulation(tw)
    tr.step(30)
    lw = dict(workload("tiny"), nx=40, nz=36, slab_k=18, ppc_ion=8, ppc_electron=8)
    las = crater.laser_from_transport(tr, lw)
    a, ions, el = _host(tr, 0), _host(las, 0), _host(las, 1)
    ka, ki, ke = (np.lexsort((d["fz"], d["fx"], d["cell"])) for d in (a, ions, el))
    for k in ("cell", "fx", "fz", "ux", "uy", "uz"):
        assert np.array_equal(ions[k][ki], a[k][ka]), k
    for k in ("cell", "fx", "fz"):
        assert np.array_equal(el[k][ke], a[k][ka]), k
    assert np.array_equal(las.get_density().cpu().numpy(), tr.get_density().cpu().numpy())
    las.step(5)
    assert las.info()["step"] == 5
    las.close()
    tr.close()


def test_new_entry_points_refuse_bad_arguments(gb):
    """Argument checks of the transport-stage entry points, before any kernel runs."""
    w = dict(workload("transport"), nx=16, nz=16, slab_k=8, ppc_ion=4)
    sim = gb.Simulation(w)
    out = torch.empty(3, dtype=torch.float32, device="cuda")
    idx = torch.zeros(1, dtype=torch.int32, device="cuda")
    half = torch.full((1,), 0.5, dtype=torch.float32, device="cuda")
    cases = [
        lambda: gb.pic_crater_profile(sim.h, 0, out.data_ptr()),                      # NULL rho0
        lambda: gb.pic_pair_force_at(sim.h, -1, idx.data_ptr(), half.data_ptr(), half.data_ptr(), 0, 1.0, 1.0,
                                     out.data_ptr()),                                 # n < 0
        lambda: gb.pic_pair_force_at(sim.h, 1, idx.data_ptr(), half.data_ptr(), half.data_ptr(), 2, 1.0, 1.0,
                                     out.data_ptr()),                                 # Morse, no stiffness
        lambda: gb.pic_pair_force_at(sim.h, 1, idx.data_ptr(), half.data_ptr(), half.data_ptr(), 3, 1.0, 1.0,
                                     out.data_ptr()),                                 # pot_mode 3
        lambda: gb.pic_pair_force_at(sim.h, 1, 0, half.data_ptr(), half.data_ptr(), 0, 1.0, 1.0,
                                     out.data_ptr()),                                 # NULL cells
        lambda: gb.pic_cell_temperature(sim.h, 0, 0, out.data_ptr()),                  # NULL scratch
        lambda: gb.pic_set_temperature(sim.h, 1, out.data_ptr(), 300.0),               # no species 1
    ]
    for call in cases:
        with pytest.raises(gb.PicError) as e:
            call()
        assert e.value.code == gb.PIC_EINVAL
    # the context stays usable
    sim.step(2)
    sim.close()
    s3 = gb.Simulation(dict(workload("tiny"), dims=3, nx=8, ny=8, nz=8, slab_k=4, ppc_ion=2, ppc_electron=2, tile=4))
    with pytest.raises(gb.PicError) as e:
        gb.pic_pair_force_at(s3.h, 1, idx.data_ptr(), half.data_ptr(), half.data_ptr(), 0, 1.0, 1.0, out.data_ptr())
    assert e.value.code == gb.PIC_ESTATE
    s3.close()


@pytest.mark.parametrize("dims, src, dst", [
    (2, (48, 1, 40, 10e-9, 20), (32, 1, 27, 15e-9, 13)),        # coarser, non-integer ratio
    (2, (30, 1, 24, 15e-9, 12), (67, 1, 50, 6.5e-9, 29)),       # finer and wider than the source
    (2, (16, 1, 12, 10e-9, 6), (16, 1, 12, 10e-9, 6)),          # the same grid
    (3, (14, 12, 16, 10e-9, 8), (9, 8, 11, 16e-9, 5)),
    (3, (9, 8, 11, 16e-9, 5), (20, 17, 25, 7e-9, 12)),
], ids=["2d-coarser", "2d-finer", "2d-same", "3d-coarser", "3d-finer"])
def test_regrid_matches_oracle(gb, dims, src, dst):
    """The conservative remap of a cell map between grids placed on each other by the slab surface
    and the laser axis, on the GPU against the oracle's definition (FP64 on both sides: 1e-12)."""
    import torch
    rng = np.random.default_rng(11)
    shape = (src[2], src[1], src[0]) if dims == 3 else (src[2], src[0])
    a = rng.uniform(300.0, 8000.0, shape)
    out = gb.regrid_cells(torch.tensor(a, device="cuda"), src, dst, 300.0, dims=dims)
    torch.cuda.synchronize()
    ref = oracle.regrid_cells(a, src, dst, 300.0, dims=dims)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12)
    dev = torch.zeros(8, dtype=torch.float64, device="cuda")
    for bad in (dict(dims=4), dict(src=(4, 1, 2, 0.0, 1)), dict(src=(4, 1, 2, 1.0, 3)), dict(dst=(0, 1, 2, 1.0, 1))):
        args = dict(dims=2, src=(4, 1, 2, 1.0, 1), dst=(4, 1, 2, 1.0, 1))
        args.update(bad)
        with pytest.raises(gb.PicError) as e:
            gb.pic_regrid_cells(args["dims"], dev.data_ptr(), args["src"], dev.data_ptr(), args["dst"], 0.0)
        assert e.value.code == gb.PIC_EINVAL


def test_two_stage_start_on_coarser_cells_matches_oracle(gb):
    """The transport stage on cells 1.5 times the laser stage's (the paper's stages use different
    cells): its atoms are re-tempered to the laser stage's ion temperature remapped onto its own
    grid; against the oracle's remap of the same map and re-tempering of the same draws (FP32 of
    one FP64 multiply: 1 ulp)."""
    from paper_1502_07722_gb300 import crater
    w, las = _laser_stage(gb)
    tw = dict(workload("transport"), nx=32, nz=27, slab_k=13, dx=1.5 * w["dx"], ppc_ion=12, T_ion_K=300.0)
    cold = gb.Simulation(tw)
    before = _host(cold, 0)
    cold.close()
    Tl = np.maximum(las.cell_temperature(0).cpu().numpy(), 300.0)
    tr = crater.transport_from_laser(las, tw)
    assert las.cell_grid() != tr.cell_grid()
    Tmap = oracle.regrid_cells(Tl, las.cell_grid(), tr.cell_grid(), 300.0)
    assert Tmap.shape == (27, 32) and Tmap.max() > 400.0       # the laser-heated cells arrive
    after = _host(tr, 0)
    ka = np.lexsort((after["fz"], after["fx"], after["cell"]))
    kb = np.lexsort((before["fz"], before["fx"], before["cell"]))
    for k in ("cell", "fx", "fz"):
        assert np.array_equal(after[k][ka], before[k][kb])
    orc = _oracle_from(tw, [before])
    orc.set_temperature(0, Tmap, 300.0)
    o = orc.get_particles(0)
    for k in ("ux", "uy", "uz"):
        ref = o[k].astype(np.float32)[kb]
        np.testing.assert_allclose(after[k][ka], ref, rtol=2 ** -23, atol=0)
    tr.close()
    las.close()

