"""Batched intensity sweep (several slabs, one persistent launch per step, CUDA graph) against the
same slabs run one at a time: identical grids and particle sets."""
import numpy as np
import pytest

from paper_1502_07722_gb300.workloads import batched_sweep, workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1502_07722_gb300 import _build
    _build.build()
    import paper_1502_07722_gb300 as m
    return m


def small_sweep():
    """Three uneven slabs with different ppc, intensities and seeds (a scaled-down sweep)."""
    out = []
    for k, (side, ppc, I0) in enumerate(((48, 8, 1e17), (72, 16, 1e18), (40, 4, 1e19))):
        out.append(workload("tiny", nx=side, nz=side, slab_k=side // 2, ppc_ion=ppc, ppc_electron=ppc,
                            laser_profile=2, w0=0.2e-6, I0=I0, t_peak=5 * 2.24e-17, seed=200 + k))
    return out


def _multiset(sim, s):
    """Particles ordered by their position (cell, fx, fz as bit patterns), then momenta."""
    p = sim.get_particles(s)
    arr = np.stack([p[k].cpu().numpy().view(np.int32) for k in ("cell", "fx", "fz", "ux", "uy", "uz")])
    return arr[:, np.lexsort(arr[::-1])]


def _same_particles(a, b):
    """The same particles up to FP32 rounding: equal counts per cell, and per-cell sums of the
    offsets and momenta equal to rounding. The batched and the single-simulation kernels are
    separate compilations of the same push; the compiler may fuse a different multiply-add pair
    in each, which moves a kick or an offset by its last bit (below the 2^-16 deposition quantum,
    so every grid stays bit-identical)."""
    ca, cb = a[0], b[0]
    n = int(max(ca.max(), cb.max())) + 1
    if not np.array_equal(np.bincount(ca, minlength=n), np.bincount(cb, minlength=n)):
        return False
    for q in range(1, 6):
        va, vb = a[q].view(np.float32).astype(np.float64), b[q].view(np.float32).astype(np.float64)
        sa, sb = np.bincount(ca, va, minlength=n), np.bincount(cb, vb, minlength=n)
        tol = (1e-6 if q < 3 else 1e-6 * np.abs(vb).max()) * np.bincount(cb, minlength=n)
        if not np.all(np.abs(sa - sb) <= tol):
            return False
    return True


def _state(sim):
    return (sim.get_density().cpu().numpy(), sim.get_current().cpu().numpy(),
            [sim.get_field(f).cpu().numpy() for f in range(6)],
            [_multiset(sim, s) for s in range(sim.nspecies)])


@pytest.mark.parametrize("timing,pot", [(False, {}), (True, {}), (False, dict(pot_mode=2, morse_a=3.0)),
                                        (False, dict(lattice=1)), (False, dict(pot_mode=3))],
                         ids=["graph", "timing", "morse", "hcp", "eam"])
def test_batch_equals_single_runs(gb, timing, pot):
    """Every slab of a batch ends with the same grids (bit for bit) and the same particles as the
    same slab run alone (graph replay and the direct-launch timing path alike, and with the Morse
    instance of the batched kernel), across cell sorts."""
    ws = [dict(w, **pot) for w in small_sweep()]
    batch = gb.Batch(ws, sort_every=3)
    if timing:
        gb.pic_batch_set_timing(batch.b, True)
    batch.step(7)
    for i, w in enumerate(ws):
        single = gb.Simulation(w, sort_every=3)
        single.step(7)
        a, b = _state(batch.slabs[i]), _state(single)
        assert np.array_equal(a[0], b[0]), f"density of slab {i}"
        assert np.array_equal(a[1], b[1]), f"current of slab {i}"
        for f in range(6):
            assert np.array_equal(a[2][f], b[2][f]), f"field {f} of slab {i}"
        for s in range(len(a[3])):
            assert _same_particles(a[3][s], b[3][s]), f"species {s} of slab {i}"
        assert batch.slabs[i].info()["step"] == 7
        single.close()
    if timing:
        ms, n = gb.pic_batch_get_timing(batch.b)
        assert ms[0] > 0 and n[0] == 7
    batch.close()


def test_batch_slab_refuses_pic_step(gb):
    batch = gb.Batch(small_sweep()[:2])
    h = batch.slabs[0].h
    assert gb.load_library().pic_step(h, 1) == gb.PIC_ESTATE
    batch.close()


def test_full_sweep_initialises_and_steps(gb):
    """The 16-slab sweep (256^2 ... 1024^2 cells, 105.6 M particles): every slab holds its
    particles, and a few steps keep the node density equal to a fresh deposit of the particles."""
    ws = batched_sweep()
    batch = gb.Batch(ws)
    total = sum(sum(s.info()["num_particles"]) for s in batch.slabs)
    assert total == 105_596_928
    batch.step(3)
    for i in (0, 7, 15):
        sl = batch.slabs[i]
        fresh, _ = sl.deposit_density()
        assert torch.equal(fresh, sl.get_density()), i
        assert fresh.sum().item() == sl.info()["num_particles"][0] * 2 ** 32
    batch.close()


def test_autotuner_picks_and_caches(gb, tmp_path, monkeypatch):
    from paper_1502_07722_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "cache.json"))
    ws = small_sweep()
    r = autotune.tune_batch(ws, tiles=(8, 16), sorts=(2, 4), warmup=1)
    assert r["tile"] in (8, 16) and r["sort_every"] in (2, 4)
    assert len(r["trials"]) == 4 and r["ms_per_step"] == min(t["ms_per_step"] for t in r["trials"])
    again = autotune.tune_batch(ws, tiles=(8, 16), sorts=(2, 4), warmup=1)
    assert again == r                      # served from the cache


def _match(x1, z1, ox, oz, nx, nz):
    """Index of the oracle particle each GPU particle is (the cell sort at the start of the step
    reorders the GPU's particles; particles of one species are distinct points, far apart compared
    with the FP32 rounding of a step). Checked to be a bijection."""
    from scipy.spatial import cKDTree
    tree = cKDTree(np.stack([np.mod(ox, nx), oz], 1), boxsize=[nx, 4 * nz])
    d, idx = tree.query(np.stack([np.mod(x1, nx), z1], 1))
    assert len(np.unique(idx)) == len(idx) and d.max() < 1e-3
    return idx


@pytest.mark.parametrize("slab", [1, 2])
def test_batch_slab_step_matches_oracle(gb, slab):
    """A slab of a batch against the FP64 oracle directly (not against the single-run GPU path):
    the three-slab sweep runs 3 steps with a cell sort every 3 steps, so the compared step starts
    with a sort that rewrites the batch's argument table. The oracle takes the slab's state before
    that step (particles, fields, step count); after one step of the batch and one of the oracle
    the particles agree to 1e-5 (matched by position: the sort reorders them), the current and the
    node density equal the oracle's deposition of the GPU's own move bit for bit, and the fields
    equal the oracle's Maxwell update from the same start and current to 1e-5."""
    pytest.importorskip("scipy")
    import oracle
    from tests.test_gpu_parity import to_global
    oracle.build()
    ws = small_sweep()
    batch = gb.Batch(ws, sort_every=3)
    batch.step(3)
    sl, w = batch.slabs[slab], ws[slab]
    nx, nz = w["nx"], w["nz"]
    orc = oracle.Oracle(w, with_particles=False)
    before = []
    for sp in (0, 1):
        before.append(to_global(sl.get_particles(sp), nx))
        orc.set_particles(sp, before[sp][0], before[sp][1], *before[sp][2])
    fields = [sl.get_field(f).cpu().numpy().astype(np.float64) for f in range(6)]
    for f, a in enumerate(fields):
        orc.set_field(f, a)
    n0 = sl.info()["step"]
    orc.set_step(n0)
    assert np.array_equal(sl.get_density().cpu().numpy(), orc.get_rho())
    batch.step(1)
    orc.step(1)
    J = np.zeros((3, nz + 1, nx), np.int64)
    for sp, sign in ((0, 1), (1, -1)):
        x1, z1, u1 = to_global(sl.get_particles(sp), nx)
        o = orc.get_particles(sp)
        idx = _match(x1, z1, o["x"], o["z"], nx, nz)
        x0, z0 = before[sp][0][idx], before[sp][1][idx]
        # displacement to 1e-5 relative plus the FP32 rounding of the offset (2^-22 cells)
        dx = np.mod(o["x"][idx] - x0 + nx / 2, nx) - nx / 2
        assert (np.abs(np.mod(x1 - o["x"][idx] + nx / 2, nx) - nx / 2) <= 1e-5 * np.abs(dx) + 2.0 ** -22).all()
        assert (np.abs(z1 - o["z"][idx]) <= 1e-5 * np.abs(o["z"][idx] - z0) + 2.0 ** -22).all()
        for c, comp in enumerate(("ux", "uy", "uz")):
            ref = o[comp][idx]
            np.testing.assert_allclose(u1[c], ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())
        oracle.deposit_current(nx, nz, sign, x0, z0, x1, z1, *[v.astype(np.float32) for v in u1], out=J)
    assert np.array_equal(sl.get_current().cpu().numpy(), J)
    x1, z1, _ = to_global(sl.get_particles(0), nx)
    assert np.array_equal(sl.get_density().cpu().numpy(), oracle.deposit_density(nx, nz, x1, z1))
    fo = oracle.Oracle(w, with_particles=False)
    for f, a in enumerate(fields):
        fo.set_field(f, a)
    fo.set_step(n0)
    fo.set_current(J)
    fo.maxwell()
    for f in range(6):
        a = sl.get_field(f).cpu().numpy().astype(np.float64)
        b = fo.get_field(f)
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())
    batch.close()
