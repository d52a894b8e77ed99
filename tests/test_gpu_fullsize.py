"""Parity at the benchmark sizes, in the launch configuration bench.py times (2048 x 2048 cells,
134,217,728 particles; 384 x 384 x 256 cells, 301,989,888 particles; tile and sort interval as in
the bench): sampled particles checked one by one against the oracle (their initial draws; one
step from the GPU's own fields and node density), and a property that holds at any size (the
incrementally updated node density equals a fresh deposit of the particles, bit for bit)."""
import numpy as np
import pytest

import oracle
from paper_1502_07722_gb300.workloads import workload

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

NSAMPLE = 3000


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1502_07722_gb300 import _build
    _build.build()
    import paper_1502_07722_gb300 as m
    return m


def _sample(sim, sp, idx):
    p = sim.get_particles(sp)
    keys = [k for k in ("cell", "fx", "fy", "fz", "ux", "uy", "uz") if k in p]
    out = {k: p[k].index_select(0, idx).cpu().numpy() for k in keys}
    del p
    torch.cuda.empty_cache()
    return out


def _coords(s, g):
    """cell index -> integer coordinates (2D: i, k; 3D: i, j, k) and positions in cells"""
    c = s["cell"].astype(np.int64)
    if "fy" in s:
        i, j, k = c % g[0], (c // g[0]) % g[1], c // (g[0] * g[1])
        return (i, j, k), (i + s["fx"].astype(np.float64), j + s["fy"].astype(np.float64),
                           k + s["fz"].astype(np.float64))
    i, k = c % g[0], c // g[0]
    return (i, k), (i + s["fx"].astype(np.float64), k + s["fz"].astype(np.float64))


def _check_init(sim, orc, w, dims):
    """Each sampled particle is one of its cell's slots: positions bit-exact, momenta to FP32."""
    rng = np.random.default_rng(17)
    for sp in range(sim.nspecies):
        n = sim.info()["num_particles"][sp]
        idx = torch.from_numpy(rng.integers(0, n, NSAMPLE)).cuda()
        s = _sample(sim, sp, idx)
        ijk, pos = _coords(s, (w["nx"], w.get("ny", 1)))
        ppc = w["ppc_ion"] if sp == 0 else w["ppc_electron"]
        u = [s[k].astype(np.float64) for k in ("ux", "uy", "uz")]
        scale = max(np.abs(a).max() for a in u)
        for q in range(NSAMPLE):
            cell = [int(a[q]) for a in ijk]
            found = False
            for slot in range(ppc):
                v = orc.init_particle(sp, *cell, slot)
                if all(v[d] == pos[d][q] for d in range(dims)):
                    for d in range(3):
                        assert abs(v[dims + d] - u[d][q]) <= 1e-6 * abs(v[dims + d]) + 1e-7 * scale
                    found = True
                    break
            assert found, (sp, q, cell)


def _check_one_step(gb, sim, orc, w, dims):
    """One step of the benchmark configuration against the oracle's push of the same particles
    from the GPU's own fields and node density (1e-5 of the displacement / momentum)."""
    rng = np.random.default_rng(29)
    idx = {}
    before = {}
    for sp in range(sim.nspecies):
        n = sim.info()["num_particles"][sp]
        idx[sp] = torch.from_numpy(rng.integers(0, n, NSAMPLE)).cuda()
        before[sp] = _sample(sim, sp, idx[sp])
    for f in range(6):
        orc.set_field(f, sim.get_field(f).cpu().numpy().astype(np.float64))
    orc.set_rho(sim.get_density().cpu().numpy())
    sim.step(1)                                           # no cell sort on this step: same order
    shape = [w["nx"]] + ([w["ny"]] if dims == 3 else []) + [w["nz"]]
    for sp in range(sim.nspecies):
        after = _sample(sim, sp, idx[sp])
        _, p0 = _coords(before[sp], (w["nx"], w.get("ny", 1)))
        _, p1 = _coords(after, (w["nx"], w.get("ny", 1)))
        u0 = [before[sp][k].astype(np.float64) for k in ("ux", "uy", "uz")]
        u1 = [after[k].astype(np.float64) for k in ("ux", "uy", "uz")]
        scale = max(np.abs(a).max() for a in u1)
        for q in range(NSAMPLE):
            v = orc.push_one(sp, [p[q] for p in p0] + [a[q] for a in u0])
            for d in range(dims):
                L = shape[d]
                disp = abs(((v[d] - p0[d][q]) + L / 2) % L - L / 2)
                err = abs(((p1[d][q] - v[d]) + L / 2) % L - L / 2)
                assert err <= 1e-5 * disp + 2.0 ** -22, (sp, q, d)
            for d in range(3):
                assert abs(u1[d][q] - v[dims + d]) <= 1e-5 * abs(v[dims + d]) + 1e-6 * scale, (sp, q, d)
    fresh, _ = sim.deposit_density()
    assert torch.equal(fresh, sim.get_density())


@pytest.mark.parametrize("name", ["large2d", "3d"])
def test_full_size_against_oracle(gb, name):
    w = workload(name)
    dims = 3 if w.get("dims") == 3 else 2
    sim = gb.Simulation(w, sort_every=40)
    orc = (oracle.Oracle3D if dims == 3 else oracle.Oracle)(w, with_particles=False)
    _check_init(sim, orc, w, dims)
    _check_one_step(gb, sim, orc, w, dims)
    info = sim.info()
    assert sum(info["num_particles"]) == (134217728 if dims == 2 else 301989888)
    sim.close()
