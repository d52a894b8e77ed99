"""Failure detection of the step, through the C ABI and without any GPU fault: the particle
kernel flags a non-finite momentum or a move of a cell or more in a status word, the host turns it
into a sticky error code, and every later call that would compute on the broken state refuses.
Invalid input is refused before it reaches a kernel."""
import numpy as np
import pytest

from paper_1502_07722_gb300.workloads import workload

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


def _rest_lattice(nx, nz, ppc_rows):
    cells = np.arange(nx * ppc_rows, dtype=np.int32)
    n = len(cells)
    f = np.full(n, 0.5, np.float32)
    z = np.zeros(n, np.float32)
    return cells, f, f.copy(), z, z.copy(), z.copy()


def test_move_of_a_cell_or_more_is_a_sticky_error(gb):
    """Transport stage, 12 fs steps: an atom at u = 0.01 (3000 km/s) would cross 3.6 cells."""
    w = workload("transport", nx=32, nz=32, slab_k=16, ppc_ion=1, T_ion_K=0.0)
    sim = gb.Simulation(w, sort_every=0)
    cell, fx, fz, ux, uy, uz = _rest_lattice(32, 32, 16)
    ux[100] = 0.01
    sim.set_particles(0, cell, fx, fz, ux, uy, uz)
    with pytest.raises(gb.PicError) as e:
        sim.step(1)
    assert e.value.code == gb.PIC_EMOVE
    with pytest.raises(gb.PicError) as e:            # sticky
        sim.step(1)
    assert e.value.code == gb.PIC_EMOVE
    with pytest.raises(gb.PicError):
        sim.energy()
    sim.close()


def test_non_finite_momentum_is_a_sticky_error(gb):
    w = workload("tiny", nx=32, nz=32, slab_k=16, ppc_ion=1, ppc_electron=1)
    sim = gb.Simulation(w, sort_every=0)
    p = sim.get_particles(1)
    uy = p["uy"].clone()
    uy[7] = float("nan")
    sim.set_particles(1, p["cell"], p["fx"], p["fz"], p["ux"], uy, p["uz"])
    with pytest.raises(gb.PicError) as e:
        sim.step(1)
    assert e.value.code == gb.PIC_ENAN
    with pytest.raises(gb.PicError) as e:
        sim.step(2)
    assert e.value.code == gb.PIC_ENAN
    sim.close()


def test_invalid_particles_are_refused_before_any_kernel(gb):
    w = workload("tiny", nx=32, nz=32, slab_k=16, ppc_ion=1, ppc_electron=1)
    sim = gb.Simulation(w)
    p = sim.get_particles(0)
    bad_cell = p["cell"].clone()
    bad_cell[3] = 32 * 32                            # one past the last cell
    with pytest.raises(gb.PicError) as e:
        sim.set_particles(0, bad_cell, p["fx"], p["fz"], p["ux"], p["uy"], p["uz"])
    assert e.value.code == gb.PIC_EINVAL
    bad_f = p["fx"].clone()
    bad_f[3] = 1.0                                   # offsets live in [0, 1)
    with pytest.raises(gb.PicError) as e:
        sim.set_particles(0, p["cell"], bad_f, p["fz"], p["ux"], p["uy"], p["uz"])
    assert e.value.code == gb.PIC_EINVAL
    # the context is unharmed: the valid state steps on
    sim.set_particles(0, p["cell"], p["fx"], p["fz"], p["ux"], p["uy"], p["uz"])
    sim.step(2)
    sim.close()


def test_particle_pile_up_beyond_the_fixed_point_range_is_a_sticky_error(gb):
    """The int64 node sums are proven exact while a block of 4 x 4 cells (the cells whose particles
    can reach one node) holds at most 1365 particles in the 2D full mode at the 2^18 J_y code. A
    host-made state piles 1200 electrons into one cell of a slab of 8 + 8 per cell: the sort that
    follows pic_set_particles finds the crowded block, and the next step reports the sticky
    PIC_EOVERFLOW; the seeded slab (256 per block) runs on."""
    extra = 1200
    w = workload("tiny", nx=32, nz=32, slab_k=16, max_particles=32 * 16 * 8 + extra)
    sim = gb.Simulation(w, sort_every=0)
    sim.step(1)                                        # the seeded slab (8 + 8 per cell) is fine
    p = sim.get_particles(1)
    n0 = p["cell"].numel()
    cell = torch.cat([p["cell"], torch.full((extra,), 5 * 32 + 7, dtype=torch.int32, device=p["cell"].device)])
    f = torch.linspace(0.05, 0.95, extra, device=p["cell"].device)
    fx, fz = torch.cat([p["fx"], f]), torch.cat([p["fz"], f.flip(0)])
    z = torch.zeros(extra, device=p["cell"].device)
    ux, uy, uz = (torch.cat([p[k], z]) for k in ("ux", "uy", "uz"))
    sim.set_particles(1, cell, fx, fz, ux, uy, uz)
    assert sim.info()["num_particles"][1] == n0 + extra
    with pytest.raises(gb.PicError) as e:
        sim.step(1)
    assert e.value.code == gb.PIC_EOVERFLOW
    with pytest.raises(gb.PicError) as e:              # sticky
        sim.step(1)
    assert e.value.code == gb.PIC_EOVERFLOW
    sim.close()
