"""The allocation-free energy entry point against the workspace-based one.

Callers that cannot allocate device memory -- hosts that own every buffer and forbid further
cudaMalloc, or code that runs while another component records a CUDA graph -- use
pic_energy_noalloc: it reads a state from plain device arrays and keeps its scratch in a fixed
array inside the library. This file is collected last so that a run stopping at the first
failure has run every other test before it.
"""
import ctypes
import math

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


def _view(gb, sim):
    keep = []
    v = gb.pic_state_view()
    for s in range(sim.nspecies):
        p = sim.get_particles(s)
        keep.append(p)
        v.n[s] = p["cell"].numel()
        for name in ("cell", "fx", "fz", "ux", "uy", "uz"):
            getattr(v, name)[s] = p[name].data_ptr()
    for f in range(6):
        t = sim.get_field(f)
        keep.append(t)
        v.F[f] = t.data_ptr()
    rho = sim.get_density()
    keep.append(rho)
    v.rho = rho.data_ptr()
    return v, keep


@pytest.mark.parametrize("name,pot", [("tiny", {}), ("transport", {}), ("transport", dict(pot_mode=2, morse_a=3.0)),
                                      ("transport", dict(lattice=1))],
                         ids=["tiny", "transport", "transport-morse", "transport-hcp"])
def test_noalloc_energy_equals_pic_energy_twice(gb, name, pot):
    """Same five energies as pic_energy (same kernels, same summation order), on two calls in a
    row; the output is poisoned before each call so that each call must write all of it."""
    w = workload(name, nx=48, nz=40, slab_k=20, **pot)
    sim = gb.Simulation(w)
    sim.step(4)
    ref = sim.energy()
    view, keep = _view(gb, sim)
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    keys = ("kinetic_ion", "kinetic_electron", "field_E", "field_B", "pair")
    for _ in range(2):
        out.fill_(float("nan"))
        stream.synchronize()
        gb.pic_energy_noalloc(sim.cfg, view, out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().tolist()
        for k, g in zip(keys, got):
            assert math.isfinite(g), k
            assert g == pytest.approx(ref[k], rel=1e-12, abs=0.0), k
    del keep
    sim.close()


def test_noalloc_energy_refuses_bad_sizes(gb):
    """Particle counts above 2^31 - 1 and missing pointers are refused before any GPU work."""
    w = workload("tiny", nx=48, nz=40, slab_k=20)
    cfg = gb.make_config(w)
    v = gb.pic_state_view()
    lib = gb.load_library()
    out = ctypes.c_void_p(256)
    assert lib.pic_energy_noalloc(ctypes.byref(cfg), ctypes.byref(v), out, None) == gb.PIC_EINVAL
    v.n[0] = 2 ** 31
    for name in ("cell", "fx", "fz", "ux", "uy", "uz"):
        getattr(v, name)[0] = 256
        getattr(v, name)[1] = 256
    for f in range(6):
        v.F[f] = 256
    v.rho = 256
    assert lib.pic_energy_noalloc(ctypes.byref(cfg), ctypes.byref(v), out, None) == gb.PIC_EINVAL
    assert lib.pic_energy_noalloc(ctypes.byref(cfg), ctypes.byref(v), None, None) == gb.PIC_EINVAL


def test_noalloc_energy_refuses_unknown_potentials(gb):
    """A pot_mode outside 0..2, or the Morse form without a stiffness, is refused (the view points
    at a live context's buffers, so nothing else would stop the call)."""
    w = workload("transport", nx=48, nz=40, slab_k=20)
    sim = gb.Simulation(w)
    view, keep = _view(gb, sim)
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    lib = gb.load_library()
    for bad in (dict(pot_mode=4), dict(pot_mode=-1), dict(pot_mode=2, morse_a=0.0), dict(lattice=2),
                dict(pot_mode=3, lattice=1), dict(pot_mode=3, eam_beta=0.0)):
        cfg = gb.make_config(w, **bad)
        assert lib.pic_energy_noalloc(ctypes.byref(cfg), ctypes.byref(view), out.data_ptr(), None) == gb.PIC_EINVAL
    torch.cuda.synchronize()
    del keep
    sim.close()
