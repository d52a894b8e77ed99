"""Checkpoint/resume and the differentiable transport stage on the GPU, through the C-ABI:
bit-exact resume from a checkpoint, and dL/dD, dL/dr0 of the adjoint kernels against the FP64
oracle's reverse-mode gradient (continuous deposition) on the same initial state."""
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
    import paper_1502_07722_gb300 as m
    return m


def _state(sim):
    ps = []
    for s in range(sim.nspecies):
        p = sim.get_particles(s)
        arr = np.stack([p[k].cpu().numpy().view(np.int32) for k in ("cell", "fx", "fz", "ux", "uy", "uz")])
        ps.append(arr[:, np.lexsort(arr[::-1])])     # a cell sort orders equal cells arbitrarily
    return (sim.get_density().cpu().numpy(), sim.get_current().cpu().numpy(),
            [sim.get_field(f).cpu().numpy() for f in range(6)], ps, sim.info()["step"])


def _equal(a, b):
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for f in range(6):
        assert np.array_equal(a[2][f], b[2][f]), f
    for s in range(len(a[3])):
        assert np.array_equal(a[3][s], b[3][s]), s
    assert a[4] == b[4]


def test_checkpoint_resume_bit_exact(gb):
    w = workload("tiny", laser_profile=2, w0=0.2e-6, I0=1e19, t_peak=5 * 2.24e-17)
    sim = gb.Simulation(w, sort_every=3)
    sim.step(5)
    ck = sim.checkpoint()
    sim.step(7)
    a = _state(sim)
    sim.restore(ck)
    assert sim.info()["step"] == 5
    sim.step(7)
    _equal(a, _state(sim))
    sim.close()


def test_checkpoint_to_disk_resumes_in_a_new_context(gb, tmp_path):
    """A host checkpoint written to a file and restored into a fresh context of the same
    configuration continues exactly like the original context (with the injected-energy sum)."""
    w = workload("tiny", laser_profile=2, w0=0.2e-6, I0=1e19, t_peak=5 * 2.24e-17)
    sim = gb.Simulation(w, sort_every=3)
    sim.step(6)
    path = tmp_path / "state.ckpt"
    sim.checkpoint(on_host=True).numpy().tofile(path)
    sim.step(5)
    a, ea = _state(sim), sim.energy()
    sim.close()
    other = gb.Simulation(w, sort_every=3, seed=w["seed"] + 99)     # a different initial slab
    buf = torch.from_numpy(np.fromfile(path, dtype=np.uint8)).pin_memory()
    other.restore(buf)
    assert other.info()["step"] == 6
    other.step(5)
    _equal(a, _state(other))
    eb = other.energy()
    for k in ("kinetic_ion", "kinetic_electron", "field_E", "field_B", "pair", "injected"):
        assert ea[k] == eb[k], k
    other.close()


def test_checkpoint_rejects_foreign_buffers(gb):
    sim = gb.Simulation(workload("tiny"))
    junk = torch.zeros(gb.pic_checkpoint_size(sim.h), dtype=torch.uint8)
    with pytest.raises(gb.PicError):
        sim.restore(junk)
    sim.close()


def small_transport(**kw):
    d = dict(nx=24, nz=24, slab_k=12, ppc_ion=4, T_ion_K=3000.0, seed=11)
    d.update(kw)
    return workload("transport", **d)


def _weights(w):
    cw = np.zeros((w["nz"] + 1, w["nx"]))
    cw[: w["slab_k"]] = -w["dx"] / w["nx"]
    return cw


def _gpu_grad(gb, w, nsteps, kin, every, grid=False, orc=None, full=False):
    """GPU loss and gradient; with grid=True the initial offsets are first rounded to the 2^-16
    deposition grid (so the GPU's fixed-point density of the initial state is the continuous one).
    orc, if given, receives the same initial state."""
    from paper_1502_07722_gb300 import diff
    o = oracle.Oracle(w, with_particles=False)
    run = diff.DiffRun(w, o.D, o.r0, None, every)
    for s in range(run.sim.nspecies):
        p = run.sim.get_particles(s)
        cell = p["cell"].cpu().numpy().astype(np.int64)
        fx = p["fx"].cpu().numpy().astype(np.float64)
        fz = p["fz"].cpu().numpy().astype(np.float64)
        if grid:
            fx = np.minimum(np.round(fx * 65536) / 65536, 65535 / 65536)
            fz = np.minimum(np.round(fz * 65536) / 65536, 65535 / 65536)
            u = [p[k].cpu().numpy() for k in ("ux", "uy", "uz")]
            run.sim.set_particles(s, cell.astype(np.int32), fx.astype(np.float32), fz.astype(np.float32), *u)
        if orc is not None:
            u = [p[k].cpu().numpy().astype(np.float64) for k in ("ux", "uy", "uz")]
            orc.set_particles(s, cell % w["nx"] + fx, cell // w["nx"] + fz, *u)
    wt = torch.tensor(_weights(w), dtype=torch.float64, device="cuda")
    L = run.forward(nsteps, wt, kin)
    gD, gR, gI = run.backward(wt, kin)
    run.close()
    return (L, gD, gR, gI) if full else (L, gD, gR)


def _both(gb, w, nsteps, kin, every=7, grid=True):
    o = oracle.Oracle(w, with_particles=False)
    g = _gpu_grad(gb, w, nsteps, kin, every, grid=grid, orc=o)
    return g, o.transport_grad(nsteps, _weights(w), kin)


def rel(a, b):
    return abs(a - b) / abs(b)


def test_adjoint_seed_only(gb):
    """Zero steps on the deposition grid: L is the node functional of the initial density,
    dL/dD = 0 and dL/dr0 = 3 L / r0 -- the oracle's to summation order."""
    (L, gD, gR), (Lo, gDo, gRo) = _both(gb, small_transport(), 0, 0.0)
    assert rel(L, Lo) < 1e-12 and rel(gR, gRo) < 1e-12
    assert gD == 0.0 and gDo == 0.0


def test_adjoint_seed_only_off_grid(gb):
    """Initial offsets off the 2^-16 grid: the fixed-point density differs from the continuous one
    by the rounding of each offset (< 2^-17 cell), ~1e-8 of L here."""
    (L, gD, gR), (Lo, gDo, gRo) = _both(gb, small_transport(), 0, 0.0, grid=False)
    assert rel(L, Lo) < 1e-7 and rel(gR, gRo) < 1e-7


@pytest.mark.parametrize("kin", [0.0, 2e3])
@pytest.mark.parametrize("nsteps", [1, 5])
def test_adjoint_few_steps_match_oracle(gb, kin, nsteps):
    """From the same initial state on the deposition grid, the GPU's fixed-point moves differ from
    the oracle's continuous ones by rounding only: gradients agree to ~1e-6."""
    (L, gD, gR), (Lo, gDo, gRo) = _both(gb, small_transport(), nsteps, kin)
    assert rel(L, Lo) < 1e-6
    assert rel(gD, gDo) < 2e-5 and rel(gR, gRo) < 2e-5


def test_adjoint_one_step_off_grid(gb):
    """Off-grid initial offsets: the quantized deposition shifts the force by ~1e-5 of a cell's
    density step; the kinetic-energy gradient stays within 1e-3."""
    (L, gD, gR), (Lo, gDo, gRo) = _both(gb, small_transport(), 1, 2e3, grid=False)
    assert rel(L, Lo) < 1e-6
    assert rel(gD, gDo) < 1e-3 and rel(gR, gRo) < 1e-3


@pytest.mark.parametrize("T", [300.0, 3000.0, 30000.0])
def test_adjoint_many_steps_match_oracle(gb, T):
    (L, gD, gR), (Lo, gDo, gRo) = _both(gb, small_transport(T_ion_K=T), 20, 2e3)
    assert rel(L, Lo) < 1e-6
    assert rel(gD, gDo) < 5e-5 and rel(gR, gRo) < 5e-5


# Runs of the reverse pass differ only in the order of the FP64 atomic sums on the nodes; read
# back into the FP32 particle adjoints, those last-bit differences move the gradients by ~1e-7.
RERUN = 1e-5


def test_adjoint_checkpoint_interval_invariance(gb):
    """The gradient does not depend on the checkpoint interval (recomputed states are the saved
    ones bit for bit)."""
    w = small_transport()
    res = [_gpu_grad(gb, w, 20, 2e3, every) for every in (1, 7, 20)]
    for L, gD, gR in res[1:]:
        assert L == res[0][0]
        assert rel(gD, res[0][1]) < RERUN and rel(gR, res[0][2]) < RERUN


def test_autograd_function(gb):
    from paper_1502_07722_gb300 import diff
    w = small_transport()
    o = oracle.Oracle(w, with_particles=False)
    D = torch.tensor(o.D, dtype=torch.float64, requires_grad=True)
    r0 = torch.tensor(o.r0, dtype=torch.float64, requires_grad=True)
    wt = torch.tensor(_weights(w), dtype=torch.float64, device="cuda")
    L = diff.transport_loss(D, r0, w, 6, wt, 2e3, 4)
    L.backward()
    _, gD, gR = _gpu_grad(gb, w, 6, 2e3, 3)
    assert rel(D.grad.item(), gD) < RERUN and rel(r0.grad.item(), gR) < RERUN


def test_adjoint_refuses_other_modes(gb):
    """With the cell sort on (the particle order changes) the adjoint is refused before any launch."""
    import ctypes
    sim = gb.Simulation(workload("tiny"), sort_every=5)
    b = gb.pic_adjoint_buffers()
    lib = gb.load_library()
    assert lib.pic_adjoint_step(sim.h, ctypes.byref(b)) == gb.PIC_ESTATE
    sim.close()


# ---- full cycle (ions, electrons, fields, laser) --------------------------------------------

def small_full(**kw):
    d = dict(nx=12, nz=14, slab_k=8, ppc_ion=2, ppc_electron=2, laser_profile=1, I0=1e18,
             t_peak=10 * 2.24e-17, T_electron_eV=5.0, seed=21)
    d.update(kw)
    return workload("tiny", **d)


def _both_full(gb, w, nsteps, kin, every=7):
    o = oracle.Oracle(w, with_particles=False)
    g = _gpu_grad(gb, w, nsteps, kin, every, grid=True, orc=o, full=True)
    return g, o.full_grad(nsteps, _weights(w), kin)


def test_full_seed_only(gb):
    (L, gD, gR, gI), (Lo, gDo, gRo, gIo) = _both_full(gb, small_full(), 0, 0.0)
    assert rel(L, Lo) < 1e-12 and rel(gR, gRo) < 1e-12
    assert gD == gDo == 0.0 and gI == gIo == 0.0


@pytest.mark.parametrize("kin", [0.0, 1e-3])
@pytest.mark.parametrize("nsteps", [1, 6, 12])
def test_full_cycle_gradient_matches_oracle(gb, kin, nsteps):
    """Same initial state on the deposition grid; the GPU runs the fixed-point FP32 cycle forward
    and the FP64 adjoint kernels backward, the oracle the continuous FP64 cycle and its exact
    reverse sweep. The I0 derivative is that of a ~1e-5 share of the kinetic energy (the pulse
    against 5 eV electrons), so the forward's FP32 and fixed-point rounding shows more there."""
    (L, gD, gR, gI), (Lo, gDo, gRo, gIo) = _both_full(gb, small_full(), nsteps, kin)
    assert rel(L, Lo) < 1e-4
    assert rel(gD, gDo) < 3e-4 and rel(gR, gRo) < 2e-4
    if gIo != 0.0:
        assert rel(gI, gIo) < 2e-2


def test_full_cycle_intensity_gradient_cold_electrons(gb):
    """Cold electrons (0.01 eV) in a stronger pulse: the absorbed energy is the pulse's, and its
    I0 derivative follows the oracle closely."""
    w = small_full(T_electron_eV=0.01, I0=1e19)
    (L, gD, gR, gI), (Lo, gDo, gRo, gIo) = _both_full(gb, w, 12, 1e-3)
    assert gIo > 0.0
    assert rel(L, Lo) < 1e-4 and rel(gI, gIo) < 2e-3


def test_full_cycle_checkpoint_interval_invariance(gb):
    w = small_full()
    res = [_gpu_grad(gb, w, 12, 1e-3, every, full=True) for every in (1, 5, 12)]
    for r in res[1:]:
        assert r[0] == res[0][0]
        for q in (1, 2, 3):
            assert rel(r[q], res[0][q]) < RERUN


def test_full_cycle_autograd(gb):
    from paper_1502_07722_gb300 import diff
    w = small_full()
    o = oracle.Oracle(w, with_particles=False)
    D = torch.tensor(o.D, dtype=torch.float64, requires_grad=True)
    r0 = torch.tensor(o.r0, dtype=torch.float64, requires_grad=True)
    I0 = torch.tensor(w["I0"], dtype=torch.float64, requires_grad=True)
    wt = torch.tensor(_weights(w), dtype=torch.float64, device="cuda")
    L = diff.pic_loss(D, r0, I0, w, 8, wt, 1e-3, 3)
    L.backward()
    _, gD, gR, gI = _gpu_grad(gb, w, 8, 1e-3, 4, full=True)
    assert rel(D.grad.item(), gD) < RERUN and rel(r0.grad.item(), gR) < RERUN and rel(I0.grad.item(), gI) < RERUN
