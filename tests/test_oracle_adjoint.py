"""Pin of the oracle's reverse-mode gradient (continuous-deposition transport stage) against
central finite differences of the same forward run (h = 1e-4 relative)."""
import numpy as np
import pytest

import oracle
from paper_1502_07722_gb300.workloads import workload


def small_transport(seed=11):
    w = workload("transport", nx=12, nz=12, slab_k=6, ppc_ion=4, T_ion_K=3000.0, seed=seed)
    return w


def crater_weights(nx, nz, ks, dx):
    """Depth functional of the smooth crater depth: -dx * (uniform weights over x) on rows k < ks."""
    cw = np.zeros((nz + 1, nx))
    cw[:ks] = -dx / nx
    return cw


@pytest.mark.parametrize("kin", [0.0, 1e3])
def test_transport_gradient_matches_central_differences(kin):
    w = small_transport()
    nsteps = 25
    cw = crater_weights(w["nx"], w["nz"], w["slab_k"], w["dx"])
    o = oracle.Oracle(w)
    D0, r00 = o.D, o.r0
    L, gD, gr0 = o.transport_grad(nsteps, cw, kin)
    ref = oracle.Oracle(w)
    assert ref.transport_loss(nsteps, cw, kin, D0, r00) == pytest.approx(L, rel=1e-13)
    for which, g in (("D", gD), ("r0", gr0)):
        v = D0 if which == "D" else r00
        h = 1e-4 * v
        args_p = (D0 + h, r00) if which == "D" else (D0, r00 + h)
        args_m = (D0 - h, r00) if which == "D" else (D0, r00 - h)
        fd = (ref.transport_loss(nsteps, cw, kin, *args_p) - ref.transport_loss(nsteps, cw, kin, *args_m)) / (2 * h)
        assert g == pytest.approx(fd, rel=1e-5), which
        assert g != 0.0


# ---- full cycle (ions, electrons, fields, laser) --------------------------------------------

def small_full(seed=21, **kw):
    d = dict(nx=12, nz=14, slab_k=8, ppc_ion=2, ppc_electron=2, laser_profile=1, I0=1e18,
             t_peak=10 * 2.24e-17, T_electron_eV=5.0, seed=seed)
    d.update(kw)
    return workload("tiny", **d)


def test_maxwell_transpose_dot_product():
    """<lam, M(F, j)> = <M^T lam, (F, j)> for random fields, currents and adjoints (antenna off),
    and the E0 derivative equals <lam, M(0, 0; E0 = 1)> (the antenna's field)."""
    w = small_full()
    o = oracle.Oracle(w, with_particles=False)
    rng = np.random.default_rng(3)
    shp = (w["nz"] + 1, w["nx"])
    F = rng.normal(size=(6,) + shp)
    j = rng.normal(size=(3,) + shp)
    lam = rng.normal(size=(6,) + shp)
    step = 9
    MF = o.maxwell_cont(F, j, 0.0, step)
    lF, lj, gE0 = o.maxwell_cont_T(lam, step)
    lhs = float((lam * MF).sum())
    rhs = float((lF * F).sum() + (lj * j).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12)
    ant = o.maxwell_cont(np.zeros((6,) + shp), np.zeros((3,) + shp), 1.0, step)
    assert np.abs(ant).max() > 0
    assert gE0 == pytest.approx(float((lam * ant).sum()), rel=1e-12)


@pytest.mark.parametrize("kin", [0.0, 1e-3])
def test_full_cycle_gradient_matches_central_differences(kin):
    """dL/dD, dL/dr0 and dL/dI0 of the reverse sweep against central differences (h = 1e-4
    relative) of the same continuous forward run. Light ions (1e-3 u) and D = 10 eV: with copper
    at the plasma time step the pair force moves an ion by less than the FP64 resolution of its
    position in 12 steps, and a finite difference of the loss would be rounding noise; the
    reverse sweep does not depend on the values (its truncation order shows as h^2 convergence)."""
    w = small_full(ion_mass_amu=1e-3, D_eV=10.0)
    nsteps = 12
    cw = crater_weights(w["nx"], w["nz"], w["slab_k"], w["dx"])
    o = oracle.Oracle(w)
    D0, r00, I00 = o.D, o.r0, w["I0"]
    L, gD, gr0, gI0 = o.full_grad(nsteps, cw, kin)
    assert o.full_loss(nsteps, cw, kin, D0, r00, I00) == pytest.approx(L, rel=1e-13)
    base = {"D": D0, "r0": r00, "I0": I00}
    for which, g in (("D", gD), ("r0", gr0), ("I0", gI0)):
        h = 1e-4 * base[which]
        p = dict(base); p[which] += h
        m = dict(base); m[which] -= h
        fd = (o.full_loss(nsteps, cw, kin, p["D"], p["r0"], p["I0"]) -
              o.full_loss(nsteps, cw, kin, m["D"], m["r0"], m["I0"])) / (2 * h)
        assert g == pytest.approx(fd, rel=2e-5), which
        assert g != 0.0


def test_full_cycle_reduces_to_transport_without_fields():
    """In the neutral-atom mode the full-cycle reverse sweep is the transport one."""
    w = small_transport()
    cw = crater_weights(w["nx"], w["nz"], w["slab_k"], w["dx"])
    a = oracle.Oracle(w).full_grad(10, cw, 1e3)
    b = oracle.Oracle(w).transport_grad(10, cw, 1e3)
    np.testing.assert_allclose(a[:3], b, rtol=1e-11)
