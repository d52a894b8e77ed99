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
