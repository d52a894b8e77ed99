"""Named synthetic copper-slab workloads (physical inputs only, no method arithmetic).

Each workload is a dict of physical parameters for a 2D3V run: grid, slab, species, laser and
pair potential. The numbers follow the paper's copper target (solid density 8.5e22 cm^-3,
10 nm cells, 800 nm pulse at normal incidence) with the sizes of the benchmark workloads. The
pulse peak time is placed at mid-run for each workload's step count (the runs are shorter
than the pulse, so the run sees the pulse centre). Dissociation energy D is an assumption:
the paper takes D and r0 from its Ref. 10 without printing them; r0 = 0 selects
r0 = n^(-1/3), so the unperturbed slab sits at the potential minimum.
"""
from __future__ import annotations

COPPER = dict(
    dx=10e-9,                  # m (transport-stage cell size in the paper)
    cfl=0.95,                  # dt = 0.95 dx / (c sqrt 2)
    dt_override=0.0,
    n_atoms=8.5e28,            # m^-3 (8.5e22 cm^-3)
    T_ion_K=300.0,
    T_electron_eV=1.0,
    ion_charge=1.0,            # Cu+
    ion_mass_amu=63.546,
    D_eV=0.41,                 # assumed (not printed in the paper)
    r0=0.0,                    # 0 -> n_atoms^(-1/3)
    c_att=1.0,
    s_rep=1.0,
    pot_mode=0,
    # embedded-atom form (pot_mode 3): Johnson's analytic nearest-neighbour EAM for copper
    # (Phys. Rev. B 37, 3924, 1988), its published fcc values used as they are on the cubic lattice
    # (an assumption: the paper names no EAM parameters)
    eam_ec=3.54, eam_phi=0.59, eam_alpha=5.09, eam_beta=5.85, eam_gamma=8.00,
    mode=0,
    **{"lambda": 800e-9},
    tau_fwhm=30e-15,
)

# dt of the copper grids: 0.95 * 10 nm / (c sqrt 2) in 2D, / (c sqrt 3) in 3D
DT_2D = 2.2407216199121996e-17
DT_3D = 1.829541541469147e-17

WORKLOADS = {
    # 64 x 64 cells, slab in the lower half, 8 + 8 ppc, plane wave 1e13 W/cm^2, 200 steps
    "tiny": dict(COPPER, nx=64, nz=64, slab_k=32, ppc_ion=8, ppc_electron=8, laser_profile=1,
                 I0=1e17, w0=0.0, t_peak=100 * DT_2D, seed=1, steps=200),
    # 2048 x 2048 cells, slab depth 1024, 32 + 32 ppc, 2 um focus at 5e13 W/cm^2, 2000 steps
    "large2d": dict(COPPER, nx=2048, nz=2048, slab_k=1024, ppc_ion=32, ppc_electron=32, laser_profile=2,
                    I0=5e17, w0=2e-6, t_peak=1000 * DT_2D, seed=2, steps=2000, sort_every=160),
    # 1024 x 1024 cells, slab depth 512, 32 + 32 ppc (33.5 M particles, state larger than L2):
    # the same per-cell load as large2d at a quarter of the size, for profiling captures
    "mid2d": dict(COPPER, nx=1024, nz=1024, slab_k=512, ppc_ion=32, ppc_electron=32, laser_profile=2,
                  I0=5e17, w0=2e-6, t_peak=1000 * DT_2D, seed=3, steps=2000),
    # 512 x 512 cells, 16 + 16 ppc, 2 um focus at 3e13 W/cm^2, 200 steps
    "diff512": dict(COPPER, nx=512, nz=512, slab_k=256, ppc_ion=16, ppc_electron=16, laser_profile=2,
                    I0=3e17, w0=2e-6, t_peak=100 * DT_2D, seed=5, steps=200),
    # differentiable form: 512 x 512 cells, 16 + 16 ppc, 2 um focus at 3e13 W/cm^2, 200 steps with a
    # checkpoint every 20. The slab fills rows k < 448 so that the antenna (row 510) is 62 cells
    # above the surface and the pulse, whose peak reaches the surface at step 100, acts within the
    # run (7,340,032 particles)
    "differentiable": dict(COPPER, nx=512, nz=512, slab_k=448, ppc_ion=16, ppc_electron=16, laser_profile=2,
                           I0=3e17, w0=2e-6, t_peak=100 * DT_2D, seed=6, steps=200),
    # 3D: 384 x 384 x 256 cells, slab in the lower 128 z-cells, 8 + 8 ppc (302 M particles),
    # Gaussian focus 1.5 um waist at 1e14 W/cm^2, 500 steps
    "3d": dict(COPPER, dims=3, nx=384, ny=384, nz=256, slab_k=128, ppc_ion=8, ppc_electron=8, laser_profile=2,
               I0=1e18, w0=1.5e-6, t_peak=250 * DT_3D, seed=3, steps=500),
    # 3D at an eighth of the size (37.7 M particles), for profiling captures
    "small3d": dict(COPPER, dims=3, nx=192, ny=192, nz=128, slab_k=64, ppc_ion=8, ppc_electron=8, laser_profile=2,
                    I0=1e18, w0=1.5e-6, t_peak=250 * DT_3D, seed=4, steps=500),
    # atomic-transport stage: neutral Cu, 12 fs steps, hot slab (pair force only, no fields)
    "transport": dict(COPPER, nx=64, nz=64, slab_k=32, ppc_ion=16, ppc_electron=0, mode=1,
                      ion_charge=0.0, T_ion_K=3000.0, dt_override=12e-15, laser_profile=0,
                      I0=0.0, w0=0.0, t_peak=0.0, seed=7, steps=1000),
    # atomic-transport crater run (paper: 10 nm cells, 12 fs steps, a 4.5-6 um wide and 0.75-1 um
    # thick copper target, several ns): 6 um x 1 um slab under 1.56 um of vacuum, 128 macro-atoms
    # per cell (7.68 M), started from the lattice temperature of a 1 um laser spot (synthetic: the
    # paper's Fig. 2 profile is not available), 250 000 steps = 3 ns
    "crater": dict(COPPER, nx=600, nz=256, slab_k=100, ppc_ion=128, ppc_electron=0, mode=1,
                   ion_charge=0.0, T_ion_K=300.0, dt_override=12e-15, laser_profile=0,
                   I0=0.0, w0=0.0, t_peak=0.0, temp_profile=1, T_spot_K=20000.0, spot_w=1e-6,
                   spot_depth=80e-9, seed=8, steps=250000),
}
# the same crater run with the Morse form of the pair force (pot_mode 2): stiffness
# a = alpha r0 = 1.3588 / A x 2.2744 A = 3.09, alpha from Girifalco and Weizer's copper Morse fit
# (Phys. Rev. 114, 687 (1959); not from the paper), r0 the cubic-lattice spacing at n0, depth D
# as for Eq. (3)
WORKLOADS["crater_morse"] = dict(WORKLOADS["crater"], pot_mode=2, morse_a=3.09)
# the crater run with the embedded-atom form (pot_mode 3, Johnson's copper values above)
WORKLOADS["crater_eam"] = dict(WORKLOADS["crater"], pot_mode=3)
# the same crater run on the hexagonal close-packed neighbour geometry (lattice 1, c axis along z)
WORKLOADS["crater_hcp"] = dict(WORKLOADS["crater"], lattice=1)
# the crater run in 3D: 3 um x 3 um x 1.6 um box, slab 1 um thick, 16 macro-atoms per cell
# (144 M), a round 1 um spot (radius from the axis through the middle of the x-y plane)
WORKLOADS["crater3d"] = dict(WORKLOADS["crater"], dims=3, nx=300, ny=300, nz=160, slab_k=100, ppc_ion=16, seed=9)


def workload(name: str, **overrides) -> dict:
    w = dict(WORKLOADS[name])
    w.update(overrides)
    return w


def batched_sweep(n=16, steps=1000):
    """Intensity sweep of independent copper slabs of uneven sizes: slab k has side
    16 * round(16 * 4^(k/15)) cells (256 ... 1024), (8, 16, 32) macroparticles per cell per
    species cycling with k, peak intensity 1e13 * 100^(k/15) W/cm^2 (log-spaced up to 1e15), the
    same pulse shape, slab in the lower half, seeds 100 + k."""
    out = []
    for k in range(n):
        side = 16 * round(16 * 4 ** (k / 15))
        ppc = (8, 16, 32)[k % 3]
        out.append(dict(COPPER, nx=side, nz=side, slab_k=side // 2, ppc_ion=ppc, ppc_electron=ppc,
                        laser_profile=2, w0=2e-6, I0=1e17 * 100 ** (k / 15), t_peak=(steps // 2) * DT_2D,
                        seed=100 + k, steps=steps))
    return out
