"""Storage order written by the cell sort, read back through the C ABI.

The sort groups a species by tile (tile-major cell key) and stores each block of B particles of a
tile's cell order (B = 1024 in 2D, 256 in 3D) column by column as a 32-row matrix, so that the
particle kernels, reading records in storage order, give the 32 lanes of a warp particles in
neighbouring cells. The test undoes that layout on the host and checks that the result is the
cell order (keys non-decreasing inside each tile), that the tiles follow each other in order, and
that in a full block every warp's 32 particles sit in 32 distinct cells when each cell holds
B / 32 particles. The layout itself changes no result: every deposit is an exact integer sum.
"""
import numpy as np
import pytest

from paper_1502_07722_gb300.workloads import workload
from tests.sort_layout import cell_key, undo_layout

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


@pytest.mark.parametrize("dims", [2, 3])
def test_sort_layout(gb, dims):
    if dims == 2:
        w = dict(workload("tiny"), ppc_ion=32, ppc_electron=32, tile=16)
        T, B, ny = 16, 1024, 1
    else:
        w = dict(workload("tiny"), dims=3, nx=24, ny=20, nz=16, slab_k=8, ppc_ion=8, ppc_electron=8, tile=10,
                 laser_profile=0)
        T, B, ny = 10, 256, 20
    sim = gb.Simulation(w)
    ppc = w["ppc_ion"]
    for sp in range(2):
        cell = sim.get_particles(sp)["cell"].cpu().numpy().astype(np.int64)
        key = cell_key(cell, w["nx"], ny, T, dims)
        ordered, starts = undo_layout(key, T ** dims, B)     # tiles contiguous, in order
        full_blocks = 0
        for a, b in zip(starts[:-1], starts[1:]):
            nt = b - a
            assert (np.diff(ordered[a:b]) >= 0).all()          # the cell order, undone
            # every cell of the initial slab holds ppc particles: a full block's warps span
            # 32 distinct cells when B / 32 == ppc
            for b0 in range(0, nt - B + 1, B):
                full_blocks += 1
                blk = cell[a + b0:a + b0 + B].reshape(B // 32, 32)
                if B // 32 == ppc:
                    assert all(len(set(row.tolist())) == 32 for row in blk)
        assert full_blocks > 0
    sim.close()
