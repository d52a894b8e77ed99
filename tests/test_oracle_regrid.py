"""Pins of the oracle's cell-map regridding (the two-stage coupling between stages on different
cells: the paper's laser-interaction run uses much finer cells than its transport run and hands
over its lattice temperature). The remap is fixed by properties any conservative remap on grids
aligned at the slab surface and the laser axis must have: identity on equal grids, exact
replication under refinement by an integer factor, the block mean under coarsening, the
hand-computed partial cover of a constant field at the grid's edge, and conservation of the
integral of (T - fill) when the destination covers the source."""
import numpy as np
import pytest

import oracle


def test_regrid_equal_grids_is_the_identity():
    rng = np.random.default_rng(1)
    a = rng.uniform(300, 5000, (7, 9))
    g = (9, 1, 7, 2.5e-9, 4)
    np.testing.assert_allclose(oracle.regrid_cells(a, g, g, -1.0), a, rtol=1e-13)
    a3 = rng.uniform(300, 5000, (5, 6, 7))
    g3 = (7, 6, 5, 1e-8, 3)
    np.testing.assert_allclose(oracle.regrid_cells(a3, g3, g3, -1.0, dims=3), a3, rtol=1e-13)


@pytest.mark.parametrize("f", [2, 3])
def test_regrid_refinement_replicates_each_cell(f):
    """Cells of dx / f: each lies inside one parent cell (the surface row and the axis are shared),
    so it takes the parent's value, for odd and even extents. (With f = 3 the edges (k - s) dx / 3
    round, leaving slivers of ~1e-16 dx of overlap with the neighbouring parent: tolerance 1e-10.)"""
    rng = np.random.default_rng(f)
    for nx, nz, surf in ((8, 6, 3), (7, 5, 2)):
        a = rng.uniform(0, 1, (nz, nx))
        fine = oracle.regrid_cells(a, (nx, 1, nz, 1.0, surf), (f * nx, 1, f * nz, 1.0 / f, f * surf), 123.0)
        np.testing.assert_allclose(fine, np.repeat(np.repeat(a, f, axis=0), f, axis=1), rtol=1e-10)
    a3 = rng.uniform(0, 1, (4, 5, 6))
    fine3 = oracle.regrid_cells(a3, (6, 5, 4, 1.0, 2), (6 * f, 5 * f, 4 * f, 1.0 / f, 2 * f), 9.0, dims=3)
    np.testing.assert_allclose(fine3, np.repeat(np.repeat(np.repeat(a3, f, 0), f, 1), f, 2), rtol=1e-10)


def test_regrid_coarsening_is_the_block_mean():
    rng = np.random.default_rng(5)
    a = rng.uniform(0, 1, (6, 8))
    coarse = oracle.regrid_cells(a, (8, 1, 6, 1.0, 4), (4, 1, 3, 2.0, 2), -7.0)
    np.testing.assert_allclose(coarse, a.reshape(3, 2, 4, 2).mean(axis=(1, 3)), rtol=1e-12)
    a3 = rng.uniform(0, 1, (4, 6, 8))
    c3 = oracle.regrid_cells(a3, (8, 6, 4, 1.0, 2), (4, 3, 2, 2.0, 1), -7.0, dims=3)
    np.testing.assert_allclose(c3, a3.reshape(2, 2, 3, 2, 4, 2).mean(axis=(1, 3, 5)), rtol=1e-12)


def test_regrid_constant_field_at_the_grid_edge():
    """Source: 4 x 4 cells of 1 (x in [-2, 2], depth [-2, 2] about a surface at row 2) at the
    constant c; destination: 3 x 3 cells of 2 (x in [-3, 3], depth [-2, 4]). Each destination
    cell is c on the part the source covers and fill elsewhere: the outer columns are half
    covered, the two lower rows (depth [-2, 0] and [0, 2]) fully, the top row not at all."""
    c, fill = 7.0, 3.0
    a = np.full((4, 4), c)
    out = oracle.regrid_cells(a, (4, 1, 4, 1.0, 2), (3, 1, 3, 2.0, 1), fill)
    # rows: depth [-2, 0], [0, 2], [2, 4]; columns: x [-3, -1], [-1, 1], [1, 3]
    cover_z = np.array([1.0, 1.0, 0.0])
    cover_x = np.array([0.5, 1.0, 0.5])
    frac = cover_z[:, None] * cover_x[None, :]
    np.testing.assert_allclose(out, c * frac + fill * (1 - frac), rtol=1e-14)


@pytest.mark.parametrize("dims", [2, 3])
def test_regrid_conserves_the_integral(dims):
    """A destination of cells 0.61 / 0.37 of the source's (no common multiple nearby) that covers
    the whole source: the integral of (T - fill) over the destination equals that over the source."""
    rng = np.random.default_rng(7 + dims)
    if dims == 2:
        a = rng.uniform(300, 3000, (11, 13))
        sg, dg = (13, 1, 11, 0.37, 6), (10, 1, 9, 0.61, 4)
    else:
        a = rng.uniform(300, 3000, (5, 6, 7))
        sg, dg = (7, 6, 5, 0.37, 3), (6, 5, 5, 0.61, 2)
    fill = 300.0
    out = oracle.regrid_cells(a, sg, dg, fill, dims=dims)
    src_int = (a - fill).sum() * sg[3] ** dims
    dst_int = (out - fill).sum() * dg[3] ** dims
    assert dst_int == pytest.approx(src_int, rel=1e-12)
    # and the destination does cover it: its extent contains the source's
    for ns, nd in ((sg[0], dg[0]), (sg[1], dg[1])) if dims == 3 else ((sg[0], dg[0]),):
        assert nd * dg[3] / 2 >= ns * sg[3] / 2
    assert dg[4] * dg[3] >= sg[4] * sg[3] and (dg[2] - dg[4]) * dg[3] >= (sg[2] - sg[4]) * sg[3]
