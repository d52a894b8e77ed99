"""Host restatement of the cell sort's storage order, for the tests: the tile-major cell key and
the block layout inside a tile (blocks of B places of the cell order stored column by column as
32-row matrices)."""
import numpy as np


def cell_key(cell, nx, ny, T, dims):
    i = cell % nx
    q = cell // nx
    if dims == 2:
        k = q
        ntx = -(-nx // T)
        return ((k // T) * ntx + i // T) * T * T + (k % T) * T + (i % T)
    j, k = q % ny, q // ny
    ntx, nty = -(-nx // T), -(-ny // T)
    tile = ((k // T) * nty + j // T) * ntx + i // T
    return ((tile * T + k % T) * T + j % T) * T + i % T


def layout_order(nt, B):
    """order[u] = place in the cell order of the particle stored at slot u of a tile of nt."""
    order = np.empty(nt, np.int64)
    for b0 in range(0, nt, B):
        nb = min(B, nt - b0)
        C = (nb + 31) // 32
        R, rem = nb // C, nb % C
        j = np.arange(nb)
        r, c = j // C, j % C
        order[b0 + c * R + np.minimum(c, rem) + r] = b0 + j
    return order


def undo_layout(key, TT, B):
    """Keys in cell order: storage order is tile-major (checked), each tile laid out by blocks."""
    tile = key // TT
    assert (np.diff(tile) >= 0).all()
    out = np.empty_like(key)
    starts = np.flatnonzero(np.r_[True, np.diff(tile) != 0, True])
    for a, b in zip(starts[:-1], starts[1:]):
        out[a + layout_order(b - a, B)] = key[a:b]
    return out, starts
