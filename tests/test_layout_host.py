"""Host checks of the storage-order helpers the GPU layout tests use: the block layout is a
permutation of every tile size, and a full block puts consecutive runs of the cell order in rows
(lane l of warp c holds place 32 l + c of a 1024-block)."""
import numpy as np

from tests.sort_layout import layout_order, undo_layout


def test_layout_is_a_permutation():
    for B in (256, 1024):
        for nt in list(range(1, 70)) + [255, 256, 257, 1023, 1024, 1025, 3000, 16384]:
            assert np.array_equal(np.sort(layout_order(nt, B)), np.arange(nt))


def test_full_block_rows():
    order = layout_order(2048, 1024)
    for blk in (0, 1):
        for c in (0, 5, 31):
            lanes = order[blk * 1024 + 32 * c: blk * 1024 + 32 * c + 32] - blk * 1024
            assert np.array_equal(lanes, 32 * np.arange(32) + c)


def test_undo_layout_round_trip():
    rng = np.random.default_rng(3)
    key = np.sort(rng.integers(0, 4 * 256, 5000))             # cell order, 4 tiles of 256 keys
    stored = np.empty_like(key)
    _, starts = undo_layout(key, 256, 1024)
    for a, b in zip(starts[:-1], starts[1:]):
        stored[a + np.argsort(layout_order(b - a, 1024))] = key[a:b]
    back, _ = undo_layout(stored, 256, 1024)
    assert np.array_equal(back, key)
