"""The box store's candidate lists, built on the host (no GPU).

The distance grid's node value is the minimum over the scene's boxes of the
box signed distance (the grid's definition, appendix "Additional
Collision-Detection Details").  The box store keeps, per cell of 16 node
intervals per axis, a list of boxes; the kernels take the minimum over the
list of the lattice cell whose lower corner lies in that cell, for all eight
corners.  So the property that makes the store exact is: for every lattice
cell, the list of its store cell holds a box reaching the minimum at each of
its eight corners.  Checked here by brute force in FP64 over every box, on a
room and on an apartment with 118 boxes, for random lattice cells and for the
cells on store-cell boundaries (where the corner at 16c + 16 is still read
with the list of store cell c)."""
import numpy as np
import pytest

from paper_2306_07552_b300 import build as B
from paper_2306_07552_b300 import gx
from paper_2306_07552_b300 import inputs as I


@pytest.fixture(scope="module")
def lib():
    B.build()
    return gx.lib()


def _sd_all(scene, nodes):
    """FP64 signed distance of every box at lattice nodes [n][3] -> [n][boxes]."""
    o = scene.grid_origin.astype(np.float64)
    p = o + nodes * np.float64(scene.grid_h)
    b = scene.boxes.astype(np.float64)
    c, e = (b[:, :3] + b[:, 3:]) / 2, (b[:, 3:] - b[:, :3]) / 2
    q = np.abs(p[:, None, :] - c[None]) - e[None]
    return np.sqrt((np.maximum(q, 0) ** 2).sum(-1)) + np.minimum(q.max(-1), 0)


def _check_cells(scene, dims, off, ids, cells):
    """cells: lattice cells [n][3] (lower corners).  Every corner's minimum
    over all boxes must be reached by a box of the store cell's list."""
    nb = len(scene.boxes)
    sc = np.minimum(cells // 16, dims - 1)
    ci = (sc[:, 2] * dims[1] + sc[:, 1]) * dims[0] + sc[:, 0]
    member = np.zeros((len(cells), nb), bool)
    for c in np.unique(ci):
        member[np.ix_(np.flatnonzero(ci == c), ids[off[c]:off[c + 1]].astype(np.int64))] = True
    worst = 0.0
    for v in range(8):
        corner = cells + np.array([v & 1, (v >> 1) & 1, v >> 2])
        sd = _sd_all(scene, corner)
        best = sd.min(1)
        listed = np.where(member, sd, np.inf).min(1)
        assert np.array_equal(listed, best), (v, np.max(listed - best))
        worst = max(worst, float(np.max(listed - best)))
    return worst


@pytest.mark.parametrize("which", ["room", "apartment"])
def test_box_store_lists_hold_the_nearest_box(lib, which):
    if which == "room":
        scene = I.room_scene(1000, 2000)
    else:
        scene = I.make_scenes(I.WORKLOADS["uneven16384_nsdf"], only=[3])[0]
    dims, off, ids = gx.box_store_lists(scene)
    n = np.asarray(scene.grid_dims, np.int64)
    assert list(dims) == [max(1, -(-(int(a) - 1) // 16)) for a in n]
    assert off[0] == 0 and np.all(np.diff(off.astype(np.int64)) >= 0)
    assert len(ids) == off[-1] and np.all(ids < len(scene.boxes))
    for c in range(len(off) - 1):          # each list sorted, no repeats
        assert np.all(np.diff(ids[off[c]:off[c + 1]].astype(np.int64)) > 0)
    lengths = np.diff(off.astype(np.int64))
    print(f"{which}: {len(scene.boxes)} boxes, {len(lengths)} store cells, list length mean "
          f"{lengths.mean():.2f}, max {lengths.max()}")
    assert lengths.min() >= 1
    assert lengths.mean() <= 0.25 * len(scene.boxes)    # the lists are selective
    rng = np.random.default_rng(3)
    cells = rng.integers(0, n - 1, (40_000, 3))
    # lattice cells whose upper corners sit on a store-cell boundary
    edge = rng.integers(0, n - 1, (8_000, 3))
    for a in range(3):
        edge[a::3, a] = np.minimum((edge[a::3, a] // 16) * 16 + 15, n[a] - 2)
    _check_cells(scene, dims, off, ids, np.concatenate([cells, edge]))


def test_box_store_lists_reject_bad_scenes(lib):
    scene = I.room_scene(1000, 2000)
    bad = I.room_scene(1000, 2000)
    bad.grid_dims = np.array([1, 5, 5], np.int32)
    with pytest.raises(gx.GxError):
        gx.box_store_lists(bad)
    bad = I.room_scene(1000, 2000)
    bad.boxes = np.zeros((0, 6), np.float32)
    with pytest.raises(gx.GxError):
        gx.box_store_lists(bad)
    gx.box_store_lists(scene)
