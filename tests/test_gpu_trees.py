"""Dependency trees of more than two generations on the GPU (Sec. 3.1.1).

Every image tile gets a three-generation tree of fragment tiles: the
generation-0 declaration names the generation-1 tiles, which declare the
generation-2 tiles, which declare the generation-3 ones.  All of a frame's
fragments are submitted in one shuffled order across generations (children
may arrive before their parents).  While one generation-3 tile is missing
the frame is refused as incomplete; once it arrives the frame composites,
and the image equals the oracle's composite of the union of the fragments
(the tree decides when a tile is complete, not how it blends)."""

import numpy as np
import pytest

from harness import scenes
from oracle import dfb_oracle as o
from paper_2305_07083_gb300 import dfb as D

from tests.gpu_helpers import GpuFrameBuffer, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-5


def three_generation_trees(sc, rng):
    """Per fragment (generation, children) and per tile the generation-0
    declaration, such that every tile with fragments has a complete tree of
    three generations (fewer when the tile has fewer than three)."""
    gen = np.zeros(sc.n, np.int32)
    children = np.zeros(sc.n, np.int32)
    declared = {}
    for t in range(sc.n_tiles):
        idx = rng.permutation(np.nonzero(sc.tile_ids == t)[0])
        n = len(idx)
        if n == 0:
            continue
        g1 = max(1, n // 3)
        g2 = (n - g1) // 2
        g3 = n - g1 - g2
        if g2 == 0:          # a generation must have a parent to declare it
            g2, g3 = g3, 0
        parts = [idx[:g1], idx[g1:g1 + g2], idx[g1 + g2:]]
        declared[t] = g1
        for level, members in enumerate(parts):
            gen[members] = level + 1
            nxt = len(parts[level + 1]) if level + 1 < 3 else 0
            # the next generation's count split at random among this one's tiles
            if len(members):
                split = rng.multinomial(nxt, np.ones(len(members)) / len(members))
                children[members] = split
    return gen, children, declared


@pytest.mark.parametrize("mode", [D.DFB_BLEND_DEPTH, D.DFB_BLEND_ORDERED])
def test_three_generations_shuffled_incomplete_then_complete(mode):
    rng = np.random.default_rng(77 + mode)
    W, H, T = 200, 136, 32
    n_tiles = (-(-W // T)) * (-(-H // T))
    counts = rng.integers(0, 9, n_tiles)
    counts[rng.random(n_tiles) < 0.2] = rng.integers(17, 30)   # some long tiles too
    sc = scenes.random_scene(W, H, T, counts, seed=31 + mode, alpha_max=0.6)
    gen, children, declared = three_generation_trees(sc, rng)
    assert gen.max() == 3
    r = to_dev(sc.rgba)
    d = to_dev(sc.depth)
    rb, db = T * T * 16, T * T * 4
    descs = [(int(sc.tile_ids[i]), float(sc.keys[i]), r.data_ptr() + i * rb,
              d.data_ptr() + i * db, 1.0, int(gen[i]), int(children[i])) for i in range(sc.n)]
    order = rng.permutation(sc.n)
    # withhold one generation-3 tile until the end
    last = int(np.nonzero(gen[order] == 3)[0][-1])
    withheld = order[last]
    first = np.delete(order, last)
    fb = GpuFrameBuffer(W, H, T, mode)
    fb.begin(0)
    for t, c in declared.items():
        D.dfb_set_tile_children(fb.h, t, c)
    D.dfb_submit_tiles_ex(fb.h, [descs[i] for i in first[: len(first) // 2]], D.DFB_PTR_DEVICE)
    D.dfb_submit_tiles_ex(fb.h, [descs[i] for i in first[len(first) // 2:]], D.DFB_PTR_DEVICE)
    with pytest.raises(D.DfbError) as e:
        fb.end()
    assert e.value.code == D.DFB_ERR_INCOMPLETE
    D.dfb_submit_tiles_ex(fb.h, [descs[withheld]], D.DFB_PTR_DEVICE)
    fb.end()
    want = o.composite_frame(W, H, T, mode, sc.tile_ids, sc.keys, sc.rgba.astype(np.float64),
                             sc.depth)
    got = fb.color().astype(np.float64)
    assert np.max(np.abs(got - want)) <= TOL
    fb.close()


def test_stray_generation_keeps_the_frame_open():
    """A generation-4 tile that no generation-3 tile declared makes the tree
    incomplete: end-of-frame refuses, launches nothing, and the frame stays
    open (a new frame cannot begin)."""
    rng = np.random.default_rng(5)
    W, H, T = 64, 64, 32
    sc = scenes.random_scene(W, H, T, np.array([6, 4, 5, 3]), seed=9)
    gen, children, declared = three_generation_trees(sc, rng)
    r = to_dev(sc.rgba)
    d = to_dev(sc.depth)
    rb, db = T * T * 16, T * T * 4
    descs = [(int(sc.tile_ids[i]), float(sc.keys[i]), r.data_ptr() + i * rb,
              d.data_ptr() + i * db, 1.0, int(gen[i]), int(children[i])) for i in range(sc.n)]
    fb = GpuFrameBuffer(W, H, T, D.DFB_BLEND_DEPTH)
    fb.begin(0)
    for t, c in declared.items():
        D.dfb_set_tile_children(fb.h, t, c)
    D.dfb_submit_tiles_ex(fb.h, descs[::-1], D.DFB_PTR_DEVICE)
    stray = descs[0][:5] + (4, 0)
    D.dfb_submit_tiles_ex(fb.h, [stray], D.DFB_PTR_DEVICE)
    launches = fb.stats()["kernel_launches"]
    with pytest.raises(D.DfbError) as e:
        fb.end()
    assert e.value.code == D.DFB_ERR_INCOMPLETE
    assert fb.stats()["kernel_launches"] == launches
    with pytest.raises(D.DfbError) as e:
        fb.begin(0)
    assert e.value.code == D.DFB_ERR_STATE
    fb.close()
