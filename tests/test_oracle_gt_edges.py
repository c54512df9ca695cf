"""Pins of the outline and occlusion-boundary oracle (oracle/gt_edges.py) against a library
morphology routine and shapes whose answer is known in closed form.  No GPU."""
import numpy as np
import pytest

from oracle import gt_edges as G


def _blocky_ids(seed, h=37, w=53, n_obj=5):
    """Random axis-aligned rectangles of ids over a background of -1 (later ones on top)."""
    rng = np.random.default_rng(seed)
    ids = np.full((h, w), -1, np.int32)
    for k in range(n_obj):
        y0, x0 = rng.integers(0, h - 4), rng.integers(0, w - 4)
        y1, x1 = y0 + rng.integers(3, h // 2), x0 + rng.integers(3, w // 2)
        ids[y0:y1, x0:x1] = k
    mask = (ids >= 0) & (ids % 2 == 0)
    return ids, mask.astype(np.uint8)


@pytest.mark.parametrize("T", [1, 2, 5, 20])
def test_outline_matches_grey_morphology(T):
    """Inner band of thickness T = transparent pixels where the (2T+1)^2 window's minimum or maximum
    id differs from the pixel's own (scipy.ndimage filters, edge-replicating borders)."""
    from scipy import ndimage

    for seed in range(4):
        ids, mask = _blocky_ids(seed)
        lo = ndimage.minimum_filter(ids, size=2 * T + 1, mode="nearest")
        hi = ndimage.maximum_filter(ids, size=2 * T + 1, mode="nearest")
        expect = ((lo != ids) | (hi != ids)) & (mask != 0)
        np.testing.assert_array_equal(G.outline(ids, mask, T), expect.astype(np.uint8))


@pytest.mark.parametrize("T", [1, 3, 7])
def test_outline_of_a_rectangle_is_its_inner_band(T):
    h, w = 40, 60
    ids = np.full((h, w), -1, np.int32)
    r0, r1, c0, c1 = 8, 30, 12, 50
    ids[r0:r1, c0:c1] = 4
    mask = (ids == 4).astype(np.uint8)
    y, x = np.mgrid[0:h, 0:w]
    inside = ids == 4
    dist = np.minimum(np.minimum(y - r0, r1 - 1 - y), np.minimum(x - c0, c1 - 1 - x))
    np.testing.assert_array_equal(G.outline(ids, mask, T), (inside & (dist < T)).astype(np.uint8))
    # a rectangle against the image border: the border itself is not an edge
    ids2 = np.full((h, w), -1, np.int32)
    ids2[:, :20] = 1
    out = G.outline(ids2, (ids2 == 1).astype(np.uint8), T)
    assert out[:, : 20 - T].sum() == 0 and (out[:, 20 - T:20] == 1).all() and out[:, 20:].sum() == 0


def test_outline_between_two_touching_objects():
    ids = np.zeros((10, 10), np.int32)
    ids[:, 5:] = 1
    out = G.outline(ids, np.ones_like(ids, np.uint8), 2)
    assert (out[:, 3:7] == 1).all() and out[:, :3].sum() == 0 and out[:, 7:].sum() == 0
    # only transparent pixels are marked
    out = G.outline(ids, (ids == 1).astype(np.uint8), 2)
    assert out[:, :5].sum() == 0 and (out[:, 5:7] == 1).all()


def test_occlusion_boundary_codes():
    h, w = 12, 16
    ids = np.full((h, w), 0, np.int32)
    ids[:, 8:] = 1
    depth = np.ones((h, w))
    mask = np.ones((h, w), np.uint8)
    # a depth step of 50 % between the halves: the nearer (left) column is the occlusion boundary
    depth[:, 8:] = 1.5
    out = G.occlusion_boundaries(ids, mask, depth, 0.05)
    assert (out[:, 7] == 1).all()          # nearer side of the jump
    assert (out[:, 8] == 2).all()          # farther side: another object without being nearer
    assert out[:, :7].sum() == 0 and out[:, 9:].sum() == 0
    # a jump below the threshold is a contact edge on both sides
    depth[:, 8:] = 1.02
    out = G.occlusion_boundaries(ids, mask, depth, 0.05)
    assert (out[:, 7] == 2).all() and (out[:, 8] == 2).all()
    # the threshold is relative to the nearer depth: 1.0 -> 1.05 is a jump at 4.8 % (not at 5.04 %)
    depth[:, 8:] = 1.05
    out = G.occlusion_boundaries(ids, mask, depth, 0.048)
    assert (out[:, 7] == 1).all()
    out = G.occlusion_boundaries(ids, mask, depth, 0.0505)
    assert (out[:, 7] == 2).all()
    # a smooth ramp inside one object (2 % per pixel): nothing
    ramp = np.tile(1.0 + 0.02 * np.arange(w), (h, 1))
    assert G.occlusion_boundaries(np.zeros((h, w), np.int32), mask, ramp, 0.05).sum() == 0
    # a hit next to a miss (background, depth inf): occlusion boundary on the hit side
    ids3 = np.full((h, w), -1, np.int32)
    ids3[3:9, 4:12] = 2
    d3 = np.full((h, w), np.inf)
    d3[3:9, 4:12] = 2.0
    out = G.occlusion_boundaries(ids3, (ids3 == 2).astype(np.uint8), d3, 0.05)
    ring = np.zeros((h, w), bool)
    ring[3:9, 4:12] = True
    ring[4:8, 5:11] = False
    np.testing.assert_array_equal(out == 1, ring)
    assert (out[~ring] == 0).all()
    # non-transparent pixels carry no code
    out = G.occlusion_boundaries(ids3, np.zeros((h, w), np.uint8), d3, 0.05)
    assert out.sum() == 0


def test_occlusion_margin_marks_near_threshold_jumps():
    d = np.ones((4, 4))
    d[:, 2:] = 1.05 * (1 + 1e-9)
    m = G.occlusion_margin(d, 0.05)
    assert m[:, 1].max() < 1e-6 and (m[:, 0] == 1.0).all()  # equal depths: a whole threshold away
