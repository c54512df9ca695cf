"""Oracle of the image-space ground-truth passes: outlines and occlusion boundaries.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): only the tests, the smoke check and the
benchmark's CPU baseline use it.  Plain NumPy, written from the definitions below, sharing nothing
with the CUDA library.

The paper lists both passes among its ground truth (Sec. III-D) without formulas:

* "Outlines Ground Truth": the edges of the transparent objects highlighted with a chosen
  thickness, e.g. 1 px or 20 px.  Reading: pixel p is on the outline of thickness T when it shows a
  transparent object (mask[p] != 0) and some pixel q of the image within Chebyshev distance T
  (max(|dx|, |dy|) <= T) shows another object or the background (instance_id[q] !=
  instance_id[p]): an inner band T pixels wide along the silhouette, including where two objects
  meet.
* "Occlusion Boundaries Ground Truth": where transparent objects touch another surface, marked
  where the depth is discontinuous (after ClearGrasp).  Reading, per transparent pixel p and its
  four edge neighbours q inside the image: a depth discontinuity between p and q is a relative jump
  |d_p - d_q| > jump_rel * min(d_p, d_q) between finite depths, or q a miss (infinite depth) while
  p is a hit.  p gets code 1 (occlusion boundary) if it is the nearer side of a discontinuity with
  some neighbour; otherwise code 2 (contact edge) if some neighbour shows another object or
  surface without a discontinuity; otherwise 0.  Non-transparent pixels get 0.
"""
from __future__ import annotations

import numpy as np


def outline(instance_id: np.ndarray, mask: np.ndarray, thickness: int) -> np.ndarray:
    """uint8 [H, W]: 1 on the outline band of thickness `thickness` (Sec. III-D "Outlines")."""
    ids = np.asarray(instance_id)
    H, W = ids.shape
    T = int(thickness)
    differs = np.zeros((H, W), dtype=bool)
    for dy in range(-T, T + 1):
        for dx in range(-T, T + 1):
            # pixels p whose neighbour p + (dx, dy) lies inside the image
            y0, y1 = max(0, -dy), min(H, H - dy)
            x0, x1 = max(0, -dx), min(W, W - dx)
            if y0 >= y1 or x0 >= x1:
                continue
            differs[y0:y1, x0:x1] |= ids[y0:y1, x0:x1] != ids[y0 + dy:y1 + dy, x0 + dx:x1 + dx]
    return (differs & (np.asarray(mask) != 0)).astype(np.uint8)


def depth_discontinuity(dp, dq, jump_rel):
    """Elementwise: a relative depth jump between finite depths, or a hit next to a miss."""
    dp = np.asarray(dp, np.float64)
    dq = np.asarray(dq, np.float64)
    both = np.isfinite(dp) & np.isfinite(dq)
    jump = np.zeros(np.broadcast(dp, dq).shape, dtype=bool)
    jump[both] = np.abs(dp[both] - dq[both]) > jump_rel * np.minimum(dp[both], dq[both])
    return jump | (np.isfinite(dp) & np.isinf(dq)) | (np.isinf(dp) & np.isfinite(dq))


def occlusion_boundaries(instance_id: np.ndarray, mask: np.ndarray, depth: np.ndarray,
                         jump_rel: float) -> np.ndarray:
    """uint8 [H, W]: 1 occlusion boundary, 2 contact edge, 0 otherwise (Sec. III-D "Occlusion
    Boundaries"), from the pixel-centre instance ids, transparency mask and Euclidean depth."""
    ids = np.asarray(instance_id)
    d = np.asarray(depth, np.float64)
    H, W = ids.shape
    nearer_side = np.zeros((H, W), dtype=bool)
    contact = np.zeros((H, W), dtype=bool)
    for dy, dx in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        y0, y1 = max(0, -dy), min(H, H - dy)
        x0, x1 = max(0, -dx), min(W, W - dx)
        if y0 >= y1 or x0 >= x1:
            continue
        dp = d[y0:y1, x0:x1]
        dq = d[y0 + dy:y1 + dy, x0 + dx:x1 + dx]
        disc = depth_discontinuity(dp, dq, jump_rel)
        nearer_side[y0:y1, x0:x1] |= disc & (dp < dq)
        contact[y0:y1, x0:x1] |= ids[y0:y1, x0:x1] != ids[y0 + dy:y1 + dy, x0 + dx:x1 + dx]
    transparent = np.asarray(mask) != 0
    out = np.zeros((H, W), dtype=np.uint8)
    out[transparent & contact] = 2
    out[transparent & nearer_side] = 1
    return out


def occlusion_margin(depth: np.ndarray, jump_rel: float) -> np.ndarray:
    """Per pixel, the smallest relative distance of a neighbour comparison to the jump threshold,
    | |d_p - d_q| - jump_rel min(d_p, d_q) | / (jump_rel min(d_p, d_q)) over the four neighbours with
    finite depths (inf where none): small values mark decisions an FP32 evaluation may take the
    other way."""
    d = np.asarray(depth, np.float64)
    H, W = d.shape
    out = np.full((H, W), np.inf)
    for dy, dx in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        y0, y1 = max(0, -dy), min(H, H - dy)
        x0, x1 = max(0, -dx), min(W, W - dx)
        if y0 >= y1 or x0 >= x1:
            continue
        dp = d[y0:y1, x0:x1]
        dq = d[y0 + dy:y1 + dy, x0 + dx:x1 + dx]
        ok = np.isfinite(dp) & np.isfinite(dq)
        thr = jump_rel * np.minimum(dp, dq)
        m = np.full(dp.shape, np.inf)
        m[ok] = np.abs(np.abs(dp[ok] - dq[ok]) - thr[ok]) / np.maximum(thr[ok], 1e-300)
        out[y0:y1, x0:x1] = np.minimum(out[y0:y1, x0:x1], m)
    return out
