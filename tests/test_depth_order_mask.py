"""The depth-order exclusion of the full-size parity tests
(helpers.depth_order_ambiguous), checked against the oracle itself: swapping
every pair of adjacent list entries whose depths lie within the rule's
relative gap changes only pixels the rule flags."""
import numpy as np

import scenes
from helpers import depth_order_ambiguous


def _swapped(proj, bins, rel):
    """The pair list with each adjacent pair of near-equal depth swapped."""
    vals = bins["vals"].copy()
    depth = proj["depth"]
    for s, e in bins["ranges"]:
        k = int(s)
        while k + 1 < e:
            a, b = vals[k], vals[k + 1]
            if abs(depth[b] - depth[a]) <= rel * abs(depth[b]):
                vals[k], vals[k + 1] = b, a
                k += 2
            else:
                k += 1
    return dict(keys=bins["keys"], vals=vals, ranges=bins["ranges"], P=bins["P"])


def test_swaps_change_only_flagged_pixels(ora):
    W, H = 96, 64
    scene = scenes.random_scene(n=20000, seed=41, xy_range=0.8, log_scale_mean=-3.2)
    # depths on a few planes, jittered far below the FP32 resolution of a
    # rotated camera: many near-equal depths overlap at the same pixels
    rng = np.random.default_rng(0)
    plane = rng.integers(0, 12, scene["means"].shape[0])
    scene["means"][:, 2] = (2.5 + 0.125 * plane + rng.uniform(-1e-7, 1e-7, plane.shape)).astype(np.float32)
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H)
    bins = ora.bin_pairs(proj)
    rel = 6e-7
    a = ora.render(proj, bins)
    b = ora.render(proj, _swapped(proj, bins, rel))
    pa = np.concatenate([a["C"], a["grads"].reshape(9, H, W)])
    pb = np.concatenate([b["C"], b["grads"].reshape(9, H, W)])
    scale = np.maximum(np.abs(pa).max(axis=(1, 2), keepdims=True), 1e-12)
    changed = np.any(np.abs(pa - pb) > 1e-6 * scale, axis=0)
    ys, xs = np.mgrid[0:H, 0:W]
    flagged = depth_order_ambiguous(proj, bins, np.stack([xs.ravel(), ys.ravel()], 1), rel=rel).reshape(H, W)
    assert changed.any()                       # the case exercises the rule
    assert not np.any(changed & ~flagged), int((changed & ~flagged).sum())
    assert flagged.mean() < 0.9
