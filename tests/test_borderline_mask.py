"""The per-pixel exclusion of the full-size parity tests
(helpers.borderline_pixel_mask), checked against the oracle itself.

A rect-borderline Gaussian is one whose tile rect FP32 rounding may move by a
tile.  Render the same projection twice: once with each such Gaussian listed
in every tile of its envelope rect, once only in the tiles of its core rect.
A pixel outside the mask must come out bit for bit the same both times, and
every pixel that differs must be in the mask."""
import numpy as np
import pytest

import scenes
from helpers import borderline_pixel_mask


def _rebin(proj, bins, rect_key):
    """The oracle's pair list with each borderline Gaussian listed in the tiles
    of proj[rect_key][i] instead of its own rect; order (tile, depth, id)."""
    tiles_x, tiles_y = proj["tiles_x"], proj["tiles_y"]
    drop = np.nonzero(proj["borderline"])[0]
    keep = ~np.isin(bins["vals"], drop.astype(np.uint32))
    keys, vals = [bins["keys"][keep]], [bins["vals"][keep]]
    dbits = proj["depth"].astype(np.float32).view(np.uint32).astype(np.uint64)
    for i in drop:
        r = proj[rect_key][i]
        if r[2] < r[0] or r[3] < r[1]:
            continue
        ty, tx = np.mgrid[r[1]:r[3] + 1, r[0]:r[2] + 1]
        t = (ty * tiles_x + tx).ravel().astype(np.uint64)
        keys.append((t << np.uint64(32)) | dbits[i])
        vals.append(np.full(t.shape, i, np.uint32))
    k, v = np.concatenate(keys), np.concatenate(vals)
    o = np.lexsort((v, k))
    k, v = k[o], v[o]
    tile = (k >> np.uint64(32)).astype(np.int64)
    T = tiles_x * tiles_y
    ranges = np.stack([np.searchsorted(tile, np.arange(T), "left"),
                       np.searchsorted(tile, np.arange(T), "right")], 1).astype(np.uint32)
    return dict(keys=k, vals=v, ranges=ranges, P=len(k))


@pytest.mark.parametrize("kw,W,H", [
    # scene-shaped (mixture) scenes where some borderline Gaussian reaches the
    # cut-off in an ambiguous tile: the 3-sigma square, not the alpha box, bounds
    # the rect of a Gaussian of high opacity
    (dict(n=50000, seed=3, opacity_logit_std=4.0, log_scale_mean=-3.0), 200, 120),
    (dict(n=100000, seed=1), 240, 136),
])
def test_mask_covers_every_changed_pixel(ora, kw, W, H):
    scene = scenes.mixture_scene(**kw)
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H)
    bins = ora.bin_pairs(proj)
    assert proj["borderline"].sum() > 0
    # the depth key of an existing pair is the FP32 depth's bit pattern
    i0 = int(bins["vals"][0])
    assert int(bins["keys"][0] & np.uint64(0xFFFFFFFF)) == int(np.float32(proj["depth"][i0]).view(np.uint32))
    wide = ora.render(proj, _rebin(proj, bins, "envelope"))
    narrow = ora.render(proj, _rebin(proj, bins, "core"))
    a = np.concatenate([wide["C"], wide["grads"].reshape(9, H, W)])
    b = np.concatenate([narrow["C"], narrow["grads"].reshape(9, H, W)])
    differs = np.any(a != b, axis=0)
    ys, xs = np.mgrid[0:H, 0:W]
    pix = np.stack([xs.ravel(), ys.ravel()], 1)
    mask = borderline_pixel_mask(proj, pix).reshape(H, W)
    assert differs.any()                      # the case exercises the mask
    assert not np.any(differs & ~mask), int((differs & ~mask).sum())
    assert mask.mean() < 0.05
