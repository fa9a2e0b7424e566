"""Shared helpers for the GPU parity tests: running the CUDA path through the C
ABI binding and comparing its outputs with the oracle's.

Tolerances (from the FP32 arithmetic of the kernels against an FP64 reference):
  colour        max-abs 2e-4 (values in [0, 1])
  derivatives   |gpu - ref| <= 1e-3 * max(|ref|, rms of the reference plane)
  upscale       |gpu - ref| <= 2e-6 * (1 + max |input|) on identical inputs
Where the 3DGS mode takes a discrete decision close to its threshold (alpha at
1/255, the 0.99 clamp, the 1e-4 termination), FP32 may legitimately go the
other way; the oracle returns every such variant and a GPU pixel passes if it
matches one of them.  Pixels with more than three such decisions, and tiles
whose Gaussian set depends on a rect edge within FP32 rounding (oracle
"borderline" Gaussians), are excluded and counted.
"""
from __future__ import annotations

import numpy as np

TOL_C = 2e-4
TOL_G = 1e-3
TOL_UP = 2e-6


def borderline_tile_mask(proj) -> np.ndarray:
    """Pixels in the tiles whose membership of a borderline Gaussian can flip
    under FP32 rounding: its envelope rect minus its core rect (the tiles in
    every perturbed rect)."""
    W, H, tile = proj["W"], proj["H"], proj["tile"]
    tx, ty = proj["tiles_x"], proj["tiles_y"]
    mt = np.zeros((ty, tx), bool)
    for i in np.nonzero(proj["borderline"])[0]:
        e, c = proj["envelope"][i], proj["core"][i]
        if e[2] < e[0]:
            continue
        sub = np.ones((e[3] - e[1] + 1, e[2] - e[0] + 1), bool)
        if c[2] >= c[0]:
            sub[c[1] - e[1]:c[3] - e[1] + 1, c[0] - e[0]:c[2] - e[0] + 1] = False
        mt[e[1]:e[3] + 1, e[0]:e[2] + 1] |= sub
    return np.repeat(np.repeat(mt, tile, 0), tile, 1)[:H, :W]


def borderline_pixel_mask(proj, pix, margin: float = 1e-3) -> np.ndarray:
    """Sampled pixels [M, 2] of (x, y) that a rect-borderline Gaussian can
    change: in a tile of its envelope rect outside its core rect, with
    alpha = opacity e^g there at or above the 1/255 cut-off (less a relative
    margin).  Where alpha is below the cut-off the Gaussian is skipped whether
    or not the tile lists it, so the pixel is the same on both sides."""
    tile = proj["tile"]
    px, py = pix[:, 0].astype(np.int64), pix[:, 1].astype(np.int64)
    tx, ty = px // tile, py // tile
    out = np.zeros(len(px), bool)
    for i in np.nonzero(proj["borderline"])[0]:
        e, c = proj["envelope"][i], proj["core"][i]
        if e[2] < e[0]:
            continue
        sel = (tx >= e[0]) & (tx <= e[2]) & (ty >= e[1]) & (ty <= e[3]) & ~out
        if c[2] >= c[0]:
            sel &= ~((tx >= c[0]) & (tx <= c[2]) & (ty >= c[1]) & (ty <= c[3]))
        if not sel.any():
            continue
        a, b, cc = proj["conic"][i]
        dx = px[sel] - proj["mean2d"][i, 0]
        dy = py[sel] - proj["mean2d"][i, 1]
        g = -0.5 * (a * dx * dx + 2.0 * b * dx * dy + cc * dy * dy)
        out[np.nonzero(sel)[0]] = proj["opacity"][i] * np.exp(g) >= (1.0 - margin) / 255.0
    return out


def depth_order_ambiguous(proj, bins, pix, rel: float = 6e-7, overlap: float = 1e-5) -> np.ndarray:
    """Sampled pixels [M, 2] of (x, y) whose front-to-back order is not unique
    under FP32 depths: among the tile-list Gaussians that reach the pixel at or
    above the 1/255 cut-off (less a relative margin), two adjacent in the
    oracle's order have depths within rel of each other (an FP32 camera-space
    z, a three-term dot product plus a translation, is within a few units in
    the last place, relative 2^-24 each, of the FP64 one), both before the
    pixel's transmittance falls below 1e-4, and overlapping enough for their
    order to matter (T alpha_i alpha_j above `overlap`: swapping two layers
    changes the blend by T alpha_i alpha_j (c_i - c_j)).  The identity rotation
    keeps the FP32 depths exact."""
    tile, tiles_x = proj["tile"], proj["tiles_x"]
    out = np.zeros(len(pix), bool)
    for m, (x, y) in enumerate(np.asarray(pix, np.int64)):
        s, e = bins["ranges"][(y // tile) * tiles_x + x // tile]
        ids = bins["vals"][s:e].astype(np.int64)
        if len(ids) < 2:
            continue
        dx = x - proj["mean2d"][ids, 0]
        dy = y - proj["mean2d"][ids, 1]
        a, b, c = proj["conic"][ids].T
        alpha = proj["opacity"][ids] * np.exp(-0.5 * (a * dx * dx + 2.0 * b * dx * dy + c * dy * dy))
        live = alpha >= (1.0 - 1e-3) / 255.0
        d, al = proj["depth"][ids][live], np.minimum(alpha[live], 0.99)
        if len(d) < 2:
            continue
        T = np.concatenate([[1.0], np.cumprod(1.0 - al)[:-1]])     # transmittance before each layer
        reach = T > 1e-4 * (1.0 - 1e-3)
        close = np.abs(np.diff(d)) <= rel * np.abs(d[1:])
        out[m] = bool(np.any(close & reach[:-1] & (T[:-1] * al[:-1] * al[1:] > overlap)))
    return out


def compare_render(C_gpu, G_gpu, ref, exclude=None, tol_c=TOL_C, tol_g=TOL_G):
    """C_gpu [3,H,W], G_gpu [3,3,H,W] or None; ref: oracle.render(..., variants=True).
    Returns (n_fail, n_checked, n_excluded, worst)."""
    C = np.asarray(C_gpu, np.float64)
    H, W = C.shape[1:]
    nk = 3 if G_gpu is None else 12
    gpu = np.concatenate([C] + ([] if G_gpu is None else [np.asarray(G_gpu, np.float64).reshape(9, H, W)]))
    gpu = gpu.transpose(1, 2, 0)                                   # H, W, nk
    var = ref["variants"][..., :nk]                                # H, W, 8, nk
    nvar = ref["nvar"]
    nominal = var[:, :, 0, :]
    rms = np.sqrt(np.mean(nominal ** 2, axis=(0, 1)))              # per plane
    diff = np.abs(gpu[:, :, None, :] - var)
    tol = np.empty_like(var)
    tol[..., :3] = tol_c
    if nk > 3:
        tol[..., 3:] = tol_g * np.maximum(np.abs(var[..., 3:]), rms[None, None, None, 3:])
    ok_v = np.all(diff <= tol, axis=-1)                            # H, W, 8
    valid_v = np.arange(8)[None, None, :] < np.maximum(nvar, 0)[:, :, None]
    ok = np.any(ok_v & valid_v, axis=-1)
    excl = nvar < 1
    if exclude is not None:
        excl = excl | exclude
    fail = ~ok & ~excl
    worst = np.where(fail[..., None], diff[:, :, 0, :] / tol[:, :, 0, :], 0).max() if fail.any() else 0.0
    return int(fail.sum()), int((~excl).sum()), int(excl.sum()), float(worst)


def compare_pixels(gpu_rows, ref, tol_c=TOL_C, tol_g=TOL_G, rms=None, exclude=None):
    """Sampled version: gpu_rows [M, 12] vs oracle.render(pixels=..., variants=True)."""
    gpu = np.asarray(gpu_rows, np.float64)
    nk = gpu.shape[1]
    var = ref["variants"][..., :nk]                                # M, 8, nk
    nvar = ref["nvar"]
    if rms is None:
        rms = np.sqrt(np.mean(var[:, 0, :] ** 2, axis=0))
    diff = np.abs(gpu[:, None, :] - var)
    tol = np.empty_like(var)
    tol[..., :3] = tol_c
    if nk > 3:
        tol[..., 3:] = tol_g * np.maximum(np.abs(var[..., 3:]), rms[None, None, 3:])
    ok_v = np.all(diff <= tol, axis=-1)
    valid_v = np.arange(8)[None, :] < np.maximum(nvar, 0)[:, None]
    ok = np.any(ok_v & valid_v, axis=-1)
    excl = nvar < 1
    if exclude is not None:
        excl = excl | exclude
    fail = ~ok & ~excl
    return int(fail.sum()), int((~excl).sum()), int(excl.sum())


def gpu_rows(C, G, pix):
    """Gather [M, 12] rows (C rgb, Cx, Cy, Cxy) at pixels [M, 2] (x, y) from device images."""
    Cn = C.cpu().numpy()
    Gn = G.cpu().numpy().reshape(9, C.shape[1], C.shape[2])
    x, y = pix[:, 0], pix[:, 1]
    return np.concatenate([Cn[:, y, x].T, Gn[:, y, x].T], axis=1)


def pairs_without(keys, vals, drop_ids):
    """Pair list with every pair of the Gaussians in drop_ids removed."""
    if len(drop_ids) == 0:
        return keys, vals
    keep = ~np.isin(vals, drop_ids)
    return keys[keep], vals[keep]
