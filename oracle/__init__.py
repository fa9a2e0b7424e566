"""FP64 CPU oracle for gradient-aware spline upscaling of 3DGS images.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are the only callers.  The product
path (the CUDA library and its binding) never imports this package, and this
package never imports the product.  It wraps ``oracle.c`` (compiled with gcc,
no fused multiply-add contraction) through ctypes.

Each wrapper names the passage of the paper it follows; see ``oracle.c`` for
the arithmetic and the readings of under-specified passages.
"""
from __future__ import annotations

import ctypes as ct
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib", platform.machine())
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_3DGS = 0
MODE_EXACT = 1
MAX_VAR = 8


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_lib/liboracle.so (plain gcc, -O2)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ct.CDLL(_LIB)
            for name in ("ora_sh_basis", "ora_project", "ora_bin", "ora_render",
                         "ora_spline_cinv", "ora_upscale", "ora_upscale_adjoint",
                         "ora_render_adjoint", "ora_project_adjoint", "ora_bicubic"):
                getattr(_lib, name).restype = ct.c_int
        return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _check(st, what):
    if st != 0:
        raise ValueError(f"oracle {what} failed with status {st}")


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# --------------------------------------------------------------------------
# Spherical harmonics (Sec. 4: view-dependent colour)
# --------------------------------------------------------------------------

def sh_basis(degree: int, dirs) -> np.ndarray:
    """Real SH basis values Y_k(dir), k = l^2 + l + m, for l <= degree."""
    lib = _load()
    d = _f64(np.reshape(dirs, (-1, 3)))
    K = (degree + 1) ** 2
    out = np.zeros((d.shape[0], K))
    _check(lib.ora_sh_basis(ct.c_int(degree), ct.c_int64(d.shape[0]), _p(d), _p(out)), "sh_basis")
    return out


# --------------------------------------------------------------------------
# Projection (Sec. 4, EWA splatting)
# --------------------------------------------------------------------------

def project(scene: dict, cam: dict, W: int, H: int, tile: int = 16, mode: int = MODE_3DGS) -> dict:
    """Project every Gaussian; FP64 on the FP32 input values."""
    lib = _load()
    n = int(scene["means"].shape[0])
    means = _f64(scene["means"])
    ls = _f64(scene["log_scales"])
    qs = _f64(scene["quats"])
    ol = _f64(scene["opacity_logits"])
    sh = _f64(scene.get("sh"))
    rgb_in = _f64(scene.get("rgb")) if sh is None else None
    deg = int(scene.get("sh_degree", 0)) if sh is not None else 0
    vm = _f64(cam["viewmat"]).reshape(16)
    out = dict(
        mean2d=np.zeros((n, 2)), cov2d=np.zeros((n, 3)), conic=np.zeros((n, 3)),
        rgb=np.zeros((n, 3)), opacity=np.zeros(n), depth=np.zeros(n),
        radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32),
        tiles_touched=np.zeros(n, np.int64), borderline=np.zeros(n, np.uint8),
        envelope=np.zeros((n, 4), np.int32), core=np.zeros((n, 4), np.int32))
    st = lib.ora_project(
        ct.c_int64(n), _p(means), _p(ls), _p(qs), _p(ol), _p(sh), ct.c_int(deg), _p(rgb_in),
        _p(vm), ct.c_double(cam["fx"]), ct.c_double(cam["fy"]), ct.c_double(cam["cx"]),
        ct.c_double(cam["cy"]), ct.c_double(cam["znear"]), ct.c_int(W), ct.c_int(H),
        ct.c_int(tile), ct.c_int(mode),
        _p(out["mean2d"]), _p(out["cov2d"]), _p(out["conic"]), _p(out["rgb"]),
        _p(out["opacity"]), _p(out["depth"]), _p(out["radius"]), _p(out["rect"]),
        _p(out["tiles_touched"]), _p(out["borderline"]), _p(out["envelope"]), _p(out["core"]))
    _check(st, "project")
    out.update(W=W, H=H, tile=tile, mode=mode,
               tiles_x=(W + tile - 1) // tile, tiles_y=(H + tile - 1) // tile)
    return out


# --------------------------------------------------------------------------
# Binning (front-to-back order per tile)
# --------------------------------------------------------------------------

def bin_pairs(proj: dict) -> dict:
    """All (tile, Gaussian) pairs sorted by (tile, FP32 depth bits, id)."""
    lib = _load()
    n = proj["depth"].shape[0]
    P = int(proj["tiles_touched"].sum())
    T = proj["tiles_x"] * proj["tiles_y"]
    keys = np.zeros(max(P, 1), np.uint64)
    vals = np.zeros(max(P, 1), np.uint32)
    ranges = np.zeros((T, 2), np.uint32)
    st = lib.ora_bin(ct.c_int64(n), _p(proj["depth"]), _p(np.ascontiguousarray(proj["rect"])),
                     ct.c_int(proj["tiles_x"]), ct.c_int(proj["tiles_y"]), ct.c_int64(P),
                     _p(keys), _p(vals), _p(ranges))
    _check(st, "bin")
    return dict(keys=keys[:P], vals=vals[:P], ranges=ranges, P=P)


# --------------------------------------------------------------------------
# Blend with screen-space derivatives (Sec. 5; supplement "Forward pass")
# --------------------------------------------------------------------------

def render(proj: dict, bins: dict, bg=(0.0, 0.0, 0.0), offset=(0.0, 0.0), pixels=None,
           variants: bool = False, nthreads: int | None = None) -> dict:
    """Render C, dC/dx, dC/dy, d2C/dxdy.

    pixels=None renders the whole image and returns planes:
        C [3,H,W], grads [3 (dx, dy, dxy), 3, H, W], state [5, H, W] (A, A_x, A_y,
        A_xy, count).  With ``pixels`` (int array [M, 2] of (x, y)) returns per-pixel
        rows: out [M, 12], state [M, 5].
    variants=True also returns, per pixel, every result an FP32 evaluation may
    legitimately produce (``nvar`` of them, up to 8; negative = too many
    near-threshold decisions, pixel not comparable) in ``variants`` [.., 8, 12].
    """
    lib = _load()
    W, H = proj["W"], proj["H"]
    if pixels is None:
        npix, pix = W * H, None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
        npix = pix.shape[0]
    out = np.zeros((npix, 12))
    state = np.zeros((npix, 5))
    nvar = np.zeros(npix, np.int32)
    var = np.zeros((npix, MAX_VAR, 12)) if variants else None
    stats = np.zeros(2, np.int64)
    bgv = _f64(np.asarray(bg, np.float64).reshape(3))
    vals = np.ascontiguousarray(bins["vals"] if bins["P"] > 0 else np.zeros(1, np.uint32))
    st = lib.ora_render(
        ct.c_int(W), ct.c_int(H), ct.c_int(proj["tile"]), ct.c_int(proj["mode"]), _p(bgv),
        ct.c_double(offset[0]), ct.c_double(offset[1]),
        _p(proj["mean2d"]), _p(proj["conic"]), _p(proj["opacity"]), _p(proj["rgb"]),
        _p(vals), _p(np.ascontiguousarray(bins["ranges"])),
        ct.c_int64(npix), _p(pix), _p(out), _p(state), _p(nvar), _p(var), _p(stats),
        ct.c_int(nthreads or default_threads()))
    _check(st, "render")
    res = dict(n_eval=int(stats[0]), n_acc=int(stats[1]), nvar=nvar)
    if pixels is None:
        planes = out.reshape(H, W, 12).transpose(2, 0, 1)
        res["C"] = np.ascontiguousarray(planes[0:3])
        res["grads"] = np.ascontiguousarray(planes[3:12].reshape(3, 3, H, W))
        res["state"] = np.ascontiguousarray(state.reshape(H, W, 5).transpose(2, 0, 1))
        res["nvar"] = nvar.reshape(H, W)
        if variants:
            res["variants"] = var.reshape(H, W, MAX_VAR, 12)
    else:
        res["out"] = out
        res["state"] = state
        if variants:
            res["variants"] = var
    return res


# --------------------------------------------------------------------------
# Spline upscale (Sec. 5 "Spline Interpolation"; supplement)
# --------------------------------------------------------------------------

def spline_cinv() -> np.ndarray:
    """C^-1 for the paper's constant 4x4 matrix C, by Gauss-Jordan elimination."""
    lib = _load()
    out = np.zeros(16)
    _check(lib.ora_spline_cinv(_p(out)), "spline_cinv")
    return out.reshape(4, 4)


def upscale(C, grads, W2: int, H2: int, pixels=None) -> np.ndarray:
    """Hermite upscale of C [3,H,W] with grads [3,3,H,W] to W2 x H2.

    Returns [3, H2, W2] (pixels=None) or [M, 3] for hi-res pixels [M, 2] of (X, Y).
    """
    lib = _load()
    C = _f64(C)
    G = _f64(grads)
    H, W = C.shape[1], C.shape[2]
    if pixels is None:
        npix, pix = W2 * H2, None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
        npix = pix.shape[0]
    out = np.zeros((npix, 3))
    st = lib.ora_upscale(ct.c_int(W), ct.c_int(H), ct.c_int(W2), ct.c_int(H2), _p(C), _p(G),
                         ct.c_int64(npix), _p(pix), _p(out))
    _check(st, "upscale")
    if pixels is None:
        return np.ascontiguousarray(out.reshape(H2, W2, 3).transpose(2, 0, 1))
    return out


# --------------------------------------------------------------------------
# Reverse mode (supplement "Backward Pass")
# --------------------------------------------------------------------------

G2D_FIELDS = ("mean_x", "mean_y", "conic_a", "conic_b", "conic_c", "opacity", "r", "g", "b")


def upscale_adjoint(dout, W: int, H: int):
    """Adjoint of ``upscale``: dout [3,H2,W2] -> (dC [3,H,W], dgrads [3,3,H,W])."""
    lib = _load()
    d = _f64(dout)
    H2, W2 = d.shape[1], d.shape[2]
    dC = np.zeros((3, H, W))
    dG = np.zeros((3, 3, H, W))
    _check(lib.ora_upscale_adjoint(ct.c_int(W), ct.c_int(H), ct.c_int(W2), ct.c_int(H2), _p(d), _p(dC), _p(dG)),
           "upscale_adjoint")
    return dC, dG


def render_adjoint(proj: dict, bins: dict, dout, bg=(0.0, 0.0, 0.0), pixels=None,
                   nthreads: int | None = None) -> dict:
    """Adjoint of ``render``: upstream dL/d(C, C_x, C_y, C_xy) -> dL/d(2D parameters).

    dout: planes (dC [3,H,W], dgrads [3,3,H,W]) for the whole image, or rows
    [M, 12] (C rgb, Cx rgb, Cy rgb, Cxy rgb) for ``pixels`` [M, 2] of (x, y).
    Returns g2d [n, 9] (columns ``G2D_FIELDS``) and ``b2f``, the image recomputed
    back to front from the tape (same layout as dout).
    """
    lib = _load()
    W, H = proj["W"], proj["H"]
    n = proj["depth"].shape[0]
    if pixels is None:
        dC, dG = dout
        rows = np.concatenate([_f64(dC).reshape(3, -1), _f64(dG).reshape(9, -1)], 0).T
        npix, pix = W * H, None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
        npix = pix.shape[0]
        rows = _f64(dout).reshape(npix, 12)
    rows = np.ascontiguousarray(rows)
    g2d = np.zeros((n, 9))
    b2f = np.zeros((npix, 12))
    bgv = _f64(np.asarray(bg, np.float64).reshape(3))
    vals = np.ascontiguousarray(bins["vals"] if bins["P"] > 0 else np.zeros(1, np.uint32))
    st = lib.ora_render_adjoint(
        ct.c_int(W), ct.c_int(H), ct.c_int(proj["tile"]), ct.c_int(proj["mode"]), _p(bgv),
        _p(proj["mean2d"]), _p(proj["conic"]), _p(proj["opacity"]), _p(proj["rgb"]),
        _p(vals), _p(np.ascontiguousarray(bins["ranges"])), ct.c_int64(n),
        ct.c_int64(npix), _p(pix), _p(rows), _p(g2d), _p(b2f), ct.c_int(nthreads or default_threads()))
    _check(st, "render_adjoint")
    res = dict(g2d=g2d)
    if pixels is None:
        planes = b2f.reshape(H, W, 12).transpose(2, 0, 1)
        res["b2f_C"] = np.ascontiguousarray(planes[0:3])
        res["b2f_grads"] = np.ascontiguousarray(planes[3:12].reshape(3, 3, H, W))
    else:
        res["b2f"] = b2f
    return res


def project_adjoint(scene: dict, cam: dict, W: int, H: int, g2d) -> dict:
    """Adjoint of ``project``: dL/d(2D parameters) [n, 9] -> dL/d(scene inputs)."""
    lib = _load()
    n = int(scene["means"].shape[0])
    sh = _f64(scene.get("sh"))
    rgb_in = _f64(scene.get("rgb")) if sh is None else None
    deg = int(scene.get("sh_degree", 0)) if sh is not None else 0
    vm = _f64(cam["viewmat"]).reshape(16)
    out = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               opacity_logits=np.zeros(n))
    if sh is not None:
        out["sh"] = np.zeros(sh.shape)
    else:
        out["rgb"] = np.zeros((n, 3))
    st = lib.ora_project_adjoint(
        ct.c_int64(n), _p(_f64(scene["means"])), _p(_f64(scene["log_scales"])), _p(_f64(scene["quats"])),
        _p(_f64(scene["opacity_logits"])), _p(sh), ct.c_int(deg), _p(rgb_in), _p(vm),
        ct.c_double(cam["fx"]), ct.c_double(cam["fy"]), ct.c_double(cam["cx"]), ct.c_double(cam["cy"]),
        ct.c_double(cam["znear"]), ct.c_int(W), ct.c_int(H), _p(np.ascontiguousarray(_f64(g2d))),
        _p(out["means"]), _p(out["log_scales"]), _p(out["quats"]), _p(out["opacity_logits"]),
        _p(out.get("sh")), _p(out.get("rgb")))
    _check(st, "project_adjoint")
    return out


def bicubic(C, W2: int, H2: int, a: float = -0.75, pixels=None) -> np.ndarray:
    """Classical bicubic (cubic convolution, parameter a) of C [3,H,W] to W2 x H2.

    Returns [3, H2, W2] (pixels=None) or [M, 3] for hi-res pixels [M, 2] of (X, Y).
    """
    lib = _load()
    C = _f64(C)
    H, W = C.shape[1], C.shape[2]
    if pixels is None:
        npix, pix = W2 * H2, None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
        npix = pix.shape[0]
    out = np.zeros((npix, 3))
    st = lib.ora_bicubic(ct.c_int(W), ct.c_int(H), ct.c_int(W2), ct.c_int(H2), _p(C), ct.c_double(a),
                         ct.c_int64(npix), _p(pix), _p(out))
    _check(st, "bicubic")
    if pixels is None:
        return np.ascontiguousarray(out.reshape(H2, W2, 3).transpose(2, 0, 1))
    return out


def render_image(scene: dict, cam: dict, W: int, H: int, tile: int = 16, mode: int = MODE_3DGS,
                 bg=(0.0, 0.0, 0.0), nthreads: int | None = None) -> dict:
    """Convenience: project, bin and render the whole image."""
    proj = project(scene, cam, W, H, tile, mode)
    bins = bin_pairs(proj)
    res = render(proj, bins, bg=bg, nthreads=nthreads)
    res["proj"] = proj
    res["bins"] = bins
    return res
