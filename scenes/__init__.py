"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only draws random numbers and builds camera descriptions; it holds
none of the method's arithmetic (no projection, blending or spline code), so the
CPU oracle and the CUDA path can both take their inputs from here without
sharing any computation.

Scenes are plain dicts of float32 numpy arrays in the layout the C ABI expects:

    means           [N, 3]   world-space centres
    log_scales      [N, 3]   per-axis log standard deviation
    quats           [N, 4]   rotation quaternion (w, x, y, z), not necessarily unit
    opacity_logits  [N]      opacity before the sigmoid
    sh              [N, K, 3] spherical-harmonics coefficients, K = (deg + 1)^2
                              (absent when the scene carries direct colours)
    rgb             [N, 3]   direct colour in [0, 1] (absent for SH scenes)
    sh_degree       int

Cameras are dicts: viewmat [4, 4] float32 row-major world->camera (x right,
y down, z forward), fx, fy, cx, cy, znear, width, height.

The workload recipes follow the paper's scene types (Sec. 6, Table 1: real
captures of about 1M-5M Gaussians rendered at 1K-5K resolution); the real
datasets are not available, so these seeded distributions stand in for them.
"""
from __future__ import annotations

import math

import numpy as np

# Y_0^0 = 1 / (2 sqrt(pi)): used only to express a desired base colour as a DC
# coefficient when drawing SH scenes (input recipe, not evaluation).
_Y00 = 0.5 / math.sqrt(math.pi)


def pinhole_camera(width: int, height: int, fov_x_deg: float = 60.0,
                   viewmat: np.ndarray | None = None, znear: float = 0.2) -> dict:
    """Pinhole camera whose horizontal field of view is ``fov_x_deg``.

    Pixel (i, j) is the continuous image point (i, j); the principal point is
    the image centre ((W - 1) / 2, (H - 1) / 2) and pixels are square.
    """
    fx = width / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))
    vm = np.eye(4, dtype=np.float32) if viewmat is None else np.asarray(viewmat, np.float32).reshape(4, 4)
    return dict(viewmat=vm.copy(), fx=float(fx), fy=float(fx),
                cx=(width - 1) / 2.0, cy=(height - 1) / 2.0, znear=float(znear),
                width=int(width), height=int(height))


def scaled_camera(cam: dict, factor: int) -> dict:
    """The same view at ``factor`` times the resolution (direct full-res render).

    With the half-pixel hi-res -> low-res map x_lo = (X + 0.5) / s - 0.5, a hi-res
    pixel centre and its low-res sample point see the same camera ray.
    """
    w, h = cam["width"] * factor, cam["height"] * factor
    return dict(viewmat=cam["viewmat"].copy(), fx=cam["fx"] * factor, fy=cam["fy"] * factor,
                cx=(w - 1) / 2.0, cy=(h - 1) / 2.0, znear=cam["znear"], width=w, height=h)


def look_at_viewmat(eye, target, up=(0.0, -1.0, 0.0)) -> np.ndarray:
    """World->camera matrix (x right, y down, z forward) looking from eye to target."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])            # rows: camera axes in world coords
    vm = np.eye(4)
    vm[:3, :3] = R
    vm[:3, 3] = -R @ eye
    return vm.astype(np.float32)


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def random_scene(n: int = 1000, seed: int = 0, sh_degree: int | None = None,
                 log_scale_mean: float = -3.0, log_scale_std: float = 0.5,
                 z_range=(2.0, 4.0), xy_range=1.0) -> dict:
    """Small random scene: the 1,000-Gaussian, 64x64 parity workload.

    means ~ U[-1,1]^2 x U[2,4], log-scales ~ N(-3, 0.5), random unit quaternions,
    opacity = sigmoid(N(0,1)), direct RGB ~ U[0,1] (or SH coefficients of the
    given degree, DC from a U[0,1] base colour and the rest N(0, 0.2)).
    """
    rng = np.random.default_rng(seed)
    means = np.empty((n, 3))
    means[:, 0:2] = rng.uniform(-xy_range, xy_range, (n, 2))
    means[:, 2] = rng.uniform(z_range[0], z_range[1], n)
    scene = dict(
        means=means.astype(np.float32),
        log_scales=rng.normal(log_scale_mean, log_scale_std, (n, 3)).astype(np.float32),
        quats=_unit_quats(rng, n).astype(np.float32),
        opacity_logits=rng.normal(0.0, 1.0, n).astype(np.float32),
    )
    if sh_degree is None:
        scene["rgb"] = rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32)
        scene["sh_degree"] = 0
    else:
        scene.update(_sh_coeffs(rng, n, sh_degree))
    return scene


def _sh_coeffs(rng, n, deg):
    k = (deg + 1) ** 2
    sh = rng.normal(0.0, 0.2, (n, k, 3))
    base = rng.uniform(0.0, 1.0, (n, 3))
    sh[:, 0, :] = (base - 0.5) / _Y00
    return dict(sh=sh.astype(np.float32), sh_degree=int(deg))


def mixture_scene(n: int = 1_500_000, seed: int = 0, components: int = 200,
                  sh_degree: int = 3, aspect=(16.0, 9.0), fov_x_deg: float = 60.0,
                  log_scale_mean: float = -4.0, log_scale_std: float = 0.7,
                  opacity_logit_std: float = 1.5) -> dict:
    """Scene-shaped workload: means from a seeded mixture of anisotropic 3D normals.

    200 components; component depth z ~ U[3, 10], centre (x, y) ~ U[-0.5, 0.5]^2 *
    z * tan(fov_x / 2) * (16/9, 1), i.e. inside the view frustum;
    component covariance R diag(exp N(log 0.4, 0.5))^2 R^T; mixture weights
    Dirichlet(1).  Per Gaussian: log-scales N(-4, 0.7), random unit quaternion,
    SH degree 3 with DC from a U[0,1] base colour and the rest N(0, 0.2),
    opacity sigmoid(N(0, 1.5)).
    """
    rng = np.random.default_rng(seed)
    t = math.tan(math.radians(fov_x_deg) / 2.0)
    zc = rng.uniform(3.0, 10.0, components)
    xc = rng.uniform(-0.5, 0.5, components) * zc * t * (aspect[0] / aspect[1])
    yc = rng.uniform(-0.5, 0.5, components) * zc * t
    centres = np.stack([xc, yc, zc], axis=1)
    weights = rng.dirichlet(np.ones(components))
    counts = rng.multinomial(n, weights)
    sig = np.exp(rng.normal(math.log(0.4), 0.5, (components, 3)))
    means = np.empty((n, 3))
    pos = 0
    for c in range(components):
        m = counts[c]
        if m == 0:
            continue
        # random orthonormal axes for the component (QR of a Gaussian matrix)
        R, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        local = rng.standard_normal((m, 3)) * sig[c]
        means[pos:pos + m] = centres[c] + local @ R.T
        pos += m
    perm = rng.permutation(n)
    means = means[perm]
    scene = dict(
        means=means.astype(np.float32),
        log_scales=rng.normal(log_scale_mean, log_scale_std, (n, 3)).astype(np.float32),
        quats=_unit_quats(rng, n).astype(np.float32),
        opacity_logits=rng.normal(0.0, opacity_logit_std, n).astype(np.float32),
    )
    scene.update(_sh_coeffs(rng, n, sh_degree))
    return scene


def subset(scene: dict, idx) -> dict:
    """Scene restricted to the Gaussians ``idx`` (same fields, same degree)."""
    out = {}
    for k, v in scene.items():
        out[k] = v[idx] if isinstance(v, np.ndarray) else v
    return out


def num_gaussians(scene: dict) -> int:
    return int(scene["means"].shape[0])


def mixture_scene_device(n: int, seed: int = 0, device: str = "cuda", components: int = 200,
                         sh_degree: int = 3, aspect=(16.0, 9.0), fov_x_deg: float = 60.0,
                         log_scale_mean: float = -4.0, log_scale_std: float = 0.7,
                         opacity_logit_std: float = 1.5) -> dict:
    """The recipe of ``mixture_scene`` drawn with torch's generator on the device
    (another random stream than the numpy one; for generating many training
    scenes quickly).  Values are torch float32 tensors on ``device``."""
    import torch
    g = torch.Generator(device=device).manual_seed(int(seed))
    kw = dict(device=device, generator=g)
    t = math.tan(math.radians(fov_x_deg) / 2.0)
    zc = 3.0 + 7.0 * torch.rand(components, **kw)
    xc = (torch.rand(components, **kw) - 0.5) * zc * t * (aspect[0] / aspect[1])
    yc = (torch.rand(components, **kw) - 0.5) * zc * t
    centres = torch.stack([xc, yc, zc], 1)
    # Dirichlet(1) weights = normalised Exp(1) draws
    w = -torch.log(torch.rand(components, **kw).clamp_min(1e-12))
    comp = torch.multinomial(w / w.sum(), n, replacement=True, generator=g)
    sig = torch.exp(math.log(0.4) + 0.5 * torch.randn(components, 3, **kw))
    # random component axes: the rotation of a uniformly random unit quaternion
    qc = torch.randn(components, 4, **kw)
    w, x, y, z = (qc / qc.norm(dim=1, keepdim=True)).unbind(1)
    R = torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                     2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                     2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1).view(components, 3, 3)
    local = torch.randn(n, 3, **kw) * sig[comp]
    means = centres[comp] + torch.einsum("nij,nj->ni", R[comp], local)
    q = torch.randn(n, 4, **kw)
    q = q / q.norm(dim=1, keepdim=True)
    k = (sh_degree + 1) ** 2
    sh = 0.2 * torch.randn(n, k, 3, **kw)
    sh[:, 0, :] = (torch.rand(n, 3, **kw) - 0.5) / _Y00
    return dict(means=means.float().contiguous(),
                log_scales=(log_scale_mean + log_scale_std * torch.randn(n, 3, **kw)).contiguous(),
                quats=q.contiguous(), opacity_logits=(opacity_logit_std * torch.randn(n, **kw)).contiguous(),
                sh=sh.contiguous(), sh_degree=int(sh_degree))


def stereo_views(seed: int = 0, pairs: int = 8, lo=(512, 512), hi=(1104, 1032), ipd: float = 0.064):
    """The batching workload's 16 views: 8 stereo pairs whose per-eye sizes are
    log-uniform between lo and hi (rounded to even), eyes 64 mm apart around the
    origin, each pair yawed by U[-0.05, 0.05] rad, looking down +z.  Returns
    ([(eye, target)] per view, [(W, H)] per view)."""
    rng = np.random.default_rng(seed)
    cams, eyes = [], []
    for _ in range(pairs):
        W = int(round(np.exp(rng.uniform(np.log(lo[0]), np.log(hi[0]))) / 2)) * 2
        H = int(round(np.exp(rng.uniform(np.log(lo[1]), np.log(hi[1]))) / 2)) * 2
        yaw = rng.uniform(-0.05, 0.05)
        for side in (-0.5, 0.5):
            eye = (side * ipd, 0.0, 0.0)
            target = (side * ipd + 6.0 * np.sin(yaw), 0.0, 6.0 * np.cos(yaw))
            eyes.append((W, H))
            cams.append((eye, target))
    return cams, eyes
