"""Python binding of libgs (include/gs.h): gradient-aware spline upscaling of
3D Gaussian Splatting images on GB300.

Argument marshalling only: every step of the path runs in the CUDA kernels of
libgs.so; PyTorch supplies device memory and streams.  Importing this package
loads the in-tree library and fails loudly if it has not been built
(``python -c "import __graft_entry__ as g; g.build()"``).

Low-level entry points carry the C names (``gs_create``, ``gs_project``,
``gs_render_with_grads``, ``gs_render``, ``gs_upscale`` ...) and take raw
pointers; :class:`Context` wraps them for torch tensors.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgs.so")

GS_OK = 0
GS_ERR_INVALID_ARG = 1
GS_ERR_CUDA = 2
GS_ERR_OOM = 3
GS_ERR_CAPACITY = 4
GS_ERR_TIMEOUT = 5
GS_ERR_DEVICE_CHECK = 6
GS_ERR_NOT_READY = 7
GS_MODE_3DGS = 0
GS_MODE_EXACT = 1
MODES = {"3dgs": GS_MODE_3DGS, "exact": GS_MODE_EXACT}
GS_FLAG_NO_HOST_WAIT = 1
GS_FLAG_BWD_RECOMPUTE = 2
GS_INJECT_NONE = 0
GS_INJECT_WAIT_EXPIRY = 1
GS_INJECT_ALLOC_FAILURE = 2
GS_VIEWS_CONFIGS = 16
GS_MLP_IN = 50
GS_MLP_HIDDEN = 64
GS_MLP_PARAMS = 7619
GS_MLP_ROW = 64


class GsGaussians(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("sh_degree", ct.c_int32), ("reserved", ct.c_int32),
                ("means", ct.c_void_p), ("log_scales", ct.c_void_p), ("quats", ct.c_void_p),
                ("opacity_logits", ct.c_void_p), ("sh", ct.c_void_p), ("rgb", ct.c_void_p)]


class GsCamera(ct.Structure):
    _fields_ = [("viewmat", ct.c_float * 16), ("fx", ct.c_float), ("fy", ct.c_float),
                ("cx", ct.c_float), ("cy", ct.c_float), ("znear", ct.c_float)]


class GsOptions(ct.Structure):
    _fields_ = [("tile", ct.c_int32), ("mode", ct.c_int32), ("bg", ct.c_float * 3),
                ("flags", ct.c_int32), ("max_pairs", ct.c_int64)]


class GsGaussianGrads(ct.Structure):
    _fields_ = [("means", ct.c_void_p), ("log_scales", ct.c_void_p), ("quats", ct.c_void_p),
                ("opacity_logits", ct.c_void_p), ("sh", ct.c_void_p), ("rgb", ct.c_void_p)]


# name -> argtypes (all return gs_status except gs_status_string / gs_last_error)
_P = ct.c_void_p
_SIGS = {
    "gs_status_string": ([ct.c_int], ct.c_char_p),
    "gs_last_error": ([_P], ct.c_char_p),
    "gs_create": ([ct.POINTER(_P), _P, ct.POINTER(GsOptions)], ct.c_int),
    "gs_destroy": ([_P], ct.c_int),
    "gs_set_stream": ([_P, _P], ct.c_int),
    "gs_set_options": ([_P, ct.POINTER(GsOptions)], ct.c_int),
    "gs_reserve": ([_P, ct.c_int64, ct.c_int32, ct.c_int32, ct.c_int64], ct.c_int),
    "gs_reserve_views": ([_P, ct.c_int64, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int64], ct.c_int),
    "gs_render_views": ([_P, ct.POINTER(GsGaussians), ct.c_int32, ct.POINTER(GsCamera), ct.POINTER(ct.c_int32),
                         ct.POINTER(ct.c_int32), ct.POINTER(_P), ct.POINTER(_P), ct.POINTER(ct.c_int32),
                         ct.POINTER(_P)], ct.c_int),
    "gs_render_views_scenes": ([_P, ct.POINTER(GsGaussians), ct.c_int32, ct.POINTER(ct.c_int32), ct.c_int32,
                                ct.POINTER(GsCamera), ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32), ct.POINTER(_P),
                                ct.POINTER(_P), ct.POINTER(ct.c_int32), ct.POINTER(_P)], ct.c_int),
    "gs_views_config": ([_P, ct.c_int32, ct.c_int32, ct.c_int32], ct.c_int),
    "gs_autotune_views_scenes": ([_P, ct.POINTER(GsGaussians), ct.c_int32, ct.POINTER(ct.c_int32), ct.c_int32,
                                  ct.POINTER(GsCamera), ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32),
                                  ct.POINTER(_P), ct.POINTER(_P), ct.POINTER(ct.c_int32), ct.POINTER(_P), ct.c_int32,
                                  ct.POINTER(ct.c_float), ct.POINTER(ct.c_int32)], ct.c_int),
    "gs_autotune_views": ([_P, ct.POINTER(GsGaussians), ct.c_int32, ct.POINTER(GsCamera), ct.POINTER(ct.c_int32),
                           ct.POINTER(ct.c_int32), ct.POINTER(_P), ct.POINTER(_P), ct.POINTER(ct.c_int32),
                           ct.POINTER(_P), ct.c_int32, ct.POINTER(ct.c_float), ct.POINTER(ct.c_int32)], ct.c_int),
    "gs_project": ([_P, ct.POINTER(GsGaussians), ct.POINTER(GsCamera), ct.c_int32, ct.c_int32], ct.c_int),
    "gs_render_binned": ([_P, _P, _P], ct.c_int),
    "gs_render_with_grads": ([_P, ct.POINTER(GsGaussians), ct.POINTER(GsCamera), ct.c_int32, ct.c_int32, _P, _P],
                             ct.c_int),
    "gs_render": ([_P, ct.POINTER(GsGaussians), ct.POINTER(GsCamera), ct.c_int32, ct.c_int32, _P], ct.c_int),
    "gs_upscale": ([_P, _P, _P, ct.c_int32, ct.c_int32, ct.c_int32, _P], ct.c_int),
    "gs_pair_count": ([_P, ct.POINTER(ct.c_int64)], ct.c_int),
    "gs_super_pair_count": ([_P, ct.POINTER(ct.c_int64)], ct.c_int),
    "gs_read_projected": ([_P, _P, _P, _P, _P, _P, _P, _P], ct.c_int),
    "gs_read_bins": ([_P, _P, _P, _P, ct.c_int64], ct.c_int),
    "gs_read_state": ([_P, _P, _P], ct.c_int),
    "gs_launch_count": ([_P, ct.POINTER(ct.c_int64)], ct.c_int),
    "gs_blend_stats": ([_P, _P], ct.c_int),
    "gs_synchronize": ([_P], ct.c_int),
    "gs_upscale_backward": ([_P, _P, ct.c_int32, ct.c_int32, ct.c_int32, _P, _P], ct.c_int),
    "gs_upscale_to": ([_P, _P, _P, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, _P], ct.c_int),
    "gs_upscale_backward_to": ([_P, _P, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, _P, _P], ct.c_int),
    "gs_upscale_bicubic": ([_P, _P, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_float, _P], ct.c_int),
    "gs_render_backward": ([_P, _P, _P, _P], ct.c_int),
    "gs_project_backward": ([_P, _P, ct.POINTER(GsGaussianGrads)], ct.c_int),
    "gs_backward": ([_P, _P, ct.c_int32, ct.POINTER(GsGaussianGrads)], ct.c_int),
    "gs_debug_inject": ([_P, ct.c_int32, ct.c_int64], ct.c_int),
    "gs_read_tile_work": ([_P, _P], ct.c_int),
    "gs_render_with_grads_noalloc": ([ct.POINTER(GsGaussians), ct.POINTER(GsCamera), ct.c_int32, ct.c_int32,
                                      ct.POINTER(GsOptions), _P, _P, _P], ct.c_int),
    "gs_upscale_mlp": ([_P, _P, _P, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, _P, _P], ct.c_int),
    "gs_mlp_samples": ([_P, _P, _P, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, _P, ct.c_int64, _P, _P, _P, _P],
                       ct.c_int),
    "gs_mlp_gradient": ([_P, _P, _P, _P, _P, ct.c_int64, _P, _P], ct.c_int),
    "gs_mlp_adam": ([_P, _P, _P, _P, _P, ct.c_int32, ct.c_float, ct.c_float, ct.c_float, ct.c_float], ct.c_int),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgs.so is not built ({LIB_PATH}); run paper_2503_14171_gb300.build.build() "
                          "or __graft_entry__.build() on a machine with nvcc")
    lib = ct.CDLL(LIB_PATH)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()


class GSError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        name = lib.gs_status_string(status).decode()
        super().__init__(f"{name}: {msg}" if msg else name)


def exported_symbols():
    return sorted(_SIGS)


# ---- thin wrappers with the C names ----------------------------------------

def gs_status_string(status: int) -> str:
    return lib.gs_status_string(status).decode()


def gs_last_error(ctx) -> str:
    return lib.gs_last_error(ctx).decode()


def gs_create(stream=None, options: GsOptions | None = None):
    h = _P()
    st = lib.gs_create(ct.byref(h), stream, ct.byref(options) if options is not None else None)
    if st != GS_OK:
        raise GSError(st, "gs_create")
    return h


def _chk(st, ctx, what):
    if st != GS_OK:
        raise GSError(st, f"{what}: {gs_last_error(ctx)}")


def gs_destroy(ctx):
    _chk(lib.gs_destroy(ctx), None, "gs_destroy")


def gs_project(ctx, g: GsGaussians, cam: GsCamera, W: int, H: int):
    _chk(lib.gs_project(ctx, ct.byref(g), ct.byref(cam), W, H), ctx, "gs_project")


def gs_render_binned(ctx, out_C: int, out_grads: int | None):
    _chk(lib.gs_render_binned(ctx, out_C, out_grads), ctx, "gs_render_binned")


def gs_render_with_grads(ctx, g: GsGaussians, cam: GsCamera, W: int, H: int, out_C: int, out_grads: int):
    _chk(lib.gs_render_with_grads(ctx, ct.byref(g), ct.byref(cam), W, H, out_C, out_grads), ctx,
         "gs_render_with_grads")


def gs_render(ctx, g: GsGaussians, cam: GsCamera, W: int, H: int, out_C: int):
    _chk(lib.gs_render(ctx, ct.byref(g), ct.byref(cam), W, H, out_C), ctx, "gs_render")


def gs_upscale(ctx, C: int, grads: int, W: int, H: int, factor: int, out: int):
    _chk(lib.gs_upscale(ctx, C, grads, W, H, factor, out), ctx, "gs_upscale")


def gs_synchronize(ctx):
    _chk(lib.gs_synchronize(ctx), ctx, "gs_synchronize")


def gs_upscale_backward(ctx, dL_dout: int, W: int, H: int, factor: int, dL_dC: int, dL_dgrads: int):
    _chk(lib.gs_upscale_backward(ctx, dL_dout, W, H, factor, dL_dC, dL_dgrads), ctx, "gs_upscale_backward")


def gs_render_backward(ctx, dL_dC: int, dL_dgrads: int | None, grad2d: int):
    _chk(lib.gs_render_backward(ctx, dL_dC, dL_dgrads, grad2d), ctx, "gs_render_backward")


def gs_project_backward(ctx, grad2d: int, out: GsGaussianGrads):
    _chk(lib.gs_project_backward(ctx, grad2d, ct.byref(out)), ctx, "gs_project_backward")


def gs_backward(ctx, dL_dout: int, factor: int, out: GsGaussianGrads):
    _chk(lib.gs_backward(ctx, dL_dout, factor, ct.byref(out)), ctx, "gs_backward")


def gs_debug_inject(ctx, what: int, value: int):
    _chk(lib.gs_debug_inject(ctx, what, value), ctx, "gs_debug_inject")


def gs_render_with_grads_noalloc(g: GsGaussians, cam: GsCamera, W: int, H: int, options: GsOptions | None,
                                 stream, out_C: int, out_grads: int):
    """Context-free render with derivatives whose scratch is a static device array."""
    st = lib.gs_render_with_grads_noalloc(ct.byref(g), ct.byref(cam), W, H,
                                          ct.byref(options) if options is not None else None, stream, out_C,
                                          out_grads)
    if st != GS_OK:
        raise GSError(st, "gs_render_with_grads_noalloc")


# ---- torch-facing helpers ----------------------------------------------------

def _torch():
    import torch
    return torch


def make_camera(cam: dict) -> GsCamera:
    c = GsCamera()
    vm = np.asarray(cam["viewmat"], np.float32).reshape(16)
    for k in range(16):
        c.viewmat[k] = float(vm[k])
    c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
    c.znear = float(cam.get("znear", 0.2))
    return c


class DeviceScene:
    """A Gaussian set resident on the GPU (fp32, contiguous) and its gs_gaussians view."""

    FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh", "rgb")

    def __init__(self, scene: dict, device="cuda", tensors: dict | None = None):
        torch = _torch()
        self.t = {}
        if tensors is not None:
            self.t = dict(tensors)
        else:
            for k in self.FIELDS:
                if k in scene and scene[k] is not None:
                    self.t[k] = torch.as_tensor(np.ascontiguousarray(scene[k], np.float32)).to(device)
        self.n = int(self.t["means"].shape[0])
        self.sh_degree = int(scene.get("sh_degree", 0)) if "sh" in self.t else 0
        self.struct = self._make()

    def _make(self) -> GsGaussians:
        g = GsGaussians()
        g.n = self.n
        g.sh_degree = self.sh_degree
        for k in self.FIELDS:
            v = self.t.get(k)
            if v is not None:
                assert v.is_contiguous() and v.dtype == _torch().float32
            setattr(g, k, v.data_ptr() if v is not None and v.numel() > 0 else None)
        return g

    def copy_from(self, host: "HostScene", non_blocking=True):
        for k, v in host.t.items():
            self.t[k].copy_(v, non_blocking=non_blocking)

    def nbytes(self) -> int:
        return sum(v.numel() * 4 for v in self.t.values())


class HostScene:
    """The same fields in pinned host memory (for end-to-end timing)."""

    def __init__(self, scene: dict):
        torch = _torch()
        self.t = {}
        for k in DeviceScene.FIELDS:
            if k in scene and scene[k] is not None:
                self.t[k] = torch.as_tensor(np.ascontiguousarray(scene[k], np.float32)).pin_memory()


class Context:
    """Owns a gs_ctx bound to a torch CUDA stream (default: the current stream)."""

    def __init__(self, mode: str | int = "3dgs", bg=(0.0, 0.0, 0.0), stream=None, max_pairs: int = 0,
                 no_host_wait: bool = False, bwd_recompute: bool = False):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("libgs needs a CUDA device")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.opt = GsOptions()
        self.opt.tile = 16
        self.opt.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        for k in range(3):
            self.opt.bg[k] = float(bg[k])
        self.opt.max_pairs = int(max_pairs)
        self.opt.flags = (GS_FLAG_NO_HOST_WAIT if no_host_wait else 0) | (GS_FLAG_BWD_RECOMPUTE if bwd_recompute
                                                                          else 0)
        self.h = gs_create(ct.c_void_p(self.stream.cuda_stream), self.opt)
        self.W = self.H = 0

    def close(self):
        if getattr(self, "h", None):
            gs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reserve(self, n: int, W: int, H: int, super_pairs: int):
        """Allocate every buffer for frames up to these sizes (needed for no_host_wait)."""
        _chk(lib.gs_reserve(self.h, int(n), int(W), int(H), int(super_pairs)), self.h, "gs_reserve")

    def reserve_views(self, n: int, V: int, W: int, H: int, super_pairs: int):
        """Buffers for gs_render_views batches of up to V views."""
        _chk(lib.gs_reserve_views(self.h, int(n), int(V), int(W), int(H), int(super_pairs)), self.h,
             "gs_reserve_views")

    def _views_outs(self, sizes, factors, outs):
        if outs is not None:
            return outs
        outs = []
        for v, (W, H) in enumerate(sizes):
            o = [self._empty(3, H, W), self._empty(3, 3, H, W)]
            if factors is not None:
                o.append(self._empty(3, H * factors[v], W * factors[v]))
            outs.append(o)
        return outs

    def render_views(self, scene, cams: list, sizes: list, factors=None, outs=None, scene_of_view=None):
        """Render len(cams) views (sizes: [(W, H)]) with derivatives in one batch;
        with factors, also upscale view v by factors[v].  scene is one
        DeviceScene (gs_render_views), or a list of them with scene_of_view[v]
        naming view v's (gs_render_views_scenes).  Returns a list of (C, G) or
        (C, G, up) per view."""
        V = len(cams)
        outs = self._views_outs(sizes, factors, outs)
        if isinstance(scene, (list, tuple)):
            sets, sov = self._scenes_args(scene, scene_of_view, V)
            _chk(lib.gs_render_views_scenes(self.h, sets, len(scene), sov, V,
                                            *self._views_args(cams, sizes, factors, outs)),
                 self.h, "gs_render_views_scenes")
        else:
            _chk(lib.gs_render_views(self.h, ct.byref(scene.struct), V,
                                     *self._views_args(cams, sizes, factors, outs)),
                 self.h, "gs_render_views")
        return outs

    @staticmethod
    def _scenes_args(scenes, scene_of_view, V):
        if scene_of_view is None or len(scene_of_view) != V:
            raise ValueError("a list of scenes needs scene_of_view with one entry per view")
        sets = (GsGaussians * len(scenes))(*[s.struct for s in scenes])
        sov = (ct.c_int32 * V)(*[int(k) for k in scene_of_view])
        return sets, sov

    @staticmethod
    def _views_args(cams, sizes, factors, outs):
        V = len(cams)
        cam_arr = (GsCamera * V)(*[make_camera(c) for c in cams])
        Ws = (ct.c_int32 * V)(*[int(w) for w, _ in sizes])
        Hs = (ct.c_int32 * V)(*[int(h) for _, h in sizes])
        pC = (_P * V)(*[o[0].data_ptr() for o in outs])
        pG = (_P * V)(*[o[1].data_ptr() for o in outs])
        fac = (ct.c_int32 * V)(*[int(f) for f in factors]) if factors is not None else None
        pU = (_P * V)(*[o[2].data_ptr() for o in outs]) if factors is not None else None
        return cam_arr, Ws, Hs, pC, pG, fac, pU

    def views_config(self, warp_map: int, schedule: int, super_side: int = 0):
        """Binning and launch shape of render_views batches (see gs_views_config)."""
        _chk(lib.gs_views_config(self.h, int(warp_map), int(schedule), int(super_side)), self.h, "gs_views_config")

    def autotune_views(self, scene, cams: list, sizes: list, factors, outs, reps: int = 5, scene_of_view=None):
        """Time every binning and launch shape of the batched views on this
        batch, keep the fastest; returns (ms per configuration, chosen
        configuration).  scene as for render_views."""
        ms = (ct.c_float * GS_VIEWS_CONFIGS)()
        best = ct.c_int32()
        V = len(cams)
        if isinstance(scene, (list, tuple)):
            sets, sov = self._scenes_args(scene, scene_of_view, V)
            _chk(lib.gs_autotune_views_scenes(self.h, sets, len(scene), sov, V,
                                              *self._views_args(cams, sizes, factors, outs), int(reps), ms,
                                              ct.byref(best)),
                 self.h, "gs_autotune_views_scenes")
        else:
            _chk(lib.gs_autotune_views(self.h, ct.byref(scene.struct), V,
                                       *self._views_args(cams, sizes, factors, outs), int(reps), ms, ct.byref(best)),
                 self.h, "gs_autotune_views")
        return list(ms), int(best.value)

    def set_options(self, mode=None, bg=None, max_pairs=None, bwd_recompute=None):
        if bwd_recompute is not None:
            self.opt.flags = (self.opt.flags & ~GS_FLAG_BWD_RECOMPUTE) | (GS_FLAG_BWD_RECOMPUTE if bwd_recompute
                                                                          else 0)
        if mode is not None:
            self.opt.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        if bg is not None:
            for k in range(3):
                self.opt.bg[k] = float(bg[k])
        if max_pairs is not None:
            self.opt.max_pairs = int(max_pairs)
        _chk(lib.gs_set_options(self.h, ct.byref(self.opt)), self.h, "gs_set_options")

    def _empty(self, *shape, dtype=None):
        torch = _torch()
        return torch.empty(*shape, dtype=dtype or torch.float32, device="cuda")

    def project(self, scene: DeviceScene, cam: dict, W: int, H: int):
        gs_project(self.h, scene.struct, make_camera(cam), W, H)
        self.W, self.H, self.n, self.scene = W, H, scene.n, scene

    def render_binned(self, grads: bool = True, out_C=None, out_grads=None):
        C = out_C if out_C is not None else self._empty(3, self.H, self.W)
        G = None
        if grads:
            G = out_grads if out_grads is not None else self._empty(3, 3, self.H, self.W)
        gs_render_binned(self.h, C.data_ptr(), G.data_ptr() if G is not None else None)
        return (C, G) if grads else C

    def render_with_grads(self, scene: DeviceScene, cam: dict, W: int, H: int, out_C=None, out_grads=None):
        C = out_C if out_C is not None else self._empty(3, H, W)
        G = out_grads if out_grads is not None else self._empty(3, 3, H, W)
        gs_render_with_grads(self.h, scene.struct, make_camera(cam), W, H, C.data_ptr(), G.data_ptr())
        self.W, self.H, self.n, self.scene = W, H, scene.n, scene
        return C, G

    def render(self, scene: DeviceScene, cam: dict, W: int, H: int, out_C=None):
        C = out_C if out_C is not None else self._empty(3, H, W)
        gs_render(self.h, scene.struct, make_camera(cam), W, H, C.data_ptr())
        self.W, self.H, self.n, self.scene = W, H, scene.n, scene
        return C

    def upscale(self, C, grads, factor: int, out=None):
        H, W = int(C.shape[-2]), int(C.shape[-1])
        assert C.is_contiguous() and grads.is_contiguous()
        o = out if out is not None else self._empty(3, H * factor, W * factor)
        gs_upscale(self.h, C.data_ptr(), grads.data_ptr(), W, H, factor, o.data_ptr())
        return o

    def upscale_to(self, C, grads, W2: int, H2: int, out=None):
        """Spline upscale to any size W2 x H2 (fractional factors)."""
        H, W = int(C.shape[-2]), int(C.shape[-1])
        assert C.is_contiguous() and grads.is_contiguous()
        o = out if out is not None else self._empty(3, H2, W2)
        _chk(lib.gs_upscale_to(self.h, C.data_ptr(), grads.data_ptr(), W, H, W2, H2, o.data_ptr()), self.h,
             "gs_upscale_to")
        return o

    def upscale_bicubic(self, C, W2: int, H2: int, a: float = -0.75, out=None):
        """Classical bicubic comparator (cubic convolution, parameter a) of the colour image."""
        H, W = int(C.shape[-2]), int(C.shape[-1])
        assert C.is_contiguous()
        o = out if out is not None else self._empty(3, H2, W2)
        _chk(lib.gs_upscale_bicubic(self.h, C.data_ptr(), W, H, W2, H2, float(a), o.data_ptr()), self.h,
             "gs_upscale_bicubic")
        return o

    def upscale_mlp(self, C, grads, W2: int, H2: int, params=None, out=None):
        """Spline plus the learned residual (params: FP32 [GS_MLP_PARAMS] on the
        device, or None for the spline alone) at any size W2 x H2."""
        H, W = int(C.shape[-2]), int(C.shape[-1])
        assert C.is_contiguous() and grads.is_contiguous()
        if params is not None:
            assert params.is_contiguous() and params.numel() == GS_MLP_PARAMS
        o = out if out is not None else self._empty(3, H2, W2)
        _chk(lib.gs_upscale_mlp(self.h, C.data_ptr(), grads.data_ptr(), W, H, W2, H2,
                                None if params is None else params.data_ptr(), o.data_ptr()), self.h,
             "gs_upscale_mlp")
        return o

    def mlp_samples(self, C, grads, W2: int, H2: int, pixels, target_image=None, out=None):
        """Training samples at output pixels (int32 [M, 2] of (X, Y) on the device):
        (features int16 [M, GS_MLP_ROW] holding BF16 bit patterns, spline [M, 3],
        target [M, 3] or None)."""
        torch = _torch()
        H, W = int(C.shape[-2]), int(C.shape[-1])
        assert pixels.dtype == torch.int32 and pixels.is_contiguous()
        M = int(pixels.shape[0])
        if out is None:
            feat = torch.empty(M, GS_MLP_ROW, dtype=torch.int16, device="cuda")
            base = self._empty(M, 3)
            tgt = self._empty(M, 3) if target_image is not None else None
        else:
            feat, base, tgt = out
        _chk(lib.gs_mlp_samples(self.h, C.data_ptr(), grads.data_ptr(), W, H, W2, H2, pixels.data_ptr(), M,
                                None if target_image is None else target_image.data_ptr(), feat.data_ptr(),
                                base.data_ptr(), None if tgt is None else tgt.data_ptr()), self.h, "gs_mlp_samples")
        return feat, base, tgt

    def mlp_gradient(self, params, feat, base, target, out=None):
        """(dL/dparams [GS_MLP_PARAMS], L as a device scalar) of the mean squared
        error over the samples."""
        torch = _torch()
        M = int(feat.shape[0])
        g, L = out if out is not None else (self._empty(GS_MLP_PARAMS), self._empty(1))
        _chk(lib.gs_mlp_gradient(self.h, params.data_ptr(), feat.data_ptr(), base.data_ptr(), target.data_ptr(), M,
                                 g.data_ptr(), None if L is None else L.data_ptr()), self.h, "gs_mlp_gradient")
        return g, L

    def mlp_adam(self, params, m, v, grads, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8):
        _chk(lib.gs_mlp_adam(self.h, params.data_ptr(), m.data_ptr(), v.data_ptr(), grads.data_ptr(), int(step),
                             float(lr), float(beta1), float(beta2), float(eps)), self.h, "gs_mlp_adam")

    def upscale_backward_to(self, dout, W: int, H: int, out=None):
        """Adjoint of upscale_to: dL/d(out) [3, H2, W2] -> (dL/dC, dL/dgrads)."""
        assert dout.is_contiguous()
        H2, W2 = int(dout.shape[-2]), int(dout.shape[-1])
        dC, dG = out if out is not None else (self._empty(3, H, W), self._empty(3, 3, H, W))
        _chk(lib.gs_upscale_backward_to(self.h, dout.data_ptr(), W, H, W2, H2, dC.data_ptr(), dG.data_ptr()),
             self.h, "gs_upscale_backward_to")
        return dC, dG

    def pair_count(self) -> int:
        P = ct.c_int64()
        _chk(lib.gs_pair_count(self.h, ct.byref(P)), self.h, "gs_pair_count")
        return int(P.value)

    def super_pair_count(self) -> int:
        P = ct.c_int64()
        _chk(lib.gs_super_pair_count(self.h, ct.byref(P)), self.h, "gs_super_pair_count")
        return int(P.value)

    def read_projected(self) -> dict:
        torch = _torch()
        n = self.n
        out = dict(mean2d=self._empty(n, 2), conic=self._empty(n, 3), rgb=self._empty(n, 3),
                   opacity=self._empty(n), depth=self._empty(n),
                   radius=self._empty(n, dtype=torch.int32), tiles_touched=self._empty(n, dtype=torch.int32))
        _chk(lib.gs_read_projected(self.h, *(out[k].data_ptr() for k in
                                             ("mean2d", "conic", "rgb", "opacity", "depth", "radius",
                                              "tiles_touched"))), self.h, "gs_read_projected")
        return out

    def read_bins(self):
        torch = _torch()
        P = self.pair_count()
        T = ((self.W + 15) // 16) * ((self.H + 15) // 16)
        keys = self._empty(max(P, 1), dtype=torch.int64)
        vals = self._empty(max(P, 1), dtype=torch.int32)
        ranges = self._empty(T, 2, dtype=torch.int32)
        _chk(lib.gs_read_bins(self.h, keys.data_ptr(), vals.data_ptr(), ranges.data_ptr(), max(P, 1)),
             self.h, "gs_read_bins")
        return keys[:P], vals[:P], ranges

    def read_state(self):
        torch = _torch()
        state = self._empty(4, self.H, self.W)
        count = self._empty(self.H, self.W, dtype=torch.int32)
        _chk(lib.gs_read_state(self.h, state.data_ptr(), count.data_ptr()), self.h, "gs_read_state")
        return state, count

    def read_tile_work(self):
        """Per-tile block durations of the last blend (units of 16 SM cycles), [tiles_y, tiles_x]."""
        torch = _torch()
        tx, ty = (self.W + 15) // 16, (self.H + 15) // 16
        out = torch.empty(ty, tx, dtype=torch.int32, device="cuda")
        _chk(lib.gs_read_tile_work(self.h, out.data_ptr()), self.h, "gs_read_tile_work")
        return out

    def blend_stats(self):
        """(pairs evaluated, pairs blended) of the current binning."""
        counts = (ct.c_int64 * 2)()
        _chk(lib.gs_blend_stats(self.h, ct.cast(counts, ct.c_void_p)), self.h, "gs_blend_stats")
        return int(counts[0]), int(counts[1])

    def launch_count(self) -> int:
        n = ct.c_int64()
        _chk(lib.gs_launch_count(self.h, ct.byref(n)), self.h, "gs_launch_count")
        return int(n.value)

    def synchronize(self):
        gs_synchronize(self.h)

    def debug_inject(self, what: int, value: int = 0):
        """Fault injection for the error-path tests (GS_INJECT_*)."""
        gs_debug_inject(self.h, what, value)

    # ---- reverse mode ----------------------------------------------------------

    def upscale_backward(self, dout, W: int, H: int, factor: int, out=None):
        """dL/d(upscaled image) [3, sH, sW] -> (dL/dC [3, H, W], dL/dgrads [3, 3, H, W])."""
        assert dout.is_contiguous()
        dC, dG = out if out is not None else (self._empty(3, H, W), self._empty(3, 3, H, W))
        gs_upscale_backward(self.h, dout.data_ptr(), W, H, factor, dC.data_ptr(), dG.data_ptr())
        return dC, dG

    def render_backward(self, dC, dG=None, out=None):
        """Adjoint of the last derivative blend: -> grad2d [n, 9] (mean_x, mean_y,
        conic a, b, c, opacity, r, g, b)."""
        assert dC.is_contiguous() and (dG is None or dG.is_contiguous())
        g2 = out if out is not None else self._empty(max(self.n, 1), 9)
        gs_render_backward(self.h, dC.data_ptr(), dG.data_ptr() if dG is not None else None, g2.data_ptr())
        return g2[:self.n]

    def _grads_like(self, out=None):
        out = out if out is not None else {k: _torch().empty_like(v) for k, v in self.scene.t.items()}
        g = GsGaussianGrads()
        for k in DeviceScene.FIELDS:
            v = out.get(k)
            setattr(g, k, v.data_ptr() if v is not None and v.numel() > 0 else None)
        return out, g

    def project_backward(self, grad2d, out=None) -> dict:
        """Adjoint of the last projection: grad2d [n, 9] -> gradients of the scene's tensors."""
        assert grad2d.is_contiguous()
        out, g = self._grads_like(out)
        gs_project_backward(self.h, grad2d.data_ptr(), g)
        return out

    def backward(self, dout, factor: int, out=None) -> dict:
        """The whole chain (upscale, blend, projection) for dL/d(upscaled image)."""
        assert dout.is_contiguous()
        out, g = self._grads_like(out)
        gs_backward(self.h, dout.data_ptr(), factor, g)
        return out


def _render_upscale_function():
    torch = _torch()

    class RenderUpscale(torch.autograd.Function):
        """Upscaled image of the Gaussians, differentiable in their tensors.

        forward(context, cam, W, H, factor, means, log_scales, quats,
        opacity_logits, colour) renders W x H with derivatives and upscales by
        factor; colour is the SH tensor [n, K, 3] (sh_degree from its K) or
        direct RGB [n, 3].  backward runs gs_backward.
        """

        @staticmethod
        def forward(actx, gctx, cam, W, H, factor, means, log_scales, quats, opacity_logits, colour):
            t = dict(means=means.contiguous(), log_scales=log_scales.contiguous(), quats=quats.contiguous(),
                     opacity_logits=opacity_logits.contiguous())
            scene = {}
            if colour.dim() == 3:
                t["sh"] = colour.contiguous()
                scene["sh_degree"] = int(round(colour.shape[1] ** 0.5)) - 1
            else:
                t["rgb"] = colour.contiguous()
            dev = DeviceScene(scene, tensors=t)
            dev.sh_degree = scene.get("sh_degree", 0) if "sh" in t else 0
            dev.struct = dev._make()
            C, G = gctx.render_with_grads(dev, cam, W, H)
            out = gctx.upscale(C, G, factor)
            actx.gctx, actx.factor, actx.dev = gctx, factor, dev
            actx.colour_key = "sh" if "sh" in t else "rgb"
            return out

        @staticmethod
        def backward(actx, dout):
            g = actx.gctx.backward(dout.contiguous(), actx.factor)
            return (None, None, None, None, None, g["means"], g["log_scales"], g["quats"], g["opacity_logits"],
                    g[actx.colour_key])

    return RenderUpscale


def render_upscale(gctx: "Context", cam: dict, W: int, H: int, factor: int, means, log_scales, quats,
                   opacity_logits, colour):
    """Differentiable render (W x H, with derivatives) + gradient-aware upscale by factor."""
    global _RenderUpscale
    if _RenderUpscale is None:
        _RenderUpscale = _render_upscale_function()
    return _RenderUpscale.apply(gctx, cam, W, H, factor, means, log_scales, quats, opacity_logits, colour)


_RenderUpscale = None
