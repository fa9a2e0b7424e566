"""gs_render_with_grads_noalloc (scratch in a static device array, no
allocation) against gs_render_with_grads on the same inputs.

The file name sorts last so that the test also runs after every other GPU test
has used (and grown) the context-based path in the same process."""
import ctypes as ct

import numpy as np
import pytest

import scenes
from helpers import TOL_C, TOL_G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    import torch
    import paper_2503_14171_gb300 as gs
    assert torch.cuda.is_available()
    return gs


def _options(gs, mode="3dgs", bg=(0.0, 0.0, 0.0)):
    o = gs.GsOptions()
    o.tile = 16
    o.mode = gs.MODES[mode]
    for k in range(3):
        o.bg[k] = float(bg[k])
    return o


def _noalloc(gs, scene, cam, W, H, opt=None, fill=None, out=None):
    import torch
    if out is None:
        out = (torch.empty(3, H, W, device="cuda"), torch.empty(3, 3, H, W, device="cuda"))
    C, G = out
    if fill is not None:
        C.fill_(fill)
        G.fill_(fill)
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    gs.gs_render_with_grads_noalloc(scene.struct, gs.make_camera(cam), W, H, opt, stream, C.data_ptr(), G.data_ptr())
    return C, G


def _refused(gs, scene, cam, W, H, opt=None):
    """The call's status; its outputs must still hold the fill value."""
    import torch
    out = (torch.full((3, H, W), 7.0, device="cuda"), torch.full((3, 3, H, W), 7.0, device="cuda"))
    with pytest.raises(gs.GSError) as e:
        _noalloc(gs, scene, cam, W, H, opt, out=out)
    torch.cuda.synchronize()
    assert bool((out[0] == 7.0).all()) and bool((out[1] == 7.0).all()), "a refused call wrote its outputs"
    return e.value.status


def _context(gs, scene, cam, W, H, mode="3dgs", bg=(0.0, 0.0, 0.0)):
    with gs.Context(mode=mode, bg=bg) as ctx:
        C, G = ctx.render_with_grads(scene, cam, W, H)
        ctx.synchronize()
    return C, G


def _assert_close(a, b):
    (Ca, Ga), (Cb, Gb) = a, b
    Ca, Ga, Cb, Gb = (t.cpu().numpy() for t in (Ca, Ga, Cb, Gb))
    assert np.all(np.isfinite(Ca)) and np.all(np.isfinite(Ga))
    assert np.max(np.abs(Ca - Cb), initial=0.0) <= TOL_C
    assert np.all(np.abs(Ga - Gb) <= TOL_G * np.maximum(1.0, np.abs(Gb)))


def _assert_identical(a, b):
    """Both paths run the same kernels on the same inputs: equal bit for bit."""
    (Ca, Ga), (Cb, Gb) = a, b
    assert np.array_equal(Ca.cpu().numpy(), Cb.cpu().numpy())
    assert np.array_equal(Ga.cpu().numpy(), Gb.cpu().numpy())


CASES = [
    # scene kwargs, W, H, mode, bg
    (dict(n=3000, seed=11, sh_degree=3), 96, 64, "3dgs", (0.0, 0.0, 0.0)),
    (dict(n=12000, seed=12, xy_range=1.2, log_scale_mean=-3.3), 200, 136, "exact", (0.2, 0.5, 0.9)),
]


def test_noalloc_two_calls_in_a_row(gs):
    """Two consecutive calls with different scenes, sizes and options, each
    equal to the context-based render."""
    got, want = [], []
    for kw, W, H, mode, bg in CASES:
        scene = gs.DeviceScene(scenes.random_scene(**kw))
        got.append(_noalloc(gs, scene, scenes.pinhole_camera(W, H), W, H, _options(gs, mode, bg)))
    for (kw, W, H, mode, bg), g in zip(CASES, got):
        scene = gs.DeviceScene(scenes.random_scene(**kw))
        want.append(_context(gs, scene, scenes.pinhole_camera(W, H), W, H, mode, bg))
    for g, w in zip(got, want):
        _assert_close(g, w)
        _assert_identical(g, w)


def test_noalloc_repeat_is_identical(gs):
    """Leftover contents of the shared array do not leak into the next call."""
    kw, W, H, mode, bg = CASES[0]
    scene = gs.DeviceScene(scenes.random_scene(**kw))
    cam = scenes.pinhole_camera(W, H)
    a = _noalloc(gs, scene, cam, W, H, _options(gs, mode, bg))
    big = gs.DeviceScene(scenes.random_scene(**CASES[1][0]))
    _noalloc(gs, big, scenes.pinhole_camera(CASES[1][1], CASES[1][2]), CASES[1][1], CASES[1][2])
    b = _noalloc(gs, scene, cam, W, H, _options(gs, mode, bg))
    assert np.array_equal(a[0].cpu().numpy(), b[0].cpu().numpy())
    assert np.array_equal(a[1].cpu().numpy(), b[1].cpu().numpy())


def test_noalloc_default_options_and_empty_scene(gs):
    scene = gs.DeviceScene(scenes.random_scene(n=500, seed=13))
    cam = scenes.pinhole_camera(40, 33)
    _assert_identical(_noalloc(gs, scene, cam, 40, 33, None), _context(gs, scene, cam, 40, 33))
    empty = gs.DeviceScene(scenes.random_scene(n=0, seed=0))
    C, G = _noalloc(gs, empty, cam, 40, 33, _options(gs, "3dgs", (0.3, 0.6, 0.1)))
    C, G = C.cpu().numpy(), G.cpu().numpy()
    assert np.allclose(C, np.array([0.3, 0.6, 0.1], np.float32)[:, None, None])
    assert not G.any()


def test_noalloc_limits(gs):
    """Sizes beyond the static array's limits are refused and nothing is written."""
    cam = scenes.pinhole_camera(64, 64)
    big = gs.DeviceScene(scenes.random_scene(n=16385, seed=14))
    assert _refused(gs, big, cam, 64, 64) == gs.GS_ERR_CAPACITY
    small = gs.DeviceScene(scenes.random_scene(n=100, seed=15))
    assert _refused(gs, small, scenes.pinhole_camera(257, 256), 257, 256) == gs.GS_ERR_CAPACITY
    assert _refused(gs, small, cam, 0, 64) == gs.GS_ERR_INVALID_ARG
    # at the limits themselves the call succeeds
    edge = gs.DeviceScene(scenes.random_scene(n=16384, seed=16, log_scale_mean=-4.0))
    cam = scenes.pinhole_camera(256, 256)
    _assert_identical(_noalloc(gs, edge, cam, 256, 256), _context(gs, edge, cam, 256, 256))


def test_noalloc_super_pair_overflow(gs):
    """Within the Gaussian and pixel limits but beyond the 262144 super-tile
    pairs: exact mode puts each of 5000 Gaussians in all 64 super-tiles of a
    4096 x 16 image (320000 pairs).  The count is known only after the
    projection; the call is still refused with its outputs untouched."""
    scene = gs.DeviceScene(scenes.random_scene(n=5000, seed=17))
    cam = scenes.pinhole_camera(4096, 16)
    assert _refused(gs, scene, cam, 4096, 16, _options(gs, "exact")) == gs.GS_ERR_CAPACITY
    # the same call in 3DGS mode fits, and equals the context path
    _assert_identical(_noalloc(gs, scene, cam, 4096, 16, _options(gs, "3dgs")),
                      _context(gs, scene, cam, 4096, 16, "3dgs"))


def test_noalloc_options(gs):
    """max_pairs is honoured as by the context path; flags are refused."""
    scene = gs.DeviceScene(scenes.random_scene(n=3000, seed=18))
    cam = scenes.pinhole_camera(96, 64)
    with gs.Context() as ctx:
        ctx.render_with_grads(scene, cam, 96, 64)
        P = ctx.pair_count()
    o = _options(gs)
    o.max_pairs = P - 1
    assert _refused(gs, scene, cam, 96, 64, o) == gs.GS_ERR_CAPACITY
    o.max_pairs = P
    _assert_identical(_noalloc(gs, scene, cam, 96, 64, o), _context(gs, scene, cam, 96, 64))
    o.max_pairs = 0
    o.flags = 1
    assert _refused(gs, scene, cam, 96, 64, o) == gs.GS_ERR_INVALID_ARG
