"""Frames without a host wait (GS_FLAG_NO_HOST_WAIT after gs_reserve): the
same outputs as the default path, device-side capacity overflow reported at
gs_synchronize, and the project -> render -> upscale step captured in a CUDA
graph and replayed on new inputs."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    import torch
    import paper_2503_14171_gb300 as gs
    assert torch.cuda.is_available()
    return gs


def _render(ctx, gs, scene, cam, W, H):
    C, G = ctx.render_with_grads(scene, cam, W, H)
    ctx.synchronize()
    return C.cpu().numpy(), G.cpu().numpy()


CASES = [
    (dict(n=3000, seed=5, sh_degree=3), 77, 45),
    (dict(n=20000, seed=3, xy_range=1.3, log_scale_mean=-3.4), 200, 136),
    (dict(n=1, seed=8), 40, 30),
]


@pytest.mark.parametrize("kw,W,H", CASES)
def test_no_wait_equals_default(gs, kw, W, H):
    scene = gs.DeviceScene(scenes.random_scene(**kw))
    cam = scenes.pinhole_camera(W, H)
    with gs.Context(bg=(0.1, 0.2, 0.3)) as ref:
        want = _render(ref, gs, scene, cam, W, H)
        P = ref.pair_count()
    with gs.Context(bg=(0.1, 0.2, 0.3), no_host_wait=True) as ctx:
        ctx.reserve(scene.n, W, H, 4 * P + 16)
        for _ in range(2):           # twice: scratch reused across frames
            got = _render(ctx, gs, scene, cam, W, H)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
        assert ctx.pair_count() == P


def test_no_wait_requires_reserve_and_bounds(gs):
    scene = gs.DeviceScene(scenes.random_scene(n=100, seed=1))
    with gs.Context(no_host_wait=True) as ctx:
        with pytest.raises(gs.GSError) as e:
            ctx.render_with_grads(scene, scenes.pinhole_camera(32, 32), 32, 32)
        assert e.value.status == gs.GS_ERR_NOT_READY
        ctx.reserve(100, 32, 32, 10000)
        with pytest.raises(gs.GSError) as e:       # image larger than reserved
            ctx.render_with_grads(scene, scenes.pinhole_camera(64, 64), 64, 64)
        assert e.value.status == gs.GS_ERR_CAPACITY
        ctx.render_with_grads(scene, scenes.pinhole_camera(32, 32), 32, 32)
        ctx.synchronize()


def test_no_wait_pair_overflow(gs):
    """Too few reserved pairs: the frame renders as background, the overflow is
    reported at gs_synchronize with the count the frame needed; a larger
    reservation then renders it exactly."""
    W, H = 96, 64
    scene = gs.DeviceScene(scenes.random_scene(n=4000, seed=2))
    cam = scenes.pinhole_camera(W, H)
    bg = (0.3, 0.6, 0.9)
    with gs.Context(bg=bg) as ref:
        want = _render(ref, gs, scene, cam, W, H)
        P = ref.pair_count()
    with gs.Context(bg=bg, no_host_wait=True) as ctx:
        ctx.reserve(scene.n, W, H, 50)
        C, G = ctx.render_with_grads(scene, cam, W, H)
        with pytest.raises(gs.GSError) as e:
            ctx.synchronize()
        assert e.value.status == gs.GS_ERR_CAPACITY
        assert np.allclose(C.cpu().numpy(), np.array(bg, np.float32)[:, None, None])
        assert not G.cpu().numpy().any()
        assert ctx.pair_count() == P
        ctx.reserve(scene.n, W, H, 4 * P)
        got = _render(ctx, gs, scene, cam, W, H)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_no_wait_max_pairs(gs):
    W, H = 64, 64
    scene = gs.DeviceScene(scenes.random_scene(n=2000, seed=4))
    cam = scenes.pinhole_camera(W, H)
    with gs.Context(no_host_wait=True, max_pairs=10) as ctx:
        ctx.reserve(scene.n, W, H, 100000)
        ctx.render_with_grads(scene, cam, W, H)
        with pytest.raises(gs.GSError) as e:
            ctx.synchronize()
        assert e.value.status == gs.GS_ERR_CAPACITY


def test_cuda_graph_capture_and_replay(gs):
    """The whole step (project, derivative blend, 2x upscale) captured once and
    replayed on new Gaussians written into the same device tensors."""
    import torch
    W, H, s = 128, 96, 2
    sc_a = scenes.random_scene(n=6000, seed=11, sh_degree=3)
    sc_b = scenes.random_scene(n=6000, seed=12, sh_degree=3)
    cam = scenes.pinhole_camera(W, H)
    stream = torch.cuda.Stream()
    dev = gs.DeviceScene(sc_a)
    with gs.Context(stream=stream, no_host_wait=True) as ctx:
        ctx.reserve(dev.n, W, H, 200000)
        C = torch.empty(3, H, W, device="cuda")
        G = torch.empty(3, 3, H, W, device="cuda")
        out = torch.empty(3, H * s, W * s, device="cuda")

        def step():
            ctx.project(dev, cam, W, H)
            ctx.render_binned(True, C, G)
            ctx.upscale(C, G, s, out=out)

        with torch.cuda.stream(stream):
            step()                                  # eager warm-up
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            step()
        for sc in (sc_a, sc_b):
            src = gs.DeviceScene(sc)
            for k, v in src.t.items():
                dev.t[k].copy_(v)
            graph.replay()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            with gs.Context() as ref:
                Cr, Gr = ref.render_with_grads(src, cam, W, H)
                want = ref.upscale(Cr, Gr, s).cpu().numpy()
            assert np.array_equal(got, want)
        ctx.synchronize()


def test_backward_after_no_wait_frame(gs):
    import torch
    W, H, s = 64, 48, 2
    scene = gs.DeviceScene(scenes.random_scene(n=800, seed=6, sh_degree=1))
    cam = scenes.pinhole_camera(W, H)
    dout = torch.randn(3, H * s, W * s, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    with gs.Context() as ref:
        ref.render_with_grads(scene, cam, W, H)
        want = {k: v.cpu().numpy() for k, v in ref.backward(dout, s).items()}
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve(scene.n, W, H, 100000)
        ctx.render_with_grads(scene, cam, W, H)
        got = {k: v.cpu().numpy() for k, v in ctx.backward(dout, s).items()}
        ctx.synchronize()
    for k in want:
        np.testing.assert_allclose(got[k], want[k], rtol=1e-4, atol=1e-5 * (np.abs(want[k]).max() + 1e-12))


def test_no_wait_beyond_persistent_sort(gs):
    """More Gaussians than the persistent depth sort holds: the one-sweep depth
    sort shares its look-back state buffer with the pair sort, which must then
    start from cleared states (regression: a no-wait frame here once sorted
    the pairs against stale states)."""
    import torch
    n = 152 * 10240 + 4096
    W, H = 96, 64
    scene = gs.DeviceScene(scenes.random_scene(n=n, seed=35, log_scale_mean=-4.5))
    cam = scenes.pinhole_camera(W, H)
    with gs.Context() as ref:
        want = _render(ref, gs, scene, cam, W, H)
        P = ref.super_pair_count()
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve(n, W, H, P + P // 4 + 64)
        for _ in range(2):
            got = _render(ctx, gs, scene, cam, W, H)   # synchronize: no device error
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    del scene
    torch.cuda.empty_cache()
