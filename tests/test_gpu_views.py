"""Batched views (gs_render_views): every view of a batch -- stereo pairs of
different sizes, one projection launch, one blend launch and one upscale
launch for all -- equals the single-view render of the same camera bit for
bit, upscales included, in every launch shape of the batched blend; the
autotuner picks the fastest shape; the batch replays from a CUDA graph; and
the reservation rules hold."""
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


def stereo_batch(sizes, ipd=0.064, target=(0.0, 0.0, 3.0)):
    """Two cameras (left, right eye) per size, looking at target."""
    cams, szs = [], []
    for k, (W, H) in enumerate(sizes):
        for side in (-0.5, 0.5):
            eye = (side * ipd + 0.05 * k, 0.02 * k, -0.2)
            cams.append(scenes.pinhole_camera(W, H, viewmat=scenes.look_at_viewmat(eye, target)))
            szs.append((W, H))
    return cams, szs


def _single(gs, scene, cam, W, H, bg, factor):
    with gs.Context(bg=bg) as ref:
        C, G = ref.render_with_grads(scene, cam, W, H)
        up = ref.upscale(C, G, factor).cpu().numpy()
        return C.cpu().numpy(), G.cpu().numpy(), up


def _check(gs, scene, cams, szs, factors, outs, bg):
    for v, (cam, (W, H)) in enumerate(zip(cams, szs)):
        C, G, up = _single(gs, scene, cam, W, H, bg, factors[v])
        assert np.array_equal(outs[v][0].cpu().numpy(), C), v
        assert np.array_equal(outs[v][1].cpu().numpy(), G), v
        assert np.array_equal(outs[v][2].cpu().numpy(), up), v


@pytest.mark.parametrize("sh", [3, None])
def test_views_equal_single_view(gs, sh):
    scene = gs.DeviceScene(scenes.random_scene(n=8000, seed=31, sh_degree=sh, xy_range=1.2))
    cams, szs = stereo_batch([(96, 64), (130, 100), (64, 64)])
    factors = [2, 2, 3, 3, 1, 1]
    bg = (0.1, 0.3, 0.5)
    with gs.Context(bg=bg, no_host_wait=True) as ctx:
        ctx.reserve_views(scene.n, len(cams), 130, 100, 400000)
        outs = ctx.render_views(scene, cams, szs, factors)
        ctx.synchronize()
    _check(gs, scene, cams, szs, factors, outs, bg)


@pytest.mark.parametrize("config", range(8))
def test_views_every_launch_shape(gs, config):
    """Each launch shape of the batched blend (warp map x schedule) gives the
    single-view images bit for bit; twice, so that the heaviest-first schedule
    runs on recorded tile durations."""
    scene = gs.DeviceScene(scenes.random_scene(n=12000, seed=36, sh_degree=2, xy_range=1.3, log_scale_mean=-3.3))
    cams, szs = stereo_batch([(150, 110), (77, 45)])
    factors = [2, 2, 3, 3]
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve_views(scene.n, len(cams), 150, 110, 600000)
        ctx.views_config(config % 2, config // 2)
        outs = ctx.render_views(scene, cams, szs, factors)
        outs = ctx.render_views(scene, cams, szs, factors, outs=outs)
        ctx.synchronize()
    _check(gs, scene, cams, szs, factors, outs, (0.0, 0.0, 0.0))


def test_views_autotune(gs):
    scene = gs.DeviceScene(scenes.random_scene(n=10000, seed=37, sh_degree=1))
    cams, szs = stereo_batch([(128, 96), (96, 64)])
    factors = [2] * 4
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve_views(scene.n, len(cams), 128, 96, 500000)
        outs = ctx.render_views(scene, cams, szs, factors)
        ms, best = ctx.autotune_views(scene, cams, szs, factors, outs, reps=3)
        assert len(ms) == gs.GS_VIEWS_CONFIGS and all(t > 0 for t in ms)
        assert 0 <= best < gs.GS_VIEWS_CONFIGS and ms[best] == min(ms)
        outs = ctx.render_views(scene, cams, szs, factors, outs=outs)   # with the chosen shape
        ctx.synchronize()
        with pytest.raises(gs.GSError) as e:
            ctx.views_config(2, 0)
        with pytest.raises(gs.GSError):
            ctx.views_config(0, 4)
        assert e.value.status == gs.GS_ERR_INVALID_ARG
    _check(gs, scene, cams, szs, factors, outs, (0.0, 0.0, 0.0))


@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_views_graph_replay(gs, schedule):
    import torch
    scene = gs.DeviceScene(scenes.random_scene(n=6000, seed=32, sh_degree=1))
    cams, szs = stereo_batch([(80, 60), (112, 80)])
    factors = [2] * 4
    stream = torch.cuda.Stream()
    with gs.Context(stream=stream, no_host_wait=True) as ctx:
        ctx.reserve_views(scene.n, 4, 112, 80, 300000)
        ctx.views_config(0, schedule)
        with torch.cuda.stream(stream):
            outs = ctx.render_views(scene, cams, szs, factors)
        torch.cuda.synchronize()
        eager = [[t.cpu().numpy() for t in o] for o in outs]
        for o in outs:
            for t in o:
                t.zero_()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            ctx.render_views(scene, cams, szs, factors, outs=outs)
        graph.replay()
        torch.cuda.synchronize()
        ctx.synchronize()
    for o, e in zip(outs, eager):
        for t, te in zip(o, e):
            assert np.array_equal(t.cpu().numpy(), te)


def test_views_rules(gs):
    scene = gs.DeviceScene(scenes.random_scene(n=500, seed=33))
    cams, szs = stereo_batch([(64, 48)])
    with gs.Context() as ctx:
        with pytest.raises(gs.GSError) as e:
            ctx.render_views(scene, cams, szs)
        assert e.value.status == gs.GS_ERR_NOT_READY
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve_views(500, 2, 64, 48, 10000)
        with pytest.raises(gs.GSError) as e:          # more views than reserved
            c3, s3 = stereo_batch([(64, 48), (32, 32)])
            ctx.render_views(scene, c3, s3)
        assert e.value.status == gs.GS_ERR_CAPACITY
        with pytest.raises(gs.GSError) as e:          # a view larger than reserved
            c2, s2 = stereo_batch([(96, 48)])
            ctx.render_views(scene, c2, s2)
        assert e.value.status == gs.GS_ERR_CAPACITY
        ctx.render_views(scene, cams, szs)
        ctx.synchronize()


def test_views_beyond_persistent_sort(gs):
    """n above the persistent depth sort's capacity (one block per SM, 10240
    Gaussians each): the views take the one-sweep sort path."""
    import torch
    n = 152 * 10240 + 4096
    scene = gs.DeviceScene(scenes.random_scene(n=n, seed=34, log_scale_mean=-4.5))
    cams, szs = stereo_batch([(64, 48)])
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve_views(n, 2, 64, 48, 4 * n)
        outs = ctx.render_views(scene, cams, szs, [2, 2])
        ctx.synchronize()
    _check(gs, scene, cams, szs, [2, 2], outs, (0.0, 0.0, 0.0))
    del outs
    torch.cuda.empty_cache()


def test_views_at_the_view_limit(gs):
    """32 views (the limit: five view bits above the 32 depth bits of the
    batched sort's keys) of a small scene at small and ragged sizes, and a
    single view (which keeps the persistent depth sort): each equals its
    single-view render bit for bit."""
    scene = gs.DeviceScene(scenes.random_scene(n=3000, seed=38, sh_degree=1, xy_range=1.1))
    sizes = [(16 + 3 * k, 12 + 2 * k) for k in range(16)]
    cams, szs = stereo_batch(sizes)
    assert len(cams) == 32
    factors = [1 + (v % 3) for v in range(32)]
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve_views(scene.n, 32, max(w for w, _ in szs), max(h for _, h in szs), 200000)
        outs = ctx.render_views(scene, cams, szs, factors)
        ctx.synchronize()
    _check(gs, scene, cams, szs, factors, outs, (0.0, 0.0, 0.0))
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve_views(scene.n, 1, 64, 48, 200000)
        one = ctx.render_views(scene, cams[:1], [(64, 48)], [2])
        ctx.synchronize()
    _check(gs, scene, cams[:1], [(64, 48)], [2], one, (0.0, 0.0, 0.0))
