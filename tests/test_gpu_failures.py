"""Failure detection on the GPU without a GPU fault: a bounded device wait that
runs out, and a scratch allocation that fails, each injected through
gs_debug_inject.  The expiry is reported at gs_synchronize as GS_ERR_TIMEOUT,
the allocation failure as GS_ERR_OOM from the call that needed the memory,
and in both cases the context renders the next frame exactly as a fresh one.
Nothing here faults, traps or hangs the GPU: the expired wait polls a device
word that nothing sets for a bounded number of polls."""
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


def _frame(ctx, scene, cam, W, H):
    C, G = ctx.render_with_grads(scene, cam, W, H)
    return C, G


def _same(a, b):
    return all(np.array_equal(x.cpu().numpy(), y.cpu().numpy()) for x, y in zip(a, b))


@pytest.mark.parametrize("polls", [1, 1000])
def test_wait_expiry_is_reported_and_the_context_recovers(gs, polls):
    scene = gs.DeviceScene(scenes.random_scene(n=4000, seed=21, sh_degree=3))
    W, H = 96, 64
    cam = scenes.pinhole_camera(W, H)
    with gs.Context() as ref:
        want = _frame(ref, scene, cam, W, H)
        ref.synchronize()
    with gs.Context() as ctx:
        _frame(ctx, scene, cam, W, H)
        ctx.synchronize()
        ctx.debug_inject(gs.GS_INJECT_WAIT_EXPIRY, polls)
        got = _frame(ctx, scene, cam, W, H)
        with pytest.raises(gs.GSError) as e:
            ctx.synchronize()
        assert e.value.status == gs.GS_ERR_TIMEOUT
        # the injected wait is outside the sort's data path: the frame itself is intact
        assert _same(got, want)
        # one-shot: the next frame is clean and its status is GS_OK
        again = _frame(ctx, scene, cam, W, H)
        ctx.synchronize()
        assert _same(again, want)


def test_wait_expiry_in_a_frame_without_host_wait(gs):
    """The same expiry inside a frame that never blocks the host: reported at
    the next gs_synchronize, the following frame clean."""
    scene = gs.DeviceScene(scenes.random_scene(n=3000, seed=22))
    W, H = 77, 45
    cam = scenes.pinhole_camera(W, H)
    with gs.Context() as ref:
        want = _frame(ref, scene, cam, W, H)
        P = ref.super_pair_count()
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve(scene.n, W, H, 2 * P + 64)
        ctx.debug_inject(gs.GS_INJECT_WAIT_EXPIRY, 100)
        _frame(ctx, scene, cam, W, H)
        with pytest.raises(gs.GSError) as e:
            ctx.synchronize()
        assert e.value.status == gs.GS_ERR_TIMEOUT
        got = _frame(ctx, scene, cam, W, H)
        ctx.synchronize()
        assert _same(got, want)


@pytest.mark.parametrize("countdown", [0, 3, 12])
def test_allocation_failure_is_reported_and_the_context_recovers(gs, countdown):
    """The scratch allocation after `countdown` successful ones fails (as if
    cudaMalloc ran out of memory): the call returns GS_ERR_OOM, and the same
    call then succeeds with the outputs of a fresh context."""
    scene = gs.DeviceScene(scenes.random_scene(n=2500, seed=23))
    W, H = 80, 48
    cam = scenes.pinhole_camera(W, H)
    with gs.Context() as ref:
        want = _frame(ref, scene, cam, W, H)
        ref.synchronize()
    with gs.Context() as ctx:
        ctx.debug_inject(gs.GS_INJECT_ALLOC_FAILURE, countdown)
        with pytest.raises(gs.GSError) as e:
            _frame(ctx, scene, cam, W, H)
        assert e.value.status == gs.GS_ERR_OOM
        assert "injected" in str(e.value)
        got = _frame(ctx, scene, cam, W, H)
        ctx.synchronize()
        assert _same(got, want)


def test_allocation_failure_in_reserve(gs):
    """gs_reserve reports the failure and leaves the context unreserved; a
    second gs_reserve succeeds."""
    scene = gs.DeviceScene(scenes.random_scene(n=500, seed=24))
    cam = scenes.pinhole_camera(32, 32)
    with gs.Context(no_host_wait=True) as ctx:
        ctx.debug_inject(gs.GS_INJECT_ALLOC_FAILURE, 5)
        with pytest.raises(gs.GSError) as e:
            ctx.reserve(500, 32, 32, 20000)
        assert e.value.status == gs.GS_ERR_OOM
        with pytest.raises(gs.GSError) as e:      # not reserved: frames without a host wait are refused
            _frame(ctx, scene, cam, 32, 32)
        assert e.value.status == gs.GS_ERR_NOT_READY
        ctx.reserve(500, 32, 32, 20000)
        _frame(ctx, scene, cam, 32, 32)
        ctx.synchronize()


def test_injection_arguments(gs):
    with gs.Context() as ctx:
        for what, value in ((gs.GS_INJECT_WAIT_EXPIRY, 0), (gs.GS_INJECT_ALLOC_FAILURE, -1), (99, 1)):
            with pytest.raises(gs.GSError) as e:
                ctx.debug_inject(what, value)
            assert e.value.status == gs.GS_ERR_INVALID_ARG
        ctx.debug_inject(gs.GS_INJECT_ALLOC_FAILURE, 0)
        ctx.debug_inject(gs.GS_INJECT_NONE)          # cancelled: the next frame allocates normally
        scene = gs.DeviceScene(scenes.random_scene(n=100, seed=25))
        _frame(ctx, scene, scenes.pinhole_camera(32, 32), 32, 32)
        ctx.synchronize()
