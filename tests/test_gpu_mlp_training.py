"""Training the learned residual on the GPU with the library's own kernels
(gs_mlp_samples, gs_mlp_gradient and gs_mlp_adam through the residual module):
the training loss falls, and on held-out scenes the spline plus the trained
residual is closer to the direct render than the spline alone."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

W, H, FACTOR = 240, 136, 4
N_GAUSS = 300_000


@pytest.fixture(scope="module")
def gs():
    import torch
    import paper_2503_14171_gb300 as gs
    assert torch.cuda.is_available()
    return gs


def _pairs(gs, ctx, seeds):
    """(C, grads, direct) per seed: the low-res render with derivatives and the
    direct render at FACTOR times the resolution."""
    cam = scenes.pinhole_camera(W, H)
    cam_hi = scenes.scaled_camera(cam, FACTOR)
    out = []
    for s in seeds:
        sc = scenes.mixture_scene_device(N_GAUSS, seed=s)
        dev = gs.DeviceScene({"sh_degree": sc["sh_degree"]}, tensors={k: v for k, v in sc.items() if k != "sh_degree"})
        C, G = ctx.render_with_grads(dev, cam, W, H)
        D = ctx.render(dev, cam_hi, W * FACTOR, H * FACTOR)
        out.append((C, G, D))
    ctx.synchronize()
    return out


def test_training_gain(gs, tmp_path):
    import torch
    from paper_2503_14171_gb300 import residual
    with gs.Context() as ctx:
        train_pairs = _pairs(gs, ctx, range(1000, 1016))
        held_out = _pairs(gs, ctx, range(2000, 2003))
        gen = torch.Generator(device="cuda").manual_seed(0)
        samples = residual.SampleSet.cat([residual.draw_samples(ctx, C, G, D, 32768, gen) for C, G, D in train_pairs])
        model = residual.ResidualMLP(ctx, seed=0)
        losses = residual.train(model, samples, steps=400, batch=16384, lr=2e-3, seed=1).cpu().numpy()
        ctx.synchronize()
        assert np.all(np.isfinite(losses))
        assert losses[-20:].mean() < 0.9 * losses[:5].mean(), (losses[:5].mean(), losses[-20:].mean())
        gain = []
        for C, G, D in held_out:
            spline = ctx.upscale_mlp(C, G, W * FACTOR, H * FACTOR)
            learned = model.upscale(C, G, W * FACTOR, H * FACTOR)
            gain.append(residual.psnr(learned, D) - residual.psnr(spline, D))
        print("held-out PSNR gain (dB):", gain, "loss", losses[0], "->", losses[-20:].mean())
        assert np.mean(gain) > 0.0, gain
        # the state round-trips through a file
        path = str(tmp_path / "mlp.pt")
        model.save(path)
        other = residual.ResidualMLP(ctx, seed=5)
        other.load(path)
        C, G, _ = held_out[0]
        a = model.upscale(C, G, W * FACTOR, H * FACTOR).cpu().numpy()
        b = other.upscale(C, G, W * FACTOR, H * FACTOR).cpu().numpy()
        assert np.array_equal(a, b) and other.t == model.t


def test_untrained_residual_is_the_spline(gs):
    import torch
    from paper_2503_14171_gb300 import residual
    with gs.Context() as ctx:
        (C, G, _), = _pairs(gs, ctx, [7])
        model = residual.ResidualMLP(ctx, seed=3)       # zero output layer
        a = model.upscale(C, G, W * 2, H * 2).cpu().numpy()
        b = ctx.upscale_to(C, G, W * 2, H * 2).cpu().numpy()
        tol = 2e-6 * (1.0 + max(C.abs().max().item(), G.abs().max().item()))
        assert np.abs(a - b).max() <= tol
        assert torch.count_nonzero(model.params).item() > 0
