"""Training and use of the learned residual on the spline upscale.

The paper's upscaler is the gradient-aware spline alone (Sec. 5).  This module
drives the optional learned part behind the C ABI (gs_upscale_mlp and the
gs_mlp_* calls): a per-output-pixel MLP 50 -> 64 -> 64 -> 3 on the spline's own
48 corner values and the sample point's local coordinates, whose output is
added to the spline.  Every numeric step runs in the library's kernels
(tensor-core forward and reverse mode, Adam); this module only holds the
parameter and moment buffers and orders the calls.

Training pairs are renders of the same scene at low resolution with
derivatives and at the output resolution directly; samples are output pixels
drawn at random from each pair (gs_mlp_samples), the target being the direct
render there.
"""
from __future__ import annotations

import math

import numpy as np

from . import GS_MLP_PARAMS, _torch

SHAPES = (("W1", (64, 50)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (3, 64)), ("b3", (3,)))


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform hidden layers (bound sqrt(6 / fan_in)), zero biases and a zero
    output layer, so the untrained residual is exactly 0 (the spline)."""
    rng = np.random.default_rng(seed)
    parts = {
        "W1": rng.uniform(-1.0, 1.0, (64, 50)) * math.sqrt(6.0 / 50.0),
        "b1": np.zeros(64),
        "W2": rng.uniform(-1.0, 1.0, (64, 64)) * math.sqrt(6.0 / 64.0),
        "b2": np.zeros(64),
        "W3": np.zeros((3, 64)),
        "b3": np.zeros(3),
    }
    flat = np.concatenate([parts[name].reshape(-1) for name, _ in SHAPES]).astype(np.float32)
    assert flat.size == GS_MLP_PARAMS
    return flat


class SampleSet:
    """Training samples on the device: BF16 feature rows [N, 64] (int16 bit
    patterns), spline values [N, 3], targets [N, 3]."""

    def __init__(self, feat, base, target):
        self.feat, self.base, self.target = feat, base, target

    def __len__(self):
        return int(self.feat.shape[0])

    @staticmethod
    def cat(sets):
        torch = _torch()
        return SampleSet(torch.cat([s.feat for s in sets]), torch.cat([s.base for s in sets]),
                         torch.cat([s.target for s in sets]))

    def permuted(self, gen):
        torch = _torch()
        idx = torch.randperm(len(self), generator=gen, device=self.feat.device)
        return SampleSet(self.feat[idx].contiguous(), self.base[idx].contiguous(), self.target[idx].contiguous())

    def slice(self, a: int, b: int):
        return SampleSet(self.feat[a:b], self.base[a:b], self.target[a:b])


def draw_samples(ctx, C, grads, direct, count: int, gen) -> SampleSet:
    """count output pixels drawn uniformly from the direct render's image plane
    (a torch.Generator on the device), as training samples of the low-res render
    (C [3, H, W], grads [3, 3, H, W]) against the direct render [3, H2, W2]."""
    torch = _torch()
    H2, W2 = int(direct.shape[1]), int(direct.shape[2])
    X = torch.randint(0, W2, (count,), generator=gen, device="cuda", dtype=torch.int32)
    Y = torch.randint(0, H2, (count,), generator=gen, device="cuda", dtype=torch.int32)
    pix = torch.stack([X, Y], 1).contiguous()
    feat, base, tgt = ctx.mlp_samples(C, grads, W2, H2, pix, target_image=direct)
    return SampleSet(feat, base, tgt)


class ResidualMLP:
    """Parameters (FP32, on the device), Adam moments and the step count."""

    def __init__(self, ctx, params=None, seed: int = 0):
        torch = _torch()
        self.ctx = ctx
        p = init_params(seed) if params is None else np.asarray(params, np.float32).reshape(-1)
        assert p.size == GS_MLP_PARAMS
        self.params = torch.as_tensor(p).cuda()
        self.m = torch.zeros(GS_MLP_PARAMS, device="cuda")
        self.v = torch.zeros(GS_MLP_PARAMS, device="cuda")
        self.t = 0
        self.grads = torch.empty(GS_MLP_PARAMS, device="cuda")
        self.loss = torch.empty(1, device="cuda")

    def step(self, batch: SampleSet, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        """One Adam step on the mean squared error of the batch; returns the
        batch loss before the step (a device scalar)."""
        self.ctx.mlp_gradient(self.params, batch.feat, batch.base, batch.target, out=(self.grads, self.loss))
        self.t += 1
        self.ctx.mlp_adam(self.params, self.m, self.v, self.grads, self.t, lr, beta1, beta2, eps)
        return self.loss

    def upscale(self, C, grads, W2: int, H2: int, out=None):
        return self.ctx.upscale_mlp(C, grads, W2, H2, params=self.params, out=out)

    def state_dict(self) -> dict:
        return {"params": self.params.detach().cpu(), "m": self.m.detach().cpu(), "v": self.v.detach().cpu(),
                "step": self.t}

    def load_state_dict(self, d: dict):
        self.params.copy_(d["params"])
        self.m.copy_(d["m"])
        self.v.copy_(d["v"])
        self.t = int(d["step"])

    def save(self, path: str):
        _torch().save(self.state_dict(), path)

    def load(self, path: str):
        self.load_state_dict(_torch().load(path))


def train(model: ResidualMLP, samples: SampleSet, steps: int, batch: int = 16384, lr: float = 2e-3,
          lr_final: float | None = None, seed: int = 0):
    """Adam on minibatches of a seeded reshuffle of the samples (one per pass),
    learning rate decayed linearly from lr to lr_final (default lr / 10).
    Returns the device losses of the steps (one tensor)."""
    torch = _torch()
    gen = torch.Generator(device="cuda").manual_seed(seed)
    lr_final = lr / 10.0 if lr_final is None else lr_final
    losses = torch.empty(steps, device="cuda")
    n = len(samples)
    batch = min(batch, n)
    data, pos = samples.permuted(gen), 0
    for k in range(steps):
        if pos + batch > n:
            data, pos = samples.permuted(gen), 0
        a = lr + (lr_final - lr) * (k / max(1, steps - 1))
        losses[k:k + 1].copy_(model.step(data.slice(pos, pos + batch), a))
        pos += batch
    return losses


def psnr(img, ref) -> float:
    """PSNR in dB of img against ref (device tensors [3, H, W]), both clipped to [0, 1]."""
    torch = _torch()
    mse = torch.mean((img.clamp(0, 1) - ref.clamp(0, 1)) ** 2).item()
    return float("inf") if mse == 0 else 10.0 * math.log10(1.0 / mse)
