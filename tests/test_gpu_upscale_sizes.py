"""GPU parity of the upscale at fractional factors (gs_upscale_to and its
adjoint gs_upscale_backward_to) and of the classical bicubic comparator
(gs_upscale_bicubic), against the FP64 oracle on the same inputs.

Tolerance: FP32 evaluation of a fixed number of weighted terms (16 for the
spline, 16 taps for the bicubic) on identical inputs, |gpu - ref| <=
TOL_UP (1 + max |input|); for the adjoint the number of summed terms grows
with the factor, so the bound scales by the (2 s + 2)^2 output pixels each
low-res value gathers."""
import numpy as np
import pytest

from helpers import TOL_UP

pytestmark = pytest.mark.gpu

SIZES = [
    (16, 12, 24, 18),      # 1.5x
    (77, 45, 100, 60),     # ragged, 1.30 x 1.33
    (33, 17, 70, 40),      # 2.12 x 2.35
    (40, 30, 40, 30),      # 1x
    (19, 23, 300, 100),    # 15.8 x 4.35
    (2, 2, 7, 3),          # smallest spline input
    (130, 70, 195, 105),   # several 64 x 16 output tiles, 1.5x
]


@pytest.fixture(scope="module")
def gs():
    import torch
    import paper_2503_14171_gb300 as gs
    assert torch.cuda.is_available()
    return gs


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda()


def _inputs(W, H, seed):
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 1, size=(3, H, W)).astype(np.float32)
    G = rng.normal(0, 0.3, size=(3, 3, H, W)).astype(np.float32)
    return C, G


@pytest.mark.parametrize("W,H,W2,H2", SIZES)
def test_upscale_fractional(gs, ora, W, H, W2, H2):
    C, G = _inputs(W, H, W2 + H2)
    want = ora.upscale(C.astype(np.float64), G.astype(np.float64), W2, H2)
    with gs.Context() as ctx:
        got = ctx.upscale_to(_t(C), _t(G), W2, H2).cpu().numpy()
    scale = 1.0 + max(np.abs(C).max(), np.abs(G).max())
    assert np.abs(got - want).max() <= TOL_UP * scale


@pytest.mark.parametrize("factor", [1, 2, 3, 4, 7, 16])
def test_upscale_to_equals_integer_factor(gs, factor):
    C, G = _inputs(45, 29, factor)
    with gs.Context() as ctx:
        a = ctx.upscale(_t(C), _t(G), factor).cpu().numpy()
        b = ctx.upscale_to(_t(C), _t(G), 45 * factor, 29 * factor).cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("a", [-0.75, -0.5])
@pytest.mark.parametrize("W,H,W2,H2", SIZES + [(1, 1, 5, 4), (3, 1, 9, 2)])
def test_bicubic(gs, ora, a, W, H, W2, H2):
    C, _ = _inputs(W, H, 7 * W2 + H2)
    want = ora.bicubic(C.astype(np.float64), W2, H2, a=a)
    with gs.Context() as ctx:
        got = ctx.upscale_bicubic(_t(C), W2, H2, a=a).cpu().numpy()
    assert np.abs(got - want).max() <= 2 * TOL_UP * (1.0 + np.abs(C).max())


@pytest.mark.parametrize("W,H,W2,H2", SIZES)
def test_upscale_backward_fractional(gs, ora, W, H, W2, H2):
    rng = np.random.default_rng(W2 * 3 + H2)
    dout = rng.normal(size=(3, H2, W2)).astype(np.float32)
    want_C, want_G = ora.upscale_adjoint(dout.astype(np.float64), W, H)
    with gs.Context() as ctx:
        dC, dG = ctx.upscale_backward_to(_t(dout), W, H)
        dC, dG = dC.cpu().numpy(), dG.cpu().numpy()
    s = max(W2 / W, H2 / H)
    scale = 1.0 + np.abs(dout).max() * (2 * s + 2) ** 2
    assert np.abs(dC - want_C).max() <= TOL_UP * scale
    assert np.abs(dG - want_G).max() <= TOL_UP * scale


def test_size_rules(gs):
    C, G = _inputs(8, 8, 0)
    with gs.Context() as ctx:
        for W2, H2 in ((7, 8), (8, 7), (8 * 16 + 1, 8), (8, 8 * 16 + 1)):
            with pytest.raises(gs.GSError) as e:
                ctx.upscale_to(_t(C), _t(G), W2, H2)
            assert e.value.status == gs.GS_ERR_INVALID_ARG
            with pytest.raises(gs.GSError) as e:
                ctx.upscale_bicubic(_t(C), W2, H2)
            assert e.value.status == gs.GS_ERR_INVALID_ARG
        with pytest.raises(gs.GSError) as e:
            ctx.upscale_bicubic(_t(C), 16, 16, a=0.5)
        assert e.value.status == gs.GS_ERR_INVALID_ARG


@pytest.mark.parametrize("W,H,W2,H2", [(960, 540, 1920, 1080), (64, 32, 64, 32), (64, 64, 128, 128),
                                       (132, 70, 264, 140), (100, 60, 150, 90), (4, 2, 5, 2), (8, 6, 8, 6),
                                       (480, 270, 1920, 1080)])
def test_tma_fed_equals_staged(gs, ora, W, H, W2, H2):
    """Frames with 16-byte rows, aligned planes and footprints of more than
    512 low-res pixels per output tile (factors up to ~2.2; the last case,
    4x, does not qualify) take the TMA-fed persistent form; the same values
    one float off a 16-byte boundary take the staged form.  Both evaluate the
    same products and sums: bit-identical outputs, and the smaller frames
    within the spline tolerance of the oracle."""
    import torch
    C, G = _inputs(W, H, W * 7 + H2)
    n3, n9 = 3 * H * W, 9 * H * W
    buf = torch.zeros(1 + n3 + n9 + 3, device="cuda")
    Cu = buf[1:1 + n3].view(3, H, W)      # 4 bytes past a 16-byte boundary
    Gu = buf[1 + n3:1 + n3 + n9].view(9, H, W)
    Cu.copy_(_t(C))
    Gu.copy_(_t(G.reshape(9, H, W)))
    assert Cu.data_ptr() % 16 != 0
    with gs.Context() as ctx:
        fed = ctx.upscale_to(_t(C), _t(G), W2, H2)
        staged = ctx.upscale_to(Cu, Gu, W2, H2)
        ctx.synchronize()
    assert torch.equal(fed, staged)
    if W * H <= 140 * 80:
        want = ora.upscale(C.astype(np.float64), G.astype(np.float64), W2, H2)
        scale = 1.0 + max(np.abs(C).max(), np.abs(G).max())
        assert np.abs(fed.cpu().numpy() - want).max() <= TOL_UP * scale
