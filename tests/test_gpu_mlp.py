"""GPU parity of the learned residual (the tcgen05 kernels behind
gs_upscale_mlp, gs_mlp_samples, gs_mlp_gradient, gs_mlp_adam) against the
FP64 oracle (oracle.mlp), through the C ABI.

Rules (helpers_mlp): the reference takes the BF16 narrowing decisions in the
kernels' precision; what remains is FP32 accumulation with derived bounds,
one BF16 step where a value sits at a rounding boundary, and samples with an
ambiguous ReLU decision left out.  The spline part of gs_upscale_mlp is held
to the spline's own tolerance, |gpu - ref| <= TOL_UP (1 + max |input|)."""
import numpy as np
import pytest

from helpers import TOL_UP
from helpers_mlp import bf16_params, forward_reference, gradient_reference, q, random_theta
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    import torch
    import paper_2503_14171_gb300 as gs
    assert torch.cuda.is_available()
    return gs


def _t(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype or np.float32)).cuda()


def _planes(W, H, seed):
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 1, size=(3, H, W)).astype(np.float32)
    G = rng.normal(0, 0.3, size=(3, 3, H, W)).astype(np.float32)
    return C, G


def _bits(feat_rows):
    """BF16 feature rows [M, 64] as float64 [M, 64]."""
    b = np.asarray(feat_rows).astype(np.int32).view(np.uint32) & 0xFFFF
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _rows(f):
    """float64 features [M, 50] holding BF16 values -> int16 rows [M, 64] of their bits."""
    bits = (np.asarray(q(f), np.float32).view(np.uint32) >> 16).astype(np.uint16)
    out = np.zeros((f.shape[0], 64), np.uint16)
    out[:, :50] = bits
    return out.view(np.int16)


SIZES = [
    (37, 23, 148, 92),     # 4x, ragged tiles of 128 output pixels
    (16, 12, 24, 18),      # 1.5x
    (64, 40, 128, 80),     # 2x
    (2, 2, 9, 7),          # smallest input
    (30, 17, 30, 17),      # 1x
    (61, 35, 244, 140),    # 4x, 267 tiles (several per CTA at small grids)
]


@pytest.mark.parametrize("W,H,W2,H2", SIZES)
def test_upscale_mlp_matches_oracle(gs, ora, W, H, W2, H2):
    C, G = _planes(W, H, W2 * 7 + H2)
    theta = bf16_params(random_theta(np.random.default_rng(W2)))
    with gs.Context() as ctx:
        got = ctx.upscale_mlp(_t(C), _t(G), W2, H2, params=_t(theta)).cpu().numpy()
        ctx.synchronize()
    f = mlp.features(C.astype(np.float64), G.astype(np.float64), W2, H2)
    ref = forward_reference(theta, f)
    spline = ora.upscale(C.astype(np.float64), G.astype(np.float64), W2, H2)
    want = spline + ref["r"].T.reshape(3, H2, W2)
    tol = TOL_UP * (1.0 + max(np.abs(C).max(), np.abs(G).max())) + ref["e3"].T.reshape(3, H2, W2)
    keep = ref["keep"].reshape(H2, W2)
    assert keep.mean() > 0.9
    bad = (np.abs(got - want) > tol) & keep[None]
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(got - want)[:, keep] / tol[:, keep])))
    # the residual is not negligible: the comparison tests the network
    assert np.abs(ref["r"]).mean() > 0.05


def test_spline_fallback_is_upscale_to(gs):
    C, G = _planes(45, 29, 1)
    with gs.Context() as ctx:
        a = ctx.upscale_mlp(_t(C), _t(G), 90, 58).cpu().numpy()
        b = ctx.upscale_to(_t(C), _t(G), 90, 58).cpu().numpy()
    assert np.array_equal(a, b)


def test_zero_network_is_the_spline(gs, ora):
    C, G = _planes(33, 20, 2)
    with gs.Context() as ctx:
        got = ctx.upscale_mlp(_t(C), _t(G), 132, 80, params=_t(np.zeros(mlp.N_PARAMS))).cpu().numpy()
    want = ora.upscale(C.astype(np.float64), G.astype(np.float64), 132, 80)
    assert np.abs(got - want).max() <= TOL_UP * (1.0 + max(np.abs(C).max(), np.abs(G).max()))


@pytest.mark.parametrize("M", [1, 1000])
def test_samples_match_oracle(gs, ora, M):
    W, H, W2, H2 = 50, 31, 200, 124
    C, G = _planes(W, H, 3)
    rng = np.random.default_rng(M)
    img = rng.uniform(0, 1, (3, H2, W2)).astype(np.float32)
    pix = np.stack([rng.integers(0, W2, M), rng.integers(0, H2, M)], 1).astype(np.int32)
    pix[0] = (W2 - 1, H2 - 1)
    with gs.Context() as ctx:
        feat, base, tgt = ctx.mlp_samples(_t(C), _t(G), W2, H2, _t(pix, np.int32), target_image=_t(img))
        ctx.synchronize()
        feat, base, tgt = feat.cpu().numpy(), base.cpu().numpy(), tgt.cpu().numpy()
    f = _bits(feat)
    want = q(mlp.features(C.astype(np.float64), G.astype(np.float64), W2, H2, pix))
    assert np.array_equal(f[:, :50], want)
    assert not f[:, 50:].any()
    spline = ora.upscale(C.astype(np.float64), G.astype(np.float64), W2, H2, pixels=pix)
    assert np.abs(base - spline).max() <= TOL_UP * (1.0 + max(np.abs(C).max(), np.abs(G).max()))
    assert np.array_equal(tgt, img[:, pix[:, 1], pix[:, 0]].T)


def test_samples_reject_outside_pixels(gs):
    C, G = _planes(8, 8, 4)
    pix = np.array([[0, 0], [16, 3]], np.int32)
    with gs.Context() as ctx:
        ctx.mlp_samples(_t(C), _t(G), 16, 16, _t(pix, np.int32))
        with pytest.raises(gs.GSError) as e:
            ctx.synchronize()
        assert e.value.status == gs.GS_ERR_DEVICE_CHECK


def _train_data(seed, M):
    rng = np.random.default_rng(seed)
    f = q(np.concatenate([rng.normal(0, 1.0, (M, 48)), rng.uniform(-0.4, 1.4, (M, 2))], 1))
    theta = bf16_params(random_theta(rng))
    base = rng.uniform(0, 1, (M, 3))
    target = base + rng.normal(0, 0.3, (M, 3))
    keep = forward_reference(theta, f)["keep"]
    return theta, f[keep], base[keep].astype(np.float32), target[keep].astype(np.float32)


@pytest.mark.parametrize("M", [100, 1000, 128 * 152 * 2 + 77])
def test_gradient_matches_oracle(gs, M):
    theta, f, base, target = _train_data(M, M)
    g_ref, bound, L_ref, eL = gradient_reference(theta, f, base, target)
    with gs.Context() as ctx:
        g, L = ctx.mlp_gradient(_t(theta), _t(_rows(f), np.int16), _t(base), _t(target))
        ctx.synchronize()
        g, L = g.cpu().numpy().astype(np.float64), float(L.cpu().numpy()[0])
    bad = np.abs(g - g_ref) > bound
    if bad.any():
        names = [n for n, s in mlp.SHAPES for _ in range(int(np.prod(s)))]
        worst = int(np.argmax(np.abs(g - g_ref) / bound))
        raise AssertionError(f"{int(bad.sum())} of {g.size} outside; worst {names[worst]} "
                             f"got {g[worst]:.6g} want {g_ref[worst]:.6g} bound {bound[worst]:.3g}")
    assert abs(L - L_ref) <= eL + 1e-7 * L_ref
    for name, a in mlp.unpack(g_ref).items():
        assert np.abs(a).max() > 0, name


def test_gradient_of_no_samples_is_zero(gs):
    theta = bf16_params(random_theta(np.random.default_rng(0)))
    import torch
    with gs.Context() as ctx:
        g = torch.full((mlp.N_PARAMS,), 7.0, device="cuda")
        L = torch.full((1,), 7.0, device="cuda")
        e = torch.empty(0, 64, dtype=torch.int16, device="cuda")
        z = torch.empty(0, 3, device="cuda")
        ctx.mlp_gradient(_t(theta), e, z, z, out=(g, L))
        ctx.synchronize()
    assert not g.cpu().numpy().any() and float(L.cpu()[0]) == 0.0


@pytest.mark.parametrize("step", [1, 7])
def test_adam_matches_oracle(gs, step):
    """The kernel receives the hyper-parameters as FP32, so the oracle gets the
    same FP32 values; each FP32 operation then rounds once (relative 2^-24)."""
    rng = np.random.default_rng(step)
    n = mlp.N_PARAMS
    theta = rng.normal(0, 0.3, n).astype(np.float32)
    m = rng.normal(0, 0.01, n).astype(np.float32) * (step > 1)
    v = (rng.uniform(0, 1e-4, n) * (step > 1)).astype(np.float32)
    g = rng.normal(0, 0.05, n).astype(np.float32)
    lr, b1, b2, eps = (float(np.float32(x)) for x in (2e-3, 0.9, 0.999, 1e-8))
    _, m_ref, v_ref = mlp.adam(theta, m, v, g, step, lr, b1, b2, eps)
    P, Mt, Vt = _t(theta), _t(m), _t(v)
    with gs.Context() as ctx:
        ctx.mlp_adam(P, Mt, Vt, _t(g), step, lr, b1, b2, eps)
        ctx.synchronize()
    u = 2.0 ** -24
    mg, vg = Mt.cpu().numpy().astype(np.float64), Vt.cpu().numpy().astype(np.float64)
    g64 = g.astype(np.float64)
    assert np.all(np.abs(mg - m_ref) <= 4 * u * (b1 * np.abs(m) + (1 - b1) * np.abs(g64)))
    assert np.all(np.abs(vg - v_ref) <= 4 * u * (b2 * v + (1 - b2) * g64 * g64))
    # the update from the kernel's own moments, with the bias corrections
    c1, c2 = 1.0 / (1.0 - b1 ** step), 1.0 / (1.0 - b2 ** step)
    upd = lr * (mg * c1) / (np.sqrt(vg * c2) + eps)
    dt = P.cpu().numpy().astype(np.float64) - theta
    assert np.all(np.abs(dt + upd) <= 12 * u * np.abs(upd) + 2 * u * np.abs(theta))


def test_mlp_argument_rules(gs):
    C, G = _planes(8, 8, 5)
    theta = _t(np.zeros(mlp.N_PARAMS))
    with gs.Context() as ctx:
        with pytest.raises(gs.GSError) as e:
            ctx.upscale_mlp(_t(C), _t(G), 7, 8, params=theta)
        assert e.value.status == gs.GS_ERR_INVALID_ARG
        with pytest.raises(gs.GSError) as e:
            ctx.mlp_adam(theta, theta, theta, theta, 0, 1e-3)
        assert e.value.status == gs.GS_ERR_INVALID_ARG
