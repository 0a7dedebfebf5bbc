"""The learned starting density on the GPU (sq3_mlp_*) against its FP64
oracle (oracle.mlp): descriptors, prediction, loss and the back-propagated
gradient of every parameter block, and Adam training.

The GPU multiplies BF16 operands (features, activations, weights) on the
tensor cores with FP32 accumulation.  BF16 keeps 8 significant bits (unit
roundoff 2^-9 = 2e-3); every layer rounds its input once, so the
prediction carries a few 1e-3 of relative error and the gradient, which
passes through the layers twice, about 1e-2.  The tolerances below are
that budget: 1e-2 relative on the density and the loss, 5e-2 relative (L2
over each parameter block) on the gradient."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2112_08639_gb300 import inputs

from gpu_common import need_gpu, sq3

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _flat(p):
    return np.concatenate([np.ravel(p[k]) for k in omlp.LAYER_NAMES]).astype(np.float32)


def _unflat(a, F):
    shapes = {"W1": (128, F), "b1": (128,), "W2": (128, 128), "b2": (128,), "W3": (128, 128),
              "b3": (128,), "w4": (128,), "b4": (1,)}
    out, i = {}, 0
    for k in omlp.LAYER_NAMES:
        n = int(np.prod(shapes[k]))
        out[k] = np.asarray(a[i:i + n], dtype=np.float64).reshape(shapes[k])
        i += n
    return out


def _bf16(x):
    """Round to the nearest BF16 value (ties to even) in float64."""
    t = torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float64)
    return t.numpy()


def _setup(seed=0, n=18):
    cfg = inputs.C1
    L = cfg.L
    pos = inputs.fcc_positions(1, disp_sigma=0.2, seed=seed)
    ctx = sq3().Context(0)
    ctx.setup_grid(n, n, n, L, L, L, 12)
    p = omlp.init_params(seed=seed)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(size=128) * 0.2
    for k in ("W1", "W2", "W3"):
        p[k] = _bf16(p[k])
    p["b4"] = np.array([0.1])
    p = _unflat(_flat(p), len(omlp.WIDTHS))        # float32-representable
    m = sq3().MLP(ctx, omlp.WIDTHS, seed=seed)
    m.set_params(_flat(p))
    m.features(pos)
    X = omlp.descriptors(n, L, pos)
    return ctx, m, p, X, pos, (L / n) ** 3


def test_parameters_round_trip_and_count():
    ctx, m, p, _, _, _ = _setup()
    assert m.n_params == 128 * len(omlp.WIDTHS) + 33281
    np.testing.assert_array_equal(m.get_params(), _flat(p))


def test_prediction_matches_oracle():
    ctx, m, p, X, pos, dV = _setup(1)
    Ne = 12.0
    rho = m.predict(Ne).cpu().numpy()
    ref = omlp.predict(p, X, Ne, dV)
    assert np.max(np.abs(rho - ref)) < 1e-2 * np.max(ref)
    assert abs(rho.sum() * dV - Ne) < 1e-10 * Ne


def test_loss_and_gradient_match_oracle():
    ctx, m, p, X, pos, dV = _setup(2)
    Ne = 12.0
    n = round((X.shape[0]) ** (1 / 3))
    from oracle import guess
    target = guess.superposition(n, inputs.C1.L, pos, Ne, 1.5)
    loss, g = m.gradient(torch.from_numpy(target).cuda(), Ne)
    Lref, gref = omlp.loss_and_grad(p, X, target, Ne, dV)
    assert abs(loss - Lref) < 1e-2 * Lref
    gg = _unflat(g, len(omlp.WIDTHS))
    for k in omlp.LAYER_NAMES:
        err = np.linalg.norm(gg[k] - gref[k]) / np.linalg.norm(gref[k])
        assert err < 5e-2, (k, err)


def test_training_on_the_gpu_tracks_the_oracle():
    """Twenty Adam steps from the same start on both sides.  The first loss
    (before any step) agrees to the BF16 budget (2 %); after that the BF16
    and FP64 trajectories drift apart (Adam's normalised steps amplify the
    rounding of small gradient components), so the GPU is only required to
    lower the loss like the oracle: below 0.8 of the start after twenty
    steps, and within 30 % of the oracle's loss there."""
    ctx, m, p, X, pos, dV = _setup(3)
    Ne = 12.0
    from oracle import guess
    n = round((X.shape[0]) ** (1 / 3))
    target = guess.superposition(n, inputs.C1.L, pos, Ne, 1.4)
    tgt = torch.from_numpy(target).cuda()
    opt = omlp.Adam(p, lr=2e-3)
    first = None
    for step in range(20):
        lg = m.train_step(tgt, Ne, 2e-3)
        lo, g = omlp.loss_and_grad(p, X, target, Ne, dV)
        opt.step(p, g)
        if first is None:
            first = lo
            assert abs(lg - lo) < 0.02 * lo
    final = m.gradient(tgt, Ne)[0]
    lo_final = omlp.loss(p, X, target, Ne, dV)
    assert final < 0.8 * first and abs(final - lo_final) < 0.3 * lo_final


def test_error_paths():
    mod = sq3()
    ctx = mod.Context(0)
    ctx.setup_grid(8, 8, 8, 4.0, 4.0, 4.0, 12)
    m = mod.MLP(ctx, [1.0, 2.0])
    with pytest.raises(mod.SQ3Error) as e:
        m.predict(3.0)                       # no features yet
    assert e.value.code == mod.ENOTSETUP
    bad = m.get_params()
    bad[5] = np.nan
    with pytest.raises(mod.SQ3Error) as e:
        m.set_params(bad)
    assert e.value.code == mod.EINVAL
    with pytest.raises(mod.SQ3Error) as e:
        mod.MLP(ctx, [1.0] * 17)
    assert e.value.code == mod.EINVAL
