"""Pins of the FP64 oracle's codec pieces: rounding against library conversions,
the block layout against coordinate-encoded fields, GELU identities, the training
gradient against finite differences, LAMB's trust-ratio invariant, and the linear
autoencoder reaching the Eckart-Young (PCA) optimum (Sec. 1).  CPU only."""
import numpy as np
import pytest
import torch

from oracle import codec as C


def test_round_bf16_matches_torch_on_fp32_values():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(C.round_bf16(x.astype(np.float64)), want)


def test_round_bf16_ties_to_even():
    u = 2.0 ** -8   # half an ulp of bf16 at 1.0
    assert C.round_bf16(1.0 + u) == 1.0
    assert C.round_bf16(1.0 + 3 * u) == 1.0 + 4 * u
    assert C.round_bf16(-(1.0 + u * 1.0000001)) == -(1.0 + 2 * u)


def test_round_fp16_matches_numpy():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(20000) * np.exp(rng.uniform(-18, 11, 20000))
    want = x.astype(np.float16).astype(np.float64)
    np.testing.assert_array_equal(C.round_fp16(x), want)


def test_block_layout_from_coordinate_encoded_fields():
    nz, ny, nx = 16, 24, 8
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    fields = [f * 1e6 + k * 1e4 + j * 1e2 + i for f in range(4)]
    X = C.pack_blocks(fields)
    NBy, NBx = ny // 8, nx // 8
    rng = np.random.default_rng(2)
    for _ in range(200):
        b = rng.integers(X.shape[0]); kk = rng.integers(2048)
        v = X[b, kk]
        f, rest = divmod(v, 1e6); kz, rest = divmod(rest, 1e4); jy, ix = divmod(rest, 1e2)
        z, r = divmod(kk, 256); ff, r = divmod(r, 64); y, x = divmod(r, 8)
        bz, r = divmod(b, NBy * NBx); by, bx = divmod(r, NBx)
        assert (f, kz, jy, ix) == (ff, 8 * bz + z, 8 * by + y, 8 * bx + x)
    for f in range(4):
        np.testing.assert_array_equal(C.unpack_field(X, (nz, ny, nx), f), fields[f])


def test_block_scales_are_powers_of_two_bracketing_the_block_max():
    rng = np.random.default_rng(3)
    st = [rng.standard_normal((16, 8, 24)) * 10.0 ** rng.uniform(-20, 5) for _ in range(4)]
    st[2][:8, :, 8:16] = 0.0                     # one all-zero block-field
    s = C.block_scales(st)
    X = C.pack_blocks(st)
    # brute force: loop over blocks and fields
    for b in range(X.shape[0]):
        for f in range(4):
            m = max(abs(v) for v in X[b, C.field_columns(f)])
            if m == 0:
                assert s[b, f] == 0
            else:
                e = np.log2(s[b, f])
                assert e == np.round(e)              # a power of two
                assert s[b, f] / 2 <= m < s[b, f]


def test_block_scale_exponent_is_clamped_for_tiny_blocks():
    st = [np.full((8, 8, 8), v) for v in (1e-40, -3e-35, 1e-28, 0.0)]
    s = C.block_scales(st)
    assert s[0, 0] == s[0, 1] == 2.0 ** -100      # clamped (maxima below 2^-101)
    assert s[0, 2] == 2.0 ** -93                  # 1e-28 = 0.99 * 2^-93: not clamped
    assert s[0, 3] == 0
    assert np.isfinite(1.0 / np.float32(s[0, 0]))


def test_normalise_per_block_bounds_and_zero_blocks():
    rng = np.random.default_rng(4)
    st = [rng.standard_normal((8, 8, 16)) * 10.0 ** (-3 * f) for f in range(4)]
    st[1][:, :, :8] = 0.0
    s = C.block_scales(st)
    Y = C.normalise(C.pack_blocks(st), s)
    for f in range(4):
        blk = np.abs(Y[:, C.field_columns(f)]).max(axis=1)
        live = s[:, f] > 0
        assert np.all((blk[live] >= 0.5) & (blk[live] < 1.0))
        assert np.all(blk[~live] == 0)
    # scaling by a power of two commutes with BF16 rounding (exactness of the scale)
    X = C.pack_blocks(st)
    sv = C.normalise(np.ones_like(X), s)         # 1/s per entry (0 where s = 0)
    np.testing.assert_array_equal(C.round_bf16(X) * sv, C.round_bf16(X * sv))


def test_gelu_identities():
    x = np.linspace(-6, 6, 1001)
    assert C.gelu(0.0) == 0.0
    np.testing.assert_allclose(C.gelu(x) - C.gelu(-x), x, atol=1e-14)   # x Phi(x) + x Phi(-x) = x
    assert C.gelu(10.0) == pytest.approx(10.0, abs=1e-15)
    assert C.gelu_prime(0.0) == 0.5
    fd = (C.gelu(x + 1e-6) - C.gelu(x - 1e-6)) / 2e-6
    np.testing.assert_allclose(C.gelu_prime(x), fd, atol=1e-8)


def _small_weights(rng, d=16, hdim=8, k=4):
    return {"W1": rng.uniform(-.5, .5, (d, hdim)), "b1": rng.uniform(-.1, .1, hdim),
            "W2": rng.uniform(-.5, .5, (hdim, k)), "b2": rng.uniform(-.1, .1, k),
            "W3": rng.uniform(-.5, .5, (k, hdim)), "b3": rng.uniform(-.1, .1, hdim),
            "W4": rng.uniform(-.5, .5, (hdim, d)), "b4": rng.uniform(-.1, .1, d)}


def test_training_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    Wt = _small_weights(rng)
    Y = rng.uniform(-1, 1, (32, 16))
    _, g = C.loss_and_grad(Wt, Y)
    eps = 1e-6
    for name in C.PARAMS:
        flat = Wt[name].ravel()
        for idx in rng.choice(flat.size, size=min(5, flat.size), replace=False):
            Wp = {k: v.copy() for k, v in Wt.items()}; Wm = {k: v.copy() for k, v in Wt.items()}
            Wp[name].ravel()[idx] += eps; Wm[name].ravel()[idx] -= eps
            fd = (C.loss_and_grad(Wp, Y)[0] - C.loss_and_grad(Wm, Y)[0]) / (2 * eps)
            assert fd == pytest.approx(g[name].ravel()[idx], rel=1e-6, abs=1e-10), (name, idx)


def test_lamb_update_norm_is_lr_times_weight_norm():
    """With zero weight decay the LAMB step of every tensor has norm lr |w|."""
    rng = np.random.default_rng(5)
    Wt = _small_weights(rng)
    opt = C.Lamb(Wt)
    for t in range(5):
        g = {k: rng.standard_normal(v.shape) for k, v in Wt.items()}
        new = opt.step(Wt, g, lr=1e-2)
        for k in Wt:
            step = np.linalg.norm(new[k] - Wt[k])
            assert step == pytest.approx(1e-2 * np.linalg.norm(Wt[k]), rel=1e-12)
        Wt = new
    # first step: bias-corrected moments give u = g / (|g| + eps), i.e. ~ sign(g)
    opt = C.Lamb(Wt)
    g = {k: rng.standard_normal(v.shape) for k, v in Wt.items()}
    new = opt.step(Wt, g, lr=1e-3)
    d = -(new["W1"] - Wt["W1"])
    assert np.all(np.sign(d) == np.sign(g["W1"]))


def test_linear_autoencoder_reaches_pca_optimum():
    """Sec. 1: a linear autoencoder learns the PCA subspace; trained with the oracle's
    gradient and LAMB it must reach the Eckart-Young error of a rank-k truncated SVD of
    the centred data, and can never go below it."""
    rng = np.random.default_rng(0)
    d, k, B = 32, 4, 256
    U = np.linalg.qr(rng.standard_normal((d, d)))[0]
    Y = (rng.standard_normal((B, d)) * np.exp(-np.arange(d) / 3.0)) @ U.T + 0.3
    s = np.linalg.svd(Y - Y.mean(0), compute_uv=False)
    opt_mse = np.sum(s[k:] ** 2) / (B * d)
    Wt = {"W1": rng.uniform(-.3, .3, (d, 8)), "b1": np.zeros(8), "W2": rng.uniform(-.3, .3, (8, k)),
          "b2": np.zeros(k), "W3": rng.uniform(-.3, .3, (k, 8)), "b3": np.zeros(8),
          "W4": rng.uniform(-.3, .3, (8, d)), "b4": np.zeros(d)}
    opt = C.Lamb(Wt)
    for it in range(4000):
        L, g = C.loss_and_grad(Wt, Y, act="linear")
        Wt = opt.step(Wt, g, 2e-2 * 0.5 ** (it // 1500))
    L, _ = C.loss_and_grad(Wt, Y, act="linear")
    assert opt_mse * (1 - 1e-9) <= L <= 1.05 * opt_mse


def test_emulated_codec_close_to_exact_and_rounded():
    rng = np.random.default_rng(6)
    from paper_2304_04781_gb300 import inputs
    Wt = inputs.codec_init(seed=1)
    Y = rng.uniform(-1, 1, (16, 2048))
    z_exact = C.encode(Wt, Y)
    z_emul = C.encode(Wt, Y, emulate=True)
    assert np.all(C.round_fp16(z_emul) == z_emul)
    rel = np.linalg.norm(z_emul - z_exact) / np.linalg.norm(z_exact)
    assert 1e-5 < rel < 2e-2
    out_e = C.decode(Wt, z_emul, emulate=True)
    out_x = C.decode(Wt, z_emul)
    assert np.linalg.norm(out_e - out_x) / np.linalg.norm(out_x) < 2e-2
    cols = C.field_columns(0)
    np.testing.assert_allclose(C.decode(Wt, z_emul, cols=cols), out_x[:, cols], rtol=1e-12, atol=1e-12)


def test_training_schedule_follows_table_2():
    """The training call's defaults (aew_codec_train through the binding) and the
    oracle's schedule are the values Table 2 prints (fixture
    tests/golden/table2_training.json)."""
    import inspect
    import json
    import os
    from paper_2304_04781_gb300 import aewave
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table2_training.json")))
    sig = inspect.signature(aewave.Solver.codec_train).parameters
    assert sig["epochs"].default == g["epochs"]
    assert sig["batch"].default == g["batch_size"]
    assert sig["lr0"].default == g["initial_learning_rate"]
    assert sig["halve_every"].default == g["learning_rate_decay_every_epochs"]
    lr0, k = g["initial_learning_rate"], g["learning_rate_decay_every_epochs"]
    for ep in range(g["epochs"]):
        assert C.lr_schedule(ep, lr0) == pytest.approx(lr0 * g["learning_rate_decay_factor"] ** (ep // k), rel=0, abs=0)


def test_weighted_training_gradient_matches_finite_differences():
    """The per-vector, per-field weighted loss: its back-propagated gradient against
    central differences, and all-one weights reproduce the plain mean squared error."""
    rng = np.random.default_rng(14)
    d = 2048
    Wt = {"W1": rng.uniform(-.05, .05, (d, 8)), "b1": rng.uniform(-.1, .1, 8),
          "W2": rng.uniform(-.5, .5, (8, 4)), "b2": rng.uniform(-.1, .1, 4),
          "W3": rng.uniform(-.5, .5, (4, 8)), "b3": rng.uniform(-.1, .1, 8),
          "W4": rng.uniform(-.5, .5, (8, d)), "b4": rng.uniform(-.1, .1, d)}
    Y = rng.uniform(-1, 1, (6, d))
    w = rng.uniform(0, 3, (6, 4))
    w[:, 1:] *= rng.integers(0, 2, (6, 3))          # some fields switched off
    L1, g1 = C.loss_and_grad(Wt, Y)
    L0, g0 = C.loss_and_grad(Wt, Y, weights=np.ones((6, 4)))
    assert L0 == L1 and all(np.array_equal(g0[k], g1[k]) for k in g1)
    _, g = C.loss_and_grad(Wt, Y, weights=w)
    eps = 1e-4   # the loss is O(1): a smaller step drowns the derivative in rounding
    for name in C.PARAMS:
        flat = Wt[name].ravel()
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            Wp = {k: v.copy() for k, v in Wt.items()}; Wm = {k: v.copy() for k, v in Wt.items()}
            Wp[name].ravel()[idx] += eps; Wm[name].ravel()[idx] -= eps
            fd = (C.loss_and_grad(Wp, Y, weights=w)[0] - C.loss_and_grad(Wm, Y, weights=w)[0]) / (2 * eps)
            assert fd == pytest.approx(g[name].ravel()[idx], rel=1e-5, abs=1e-10), (name, idx)
