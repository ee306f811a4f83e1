"""Pins of the FP64 oracle for compression in time (Sec. 3.2) and of the codec's forward
pass: the window layout against coordinate-encoded strain histories, the vector scales
by brute force, the rank-k GELU code against the Eckart-Young optimum and against data
that lie in a k-dimensional affine subspace, the compressed history and gradient with a
code that is exact on its data, and the training loss against the forward pass it
differentiates.  CPU only."""
import numpy as np
import pytest
from scipy.special import erf

from oracle import codec as C
from oracle import codec_time as CT
from oracle import wave as W
from paper_2304_04781_gb300 import inputs


def _coord_history(nt, shape):
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return [n * 1e6 + k * 1e4 + j * 1e2 + i + 0.5 for n in range(nt)]


def test_window_layout_from_coordinate_encoded_history():
    shape = (6, 16, 24)
    nt = 37                                       # three windows, the last one partial
    hist = _coord_history(nt, shape)
    NBy, NBx = shape[1] // 8, shape[2] // 8
    rng = np.random.default_rng(0)
    for tb in range(CT.n_windows(nt)):
        X = CT.window_vectors(hist, shape, tb)
        assert X.shape == (CT.nvectors(shape), 2048)
        for _ in range(300):
            v = rng.integers(X.shape[0]); kk = rng.integers(2048)
            t, r = divmod(kk, 128); z, r = divmod(r, 64); y, x = divmod(r, 8)
            bz, r2 = divmod(v, NBy * NBx); by, bx = divmod(r2, NBx)
            n = 16 * tb + t
            if n >= nt:
                assert X[v, kk] == 0.0           # beyond the last state: zero padding
                continue
            val = X[v, kk] - 0.5
            nn, rest = divmod(val, 1e6); kz, rest = divmod(rest, 1e4); jy, ix = divmod(rest, 1e2)
            assert (nn, kz, jy, ix) == (n, 2 * bz + z, 8 * by + y, 8 * bx + x)
        E = CT.unpack(X, shape)
        for t in range(16):
            if 16 * tb + t < nt:
                np.testing.assert_array_equal(E[t], hist[16 * tb + t])
            else:
                assert not E[t].any()


def test_vector_scales_bracket_the_vector_max_by_brute_force():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((50, 2048)) * 10.0 ** rng.uniform(-30, 5, (50, 1))
    X[7] = 0.0
    X[8] = 1e-40
    s = CT.vector_scales(X)
    for v in range(50):
        m = max(abs(a) for a in X[v])
        if m == 0:
            assert s[v] == 0
        elif m < 2.0 ** -101:
            assert s[v] == 2.0 ** -100           # exponent clamp (1/s finite in FP32)
        else:
            e = np.log2(s[v])
            assert e == np.round(e) and s[v] / 2 <= m < s[v]
    Y = CT.normalise(X, s)
    assert np.abs(Y).max() < 1.0 and not Y[7].any()


def test_emulated_encoder_inputs_round_when_written_then_scale_exactly():
    rng = np.random.default_rng(21)
    X = rng.standard_normal((6, 2048)) * 10.0 ** rng.uniform(-20, 5, (6, 1))
    X[5, :100] = 1e-40                      # below BF16's normal range
    s = CT.vector_scales(X)
    Y = CT.encoder_inputs(X, s, emulate=True)
    np.testing.assert_array_equal(Y, C.round_bf16(X) / s[:, None])
    # for normal values it is the same as normalising first and rounding once
    np.testing.assert_array_equal(Y[:5], C.round_bf16(X[:5] / s[:5, None]))
    np.testing.assert_array_equal(CT.encoder_inputs(X, s), X / s[:, None])


def test_pca_codec_reproduces_data_in_a_k_dimensional_affine_subspace():
    rng = np.random.default_rng(2)
    k = 12
    basis = rng.standard_normal((k, 2048))
    mu = rng.standard_normal(2048)
    Y = rng.standard_normal((200, k)) @ basis * 0.1 + mu
    Wt = CT.pca_codec(Y, k)
    Z = C.encode(Wt, Y)
    np.testing.assert_allclose(C.decode(Wt, Z), Y, rtol=0, atol=1e-9 * np.abs(Y).max())
    # the latent is the coordinate vector (y - mu_w) V: it reproduces the centred data
    Yc = Y - Y.mean(0)
    V = Wt["W1"][:, :k]
    np.testing.assert_allclose(Z, Yc @ V, rtol=0, atol=1e-9 * np.abs(Z).max())
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-10)


@pytest.mark.parametrize("weighted", [False, True])
def test_pca_codec_error_is_the_eckart_young_tail(weighted):
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((400, 2048)) * np.linspace(3.0, 0.1, 2048) + 0.2
    w = rng.uniform(0.1, 3.0, 400) if weighted else np.ones(400)
    k = 40
    Wt = CT.pca_codec(Y, k, w if weighted else None)
    R = C.decode(Wt, C.encode(Wt, Y))
    err = float((w[:, None] * (R - Y) ** 2).sum())
    mu = (w[:, None] * Y).sum(0) / w.sum()
    lam = np.sort(np.linalg.eigvalsh(((Y - mu) * w[:, None]).T @ (Y - mu)))[::-1]
    assert err == pytest.approx(lam[k:].sum(), rel=1e-9)
    # and no other rank-k code of the same form does better: a perturbed basis is worse
    Wp = {kk: v.copy() for kk, v in Wt.items()}
    Q, _ = np.linalg.qr(Wt["W1"][:, :k] + 1e-2 * rng.standard_normal((2048, k)))
    Wp["W1"] = np.concatenate([Q, -Q], 1)
    Wp["W4"] = np.concatenate([Q.T, -Q.T], 0)
    Wp["b1"] = np.concatenate([-mu @ Q, mu @ Q])
    Rp = C.decode(Wp, C.encode(Wp, Y))
    assert float((w[:, None] * (Rp - Y) ** 2).sum()) > err


def _small_problem(nt=40):
    shape = (16, 16, 16)
    rec = inputs.receiver_grid(16, 16, 16)
    prob = W.Problem(shape=shape, h=10.0, nt=nt, rec=rec)
    c = inputs.velocity_model(shape, 10.0, seed=5)
    return prob, c


def test_compressed_history_and_gradient_with_a_code_exact_on_its_data():
    """Windows, tail padding, scales and boundary handling of the compressed history:
    with a code that reproduces every normalised vector of this history (k = number of
    vectors), the decoded history is the stored one and the compressed gradient is the
    full-storage gradient."""
    prob, c = _small_problem(nt=40)                 # windows of 16, 16 and 8 states
    d, states = W.forward_states(prob, c)
    e_hist = [st[0] for st in states]
    Ys = []
    for tb in range(CT.n_windows(prob.nt)):
        X = CT.window_vectors(e_hist, prob.shape, tb)
        Ys.append(CT.normalise(X, CT.vector_scales(X)))
    Y = np.concatenate(Ys)
    Wt = CT.pca_codec(Y, Y.shape[0])
    eh = CT.compressed_e_history(Wt, e_hist)
    assert len(eh) == prob.nt
    emax = max(float(np.abs(e).max()) for e in e_hist)
    for n in range(prob.nt):
        np.testing.assert_allclose(eh[n], e_hist[n], rtol=0, atol=1e-9 * emax)
    d_obs, _, _ = W.forward(prob, inputs.bump_model(c))
    J, g_full, _ = W.gradient(prob, c, d_obs)
    _, g_ae, _ = W.gradient(prob, c, d_obs, e_of=lambda n: eh[n])
    assert np.linalg.norm(g_ae - g_full) / np.linalg.norm(g_full) < 1e-9
    # with the GPU's rounding emulated the history stays close (BF16 / FP16 operands)
    eh16 = CT.compressed_e_history(Wt, e_hist, emulate=True)
    num = sum(float(np.sum((a - b) ** 2)) for a, b in zip(eh16, e_hist))
    den = sum(float(np.sum(b ** 2)) for b in e_hist)
    assert np.sqrt(num / den) < 2e-2


def test_compressed_history_keeps_the_exact_zero_initial_state():
    """e^0 = 0 (Eq. (2)) is not decoded: with a code that is not exact, window 0 decodes
    its slot 0 to nonzero values, but the history's first entry stays exactly 0."""
    prob, c = _small_problem(nt=40)
    _, states = W.forward_states(prob, c)
    e_hist = [st[0] for st in states]
    Y = []
    for tb in range(3):      # later windows have nonzero first slots
        X = CT.window_vectors(e_hist, prob.shape, tb)
        Y.append(CT.normalise(X, CT.vector_scales(X)))
    Wt = CT.pca_codec(np.concatenate(Y), 4)       # far from exact
    assert np.abs(CT.roundtrip_window(Wt, e_hist, prob.shape, 0)[0]).max() > 0
    eh = CT.compressed_e_history(Wt, e_hist)
    assert not eh[0].any() and eh[1].any()


def test_compressed_history_zeroes_boundary_nodes():
    shape = (8, 8, 8)
    rng = np.random.default_rng(6)
    hist = [rng.standard_normal(shape) for _ in range(16)]
    X = CT.window_vectors(hist, shape, 0)
    Y = CT.normalise(X, CT.vector_scales(X))
    Wt = CT.pca_codec(Y, Y.shape[0])
    E = CT.roundtrip_window(Wt, hist, shape, 0)
    for t in range(16):
        assert not E[t][[0, -1]].any() and not E[t][:, [0, -1]].any() and not E[t][:, :, [0, -1]].any()
        np.testing.assert_allclose(E[t][1:-1, 1:-1, 1:-1], hist[t][1:-1, 1:-1, 1:-1], atol=1e-9)


# --------------------------------------------------------------------------------------
# The space codec's forward pass (encode, decode, roundtrip_e)
# --------------------------------------------------------------------------------------
def _codec(seed, n_lat=16):
    return {k: v.astype(np.float64) for k, v in inputs.codec_init(seed, n_lat=n_lat).items()}


@pytest.mark.parametrize("act", ["gelu", "linear"])
def test_training_loss_is_the_error_of_decode_after_encode(act):
    """loss_and_grad differentiates its own copy of the forward pass: its loss must be
    the mean squared error of decode(encode(Y)) (exact mode), plain and weighted."""
    rng = np.random.default_rng(7)
    Wt = _codec(8)
    for k in ("b1", "b2", "b3", "b4"):
        Wt[k] = rng.standard_normal(Wt[k].shape) * 0.1
    Y = rng.uniform(-1, 1, (24, 2048))
    if act == "linear":
        lin = lambda a: a
        h = (Y @ Wt["W1"] + Wt["b1"]) @ Wt["W2"] + Wt["b2"]
        R = lin(h @ Wt["W3"] + Wt["b3"]) @ Wt["W4"] + Wt["b4"]
    else:
        R = C.decode(Wt, C.encode(Wt, Y))
    loss, _ = C.loss_and_grad(Wt, Y, act=act)
    assert loss == pytest.approx(float(np.mean((R - Y) ** 2)), rel=1e-12)
    w = rng.uniform(0.0, 2.0, (24, 4))
    fcol = (np.arange(2048) >> 6) & 3
    lw, _ = C.loss_and_grad(Wt, Y, act=act, weights=w)
    assert lw == pytest.approx(float(np.mean(w[:, fcol] * (R - Y) ** 2)), rel=1e-12)


def test_decode_columns_are_the_full_decoders_columns():
    rng = np.random.default_rng(9)
    Wt = _codec(10)
    Z = rng.standard_normal((7, 16))
    full = C.decode(Wt, Z)
    cols = C.field_columns(0)
    np.testing.assert_allclose(C.decode(Wt, Z, cols=cols), full[:, cols], rtol=1e-13, atol=0)
    np.testing.assert_allclose(C.decode(Wt, Z, cols=cols, emulate=True),
                               C.decode(Wt, Z, emulate=True)[:, cols], rtol=1e-13, atol=0)


def test_encoder_layers_in_order_with_gelu_only_on_the_hidden_layer():
    """encode = (GELU(y W1 + b1)) W2 + b2: a GELU on the latent, or the layers swapped,
    changes the result (checked against the written-out composition)."""
    rng = np.random.default_rng(11)
    Wt = _codec(12)
    Wt["b2"] = rng.standard_normal(16)
    Y = rng.uniform(-1, 1, (5, 2048))
    a = Y @ Wt["W1"] + Wt["b1"]
    want = (a * 0.5 * (1 + erf(a / np.sqrt(2)))) @ Wt["W2"] + Wt["b2"]
    np.testing.assert_allclose(C.encode(Wt, Y), want, rtol=1e-12, atol=1e-14)


def test_roundtrip_e_unpacks_scales_and_zeroes_the_boundary():
    """roundtrip_e with a code exact on the state's own normalised block vectors returns
    the interior of the strain field (coordinate-encoded, every block scaled)."""
    shape = (16, 16, 16)
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rng = np.random.default_rng(13)
    state = [(k * 1e4 + j * 1e2 + i + 1.0) * 10.0 ** (-3 * f) * rng.uniform(0.5, 2.0) for f in range(4)]
    s = C.block_scales(state)
    Y = C.normalise(C.pack_blocks(state), s)
    Wt = CT.pca_codec(Y, Y.shape[0])
    e = C.roundtrip_e(Wt, state)
    inner = np.zeros(shape)
    inner[1:-1, 1:-1, 1:-1] = state[0][1:-1, 1:-1, 1:-1]
    np.testing.assert_allclose(e, inner, rtol=1e-9, atol=1e-9)
    assert not e[0].any() and not e[:, -1].any() and not e[:, :, 0].any()


# --------------------------------------------------------------------------------------
# The paper's normalisation and activation (Sec. 3.3): min-max to [0, 1], ELU
# --------------------------------------------------------------------------------------
def test_elu_is_continuous_with_unit_slope_at_zero_and_tends_to_minus_one():
    x = np.linspace(-30, 30, 60001)
    y, dy = C.elu(x), C.elu_prime(x)
    assert np.all(y[x >= 0] == x[x >= 0])
    assert np.all(np.diff(y) >= 0)                      # increasing (flat in FP64 below -37)
    assert np.all(np.diff(y[x > -20]) > 0)
    assert abs(C.elu(-1e-12) + 1e-12) < 1e-20 and C.elu_prime(-1e-12) == pytest.approx(1.0)
    assert C.elu(-40.0) == pytest.approx(-1.0, abs=1e-15)
    h = 1e-6
    mid = x[(np.abs(x) > 1e-3)]
    fd = (C.elu(mid + h) - C.elu(mid - h)) / (2 * h)
    np.testing.assert_allclose(C.elu_prime(mid), fd, rtol=1e-7, atol=1e-9)


def test_elu_training_gradient_matches_finite_differences():
    rng = np.random.default_rng(31)
    d = 2048
    Wt = {"W1": rng.uniform(-.05, .05, (d, 8)), "b1": rng.uniform(-.5, .5, 8),
          "W2": rng.uniform(-.5, .5, (8, 4)), "b2": rng.uniform(-.1, .1, 4),
          "W3": rng.uniform(-.5, .5, (4, 8)), "b3": rng.uniform(-.5, .5, 8),
          "W4": rng.uniform(-.5, .5, (8, d)), "b4": rng.uniform(-.1, .1, d)}
    Y = rng.uniform(0, 1, (6, d))
    L, g = C.loss_and_grad(Wt, Y, act="elu")
    assert L == pytest.approx(float(np.mean((C.decode(Wt, C.encode(Wt, Y, act="elu"), act="elu") - Y) ** 2)),
                              rel=1e-12)
    eps = 1e-4
    for name in C.PARAMS:
        flat = Wt[name].ravel()
        for idx in rng.choice(flat.size, size=min(3, flat.size), replace=False):
            Wp = {k: v.copy() for k, v in Wt.items()}; Wm = {k: v.copy() for k, v in Wt.items()}
            Wp[name].ravel()[idx] += eps; Wm[name].ravel()[idx] -= eps
            fd = (C.loss_and_grad(Wp, Y, act="elu")[0] - C.loss_and_grad(Wm, Y, act="elu")[0]) / (2 * eps)
            assert fd == pytest.approx(g[name].ravel()[idx], rel=1e-5, abs=1e-10), (name, idx)


def test_minmax_normalisation_spans_zero_to_one_and_inverts_exactly():
    rng = np.random.default_rng(32)
    X = rng.standard_normal((40, 2048)) * 10.0 ** rng.uniform(-12, 2, (40, 1)) + rng.uniform(-1, 1, (40, 1))
    X[5] = 0.25                                          # constant vector
    X[6] = 3e-9 * rng.standard_normal(2048)              # range below beta
    mn, r = CT.minmax_scales(X)
    Y = CT.minmax_normalise(X, mn, r)
    big = np.ptp(X, axis=1) > CT.BETA
    assert np.all(Y >= 0) and np.all(Y[big].max(1) == pytest.approx(1.0)) and np.all(Y.min(1) == 0.0)
    assert r[5] == CT.BETA and not Y[5].any()
    assert r[6] == CT.BETA                               # small range: the floor is the range
    assert Y[6].max() == pytest.approx(np.ptp(X[6]) / CT.BETA) and Y[6].max() < 1.0
    np.testing.assert_allclose(Y * r[:, None] + mn[:, None], X, rtol=1e-15, atol=1e-15 * np.abs(X).max())


def test_minmax_history_with_a_code_exact_on_its_data():
    prob, c = _small_problem(nt=40)
    _, states = W.forward_states(prob, c)
    e_hist = [st[0] for st in states]
    Ys = []
    for tb in range(CT.n_windows(prob.nt)):
        X = CT.window_vectors(e_hist, prob.shape, tb)
        mn, r = CT.minmax_scales(X, beta=1e-30)
        Ys.append(CT.minmax_normalise(X, mn, r))
    Y = np.concatenate(Ys)
    Wt = CT.pca_codec(Y, Y.shape[0])
    eh = CT.compressed_e_history(Wt, e_hist, norm="minmax", beta=1e-30)
    emax = max(float(np.abs(e).max()) for e in e_hist)
    for n in range(prob.nt):
        np.testing.assert_allclose(eh[n], e_hist[n], rtol=0, atol=1e-8 * emax)
    # with the paper's absolute beta = 1e-7 these states (|e| ~ 1e-7 and below) are
    # mostly squeezed under the floor of the range: the vectors are not scaled to [0, 1]
    mn, r = CT.minmax_scales(CT.window_vectors(e_hist, prob.shape, 1))
    assert np.mean(r == CT.BETA) > 0.5


def test_bf16_history_rounds_to_bf16_and_its_gradient_stays_close():
    """The adjoint-type sweeps read the decoded strain as BF16 (R34): values already in
    BF16 pass unchanged, a value halfway between two BF16 numbers goes to the even one,
    e^0 stays exactly 0, and the gradient computed from the BF16 history differs from the
    FP64 one by no more than BF16's relative step (2^-8) bounds."""
    one = np.array([1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 0.0])
    out = CT.bf16_history([one])[0]
    np.testing.assert_array_equal(out, [1.0, 1.0 + 2.0 ** -7, 1.0, 1.0 + 2 * 2.0 ** -7, -2.5, 0.0])
    prob, c = _small_problem(nt=40)
    d, states = W.forward_states(prob, c)
    e_hist = [st[0] for st in states]
    eb = CT.bf16_history(e_hist)
    assert not np.any(eb[0])
    rel = max(float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)) for a, b in zip(eb[1:], e_hist[1:]))
    assert rel <= 2.0 ** -8
    d_obs, _, _ = W.forward(prob, inputs.bump_model(c))
    _, g_full, _ = W.gradient(prob, c, d_obs)
    _, g_b, _ = W.gradient(prob, c, d_obs, e_of=lambda n: eb[n])
    err = np.linalg.norm(g_b - g_full) / np.linalg.norm(g_full)
    assert 0 < err < 2.0 ** -8
    # the Gauss-Newton HVP with a separate adjoint history: the default reads one history
    dc = inputs.direction(prob.shape, prob.h, seed=3)
    H1 = W.hessvec_gn(prob, c, dc, lambda n: e_hist[n])
    H2 = W.hessvec_gn(prob, c, dc, lambda n: e_hist[n], e_adj_of=lambda n: e_hist[n])
    np.testing.assert_array_equal(H1, H2)
    H3 = W.hessvec_gn(prob, c, dc, lambda n: e_hist[n], e_adj_of=lambda n: eb[n])
    assert 0 < np.linalg.norm(H3 - H1) / np.linalg.norm(H1) < 2.0 ** -8
