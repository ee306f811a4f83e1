"""GPU parity of the tcgen05 codec, the snapshot packing (Algorithm 1), the training
step (MSE + LAMB) and the autoencoder-compressed gradient / GN-HVP against the FP64
oracle.

Tolerances.  The oracle's emulated mode rounds exactly where the GPU rounds (BF16 /
FP16 operands, BF16 hidden activations, FP16 latent), so the two differ only by
FP32-vs-FP64 accumulation order (relative ~1e-6 per dot product of length 2048) and
by the RNE rounding flips that this causes at BF16 boundaries of the hidden layer
(one BF16 ulp, 2^-8 relative, on a ~1e-6/2^-8 ~ 1e-3 fraction of hidden values).
Outputs therefore agree to ~1e-4 in rel-L2; the tests allow 2e-3.
"""
import numpy as np
import pytest
import torch

from oracle import codec as C
from oracle import wave as W
from paper_2304_04781_gb300 import inputs

from .helpers import cuda, host, relerr, setup, solver

pytestmark = pytest.mark.gpu

CODEC_TOL = 2e-3


def _state(shape, seed):
    st = inputs.smooth_state(shape, 10.0, seed=seed)
    st[0] = W.interior(st[0])
    return [a.astype(np.float32).astype(np.float64) for a in st]


@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 64, 64), (40, 48, 56)])
@pytest.mark.parametrize("n_lat", [64, 32])
def test_encode_matches_oracle(shape, n_lat):
    prob, _, _ = setup(shape, 4, 16)
    s = solver(prob, storage="ae", n_lat=n_lat)
    Wt = inputs.codec_init(seed=1, n_lat=n_lat)
    s.codec_set(Wt)
    st = _state(shape, seed=4)
    st[2][:8, :8, :] = 0.0          # block-fields that are exactly zero (scale 0)
    st[3] *= 1e-12                  # a field many orders of magnitude smaller
    st[1][8:16, :8, :8] *= 1e-36    # a block of FP32 subnormals (clamped scale)
    st = [a.astype(np.float32).astype(np.float64) for a in st]
    lat, bm = s.codec_encode([cuda(a) for a in st])
    z = lat.float().cpu().numpy().astype(np.float64)
    sc = C.block_scales(st)
    z_ref = C.encode(Wt, C.normalise(C.pack_blocks(st), sc), emulate=True)
    assert z.shape == z_ref.shape
    assert relerr(z, z_ref) < CODEC_TOL
    # block maxima are exact (max of the same FP32 values)
    Xa = np.abs(C.pack_blocks(st))
    bm_ref = np.stack([Xa[:, C.field_columns(f)].max(1) for f in range(4)], 1)
    np.testing.assert_array_equal(host(bm), bm_ref)


def test_activation_meets_its_error_bound():
    """GELU as the encoder and decoder kernels evaluate it (Phi from Abramowitz & Stegun
    eq. 7.1.28, |erf error| <= 3e-7, one approximate reciprocal) and the derivative the
    training kernels use (erff), against the exact FP64 functions over the range the
    hidden layers see and beyond.  In FP32 the 16th power multiplies the rounding of its
    base by 16, so |dPhi| <= 1e-6 (about 1e-3 of the BF16 rounding the activations take
    next) and |dGELU| <= 1e-6 |x| + one FP32 rounding of the product; both tails go to 0
    and x, and 0 maps to 0.  The kernels take GELU two values at a time on paired FP32
    lanes; the probe returns NaN wherever that differs in any bit from the scalar form."""
    from scipy.special import erf
    from paper_2304_04781_gb300 import aewave
    x = np.concatenate([np.linspace(-12.0, 12.0, 480001), [0.0, -0.0, 1e-30, -1e-30, 40.0, -40.0,
                                                          1e6, -1e6]]).astype(np.float32)
    y, dy = aewave.activation_probe(torch.from_numpy(x).cuda())
    y, dy = host(y), host(dy)
    assert not np.any(np.isnan(y)), "paired-lane GELU differs from the scalar form"
    xd = x.astype(np.float64)
    phi = 0.5 * (1.0 + erf(xd / np.sqrt(2.0)))
    g = xd * phi
    assert np.all(np.abs(y - g) <= 1e-6 * np.abs(xd) + 2.0 ** -23 * np.abs(g) + 1e-37)
    gp = phi + xd * np.exp(-0.5 * xd * xd) / np.sqrt(2.0 * np.pi)
    assert np.all(np.abs(dy - gp) <= 1e-6 + 2.0 ** -20 * np.abs(xd * (gp - phi)))
    assert np.all(y[x == 0] == 0.0)
    # x = 40, -40, 1e6, -1e6: the upper tail gives x itself, the lower tail 0
    assert y[-4] == 40.0 and y[-3] == 0.0 and y[-2] == 1e6 and y[-1] == 0.0


@pytest.mark.parametrize("n", [64, 210, 700])
def test_pair_gemm_matches_single_sm_gemm(n, monkeypatch):
    """The encoder's wide layer on SM pairs (cta_group::2: M = 256 MMAs reading both
    CTAs' shared memories, rows 128-255 accumulated in the odd CTA's TMEM) gives the
    latents of the single-SM kernel bit for bit: every output is the same K-ordered FP32
    sum of the same BF16 products.  Ragged row counts leave the odd CTA's rows wholly
    (64) or partly (210, 700) past the end."""
    prob, _, _ = setup((32, 32, 32), 4, 16)
    Wt = inputs.codec_init(seed=3, n_lat=64)
    rng = np.random.default_rng(n)
    vec = torch.from_numpy(rng.uniform(-1.0, 1.0, (n, 2048)).astype(np.float32))
    vec = vec.to(torch.bfloat16).cuda()
    lat = {}
    for pair in ("1", "0"):
        monkeypatch.setenv("AEW_GEMM_PAIR", pair)   # read when the handle's codec is made
        s = solver(prob, storage="ae")
        s.codec_set(Wt)
        lat[pair] = s.codec_encode_vectors(vec).view(torch.int16).cpu()
        s.close()
    assert torch.equal(lat["1"], lat["0"])
    Z = C.encode(Wt, vec.double().cpu().numpy(), emulate=True)
    assert relerr(lat["1"].view(torch.float16).double().numpy(), Z) < CODEC_TOL


def test_latents_must_be_32_byte_aligned():
    """The latent epilogue stores 32 bytes per lane at once: an output pointer off a
    32-byte boundary is refused on the host (AEW_E_ARG), before any kernel runs."""
    from paper_2304_04781_gb300 import aewave
    prob, _, _ = setup((32, 32, 32), 4, 16)
    s = solver(prob, storage="ae")
    s.codec_set(inputs.codec_init(seed=3, n_lat=64))
    vec = torch.zeros((64, 2048), dtype=torch.bfloat16, device="cuda")
    lat = torch.zeros((65, 64), dtype=torch.float16, device="cuda")
    rc = aewave.lib().aew_codec_encode_vectors(s._h, vec.data_ptr(), 64, lat.data_ptr() + 16,
                                               aewave._stream())
    assert aewave._ERRORS[rc] == "AEW_E_ARG"
    torch.cuda.synchronize()
    assert not torch.any(lat)   # nothing written
    s.close()


@pytest.mark.parametrize("n_lat", [64, 32])
def test_decode_matches_oracle(n_lat):
    shape = (40, 48, 56)
    prob, _, _ = setup(shape, 4, 16)
    s = solver(prob, storage="ae", n_lat=n_lat)
    Wt = inputs.codec_init(seed=2, n_lat=n_lat)
    s.codec_set(Wt)
    Z = C.round_fp16(inputs.random_latents(s.nblocks, n_lat, seed=5).astype(np.float64))
    lat = torch.from_numpy(Z.astype(np.float16)).cuda()
    out = host(s.codec_decode(lat))
    ref = C.decode(Wt, Z, emulate=True)
    assert relerr(out, ref) < CODEC_TOL
    # strain part scattered to the grid, times each block's power-of-two scale, zero on
    # the boundary
    rng = np.random.default_rng(9)
    bm = (rng.uniform(0.5, 1.0, (s.nblocks, 4)) * 10.0 ** rng.integers(-12, 3, (s.nblocks, 4))).astype(np.float32)
    bm[3, 0] = 0.0
    e = host(s.codec_decode_e(lat, cuda(bm)))
    _, ex = np.frexp(bm[:, 0].astype(np.float64))
    sb = np.where(bm[:, 0] > 0, np.ldexp(1.0, np.maximum(ex, C.EXP_MIN)), 0.0)
    Xe = np.zeros_like(ref)
    cols = C.field_columns(0)
    Xe[:, cols] = ref[:, cols] * sb[:, None]
    e_ref = W.interior(C.unpack_field(Xe, shape, 0))
    assert relerr(e, e_ref) < CODEC_TOL
    assert np.all(e[0] == 0) and np.all(e[:, :, -1] == 0)
    # block by block, in each block's own units (the scales span 14 decades, so the
    # global norm alone would not see a wrong scale on a small block)
    z = np.zeros(shape)
    Pe = C.pack_blocks([e, z, z, z])[:, cols]
    Pr = C.pack_blocks([e_ref, z, z, z])[:, cols]
    nr = np.linalg.norm(Pr, axis=1)
    live = nr > 0
    assert np.all(Pe[~live] == 0)
    blk = np.linalg.norm(Pe[live] - Pr[live], axis=1) / nr[live]
    assert blk.max() < 5 * CODEC_TOL, blk.max()


def test_snapshots_match_packing():
    """Algorithm 1: every 10th state cut into blocks, each field of each block divided by
    its power-of-two scale, packed by the forward step that reads the state.  The
    reference is the oracle's packing and exact power-of-two normalisation of the same
    states advanced by the plain step, rounded once to BF16 as the kernel rounds.  The two step variants may contract
    m e differently, so their FP32 states can differ in the last bit: the block maxima
    must agree to a few FP32 ulps and the BF16 codes bit for bit except, rarely, one
    BF16 ulp where such a difference crosses a rounding boundary."""
    shape = (32, 32, 32)
    prob, c, _ = setup(shape, 41, 16)
    s = solver(prob, storage="ae")
    snaps, bm = s.snapshots(cuda(c), every=10, max_vectors=4 * 64, with_scales=True)
    assert snaps.shape == (4 * 64, 2048)
    st = [torch.zeros(shape, device="cuda") for _ in range(4)]
    cc = cuda(c)
    wav = W.default_wavelet(prob)
    got = snaps.view(torch.int16).cpu().numpy().view(np.uint16)
    for q in range(4):
        s.propagate(cc, st, 10 * q, 10, wavelet=wav[10 * q: 10 * q + 10])
        hs = [host(t) for t in st]
        X = C.pack_blocks(hs)
        sc = C.block_scales(hs)
        Y = C.normalise(X, sc)                       # exact: scales are powers of two
        want = torch.from_numpy(Y).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        g = got[64 * q: 64 * (q + 1)]
        assert np.mean(g == want) > 0.999
        gv = torch.from_numpy(g.view(np.int16)).view(torch.bfloat16).double().numpy()
        wv = torch.from_numpy(want.view(np.int16)).view(torch.bfloat16).double().numpy()
        assert np.all(np.abs(gv - wv) <= 2.0 ** -7 * np.maximum(np.abs(gv), np.abs(wv)))
        Xa = np.abs(X)
        bm_ref = np.stack([Xa[:, C.field_columns(f)].max(1) for f in range(4)], 1)
        np.testing.assert_allclose(host(bm[64 * q: 64 * (q + 1)]), bm_ref, rtol=1e-6, atol=0)


@pytest.mark.parametrize("every", [1, 3])
def test_snapshots_without_caller_maxima_match_with_them(every):
    """Without a block-maxima buffer the steps hand the maxima on through two alternating
    scratch slices (a step reads one state's and writes the next one's); the packed
    vectors must equal those written when the caller keeps the maxima, including every
    = 1, where each step both reads and writes maxima, and a budget that stops mid-run."""
    shape = (24, 32, 40)
    prob, c, _ = setup(shape, 14, 16)
    s = solver(prob, storage="ae")
    nb = s.nblocks
    budget = 5 * nb if every == 1 else 4 * nb
    with_bm, bm = s.snapshots(cuda(c), every=every, max_vectors=budget, with_scales=True)
    without = s.snapshots(cuda(c), every=every, max_vectors=budget)
    assert with_bm.shape == without.shape and with_bm.shape[0] in (budget, 4 * nb)
    assert torch.equal(with_bm.view(torch.int16), without.view(torch.int16))
    assert torch.all(bm >= 0) and torch.any(bm > 0)


@pytest.mark.parametrize("weighted", [False, True])
def test_training_steps_match_oracle(weighted):
    """10 LAMB steps on one batch of 256 snapshot-like vectors (lr 1e-3), with the plain
    mean squared error and with per-vector, per-field weights (some fields off)."""
    shape = (32, 32, 32)
    prob, _, _ = setup(shape, 4, 16)
    s = solver(prob, storage="ae")
    Wt = inputs.codec_init(seed=3)
    s.codec_set(Wt)
    rng = np.random.default_rng(7)
    st = _state((32, 32, 64), seed=6)
    Y = C.normalise(C.pack_blocks(st), [np.abs(a).max() for a in st])[:128]
    Y = np.concatenate([Y, rng.uniform(-1, 1, (128, 2048)) * 0.3])
    Y = C.round_bf16(Y)
    batch = torch.from_numpy(Y.astype(np.float32)).to(torch.bfloat16).cuda()
    w = None
    if weighted:
        w = rng.uniform(0.1, 3.0, (256, 4)).astype(np.float32)
        w[::2, 1:] = 0.0                          # strain only for every other vector
    wdev = None if w is None else torch.from_numpy(w).cuda()
    Wo = {k: v.astype(np.float64) for k, v in Wt.items()}
    opt = C.Lamb(Wo)
    for it in range(10):
        loss = s.train_step(batch, 1e-3, weights=wdev)
        L_ref, g = C.loss_and_grad(Wo, Y, emulate=True, weights=w)
        Wo = opt.step(Wo, g, 1e-3)
        assert abs(loss - L_ref) <= 1e-3 * L_ref, (it, loss, L_ref)
    Wg = s.codec_get()
    # weights concentrate the gradient on fewer vectors, so less of the BF16 rounding of
    # the back-propagated errors averages out in the bias sums
    tol = 2e-3 if weighted else 1e-3
    for k in C.PARAMS:
        assert relerr(Wg[k], Wo[k]) < tol, k
        moved = relerr(Wo[k], Wt[k])
        if np.linalg.norm(Wt[k]) > 0:
            assert moved > 1e-3, k   # the parameters did change


@pytest.fixture(scope="module")
def ae_case():
    prob, c, _ = setup((32, 32, 32), 200, 16, seed=0)
    ctrue = inputs.bump_model(c, prob.h).astype(np.float32).astype(np.float64)
    d_obs, _, _ = W.forward(prob, ctrue)
    Wt = inputs.codec_init(seed=4)
    return prob, c, d_obs, Wt


def test_ae_gradient_matches_oracle_ae_gradient(ae_case):
    """Same weights on both sides; the oracle decodes its own FP64 states (emulated
    rounding).  This checks the compressed pipeline (packing and block maxima inside the
    forward step, encoder on the side stream, latent store, decode, accumulation) end to
    end."""
    prob, c, d_obs, Wt = ae_case
    s = solver(prob, storage="ae")
    s.codec_set(Wt)
    J, g = s.gradient(cuda(c), cuda(d_obs))
    d, states = W.forward_states(prob, c)
    ehat = C.compressed_e_history(Wt, states, emulate=True)
    J_ref, g_ref, _ = W.gradient(prob, c, d_obs, e_of=lambda n: ehat[n])
    assert abs(J - J_ref) / J_ref < 1e-4
    eg = relerr(host(g), g_ref)
    # the HVP reuses the stored latents
    dc = inputs.direction(prob.shape, prob.h, seed=20).astype(np.float32).astype(np.float64)
    H = host(s.hessvec(cuda(dc)))
    H_ref = W.hessvec_gn(prob, c, dc, lambda n: ehat[n])
    eh = relerr(H, H_ref)
    print(f"AE parity (random codec, 32^3): gradient {eg:.2e}, HVP {eh:.2e}")
    # random weights decode noise, whose GN-HVP (applied twice) cancels more than the
    # gradient: measured 3.6e-4 / 1.4e-3; the trained codec's parity is held to 1e-3
    # for both below
    assert eg < 1e-3 and eh < 2e-3
    st = s.stats()
    assert st["latent_bytes"] == prob.nt * 64 * 64 * 2


def test_roundtrip_of_one_state_matches_oracle(ae_case):
    """Encode then decode the strain of one state with per-block scales (standalone path)."""
    prob, c, d_obs, Wt = ae_case
    s = solver(prob, storage="ae")
    s.codec_set(Wt)
    _, states = W.forward_states(prob, c)
    n = 150
    e_ref = C.roundtrip_e(Wt, states[n], emulate=True)
    lat, bm = s.codec_encode([cuda(a) for a in states[n]])
    e = host(s.codec_decode_e(lat, bm))
    er = relerr(e, e_ref)
    print(f"one-state roundtrip parity: {er:.2e}")
    assert er < 2 * CODEC_TOL


def test_trained_codec_gradient_and_hvp_match_oracle():
    """The committed trained codec (weights/codec_64.npz, 8 draws at 128^3 x 1000) in the
    compressed gradient and GN-HVP at 64^3 x 160 steps, against the oracle with the same
    weights: trained activations exercise other BF16 ranges than random weights."""
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2304_04781_gb300",
                        "weights", "codec_64.npz")
    z = np.load(path)
    Wt = {k: z[k] for k in C.PARAMS}
    prob, c, _ = setup((64, 64, 64), 160, 16, seed=3)
    ctrue = inputs.bump_model(c, prob.h).astype(np.float32).astype(np.float64)
    d_obs, _, _ = W.forward(prob, ctrue)
    s = solver(prob, storage="ae")
    s.codec_set(Wt)
    J, g = s.gradient(cuda(c), cuda(d_obs))
    _, states = W.forward_states(prob, c)
    ehat = C.compressed_e_history(Wt, states, emulate=True)
    J_ref, g_ref, _ = W.gradient(prob, c, d_obs, e_of=lambda n: ehat[n])
    dc = inputs.direction(prob.shape, prob.h, seed=21).astype(np.float32).astype(np.float64)
    H = host(s.hessvec(cuda(dc)))
    H_ref = W.hessvec_gn(prob, c, dc, lambda n: ehat[n])
    eg, eh = relerr(host(g), g_ref), relerr(H, H_ref)
    print(f"AE parity (trained codec, 64^3): gradient {eg:.2e}, HVP {eh:.2e}")
    assert abs(J - J_ref) / J_ref < 1e-4
    assert eg < 1e-3 and eh < 1e-3
