"""GPU parity of compression in time (Sec. 3.2) against the FP64 oracle
(oracle/codec_time.py) with the same weights: the window packing of the standalone
encoder and of the forward step (Algorithm 1's window snapshots), the window encoder
and decoder on tcgen05, and the time-codec compressed gradient, Jacobian-vector product
and GN-HVP end to end (latents of every window on the side stream, decoded windows
read by the adjoint and incremental steps).

Tolerances as in test_gpu_codec.py: the oracle's emulated mode rounds where the GPU
rounds (BF16 operands and hidden activations, FP16 latents), so the two differ by
accumulation order and the BF16 rounding flips it causes: ~1e-4 rel-L2, allowed 2e-3
for a codec output and 1e-3 for the gradient and HVP, whose time sums average them.
"""
import numpy as np
import pytest
import torch

from oracle import codec as C
from oracle import codec_time as CT
from oracle import wave as W
from paper_2304_04781_gb300 import inputs

from .helpers import cuda, host, relerr, setup, solver

pytestmark = pytest.mark.gpu

CODEC_TOL = 2e-3


def _f32(W):
    return {k: np.asarray(v, np.float32) for k, v in W.items()}


def _window_fields(shape, nsteps, seed):
    """nsteps strain fields with amplitudes over 40 decades, a zero region and a region
    of FP32 subnormals (clamped vector scales)."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(nsteps):
        e = inputs.smooth_state(shape, 10.0, seed=seed + t)[0] * 10.0 ** rng.uniform(-30, 3)
        e = W.interior(e)
        e[:4, :8, :16] = 0.0
        e[4:6, 8:16, :8] *= 1e-38
        out.append(e.astype(np.float32).astype(np.float64))
    return out


@pytest.mark.parametrize("shape,nsteps", [((32, 32, 32), 16), ((24, 40, 56), 11)])
def test_window_encode_and_decode_match_oracle(shape, nsteps):
    prob, _, _ = setup(shape, 4, 16)
    s = solver(prob, storage="full", codec="time")
    Wt = inputs.codec_init(seed=2, n_hid=1024, n_lat=512)
    rng = np.random.default_rng(3)
    for k in ("b1", "b2", "b3", "b4"):
        Wt[k] = (0.1 * rng.standard_normal(Wt[k].shape)).astype(np.float32)
    s.codec_set(Wt)
    es = _window_fields(shape, nsteps, seed=11)
    lat, vmax = s.codec_encode_window(cuda(np.stack(es)))
    X = CT.pack(es, shape)
    # vector maxima are exact (max of the same FP32 values)
    np.testing.assert_array_equal(host(vmax), np.abs(X).max(1))
    sv = CT.vector_scales(X)
    z_ref = C.encode(Wt, CT.encoder_inputs(X, sv, emulate=True), emulate=True)
    z = host(lat.float())
    assert relerr(z, z_ref) < CODEC_TOL
    # decoder from the GPU's own latents, scaled back per vector, scattered per step
    e_dec = host(s.codec_decode_window(lat, vmax))
    Xh = C.decode(Wt, z, emulate=True) * sv[:, None]
    E_ref = CT.unpack(Xh, shape)
    for t in range(16):
        E_ref[t] = CT.interior(E_ref[t])
    assert e_dec.shape == (16,) + shape
    assert relerr(e_dec, E_ref) < CODEC_TOL
    # every vector on its own, in its own units (a misplaced window slot shows here)
    D = CT.pack(list(e_dec), shape)
    R = CT.pack(list(E_ref), shape)
    nz = np.linalg.norm(R, axis=1) > 0
    per = np.linalg.norm(D - R, axis=1)[nz] / np.linalg.norm(R, axis=1)[nz]
    assert np.percentile(per, 99) < 1e-2


def test_window_snapshots_match_oracle_packing():
    """Algorithm 1 with the time codec: every second complete window, packed by the
    forward steps that write its states and normalised once it is complete.  The
    reference is the oracle's window packing and exact power-of-two normalisation of the
    same states advanced one step at a time by the plain step, rounded once to BF16.
    Each state is stored in BF16 when written and divided by the window's power-of-two
    scale once the window is complete (exact), as the oracle's emulated mode defines.
    The step variants may contract m e differently, so their FP32 states can differ in
    the last bit: the maxima agree to FP32 ulps and the BF16 codes bit for bit except,
    rarely, one BF16 ulp where such a difference crosses a rounding boundary."""
    prob, c, _ = setup((32, 32, 48), 100, 16, seed=1)
    s = solver(prob, storage="full", codec="time")
    vec, vm = s.snapshots(cuda(c), every=2, max_vectors=10 * s.nvec, with_scales=True)
    wins = [tb for tb in range(CT.n_windows(prob.nt)) if tb % 2 == 0 and 16 * tb + 15 <= prob.nt - 1]
    assert wins == [0, 2, 4] and vec.shape[0] == len(wins) * s.nvec
    st = [torch.zeros(prob.shape, device="cuda") for _ in range(4)]
    cc = cuda(c)
    wav = W.default_wavelet(prob)
    e_hist = [np.zeros(prob.shape)]
    for n in range(16 * wins[-1] + 15):
        s.propagate(cc, st, n, 1, wavelet=wav[n:n + 1])
        e_hist.append(host(st[0]))
    X = np.concatenate([CT.window_vectors(e_hist, prob.shape, tb) for tb in wins])
    np.testing.assert_allclose(host(vm), np.abs(X).max(1), rtol=1e-6, atol=0)
    want = torch.from_numpy(CT.encoder_inputs(X, CT.vector_scales(X), emulate=True)).to(torch.bfloat16)
    got = vec.cpu()
    g16 = got.view(torch.int16).numpy()
    w16 = want.view(torch.int16).numpy()
    assert np.mean(g16 == w16) > 0.999
    gv, wv = got.double().numpy(), want.double().numpy()
    assert np.all(np.abs(gv - wv) <= 2.0 ** -7 * np.maximum(np.abs(gv), np.abs(wv)))


@pytest.fixture(scope="module")
def tcase():
    """32^3 x 120 steps (7 windows and a partial eighth), a codec that is the optimal
    rank-512 code of this run's own normalised windows (realistic activations)."""
    prob, c, _ = setup((32, 32, 32), 120, 16, seed=0)
    ctrue = inputs.bump_model(c, prob.h).astype(np.float32).astype(np.float64)
    d_obs, _, _ = W.forward(prob, ctrue)
    _, states = W.forward_states(prob, c)
    e_hist = [st[0] for st in states]
    Y = []
    for tb in range(CT.n_windows(prob.nt)):
        X = CT.window_vectors(e_hist, prob.shape, tb)
        Y.append(CT.normalise(X, CT.vector_scales(X)))
    Wt = _f32(CT.pca_codec(np.concatenate(Y), 512))
    return prob, c, d_obs, e_hist, Wt


def test_time_ae_gradient_jvp_and_hvp_match_oracle(tcase):
    prob, c, d_obs, e_hist, Wt = tcase
    s = solver(prob, storage="ae", codec="time")
    s.codec_set(Wt)
    J, g = s.gradient(cuda(c), cuda(d_obs))
    ehat = CT.compressed_e_history(Wt, e_hist, emulate=True)
    eadj = CT.bf16_history(ehat)        # the sweeps read the decoded strain as BF16 (R34)
    J_ref, g_ref, _ = W.gradient(prob, c, d_obs, e_of=lambda n: eadj[n])
    assert abs(J - J_ref) / J_ref < 1e-4
    err_g = relerr(host(g), g_ref)
    _, g_fp32, _ = W.gradient(prob, c, d_obs, e_of=lambda n: ehat[n])
    print(f"time-codec AE gradient parity: {err_g:.2e} (vs the FP32-read history "
          f"{relerr(host(g), g_fp32):.2e})")
    assert err_g < 1e-3
    dc = inputs.direction(prob.shape, prob.h, seed=20).astype(np.float32).astype(np.float64)
    dd = host(s.jvp(cuda(dc)))
    dd_ref = W.incremental_forward(prob, c, dc, lambda n: eadj[n])
    assert relerr(dd, dd_ref) < 1e-3
    H = host(s.hessvec(cuda(dc)))
    H_ref = W.hessvec_gn(prob, c, dc, lambda n: eadj[n])
    assert relerr(H, H_ref) < 1e-3
    st = s.stats()
    nwin = CT.n_windows(prob.nt)
    assert st["latent_bytes"] == nwin * s.nvec * 512 * 2
    # this code is close to exact on its own run: the compressed gradient is near the
    # full-storage one
    _, g_full, _ = W.gradient(prob, c, d_obs)
    assert relerr(host(g), g_full) < 2e-2


def test_time_ae_gradient_is_deterministic_and_repeatable(tcase):
    prob, c, d_obs, _, Wt = tcase
    s = solver(prob, storage="ae", codec="time")
    s.codec_set(Wt)
    _, g1 = s.gradient(cuda(c), cuda(d_obs))
    g1 = host(g1)
    _, g2 = s.gradient(cuda(c), cuda(d_obs))
    np.testing.assert_array_equal(host(g2), g1)


def test_time_codec_configuration_errors():
    from paper_2304_04781_gb300 import aewave
    prob, _, _ = setup((32, 32, 32), 8, 16)
    with pytest.raises(aewave.AewError) as ei:
        solver(prob, storage="ae", codec="time", n_lat=64)
    assert ei.value.code == -1
    p2, _, _ = setup((32, 32, 28), 8, 16)   # nx = 28: not a multiple of 8
    with pytest.raises(aewave.AewError) as ei:
        solver(p2, storage="ae", codec="time")
    assert ei.value.code == -1
    s = solver(prob, storage="ae", codec="time")
    with pytest.raises(aewave.AewError) as ei:   # space-codec call on a time-codec handle
        s.codec_encode([torch.zeros(prob.shape, device="cuda")] * 4)
    assert ei.value.code == -1


def test_bf16_strain_boxes_across_x_tiles_match_oracle():
    """The sweeps' BF16 e^n boxes (the adjoint's own-node box and the incremental
    forward's box with its 8-wide x halo, R34) on a grid two CTA tiles wide in x, so the
    halo between the tiles carries data: gradient, JVP and GN-HVP against the oracle's
    BF16-read history.  The source sits at x = 128, on the boundary between the tiles,
    and in 96 steps the wave reaches the nearest of 64 receivers (the gradient spans
    x = 109 .. 145)."""
    prob, c, _ = setup((16, 16, 256), 96, 64, seed=4)
    ctrue = inputs.bump_model(c, prob.h).astype(np.float32).astype(np.float64)
    d_obs, _, _ = W.forward(prob, ctrue)
    _, states = W.forward_states(prob, c)
    e_hist = [st[0] for st in states]
    Y = []
    for tb in range(CT.n_windows(prob.nt)):
        X = CT.window_vectors(e_hist, prob.shape, tb)
        Y.append(CT.normalise(X, CT.vector_scales(X)))
    Wt = _f32(CT.pca_codec(np.concatenate(Y), 512))
    s = solver(prob, storage="ae", codec="time")
    s.codec_set(Wt)
    _, g = s.gradient(cuda(c), cuda(d_obs))
    eb = CT.bf16_history(CT.compressed_e_history(Wt, e_hist, emulate=True))
    _, g_ref, _ = W.gradient(prob, c, d_obs, e_of=lambda n: eb[n])
    dc = inputs.direction(prob.shape, prob.h, seed=21).astype(np.float32).astype(np.float64)
    dd = host(s.jvp(cuda(dc)))
    dd_ref = W.incremental_forward(prob, c, dc, lambda n: eb[n])
    H = host(s.hessvec(cuda(dc)))
    H_ref = W.hessvec_gn(prob, c, dc, lambda n: eb[n])
    errs = (relerr(host(g), g_ref), relerr(dd, dd_ref), relerr(H, H_ref))
    print(f"two x tiles, BF16 boxes: gradient {errs[0]:.2e}, JVP {errs[1]:.2e}, HVP {errs[2]:.2e}")
    assert max(errs) < 1e-3
