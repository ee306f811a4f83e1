"""GPU parity of the paper's codec variant (Sec. 3.3) on the time codec: per-vector
min-max normalisation to [0, 1] (offset and range kept in FP64, range floored at beta)
and the ELU activation, against the FP64 oracle with the same weights -- window encode
and decode, ELU training steps, and the compressed gradient."""
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


def _fields(shape, nsteps, seed):
    rng = np.random.default_rng(seed)
    out = []
    for t in range(nsteps):
        e = inputs.smooth_state(shape, 10.0, seed=seed + t)[0] * 10.0 ** rng.uniform(-9, -6)
        e = W.interior(e) + 3e-8 * (t % 3)               # offsets: the min is not -max
        out.append(e.astype(np.float32).astype(np.float64))
    return out


@pytest.mark.parametrize("act", ["gelu", "elu"])
@pytest.mark.parametrize("beta", [1e-7, 1e-30])
def test_minmax_window_encode_and_decode_match_oracle(act, beta):
    shape = (16, 24, 32)
    prob, _, _ = setup(shape, 4, 16)
    s = solver(prob, storage="full", codec="time", norm="minmax", act=act, beta=beta)
    Wt = inputs.codec_init(seed=12, n_hid=1024, n_lat=512)
    s.codec_set(Wt)
    es = _fields(shape, 13, seed=21)
    lat, sc = s.codec_encode_window(cuda(np.stack(es)))
    X16 = C.round_bf16(CT.pack(es, shape))
    mn, r = CT.minmax_scales(X16, beta)
    sc = sc.cpu().numpy()
    np.testing.assert_array_equal(sc[0], mn)             # minimum of the stored BF16 values
    np.testing.assert_allclose(sc[1], r, rtol=1e-15, atol=0)
    Y = C.round_bf16(C.round_fp32(CT.minmax_normalise(X16, mn, r)))
    z_ref = C.encode(Wt, Y, emulate=True, act=act)
    z = host(lat.float())
    assert relerr(z, z_ref) < CODEC_TOL
    e_dec = host(s.codec_decode_window(lat, torch.from_numpy(sc).cuda()))
    Xh = C.decode(Wt, z, emulate=True, act=act) * r[:, None] + mn[:, None]
    E_ref = CT.unpack(Xh, shape)
    for t in range(16):
        E_ref[t] = CT.interior(E_ref[t])
    assert relerr(e_dec, E_ref) < CODEC_TOL


def test_elu_training_steps_match_oracle():
    prob, _, _ = setup((32, 32, 32), 4, 16)
    s = solver(prob, storage="full", codec="time", act="elu")
    Wt = inputs.codec_init(seed=13, n_hid=1024, n_lat=512)
    rng = np.random.default_rng(14)
    for k in ("b1", "b3"):
        Wt[k] = (0.3 * rng.standard_normal(Wt[k].shape)).astype(np.float32)   # both ELU branches
    s.codec_set(Wt)
    Y = C.round_bf16(rng.uniform(0, 1, (256, 2048)))
    ydev = torch.from_numpy(Y.astype(np.float32)).to(torch.bfloat16).cuda()
    Wo = {k: v.astype(np.float64) for k, v in Wt.items()}
    opt = C.Lamb(Wo)
    for it in range(3):
        loss = s.train_step(ydev, 1e-3)
        L, g = C.loss_and_grad(Wo, Y, emulate=True, act="elu")
        assert abs(loss - L) <= 2e-3 * L, (it, loss, L)
        Wo = opt.step(Wo, g, 1e-3)
    Wg = s.codec_get()
    for k in C.PARAMS:
        tol = 1e-2 if k in ("b1", "b2", "b3") else 2e-3
        assert relerr(Wg[k], Wo[k]) < tol, k


def test_minmax_compressed_gradient_matches_oracle():
    """Min-max windows (beta scaled to this workload's amplitudes) with the optimal
    rank-512 code of the run's own normalised windows, end to end."""
    beta = 1e-30
    prob, c, _ = setup((32, 32, 32), 120, 16, seed=0)
    ctrue = inputs.bump_model(c, prob.h).astype(np.float32).astype(np.float64)
    d_obs, _, _ = W.forward(prob, ctrue)
    _, states = W.forward_states(prob, c)
    e_hist = [st[0] for st in states]
    Y = []
    for tb in range(CT.n_windows(prob.nt)):
        X = CT.window_vectors(e_hist, prob.shape, tb)
        mn, r = CT.minmax_scales(X, beta)
        Y.append(CT.minmax_normalise(X, mn, r))
    Wt = {k: v.astype(np.float32) for k, v in CT.pca_codec(np.concatenate(Y), 512).items()}
    s = solver(prob, storage="ae", codec="time", norm="minmax", beta=beta)
    s.codec_set(Wt)
    J, g = s.gradient(cuda(c), cuda(d_obs))
    ehat = CT.bf16_history(CT.compressed_e_history(Wt, e_hist, emulate=True, norm="minmax",
                                                      beta=beta))
    J_ref, g_ref, _ = W.gradient(prob, c, d_obs, e_of=lambda n: ehat[n])
    err = relerr(host(g), g_ref)
    print(f"min-max AE gradient parity (32^3): {err:.2e}")
    assert abs(J - J_ref) / J_ref < 1e-4
    assert err < 1e-3
