"""GPU parity of the full Newton Hessian-vector product (aew_hessvec_full: Sec. 4's
incremental forward and incremental adjoint problems with the second-order terms)
against the FP64 oracle (oracle.wave.hessvec_full), with full storage (exact
histories) and with the time codec (forward and incremental strain both compressed,
the oracle decoding its own FP64 histories with the same weights), and its reduction to
the Gauss-Newton product at zero residual."""
import numpy as np
import pytest

from oracle import codec_time as CT
from oracle import wave as W
from paper_2304_04781_gb300 import inputs

from .helpers import cuda, host, relerr, setup, solver

pytestmark = pytest.mark.gpu


def _case(shape, nt, seed):
    prob, c, _ = setup(shape, nt, 16, seed=seed)
    ctrue = inputs.bump_model(c, prob.h, amp=0.2).astype(np.float32).astype(np.float64)
    d_obs, _, _ = W.forward(prob, ctrue)
    dc = inputs.direction(prob.shape, prob.h, seed=50).astype(np.float32).astype(np.float64)
    return prob, c, d_obs, dc


def test_full_newton_hvp_full_storage_matches_oracle():
    prob, c, d_obs, dc = _case((32, 32, 32), 100, 6)
    s = solver(prob, storage="full")
    s.gradient(cuda(c), cuda(d_obs))
    H = host(s.hessvec_full(cuda(dc)))
    _, states = W.forward_states(prob, c)
    H_ref = W.hessvec_full(prob, c, d_obs, dc, lambda n: states[n][0])
    err = relerr(H, H_ref)
    Hgn = host(s.hessvec(cuda(dc)))
    print(f"full Newton HVP parity (full storage, 32^3): {err:.2e}; "
          f"Gauss-Newton differs by {relerr(Hgn, H_ref):.2e}")
    assert err < 1e-4
    assert relerr(Hgn, H_ref) > 1e-3          # the second-order terms are exercised


def test_full_newton_equals_gauss_newton_at_zero_residual():
    prob, c, _, dc = _case((32, 32, 32), 80, 7)
    s = solver(prob, storage="full")
    d = s.forward(cuda(c))
    s.gradient(cuda(c), d)                     # zero residual
    Hf = host(s.hessvec_full(cuda(dc)))
    Hg = host(s.hessvec(cuda(dc)))
    assert relerr(Hf, Hg) < 1e-5


def test_full_newton_hvp_time_codec_matches_oracle():
    prob, c, d_obs, dc = _case((32, 32, 32), 120, 8)
    _, states = W.forward_states(prob, c)
    e_hist = [st[0] for st in states]
    Y = []
    for tb in range(CT.n_windows(prob.nt)):
        X = CT.window_vectors(e_hist, prob.shape, tb)
        Y.append(CT.normalise(X, CT.vector_scales(X)))
    Wt = {k: v.astype(np.float32) for k, v in CT.pca_codec(np.concatenate(Y), 512).items()}
    s = solver(prob, storage="ae", codec="time")
    s.codec_set(Wt)
    s.gradient(cuda(c), cuda(d_obs))
    H = host(s.hessvec_full(cuda(dc)))
    # the sweeps read both decoded histories as BF16 (R34).  The GPU's FP32 decoder sums
    # and the oracle's emulation land on different sides of a BF16 rounding boundary for
    # a few percent of the values (one BF16 step, 2^-8, each), twice over for the
    # incremental strain (encoded and decoded again): about 8e-4 here.  Reading FP32
    # anywhere instead gives 1.2e-3 to 1.8e-3.
    ehat = CT.bf16_history(CT.compressed_e_history(Wt, e_hist, emulate=True))
    e_of = lambda n: ehat[n]
    _, de_hist = W.incremental_forward_states(prob, c, dc, e_of)
    dehat = CT.bf16_history(CT.compressed_e_history(Wt, de_hist, emulate=True))
    H_ref = W.hessvec_full(prob, c, d_obs, dc, e_of, de_of=lambda n: dehat[n])
    err = relerr(H, H_ref)
    # the compressed result against the exact full Newton HVP
    H_exact = W.hessvec_full(prob, c, d_obs, dc, lambda n: e_hist[n])
    print(f"full Newton HVP parity (time codec, 32^3): {err:.2e}; "
          f"vs exact: {relerr(H, H_exact):.2e}")
    assert err < 1e-3
    # a second call reuses the gradient's latents and gives the same result
    H2 = host(s.hessvec_full(cuda(dc)))
    np.testing.assert_array_equal(H2, H)


def test_full_newton_needs_a_supported_storage():
    from paper_2304_04781_gb300 import aewave
    prob, c, d_obs, dc = _case((32, 32, 32), 20, 9)
    s = solver(prob, storage="revolve", n_checkpoints=4)
    s.gradient(cuda(c), cuda(d_obs))
    with pytest.raises(aewave.AewError) as ei:
        s.hessvec_full(cuda(dc))
    assert ei.value.code == -1
    s2 = solver(prob, storage="full")
    with pytest.raises(aewave.AewError) as ei:   # no gradient yet
        s2.hessvec_full(cuda(dc))
    assert ei.value.code == -5
