"""GPU parity of the MAP machinery -- the BiLaplacian prior of Sec. 2 and the Newton-CG
and DIAS drivers of Sec. 4.3 -- against the FP64 oracle (oracle.newton): the prior's
elliptic operator and its inverse (exact in the oracle by the DCT-II), Newton-CG
iterates with the Gauss-Newton and the full misfit Hessian, the projected DIAS-F
problem, and the active subspace from prior-sample gradients."""
import numpy as np
import pytest

from oracle import newton as NW
from oracle import wave as W
from paper_2304_04781_gb300 import inputs

from .helpers import cuda, host, relerr, setup, solver

pytestmark = pytest.mark.gpu


def _grid_solver(shape):
    prob, _, _ = setup(shape, 4, 4)
    return prob, solver(prob, storage="full")


@pytest.mark.parametrize("shape", [(20, 24, 28), (12, 16, 260)])
@pytest.mark.parametrize("alpha,theta", [(1.0, 0.0), (2e-3, 6400.0), (0.5, 100.0)])
def test_prior_apply_matches_oracle(alpha, theta, shape):
    # nx = 260: rows of 65 float4, so a warp takes three passes along x and the
    # neighbours across each 128-node stretch come from the loads of lanes 0 and 31
    prob, s = _grid_solver(shape)
    for q in (inputs.velocity_model(prob.shape, prob.h, seed=4),
              inputs.white_noise(1, prob.shape, seed=5)[0]):
        q = q.astype(np.float32).astype(np.float64)
        got = host(s.prior_apply(cuda(q), alpha, theta))
        ref = NW.prior_apply(q, prob.h, alpha, theta)
        assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("theta", [0.0, 1600.0, 6400.0])
def test_prior_solve_matches_the_exact_dct_inverse(theta):
    prob, s = _grid_solver((20, 24, 28))
    w = inputs.white_noise(1, prob.shape, seed=6)[0].astype(np.float64)
    x, it = s.prior_solve(cuda(w), 0.5, theta, rtol=1e-7)
    ref = NW.prior_solve(w, prob.h, 0.5, theta)
    err = relerr(host(x), ref)
    # the true residual of the FP32 iterate, in FP64
    res = relerr(NW.prior_apply(host(x), prob.h, 0.5, theta), w)
    print(f"prior solve theta={theta}: {it} iterations, error {err:.2e}, residual {res:.2e}")
    assert err < 2e-5 and res < 2e-6
    if theta == 0.0:
        assert it == 8     # exact after one iteration, seen at the first check


def test_prior_solve_of_zero_and_argument_errors():
    prob, s = _grid_solver((8, 8, 8))
    import torch
    z = torch.zeros(prob.shape, device="cuda")
    x, it = s.prior_solve(z, 1.0, 10.0)
    assert it == 0 and not torch.any(x)
    from paper_2304_04781_gb300.aewave import AewError
    with pytest.raises(AewError, match="AEW_E_ARG"):
        s.prior_apply(z, 0.0, 1.0)
    with pytest.raises(AewError, match="AEW_E_ARG"):
        s.prior_solve(z, 1.0, -1.0)
    with pytest.raises(AewError, match="AEW_E_NOCONVERGE"):
        s.prior_solve(cuda(inputs.white_noise(1, prob.shape, seed=1)[0]), 1e-3, 6400.0,
                      rtol=1e-7, max_iter=3)


def _map_case():
    prob, c0, _ = setup((16, 16, 16), 80, 16, seed=3)
    c_true = inputs.bump_model(c0, prob.h, amp=0.1).astype(np.float32).astype(np.float64)
    d_obs, _, _ = W.forward(prob, c_true)
    return prob, c0, d_obs


def _compare(hist, hist_ref, c, q_ref, c_init, tol):
    assert len(hist) == len(hist_ref)
    for a, b in zip(hist, hist_ref):
        assert a["cg_iters"] == b[2] and a["step"] == b[3]
        assert abs(a["cost"] - b[0]) <= 1e-4 * b[0]
        assert abs(a["gnorm"] - b[1]) <= 1e-3 * b[1]
    err = relerr(c - c_init, q_ref - c_init)
    print(f"Newton-CG update parity: {err:.2e}; costs {[h['cost'] for h in hist]}")
    assert err < tol


@pytest.mark.parametrize("full", [False, True])
def test_newton_cg_matches_oracle(full):
    prob, c0, d_obs = _map_case()
    kw = dict(alpha=1e-10, theta=6400.0, newton_iters=3 if not full else 2, cg_max=10,
              full_hessian=full)
    s = solver(prob, storage="full")
    c = cuda(c0)
    hist = s.newton_cg(c, cuda(d_obs), cuda(c0), **kw)
    q_ref, hist_ref = NW.newton_cg(prob, c0, d_obs, c0, NW.NewtonCfg(**kw))
    _compare(hist, hist_ref, host(c), q_ref, c0, 1e-4)
    assert hist[-1]["cost"] < 0.5 * hist[0]["cost"]


def test_projected_newton_cg_matches_oracle():
    prob, c0, d_obs = _map_case()
    W1 = inputs.orthonormal_rows(3, c0.size, seed=8).astype(np.float32).astype(np.float64)
    kw = dict(alpha=1e-10, theta=6400.0, newton_iters=2, cg_max=8)
    s = solver(prob, storage="full")
    c = cuda(c0)
    hist = s.newton_cg(c, cuda(d_obs), cuda(c0), W1=cuda(W1), **kw)
    q_ref, hist_ref = NW.newton_cg(prob, c0, d_obs, c0, NW.NewtonCfg(**kw),
                                   proj=NW.projector(W1, prob.shape))
    _compare(hist, hist_ref, host(c), q_ref, c0, 1e-4)


def test_failed_line_search_stops_without_moving():
    prob, c0, d_obs = _map_case()
    kw = dict(alpha=1e-10, theta=6400.0, newton_iters=3, cg_max=5, c1=0.999999,
              max_backtracks=1)
    s = solver(prob, storage="full")
    c = cuda(c0)
    hist = s.newton_cg(c, cuda(d_obs), cuda(c0), **kw)
    q_ref, hist_ref = NW.newton_cg(prob, c0, d_obs, c0, NW.NewtonCfg(**kw))
    assert len(hist) == len(hist_ref) == 1 and hist[0]["step"] == 0.0
    assert hist[0]["backtracks"] == 1
    np.testing.assert_array_equal(host(c), c0)


def test_a_trial_beyond_the_stability_bound_is_backtracked():
    # a weak prior and a start 15% above the prior mean: the full Newton step leaves the
    # stability bound in the oracle's and the library's line search alike, and both
    # halve it
    # (here the first two trials reach max c = 5107 and 3637 m/s, above the bound of
    # 3464 m/s, and the third passes)
    prob, c0, d_obs = _map_case()
    start = (1.15 * c0).astype(np.float32).astype(np.float64)
    kw = dict(alpha=1e-12, theta=6400.0, newton_iters=2, cg_max=20)
    q_ref, hist_ref = NW.newton_cg(prob, start, d_obs, c0, NW.NewtonCfg(**kw))
    assert hist_ref[0][3] == 0.25
    s = solver(prob, storage="full")
    c = cuda(start)
    hist = s.newton_cg(c, cuda(d_obs), cuda(c0), **kw)
    assert hist[0]["backtracks"] == 2
    _compare(hist, hist_ref, host(c), q_ref, start, 1e-4)


def test_gtol_stops_early_and_bad_settings_are_rejected():
    prob, c0, d_obs = _map_case()
    s = solver(prob, storage="full")
    c = cuda(c0)
    hist = s.newton_cg(c, cuda(d_obs), cuda(c0), 1e-10, 6400.0, newton_iters=6, cg_max=10,
                       gtol=0.2)
    assert 1 <= len(hist) < 6
    from paper_2304_04781_gb300.aewave import AewError
    with pytest.raises(AewError, match="AEW_E_ARG"):
        s.newton_cg(c, cuda(d_obs), cuda(c0), 1e-10, 6400.0, cg_max=0)


def _sample_alpha(prob, theta, std):
    """alpha whose prior samples A^{-1} w have pointwise std `std` on average."""
    sym = NW.prior_symbol(prob.shape, prob.h, 1.0, theta)
    return float(np.sqrt(np.mean(1.0 / sym ** 2)) / std)


def test_dias_subspace_matches_oracle():
    prob, c0, d_obs = _map_case()
    theta = 6400.0
    alpha_s = _sample_alpha(prob, theta, 40.0)
    N, r = 6, 3
    noise = inputs.white_noise(N, prob.shape, seed=9)
    s = solver(prob, storage="full")
    lam, W1, G = s.dias_subspace(cuda(c0), cuda(d_obs), cuda(noise), alpha_s, theta, r)
    grads = NW.dias_samples(prob, c0, d_obs, NW.NewtonCfg(alpha=alpha_s, theta=theta),
                            noise.astype(np.float64))
    for i in range(N):
        assert relerr(host(G[i]).reshape(prob.shape), grads[i]) < 1e-4
    lam_ref, W1_ref = NW.active_subspace(grads, r)
    Gm = np.stack([g.ravel() for g in grads], 1)
    lam_all = np.linalg.eigvalsh(Gm.T @ Gm / N)[::-1]
    np.testing.assert_allclose(lam, lam_all, rtol=1e-3, atol=1e-6 * lam_all[0])
    W1g = host(W1)
    np.testing.assert_allclose(W1g @ W1g.T, np.eye(r), atol=1e-5)
    sv = np.linalg.svd(W1g @ W1_ref.T, compute_uv=False)
    print(f"DIAS eigenvalues {lam[:r]}, subspace cosines {sv}")
    assert sv.min() > 1 - 1e-4


def test_newton_cg_with_checkpointing_equals_full_storage_bitwise():
    # revolve's gradient and HVP equal full storage's bit for bit, and its trial
    # gradients run the adjoint half too (the gate tests the misfit at the end): the
    # Newton iterates must agree exactly
    prob, c0, d_obs = _map_case()
    kw = dict(alpha=1e-10, theta=6400.0, newton_iters=2, cg_max=6)
    out = []
    for storage, extra in (("full", {}), ("revolve", {"n_checkpoints": 6})):
        s = solver(prob, storage=storage, **extra)
        c = cuda(c0)
        hist = s.newton_cg(c, cuda(d_obs), cuda(c0), **kw)
        out.append((host(c), hist))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


def test_newton_cg_with_the_time_codec_tracks_full_storage():
    # the compressed history (a code fitted to this run's own windows) in every gradient,
    # trial gradient (stopped after its forward solve when the misfit fails) and HVP
    from oracle import codec_time as CT
    prob, c0, _ = setup((32, 32, 32), 96, 16, seed=2)
    c_true = inputs.bump_model(c0, prob.h, amp=0.1).astype(np.float32).astype(np.float64)
    d_obs, _, _ = W.forward(prob, c_true)
    _, states = W.forward_states(prob, c0)
    e_hist = [st[0] for st in states]
    Y = []
    for tb in range(CT.n_windows(prob.nt)):
        X = CT.window_vectors(e_hist, prob.shape, tb)
        Y.append(CT.normalise(X, CT.vector_scales(X)))
    Wt = {k: v.astype(np.float32) for k, v in CT.pca_codec(np.concatenate(Y), 512).items()}
    kw = dict(alpha=1e-10, theta=6400.0, newton_iters=3, cg_max=6)
    ae = solver(prob, storage="ae", codec="time")
    ae.codec_set(Wt)
    c_ae = cuda(c0)
    h_ae = ae.newton_cg(c_ae, cuda(d_obs), cuda(c0), **kw)
    fu = solver(prob, storage="full")
    c_fu = cuda(c0)
    h_fu = fu.newton_cg(c_fu, cuda(d_obs), cuda(c0), **kw)
    assert [h["cg_iters"] for h in h_ae] == [h["cg_iters"] for h in h_fu]
    assert h_ae[-1]["cost"] < 0.5 * h_ae[0]["cost"]
    err = relerr(host(c_ae) - c0, host(c_fu) - c0)
    print(f"Newton-CG, time codec vs full storage: update {err:.2e}; costs "
          f"{[h['cost'] for h in h_ae]} vs {[h['cost'] for h in h_fu]}")
    assert err < 2e-2


def test_argument_errors_of_the_map_calls():
    import torch
    from paper_2304_04781_gb300.aewave import AewError
    prob, c0, d_obs = _map_case()
    s = solver(prob, storage="full")
    c, d, q0 = cuda(c0), cuda(d_obs), cuda(c0)
    n = c0.size
    noise = torch.zeros((2, n), device="cuda")
    with pytest.raises(AewError, match="AEW_E_ARG"):           # r > N
        s.dias_subspace(c, d, noise, 1.0, 100.0, 3)
    with pytest.raises(AewError, match="AEW_E_ARG"):           # N > 64
        s.dias_subspace(c, d, torch.zeros((65, n), device="cuda"), 1.0, 100.0, 2)
    with pytest.raises(AewError, match="AEW_E_ARG"):           # r > 32 rows of W1
        s.newton_cg(c, d, q0, 1e-10, 6400.0, W1=torch.zeros((33, n), device="cuda"))
    buf = torch.zeros(n + 1, device="cuda")
    with pytest.raises(AewError, match="16-byte aligned"):     # a vector off by one float
        s.prior_solve(buf[1:].view(prob.shape), 1.0, 100.0)
    with pytest.raises(AewError, match="AEW_E_ARG"):
        s.newton_cg(c, d, q0, 1e-10, 6400.0, eta_max=0.0)
    # the handle stays usable after the errors
    J, _ = s.gradient(c, d)
    assert J > 0
