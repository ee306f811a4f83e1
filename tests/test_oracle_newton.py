"""Pins of the FP64 oracle's Newton-CG MAP solve with the BiLaplacian prior and of DIAS
(oracle/newton.py): the prior operator's symmetry, definiteness and exact DCT-II
eigenstructure, its exact inverse, the regularised gradient, the Newton-CG iteration
(descent, Armijo steps, the gradient reduced), and the active subspace against a dense
eigendecomposition.  CPU only."""
import numpy as np
import pytest
from scipy.fft import idctn

from oracle import newton as NW
from oracle import wave as W
from paper_2304_04781_gb300 import inputs


def _dense(op, shape):
    n = int(np.prod(shape))
    M = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n); e[k] = 1.0
        M[:, k] = op(e.reshape(shape)).ravel()
    return M


def test_neumann_laplacian_is_symmetric_semidefinite_with_constant_kernel():
    shape, h = (3, 4, 5), 10.0
    L = _dense(lambda q: NW.laplacian_neumann(q, h), shape)
    np.testing.assert_allclose(L, L.T, atol=1e-15)
    ev = np.linalg.eigvalsh(L)
    assert ev.max() < 1e-12 and np.sum(np.abs(ev) < 1e-12) == 1   # one zero mode: constants
    np.testing.assert_allclose(L @ np.ones(L.shape[0]), 0.0, atol=1e-15)


def test_prior_operator_eigenpairs_are_the_dct_modes():
    shape, h, alpha, theta = (6, 5, 7), 10.0, 2.0, 300.0
    sym = NW.prior_symbol(shape, h, alpha, theta)
    for p in [(0, 0, 0), (1, 0, 0), (0, 3, 2), (5, 4, 6), (2, 1, 3)]:
        c = np.zeros(shape); c[p] = 1.0
        mode = idctn(c, type=2, norm="ortho")          # cos(pi p (i + 1/2) / N) per axis
        np.testing.assert_allclose(NW.prior_apply(mode, h, alpha, theta), sym[p] * mode,
                                   rtol=0, atol=1e-12 * sym[p])
    A = _dense(lambda q: NW.prior_apply(q, h, alpha, theta), shape)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(A)), np.sort(sym.ravel()), rtol=1e-12)
    assert sym.min() == pytest.approx(alpha)             # the constant mode


def test_prior_solve_inverts_the_operator():
    rng = np.random.default_rng(1)
    shape, h, alpha, theta = (10, 12, 8), 10.0, 1e-3, 6400.0
    w = rng.standard_normal(shape)
    x = NW.prior_solve(w, h, alpha, theta)
    np.testing.assert_allclose(NW.prior_apply(x, h, alpha, theta), w, rtol=0, atol=1e-10 * np.abs(w).max())


def test_regularisation_gradient_and_projection():
    rng = np.random.default_rng(2)
    shape, h, alpha, theta = (6, 6, 6), 10.0, 0.3, 50.0
    q, q0, dq = (rng.standard_normal(shape) for _ in range(3))
    g = NW.regularisation_grad(q, q0, h, alpha, theta)
    eps = 1e-3
    fd = (NW.regularisation(q + eps * dq, q0, h, alpha, theta)
          - NW.regularisation(q - eps * dq, q0, h, alpha, theta)) / (2 * eps)
    assert fd == pytest.approx(float(np.sum(g * dq)), rel=1e-9)      # a quadratic: exact
    Q, _ = np.linalg.qr(rng.standard_normal((q.size, 3)))
    P = NW.projector(Q.T, shape)
    np.testing.assert_allclose(P(P(q)), P(q), atol=1e-12)             # idempotent
    assert float(np.sum(P(q) * dq)) == pytest.approx(float(np.sum(q * P(dq))), rel=1e-12)
    gp = NW.regularisation_grad(q, q0, h, alpha, theta, P)
    fdp = (NW.regularisation(q + eps * dq, q0, h, alpha, theta, P)
           - NW.regularisation(q - eps * dq, q0, h, alpha, theta, P)) / (2 * eps)
    assert fdp == pytest.approx(float(np.sum(gp * dq)), rel=1e-9)


def _map_problem():
    shape = (16, 16, 16)
    prob = W.Problem(shape=shape, h=10.0, nt=80, rec=inputs.receiver_grid(16, 16, 16))
    c_true = inputs.bump_model(inputs.velocity_model(shape, 10.0, seed=3), 10.0, amp=0.1)
    d_obs, _, _ = W.forward(prob, c_true)
    q0 = inputs.velocity_model(shape, 10.0, seed=3)
    return prob, d_obs, q0


def test_newton_cg_descends_with_armijo_steps_and_reduces_the_gradient():
    prob, d_obs, q0 = _map_problem()
    cfg = NW.NewtonCfg(alpha=1e-10, theta=6400.0, newton_iters=4, cg_max=10)
    q, hist = NW.newton_cg(prob, q0, d_obs, q0, cfg)
    costs = [h[0] for h in hist] + [NW.cost(prob, q, d_obs, q0, cfg)]
    assert all(b < a for a, b in zip(costs, costs[1:]))           # monotone descent
    assert costs[-1] < 0.05 * costs[0]
    Jm, gm, _ = W.gradient(prob, q, d_obs)
    g = gm + NW.regularisation_grad(q, q0, prob.h, cfg.alpha, cfg.theta)
    assert np.linalg.norm(g) < 0.1 * hist[0][1]
    assert all(h[2] >= 1 for h in hist) and all(0 < h[3] <= 1 for h in hist)
    # no projection and an empty active subspace are the same problem
    P0 = NW.projector(np.zeros((0, q.size)), q.shape)
    np.testing.assert_array_equal(P0(q), q)


def test_newton_step_on_a_pure_regularisation_problem_is_exact():
    # data from q0 itself, so the misfit and its gradient vanish at q0; with theta = 0
    # the prior Hessian is alpha^2 I, which at alpha = 1e-3 dwarfs the misfit's
    # Hessian, so one Newton step with a tight CG solve lands on q0 up to the misfit's
    # relative share (~1e-7)
    prob, _, q0 = _map_problem()
    d_obs, _, _ = W.forward(prob, q0)
    rng = np.random.default_rng(4)
    dq = NW.prior_solve(rng.standard_normal(q0.shape), prob.h, 1.0, 6400.0)
    dq *= 20.0 / np.abs(dq).max()
    cfg = NW.NewtonCfg(alpha=1e-3, theta=0.0, newton_iters=1, cg_max=5, eta_max=1e-12)
    q, hist = NW.newton_cg(prob, q0 + dq, d_obs, q0, cfg)
    assert hist[0][3] == 1.0
    assert np.abs(q - q0).max() < 1e-5 * np.abs(dq).max()


def test_active_subspace_matches_a_dense_eigendecomposition():
    rng = np.random.default_rng(5)
    shape = (4, 5, 6)
    grads = [rng.standard_normal(shape) * np.linspace(3, 0.2, 120).reshape(shape) for _ in range(9)]
    lam, W1 = NW.active_subspace(grads, 4)
    G = np.stack([g.ravel() for g in grads], 1)
    C = G @ G.T / G.shape[1]
    ev, V = np.linalg.eigh(C)
    np.testing.assert_allclose(lam, ev[::-1][:4], rtol=1e-10)
    np.testing.assert_allclose(W1 @ W1.T, np.eye(4), atol=1e-10)
    np.testing.assert_allclose(W1.T @ W1, V[:, ::-1][:, :4] @ V[:, ::-1][:, :4].T, atol=1e-10)


def test_stability_bound_and_a_failed_line_search():
    prob, d_obs, q0 = _map_problem()
    bound = (1.0 / np.sqrt(3.0)) * prob.h / prob.dt
    q = np.full(prob.shape, 2000.0)
    assert NW.stable(prob, q)
    q[3, 4, 5] = bound
    assert NW.stable(prob, q)
    q[3, 4, 5] = bound * (1 + 1e-12)
    assert not NW.stable(prob, q)
    q[3, 4, 5] = 0.0
    assert not NW.stable(prob, q)
    # c1 near 1 asks for the linear model's whole decrease, which a Newton step on a
    # curved cost does not give: no trial passes, nothing moves, the iteration stops
    cfg = NW.NewtonCfg(alpha=1e-10, theta=6400.0, newton_iters=3, cg_max=5, c1=0.999999,
                       max_backtracks=1)
    q, hist = NW.newton_cg(prob, q0, d_obs, q0, cfg)
    assert len(hist) == 1 and hist[0][3] == 0.0
    np.testing.assert_array_equal(q, q0)
