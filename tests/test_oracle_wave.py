"""Pins of the FP64 oracle's solver, adjoint and Hessian against what the mathematics
fixes: exact discrete eigenmodes, exact energy conservation, second-order
convergence to the continuum standing wave, the adjoint identity, central finite
differences and the Gauss-Newton identities.  CPU only."""
import math

import numpy as np
import pytest

from oracle import wave as W
from paper_2304_04781_gb300 import inputs


def _problem(n=16, nt=120, nrec=16, **kw):
    rec = inputs.receiver_grid(n, n, nrec)
    return W.Problem(shape=(n, n, n), h=10.0, nt=nt, rec=rec, **kw)


# ---------------------------------------------------------------------------- source
def test_ricker_peak_and_zero_crossings():
    f0, t0 = 25.0, 0.04
    sig = 1.0 / (math.sqrt(2.0) * math.pi * f0)
    assert W.ricker(t0, f0, t0) == pytest.approx(1.0, abs=1e-15)
    assert abs(W.ricker(t0 + sig, f0, t0)) < 1e-15
    assert abs(W.ricker(t0 - sig, f0, t0)) < 1e-15
    # spectrum peaks at f0: the standard form (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2)
    tau = np.linspace(-0.05, 0.05, 101)
    std = (1 - 2 * (math.pi * f0 * tau) ** 2) * np.exp(-(math.pi * f0 * tau) ** 2)
    np.testing.assert_allclose(W.ricker(t0 + tau, f0, t0), std, rtol=0, atol=1e-14)


# ---------------------------------------------------------------------------- operators
def _dense(op, n_in, shape):
    cols = []
    for k in range(n_in):
        x = np.zeros(n_in); x[k] = 1.0
        cols.append(op(x))
    return np.array(cols).T


def test_div_is_minus_grad_transpose_on_interior():
    shape = (4, 5, 6)
    N = int(np.prod(shape))
    h = 0.7
    inside = np.zeros(shape, bool); inside[1:-1, 1:-1, 1:-1] = True
    G = _dense(lambda x: np.concatenate([a.ravel() for a in W.grad_op(x.reshape(shape), h)]), N, shape)
    D = _dense(lambda x: W.div_op(*(x[i * N:(i + 1) * N].reshape(shape) for i in range(3)), h).ravel(),
               3 * N, shape)
    idx = np.flatnonzero(inside.ravel())
    np.testing.assert_allclose(D[idx, :], -G[:, idx].T, atol=1e-14)
    # D never writes boundary nodes
    assert np.all(D[~inside.ravel(), :] == 0)


def test_explicit_transposes():
    shape = (5, 6, 7)
    rng = np.random.default_rng(1)
    f, mu = rng.standard_normal(shape), rng.standard_normal(shape)
    l = [rng.standard_normal(shape) for _ in range(3)]
    v = [rng.standard_normal(shape) for _ in range(3)]
    h = 1.3
    lhs = sum(np.sum(a * b) for a, b in zip(W.grad_op(f, h), l))
    rhs = np.sum(f * W.grad_op_T(*l, h))
    assert lhs == pytest.approx(rhs, rel=1e-13)
    lhs = np.sum(W.div_op(*v, h) * mu)
    rhs = sum(np.sum(a * b) for a, b in zip(v, W.div_op_T(mu, h)))
    assert lhs == pytest.approx(rhs, rel=1e-13)


# ---------------------------------------------------------------------------- eigenmode
def eigenmode_setup(shape, h, c, p_modes, nt, cfl=0.5, cmax=3000.0):
    """Exact discrete standing wave of the scheme (derived from the update equations):
    S = prod sin(pi p_a x_a / L_a) with L_a = (N_a-1) h satisfies -D G S = lam S with
    lam = sum (4/h^2) sin^2(pi p_a h / (2 L_a)); then e^n = S cos(w n dt),
    v^n = m dt / (2 sin(w dt/2)) G S sin(w (n - 1/2) dt), sin(w dt/2) = c dt sqrt(lam)/2."""
    prob = W.Problem(shape=shape, h=h, nt=nt, cfl=cfl, cmax=cmax, rec=np.zeros((0, 3), int))
    dt = prob.dt
    axes = []
    lam = 0.0
    for ax, (N, p) in enumerate(zip(shape, p_modes)):
        L = (N - 1) * h
        x = np.arange(N) * h
        axes.append(np.sin(math.pi * p * x / L))
        lam += 4.0 / h ** 2 * math.sin(math.pi * p * h / (2 * L)) ** 2
    S = axes[0][:, None, None] * axes[1][None, :, None] * axes[2][None, None, :]
    m = c * c
    w = 2.0 / dt * math.asin(c * dt * math.sqrt(lam) / 2.0)
    A = m * dt / (2.0 * math.sin(w * dt / 2.0))
    G = W.grad_op(S, h)

    def state(n):
        return (S * math.cos(w * n * dt),) + tuple(A * g * math.sin(w * (n - 0.5) * dt) for g in G)

    return prob, S, state


def test_exact_discrete_eigenmode():
    shape, h, c = (12, 10, 14), 10.0, 2100.0
    prob, S, state = eigenmode_setup(shape, h, c, (2, 1, 3), nt=200)
    cfield = np.full(shape, c)
    _, final, _ = W.forward(prob, cfield, wavelet=np.zeros(prob.nt), state0=state(0))
    ref = state(prob.nt)
    for got, want in zip(final, ref):
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err < 1e-12, err


def test_energy_conserved_without_source():
    shape, h = (14, 13, 12), 10.0
    prob = W.Problem(shape=shape, h=h, nt=200, rec=np.zeros((0, 3), int))
    c = inputs.velocity_model(shape, h, seed=5)
    m = c * c
    st = inputs.smooth_state(shape, h, seed=3)
    e0 = W.interior(st[0] * 1e-3)
    state0 = (e0, st[1], st[2], st[3])
    zero = np.zeros(prob.nt)
    E = []
    cur = state0
    for n in range(prob.nt):
        nxt = W.forward_step(prob, m, *cur, 0.0)
        E.append(W.energy(m, cur[0], cur[1:], nxt[1:]))
        cur = nxt
    E = np.array(E)
    assert np.max(np.abs(E - E[0])) / abs(E[0]) < 1e-13
    # the energy is not trivially constant: both parts change over time
    kin = [0.5 * np.sum(m * x * x) for x in [state0[0], cur[0]]]
    assert abs(kin[1] - kin[0]) > 1e-3 * abs(E[0])


def test_second_order_convergence_to_continuum_standing_wave():
    """e = S cos(w_c t), v = c^2 grad S sin(w_c t) / w_c with w_c = c pi sqrt(sum (p/L)^2).
    At fixed L and CFL the nodal error must fall by 4x per halving of h."""
    L, c, p = 80.0, 2000.0, (1, 1, 1)
    wc = c * math.pi * math.sqrt(sum((q / L) ** 2 for q in p))
    errs = []
    for N, nt in ((9, 12), (17, 24), (33, 48)):
        h = L / (N - 1)
        prob = W.Problem(shape=(N, N, N), h=h, nt=nt, rec=np.zeros((0, 3), int))
        dt = prob.dt
        x = np.arange(N) * h
        xf = x + 0.5 * h
        s = np.sin(math.pi * x / L); cf = math.pi / L * np.cos(math.pi * xf / L)
        S = s[:, None, None] * s[None, :, None] * s[None, None, :]
        # continuum grad S sampled at the face centres (last face unused -> 0)
        gx = s[:, None, None] * s[None, :, None] * cf[None, None, :]
        gy = s[:, None, None] * cf[None, :, None] * s[None, None, :]
        gz = cf[:, None, None] * s[None, :, None] * s[None, None, :]
        for g, ax in ((gx, 2), (gy, 1), (gz, 0)):
            sl = [slice(None)] * 3; sl[ax] = -1
            g[tuple(sl)] = 0.0
        amp = c * c / wc * math.sin(-wc * dt / 2.0)
        state0 = (S, amp * gx, amp * gy, amp * gz)
        _, final, _ = W.forward(prob, np.full(S.shape, c), wavelet=np.zeros(nt), state0=state0)
        exact = S * math.cos(wc * nt * dt)
        errs.append(np.max(np.abs(final[0] - exact)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.7 < r1 < 4.3 and 3.7 < r2 < 4.3, (errs, r1, r2)


# ---------------------------------------------------------------------------- adjoint
def test_adjoint_identity_source_to_receiver():
    prob = _problem(n=16, nt=80)
    c = inputs.velocity_model(prob.shape, prob.h, seed=0)
    rng = np.random.default_rng(2)
    w = rng.standard_normal(prob.nt)
    r = rng.standard_normal((prob.nt + 1, prob.nrec, 3)); r[0] = 0
    d, _, states = W.forward(prob, c, wavelet=w, keep_states=True)
    _, sgrad = W.adjoint(prob, c, lambda n: states[n][0], r, want_source_grad=True)
    lhs = float(np.sum(d[1:] * r[1:]))
    rhs = float(np.dot(w, sgrad))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_adjoint_identity_parameter_jacobian():
    prob = _problem(n=16, nt=120)
    c = inputs.velocity_model(prob.shape, prob.h, seed=0)
    dc = inputs.direction(prob.shape, prob.h, seed=11)
    d, states = W.forward_states(prob, c)
    e_of = lambda n: states[n][0]
    rng = np.random.default_rng(4)
    r = rng.standard_normal(d.shape); r[0] = 0
    Jdc = W.incremental_forward(prob, c, dc, e_of)
    JTr = W.jacobian_transpose(prob, c, r, e_of)
    lhs = float(np.sum(Jdc[1:] * r[1:]))
    rhs = float(np.sum(dc * JTr))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _misfit_at(prob, c, d_obs):
    d, _, _ = W.forward(prob, c)
    return W.misfit(d, d_obs)


def test_gradient_matches_central_differences_16cubed():
    prob = _problem(n=16, nt=120)
    c = inputs.velocity_model(prob.shape, prob.h, seed=0)
    d_obs, _, _ = W.forward(prob, inputs.bump_model(c, prob.h))
    J, g, _ = W.gradient(prob, c, d_obs)
    assert J > 0
    # central differences err by ~140 (eps/|c|)^2 relative here (measured scaling), so
    # eps = 1e-6 |c| leaves ~1e-10; FP64 round-off in J is far below that.
    eps = 1e-6 * np.abs(c).max()
    for k in range(8):
        dc = inputs.direction(prob.shape, prob.h, seed=10 + k)
        fd = (_misfit_at(prob, c + eps * dc, d_obs) - _misfit_at(prob, c - eps * dc, d_obs)) / (2 * eps)
        ad = float(np.sum(g * dc))
        assert abs(fd - ad) <= 1e-8 * abs(ad), (k, fd, ad)


def test_gauss_newton_identities():
    prob = _problem(n=16, nt=120)
    c = inputs.velocity_model(prob.shape, prob.h, seed=0)
    d, states = W.forward_states(prob, c)
    e_of = lambda n: states[n][0]
    dc1 = inputs.direction(prob.shape, prob.h, seed=20)
    dc2 = inputs.direction(prob.shape, prob.h, seed=21)
    H1 = W.hessvec_gn(prob, c, dc1, e_of)
    H2 = W.hessvec_gn(prob, c, dc2, e_of)
    # (i) <dc, H dc> = |J dc|^2 with J dc from the incremental forward alone
    Jdc = W.incremental_forward(prob, c, dc1, e_of)
    q = float(np.sum(dc1 * H1))
    assert q == pytest.approx(float(np.sum(Jdc[1:] ** 2)), rel=1e-10)
    # (ii) symmetry
    a, b = float(np.sum(dc2 * H1)), float(np.sum(dc1 * H2))
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))


def test_gauss_newton_equals_gradient_derivative_at_zero_residual():
    """With d_obs = F(c) the residual vanishes, so GN = full Hessian at c and the central
    difference of the gradient must reproduce H dc (to O(eps^2))."""
    prob = _problem(n=16, nt=120)
    c = inputs.velocity_model(prob.shape, prob.h, seed=0)
    d_obs, states = W.forward_states(prob, c)
    dc = inputs.direction(prob.shape, prob.h, seed=30)
    H = W.hessvec_gn(prob, c, dc, lambda n: states[n][0])
    eps = 1e-4 * np.abs(c).max()
    _, gp, _ = W.gradient(prob, c + eps * dc, d_obs)
    _, gm, _ = W.gradient(prob, c - eps * dc, d_obs)
    fd = (gp - gm) / (2 * eps)
    err = np.linalg.norm(fd - H) / np.linalg.norm(H)
    assert err < 1e-6, err


def test_wrong_adjoint_is_caught():
    """A planted sign error in the transpose breaks the identity (the pin is sharp)."""
    prob = _problem(n=12, nt=60)
    c = inputs.velocity_model(prob.shape, prob.h, seed=0)
    dc = inputs.direction(prob.shape, prob.h, seed=11)
    d, states = W.forward_states(prob, c)
    rng = np.random.default_rng(4)
    r = rng.standard_normal(d.shape); r[0] = 0
    Jdc = W.incremental_forward(prob, c, dc, lambda n: states[n][0])
    bad = lambda n: -states[n][0] if n % 7 == 3 else states[n][0]
    JTr = W.jacobian_transpose(prob, c, r, bad)
    lhs, rhs = float(np.sum(Jdc[1:] * r[1:])), float(np.sum(dc * JTr))
    assert abs(lhs - rhs) > 1e-6 * abs(lhs)


# ---------------------------------------------------------------------------- full Newton
def test_full_hessian_equals_gradient_derivative_at_nonzero_residual():
    """The full Newton HVP is the derivative of the gradient: at a nonzero residual (data
    from the bump model) the central difference of the gradient reproduces H dc to
    O(eps^2), while the Gauss-Newton product does not."""
    prob = _problem(n=16, nt=120)
    c = inputs.velocity_model(prob.shape, prob.h, seed=0)
    d_obs, _, _ = W.forward(prob, inputs.bump_model(c, prob.h, amp=0.2))
    _, states = W.forward_states(prob, c)
    e_of = lambda n: states[n][0]
    dc = inputs.direction(prob.shape, prob.h, seed=31)
    H = W.hessvec_full(prob, c, d_obs, dc, e_of)
    # the difference errs by ~0.18 (eps/|c|)^2 relative (measured: 1.8e-6 at 1e-4 and
    # 1.8e-8 at 1e-5, an exact eps^2 scaling), far above FP64 round-off at 1e-5
    eps = 1e-5 * np.abs(c).max()
    _, gp, _ = W.gradient(prob, c + eps * dc, d_obs)
    _, gm, _ = W.gradient(prob, c - eps * dc, d_obs)
    fd = (gp - gm) / (2 * eps)
    err = np.linalg.norm(fd - H) / np.linalg.norm(H)
    assert err < 1e-7, err
    Hgn = W.hessvec_gn(prob, c, dc, e_of)
    assert np.linalg.norm(fd - Hgn) / np.linalg.norm(fd) > 1e-3    # the residual terms matter


def test_full_hessian_is_symmetric_and_reduces_to_gauss_newton_at_zero_residual():
    prob = _problem(n=16, nt=80)
    c = inputs.velocity_model(prob.shape, prob.h, seed=1)
    _, states = W.forward_states(prob, c)
    e_of = lambda n: states[n][0]
    dc1 = inputs.direction(prob.shape, prob.h, seed=40)
    dc2 = inputs.direction(prob.shape, prob.h, seed=41)
    d_obs, _, _ = W.forward(prob, inputs.bump_model(c, prob.h, amp=0.2))
    H1 = W.hessvec_full(prob, c, d_obs, dc1, e_of)
    H2 = W.hessvec_full(prob, c, d_obs, dc2, e_of)
    a, b = float(np.sum(dc2 * H1)), float(np.sum(dc1 * H2))
    assert abs(a - b) <= 1e-10 * max(abs(a), abs(b))
    d0, _, _ = W.forward(prob, c)                     # zero residual
    Hf = W.hessvec_full(prob, c, d0, dc1, e_of)
    Hg = W.hessvec_gn(prob, c, dc1, e_of)
    np.testing.assert_allclose(Hf, Hg, rtol=0, atol=1e-12 * np.abs(Hg).max())


def test_incremental_strain_history_matches_the_jacobian_product():
    prob = _problem(n=12, nt=50)
    c = inputs.velocity_model(prob.shape, prob.h, seed=2)
    _, states = W.forward_states(prob, c)
    dc = inputs.direction(prob.shape, prob.h, seed=42)
    dd, hist = W.incremental_forward_states(prob, c, dc, lambda n: states[n][0])
    np.testing.assert_array_equal(dd, W.incremental_forward(prob, c, dc, lambda n: states[n][0]))
    assert len(hist) == prob.nt and not hist[0].any()
    # de^n is the derivative of e^n: central difference of two forward solves
    eps = 1e-5 * np.abs(c).max()
    _, sp = W.forward_states(prob, c + eps * dc)
    _, sm = W.forward_states(prob, c - eps * dc)
    n = 40
    fd = (sp[n][0] - sm[n][0]) / (2 * eps)
    assert np.linalg.norm(fd - hist[n]) <= 1e-6 * np.linalg.norm(hist[n])


# ------------------------------------------------------------------ smoothed source
def test_source_weights_are_a_normalised_symmetric_gaussian():
    prob = _problem(n=16, nt=4)
    prob.src_sigma = 20.0
    R, w = W.source_weights(prob)
    assert R == 6 and w.shape == (13, 13, 13)
    assert abs(w.sum() - 1.0) < 1e-14
    np.testing.assert_allclose(w, w[::-1], atol=0)
    np.testing.assert_allclose(w, w.transpose(2, 1, 0), atol=1e-18)
    # the ratio of neighbouring weights along an axis is exp(-(2a + 1) h^2 / (2 sigma^2))
    a = 2
    ratio = w[R, R, R + a + 1] / w[R, R, R + a]
    assert ratio == pytest.approx(np.exp(-(2 * a + 1) * prob.h ** 2 / (2 * 20.0 ** 2)), rel=1e-12)


def test_smoothed_source_is_the_weighted_sum_of_point_sources():
    # the wave equation is linear in the source: a source spread over the 125 faces of a
    # two-face box gives the weighted sum of 125 point-source solves, face by face
    prob = _problem(n=16, nt=30)
    prob.src_sigma = 4.0
    c = inputs.velocity_model(prob.shape, prob.h, seed=0)
    R, w = W.source_weights(prob)
    assert R == 2
    d_s, (e_s, *_), _ = W.forward(prob, c)
    i, j, k = prob.src
    d_sum = np.zeros_like(d_s)
    e_sum = np.zeros(prob.shape)
    for cz in range(-R, R + 1):
        for by in range(-R, R + 1):
            for ax in range(-R, R + 1):
                q = W.Problem(shape=prob.shape, h=prob.h, nt=prob.nt, rec=prob.rec,
                              src=(i + ax, j + by, k + cz))
                d_p, (e_p, *_), _ = W.forward(q, c)
                d_sum += w[cz + R, by + R, ax + R] * d_p
                e_sum += w[cz + R, by + R, ax + R] * e_p
    np.testing.assert_allclose(d_s, d_sum, rtol=0, atol=1e-12 * np.abs(d_s).max())
    np.testing.assert_allclose(e_s, e_sum, rtol=0, atol=1e-12 * np.abs(e_s).max())


def test_smoothed_source_adjoint_identity_and_point_limit():
    prob = _problem(n=16, nt=60)
    prob.src_sigma = 15.0
    c = inputs.velocity_model(prob.shape, prob.h, seed=0)
    rng = np.random.default_rng(2)
    w = rng.standard_normal(prob.nt)
    r = rng.standard_normal((prob.nt + 1, prob.nrec, 3)); r[0] = 0
    d, _, states = W.forward(prob, c, wavelet=w, keep_states=True)
    _, sgrad = W.adjoint(prob, c, lambda n: states[n][0], r, want_source_grad=True)
    lhs = float(np.sum(d[1:] * r[1:]))
    assert abs(lhs - float(np.dot(w, sgrad))) <= 1e-12 * abs(lhs)
    # a very narrow Gaussian is the point source
    prob.src_sigma = 1.0
    d1, _, _ = W.forward(prob, c)
    prob.src_sigma = 0.0
    d0, _, _ = W.forward(prob, c)
    np.testing.assert_allclose(d1, d0, rtol=0, atol=1e-14 * np.abs(d0).max())
