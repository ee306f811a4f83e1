"""FP64 oracle for the Newton-CG MAP solve with the BiLaplacian prior and for DIAS
regularisation (the paper's Sec. 2 objective and Sec. 4.3).

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference legs may import this module; it shares no code with the CUDA
path.

Prior (Sec. 2, Eq. (4); readings R17, R29): the elliptic operator
    A q = alpha (q - theta Lap_N q)
with Lap_N the node-centred Laplacian with zero-flux (Neumann) boundaries -- each node
sums (q_nb - q_i) / h^2 over the neighbours it has -- is symmetric positive definite,
and the prior precision is its square: the regularisation is
    R(q) = 1/2 |A (q - q0)|^2.
Lap_N is diagonalised by the type-II discrete cosine transform, so A^{-1} (and prior
samples q0 + A^{-1} w, w white noise) are exact here.

MAP (Sec. 2): minimise J(q) = misfit(q) + R(q) by inexact Newton-CG: each Newton step
solves (H_misfit + A^2) p = -g by conjugate gradients, stopped at a relative residual
eta = min(eta_max, sqrt(|g| / |g_0|)) (Eisenstat-Walker, eta_max = 0.5), then an Armijo backtracking line
search (c1 = 1e-4, step halved).  A trial point outside the wave solver's stability
bound (c dt / h > 1/sqrt(3), or c <= 0 anywhere) fails the test like a cost increase.  If
no trial passes, the step is not taken and the iteration stops.  H_misfit is the
Gauss-Newton Hessian (or the full one).

DIAS-F (Sec. 4.3): the active subspace of C = (1/N) sum_i grad f(q_i) grad f(q_i)^T
over N gradient samples at q_i = q_MAP + A^{-1} w_i (the two-step algorithm: centred at
the MAP point), its r leading eigenvectors W1 (found from the N x N Gram matrix of the
samples), the projector P = I - W1 W1^T, and the DIAS problem with the approximate
projected regularisation 1/2 (q - q0)^T P A^2 P (q - q0), solved by Newton-CG from
q_MAP.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.fft import dctn, idctn

from . import wave as W


# --------------------------------------------------------------------------------------
# BiLaplacian prior
# --------------------------------------------------------------------------------------
def laplacian_neumann(q: np.ndarray, h: float) -> np.ndarray:
    """Node-centred Laplacian with zero-flux boundaries: sum over the neighbours a node
    has of (q_nb - q_i) / h^2."""
    out = np.zeros_like(q, dtype=np.float64)
    for ax in range(3):
        d = np.diff(q, axis=ax) / (h * h)       # q[i+1] - q[i] on each interior face
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        out[tuple(lo)] += d
        out[tuple(hi)] -= d
    return out


def prior_apply(q: np.ndarray, h: float, alpha: float, theta: float) -> np.ndarray:
    """A q = alpha (q - theta Lap_N q)."""
    return alpha * (q - theta * laplacian_neumann(q, h))


def prior_symbol(shape, h: float, alpha: float, theta: float) -> np.ndarray:
    """Eigenvalues of A on the DCT-II modes cos(pi p (i + 1/2) / N) of each axis:
    alpha (1 + theta sum_a (4 / h^2) sin^2(pi p_a / (2 N_a)))."""
    lam = np.zeros(shape)
    for ax, n in enumerate(shape):
        p = np.arange(n)
        s = (4.0 / (h * h)) * np.sin(np.pi * p / (2.0 * n)) ** 2
        sh = [1, 1, 1]
        sh[ax] = n
        lam = lam + s.reshape(sh)
    return alpha * (1.0 + theta * lam)


def prior_solve(w: np.ndarray, h: float, alpha: float, theta: float) -> np.ndarray:
    """A^{-1} w, exactly, by the DCT-II diagonalisation."""
    sym = prior_symbol(w.shape, h, alpha, theta)
    return idctn(dctn(w, type=2, norm="ortho") / sym, type=2, norm="ortho")


def regularisation(q, q0, h, alpha, theta, proj=None) -> float:
    """1/2 |A (q - q0)|^2, or with a projector P: 1/2 (q - q0)^T P A^2 P (q - q0)."""
    d = q - q0
    if proj is not None:
        d = proj(d)
    a = prior_apply(d, h, alpha, theta)
    return 0.5 * float(np.sum(a * a))


def regularisation_grad(q, q0, h, alpha, theta, proj=None) -> np.ndarray:
    """A^2 (q - q0) (A symmetric), or P A^2 P (q - q0)."""
    d = q - q0
    if proj is not None:
        d = proj(d)
    g = prior_apply(prior_apply(d, h, alpha, theta), h, alpha, theta)
    return proj(g) if proj is not None else g


# --------------------------------------------------------------------------------------
# Newton-CG
# --------------------------------------------------------------------------------------
@dataclass
class NewtonCfg:
    alpha: float
    theta: float
    newton_iters: int = 5
    cg_max: int = 20
    full_hessian: bool = False     # False: Gauss-Newton misfit Hessian
    c1: float = 1e-4
    max_backtracks: int = 10
    eta_max: float = 0.5           # cap of the Eisenstat-Walker forcing term


def stable(p: W.Problem, q) -> bool:
    """q is a wave speed the leapfrog scheme can run: positive, and max q dt / h within
    the 3-D stability bound 1/sqrt(3)."""
    return bool(np.all(q > 0) and q.max() * p.dt / p.h <= 1.0 / np.sqrt(3.0))


def cost(p: W.Problem, q, d_obs, q0, cfg: NewtonCfg, proj=None) -> float:
    d, _, _ = W.forward(p, q)
    return W.misfit(d, d_obs) + regularisation(q, q0, p.h, cfg.alpha, cfg.theta, proj)


def newton_cg(p: W.Problem, q: np.ndarray, d_obs, q0, cfg: NewtonCfg, proj=None):
    """Inexact Newton-CG (see the module docstring); returns (q, history) with one entry
    (cost, |g|, cg iterations, step length) per Newton iteration (step 0: the line search
    found no acceptable step and the iteration stopped)."""
    q = np.array(q, dtype=np.float64)
    hist = []
    g0n = None
    for it in range(cfg.newton_iters):
        Jm, gm, _ = W.gradient(p, q, d_obs)
        g = gm + regularisation_grad(q, q0, p.h, cfg.alpha, cfg.theta, proj)
        J = Jm + regularisation(q, q0, p.h, cfg.alpha, cfg.theta, proj)
        gn = float(np.linalg.norm(g))
        g0n = gn if g0n is None else g0n
        eta = min(cfg.eta_max, np.sqrt(gn / g0n))
        _, states = W.forward_states(p, q)
        e_of = lambda n: states[n][0]

        def hess(v):
            hm = (W.hessvec_full(p, q, d_obs, v, e_of) if cfg.full_hessian
                  else W.hessvec_gn(p, q, v, e_of))
            return hm + regularisation_grad(v, np.zeros_like(v), p.h, cfg.alpha, cfg.theta, proj)

        # conjugate gradients on H x = -g from x = 0
        x = np.zeros_like(q)
        r = -g.copy()
        d = r.copy()
        rr = float(np.sum(r * r))
        k = 0
        for k in range(1, cfg.cg_max + 1):
            Hd = hess(d)
            dHd = float(np.sum(d * Hd))
            if dHd <= 0:          # negative curvature: keep the current iterate
                k -= 1
                break
            a = rr / dHd
            x = x + a * d
            r = r - a * Hd
            rr_new = float(np.sum(r * r))
            if np.sqrt(rr_new) <= eta * gn:
                break
            d = r + (rr_new / rr) * d
            rr = rr_new
        if not np.any(x):
            x = -g
        # Armijo backtracking
        slope = float(np.sum(g * x))
        step = 1.0
        accepted = False
        for _ in range(cfg.max_backtracks):
            qt = q + step * x
            if stable(p, qt) and cost(p, qt, d_obs, q0, cfg, proj) <= J + cfg.c1 * step * slope:
                accepted = True
                break
            step *= 0.5
        if not accepted:        # no sufficient decrease along x: stop where we are
            hist.append((J, gn, k, 0.0))
            break
        q = q + step * x
        hist.append((J, gn, k, step))
    return q, hist


# --------------------------------------------------------------------------------------
# DIAS
# --------------------------------------------------------------------------------------
def active_subspace(grads, r: int):
    """Leading r eigenpairs of C = (1/N) sum_i g_i g_i^T from the N x N Gram matrix
    M = G^T G / N of the sample gradients G = [g_1 ... g_N]: C's eigenvectors are
    G u_k / sqrt(N lambda_k) for M's eigenpairs (lambda_k, u_k).  Returns (lambda[:r],
    W1 [r][n] rows orthonormal)."""
    G = np.stack([np.ravel(g) for g in grads], axis=1)          # n x N
    N = G.shape[1]
    M = G.T @ G / N
    lam, U = np.linalg.eigh(M)
    lam, U = lam[::-1], U[:, ::-1]
    W1 = (G @ U[:, :r]) / np.sqrt(N * lam[:r])
    return lam[:r], W1.T


def projector(W1: np.ndarray, shape):
    """x -> P x = x - W1^T (W1 x): the projection onto the inactive subspace."""
    def proj(x):
        v = np.ravel(x)
        return (v - W1.T @ (W1 @ v)).reshape(shape)
    return proj


def dias_samples(p: W.Problem, q_map, d_obs, cfg: NewtonCfg, noise):
    """Misfit gradients at q_MAP + A^{-1} w_i for the white-noise fields w_i in noise."""
    out = []
    for w in noise:
        qi = q_map + prior_solve(w, p.h, cfg.alpha, cfg.theta)
        _, g, _ = W.gradient(p, qi, d_obs)
        out.append(g)
    return out
