"""FP64 oracle: staggered leapfrog acoustic solver, discrete adjoint, Gauss-Newton HVP.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference legs may import this module. It shares no code with the CUDA
path and is written to be read against the paper, not to be fast.

What it computes (Sec. 2, Eq. (1) with rho = 1 and m := c^2):
    dv/dt - grad(m e) = s,      de/dt - div v = 0,      e = 0 on the boundary,
discretised on a structured grid of nz x ny x nx nodes with spacing h:

* e and m live on nodes [k][j][i]; e is identically 0 on boundary nodes (the
  traction-free condition of Sec. 2).
* vx lives on x-faces (i+1/2, j, k), stored at index [k][j][i] for i = 0..nx-2;
  the last face i = nx-1 is unused and stays 0. vy, vz likewise.
* G f = forward differences onto faces; D v = backward differences onto interior
  nodes.  With e restricted to interior nodes, D = -G^T exactly.
* one leapfrog step, n -> n+1 (v^n lives at t_{n-1/2}, e^n at t_n = n dt):
      v^{n+1} = v^n + dt (G(m e^n) + s^n)
      e^{n+1} = e^n + dt D v^{n+1}
      d^{n+1} = B v^{n+1}       (velocity at the receivers, the map F = B A)
* misfit J = 1/2 sum_{n=1..nt} |d^n - d_obs^n|^2  (Eq. (3), noise covariance I,
  prior term excluded).

The adjoint is the reverse-mode derivative of exactly these operations, written with
explicit transposes G^T and D^T (not with the identity D = -G^T, so that the
adjoint-identity test checks the transposes). dJ/dc = 2 c (dJ/dm).

The incremental forward / incremental adjoint problems of Sec. 4 give the
Gauss-Newton Hessian-vector product H dc = J_F^T J_F dc, and with the second-order
terms (the first-order adjoint times the incremental strain, and its source in the
second-order adjoint) the full Newton Hessian-vector product.

The autoencoder variant (Sec. 3) replaces the stored forward strain e^n in the
adjoint and incremental problems by its decoded approximation; the solve functions accept an
``e_of`` callback that supplies e^n for step n, so the same code runs full storage
and compressed storage.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math
from typing import Callable, Optional, Sequence

import numpy as np


# --------------------------------------------------------------------------------------
# Problem description
# --------------------------------------------------------------------------------------
@dataclass
class Problem:
    """Grid, time stepping, source and receivers.  Arrays are [nz][ny][nx]."""

    shape: tuple            # (nz, ny, nx)
    h: float                # grid spacing [m]
    nt: int                 # number of time steps
    cfl: float = 0.5
    cmax: float = 3000.0    # dt = cfl h / cmax
    src: tuple = None       # source node (i, j, k); force on its z-face
    src_sigma: float = 0.0  # Gaussian smoothing of the source in space [m] (0: point)
    f0: float = 25.0        # Ricker peak frequency [Hz]
    t0: Optional[float] = None   # Ricker centre time, default 1/f0
    rec: np.ndarray = field(default=None)   # int [nrec][3] of (i, j, k)

    def __post_init__(self):
        nz, ny, nx = self.shape
        if self.src is None:
            self.src = (nx // 2, ny // 2, nz // 2)
        if self.t0 is None:
            self.t0 = 1.0 / self.f0
        if self.rec is None:
            self.rec = np.zeros((0, 3), dtype=np.int64)
        self.rec = np.asarray(self.rec, dtype=np.int64).reshape(-1, 3)

    @property
    def dt(self) -> float:
        return self.cfl * self.h / self.cmax

    @property
    def nrec(self) -> int:
        return self.rec.shape[0]


def ricker(t, f0: float, t0: float):
    """Ricker wavelet of Sec. 4.1: (1 - tau^2/sig^2) exp(-tau^2/(2 sig^2)), tau = t - t0.

    sig = 1/(sqrt(2) pi f0), which makes the spectrum peak at f0.
    """
    sig = 1.0 / (math.sqrt(2.0) * math.pi * f0)
    tau = np.asarray(t, dtype=np.float64) - t0
    return (1.0 - tau * tau / (sig * sig)) * np.exp(-tau * tau / (2.0 * sig * sig))


def default_wavelet(p: Problem) -> np.ndarray:
    """s^n for n = 0..nt-1: the z-force -R(n dt) (direction [0, 0, -1], Sec. 4.1)."""
    return -ricker(np.arange(p.nt) * p.dt, p.f0, p.t0)


# --------------------------------------------------------------------------------------
# Difference operators and their transposes
# --------------------------------------------------------------------------------------
def grad_op(f: np.ndarray, h: float):
    """G f: forward differences of a node field onto the x-, y- and z-faces."""
    gx = np.zeros_like(f)
    gy = np.zeros_like(f)
    gz = np.zeros_like(f)
    gx[:, :, :-1] = (f[:, :, 1:] - f[:, :, :-1]) / h
    gy[:, :-1, :] = (f[:, 1:, :] - f[:, :-1, :]) / h
    gz[:-1, :, :] = (f[1:, :, :] - f[:-1, :, :]) / h
    return gx, gy, gz


def div_op(vx: np.ndarray, vy: np.ndarray, vz: np.ndarray, h: float) -> np.ndarray:
    """D v: backward differences of the face fields onto interior nodes (0 elsewhere)."""
    out = np.zeros_like(vx)
    c = (slice(1, -1),) * 3
    out[c] = ((vx[1:-1, 1:-1, 1:-1] - vx[1:-1, 1:-1, :-2])
              + (vy[1:-1, 1:-1, 1:-1] - vy[1:-1, :-2, 1:-1])
              + (vz[1:-1, 1:-1, 1:-1] - vz[:-2, 1:-1, 1:-1])) / h
    return out


def interior(f: np.ndarray) -> np.ndarray:
    """Copy of f with boundary nodes set to 0 (the e = 0 boundary condition)."""
    out = np.zeros_like(f)
    out[1:-1, 1:-1, 1:-1] = f[1:-1, 1:-1, 1:-1]
    return out


def grad_op_T(lx: np.ndarray, ly: np.ndarray, lz: np.ndarray, h: float) -> np.ndarray:
    """G^T: each used face value (lf[i] for i <= n-2) goes +1/h to node i+1, -1/h to node i."""
    out = np.zeros_like(lx)
    out[:, :, 1:] += lx[:, :, :-1] / h
    out[:, :, :-1] -= lx[:, :, :-1] / h
    out[:, 1:, :] += ly[:, :-1, :] / h
    out[:, :-1, :] -= ly[:, :-1, :] / h
    out[1:, :, :] += lz[:-1, :, :] / h
    out[:-1, :, :] -= lz[:-1, :, :] / h
    return out


def div_op_T(mu: np.ndarray, h: float):
    """D^T: interior node value mu[i] goes +1/h to face i and -1/h to face i-1."""
    mi = interior(mu)
    ax = mi / h
    ay = mi / h
    az = mi / h
    ax[:, :, :-1] -= mi[:, :, 1:] / h
    ay[:, :-1, :] -= mi[:, 1:, :] / h
    az[:-1, :, :] -= mi[1:, :, :] / h
    return ax, ay, az


# --------------------------------------------------------------------------------------
# Forward solve
# --------------------------------------------------------------------------------------
def _sample(p: Problem, vx, vy, vz) -> np.ndarray:
    """B v: the three velocity components at each receiver node's faces, [nrec][3]."""
    i, j, k = p.rec[:, 0], p.rec[:, 1], p.rec[:, 2]
    return np.stack([vx[k, j, i], vy[k, j, i], vz[k, j, i]], axis=1)


def source_weights(p: Problem):
    """The source's spatial weights on the z-faces (Sec. 4.1's box problem smooths the
    source by a narrow Gaussian in space).  Returns (R, w): the faces (i + a, j + b,
    k + c + 1/2) for |a|, |b|, |c| <= R around the source face (i, j, k + 1/2) get
    w[c + R][b + R][a + R] proportional to exp(-r^2 / (2 sigma^2)), r the distance
    between the face centres, normalised to sum 1 (so that sigma -> 0 is the point
    source); R = ceil(3 sigma / h).  A point source is R = 0, w = [[[1]]]."""
    if p.src_sigma <= 0.0:
        return 0, np.ones((1, 1, 1))
    R = int(math.ceil(3.0 * p.src_sigma / p.h))
    o = np.arange(-R, R + 1) * p.h
    r2 = o[:, None, None] ** 2 + o[None, :, None] ** 2 + o[None, None, :] ** 2
    w = np.exp(-r2 / (2.0 * p.src_sigma ** 2))
    return R, w / w.sum()


def forward_step(p: Problem, m, e, vx, vy, vz, s_n: float):
    """One leapfrog step (see module docstring); returns the new (e, vx, vy, vz)."""
    dt, h = p.dt, p.h
    gx, gy, gz = grad_op(m * e, h)
    vx = vx + dt * gx
    vy = vy + dt * gy
    vz = vz + dt * gz
    i, j, k = p.src
    R, w = source_weights(p)
    vz[k - R:k + R + 1, j - R:j + R + 1, i - R:i + R + 1] += dt * s_n * w
    e = interior(e + dt * div_op(vx, vy, vz, h))
    return e, vx, vy, vz


def forward(p: Problem, c: np.ndarray, wavelet: Optional[np.ndarray] = None,
            state0=None, keep_states: bool = False, on_state: Optional[Callable] = None):
    """Forward solve.  Returns d [nt+1][nrec][3] (d[0] = B v^0) and the final state.

    keep_states: also return the list of (e^n, vx^n, vy^n, vz^n) for n = 0..nt-1.
    on_state(n, e, vx, vy, vz): called with every state n = 0..nt-1 (before step n).
    """
    m = c.astype(np.float64) ** 2
    if wavelet is None:
        wavelet = default_wavelet(p)
    if state0 is None:
        e = np.zeros(p.shape); vx = np.zeros(p.shape); vy = np.zeros(p.shape); vz = np.zeros(p.shape)
    else:
        e, vx, vy, vz = (np.array(a, dtype=np.float64) for a in state0)
    d = np.zeros((p.nt + 1, p.nrec, 3))
    d[0] = _sample(p, vx, vy, vz)
    states = [] if keep_states else None
    for n in range(p.nt):
        if keep_states:
            states.append((e, vx, vy, vz))
        if on_state is not None:
            on_state(n, e, vx, vy, vz)
        e, vx, vy, vz = forward_step(p, m, e, vx, vy, vz, wavelet[n])
        d[n + 1] = _sample(p, vx, vy, vz)
    return d, (e, vx, vy, vz), states


def misfit(d: np.ndarray, d_obs: np.ndarray) -> float:
    """J = 1/2 sum_{n>=1} |d^n - d_obs^n|^2."""
    r = d[1:] - d_obs[1:]
    return 0.5 * float(np.sum(r * r))


# --------------------------------------------------------------------------------------
# Adjoint solve (reverse mode of forward_step, steps taken in reverse order)
# --------------------------------------------------------------------------------------
def adjoint(p: Problem, c: np.ndarray, e_of: Callable[[int], np.ndarray],
            resid: np.ndarray, want_source_grad: bool = False):
    """Adjoint of the forward solve for a receiver residual r = resid[n], n = 1..nt.

    e_of(n) supplies the forward strain e^n (stored, recomputed or decoded).
    Returns dJ/dm as a node field (and dJ/ds^n if asked).

    Reverse of step n, with lam = adjoint of v^{n+1}, mu = adjoint of e^{n+1}:
        lam += B^T r^{n+1}               (record)
        lam += dt D^T mu                 (strain update)
        q    = G^T lam
        mbar += dt e^n q                 (dJ/dm from G(m e^n))
        mu   = interior(mu + dt m q)     (now the adjoint of e^n)
    lam then is the adjoint of v^n.
    """
    dt, h = p.dt, p.h
    m = c.astype(np.float64) ** 2
    lx = np.zeros(p.shape); ly = np.zeros(p.shape); lz = np.zeros(p.shape)
    mu = np.zeros(p.shape)
    mbar = np.zeros(p.shape)
    sgrad = np.zeros(p.nt)
    ri, rj, rk = p.rec[:, 0], p.rec[:, 1], p.rec[:, 2]
    si, sj, sk = p.src
    R, w_src = source_weights(p)
    for n in range(p.nt - 1, -1, -1):
        r = resid[n + 1]
        np.add.at(lx, (rk, rj, ri), r[:, 0])
        np.add.at(ly, (rk, rj, ri), r[:, 1])
        np.add.at(lz, (rk, rj, ri), r[:, 2])
        ax, ay, az = div_op_T(mu, h)
        lx = lx + dt * ax
        ly = ly + dt * ay
        lz = lz + dt * az
        q = grad_op_T(lx, ly, lz, h)
        mbar += dt * e_of(n) * q
        mu = interior(mu + dt * m * q)
        sgrad[n] = dt * float(np.sum(w_src * lz[sk - R:sk + R + 1, sj - R:sj + R + 1,
                                                 si - R:si + R + 1]))
    if want_source_grad:
        return mbar, sgrad
    return mbar


def gradient(p: Problem, c: np.ndarray, d_obs: np.ndarray, wavelet=None, e_of=None):
    """Full-storage gradient: returns (J, dJ/dc, d).  e_of overrides the stored e^n."""
    d, _, states = forward(p, c, wavelet, keep_states=True)
    J = misfit(d, d_obs)
    resid = d - d_obs
    if e_of is None:
        e_of = lambda n: states[n][0]
    mbar = adjoint(p, c, e_of, resid)
    return J, 2.0 * c * mbar, d


# --------------------------------------------------------------------------------------
# Incremental forward / Gauss-Newton Hessian-vector product (Sec. 4)
# --------------------------------------------------------------------------------------
def incremental_forward(p: Problem, c: np.ndarray, dc: np.ndarray,
                        e_of: Callable[[int], np.ndarray]) -> np.ndarray:
    """Linearised forward solve J_F dc: returns dd [nt+1][nrec][3].

    With dm = 2 c dc, differentiating forward_step gives
        dv^{n+1} = dv^n + dt G(m de^n + dm e^n)
        de^{n+1} = de^n + dt D dv^{n+1}
        dd^{n+1} = B dv^{n+1}
    which needs the forward strain e^n at every step (stored or decoded).
    """
    dt, h = p.dt, p.h
    m = c.astype(np.float64) ** 2
    dm = 2.0 * c * dc
    de = np.zeros(p.shape); dvx = np.zeros(p.shape); dvy = np.zeros(p.shape); dvz = np.zeros(p.shape)
    dd = np.zeros((p.nt + 1, p.nrec, 3))
    for n in range(p.nt):
        gx, gy, gz = grad_op(m * de + dm * e_of(n), h)
        dvx = dvx + dt * gx
        dvy = dvy + dt * gy
        dvz = dvz + dt * gz
        de = interior(de + dt * div_op(dvx, dvy, dvz, h))
        dd[n + 1] = _sample(p, dvx, dvy, dvz)
    return dd


def jacobian_transpose(p: Problem, c: np.ndarray, r: np.ndarray,
                       e_of: Callable[[int], np.ndarray]) -> np.ndarray:
    """J_F^T r = 2 c (dJ/dm) for a receiver-space vector r [nt+1][nrec][3]."""
    return 2.0 * c * adjoint(p, c, e_of, r)


def hessvec_gn(p: Problem, c: np.ndarray, dc: np.ndarray,
               e_of: Callable[[int], np.ndarray],
               e_adj_of: Optional[Callable[[int], np.ndarray]] = None) -> np.ndarray:
    """Gauss-Newton Hessian-vector product J_F^T J_F dc (incremental fwd + adjoint).
    e_adj_of (default e_of) is the forward strain history the incremental adjoint reads,
    for histories stored at a different precision for the adjoint-type sweeps."""
    dd = incremental_forward(p, c, dc, e_of)
    return jacobian_transpose(p, c, dd, e_adj_of if e_adj_of is not None else e_of)


def incremental_forward_states(p: Problem, c: np.ndarray, dc: np.ndarray,
                               e_of: Callable[[int], np.ndarray]):
    """The incremental forward solve of incremental_forward, also returning the
    incremental strain history de^n, n = 0..nt-1 (de^0 = 0)."""
    dt, h = p.dt, p.h
    m = c.astype(np.float64) ** 2
    dm = 2.0 * c * dc
    de = np.zeros(p.shape); dvx = np.zeros(p.shape); dvy = np.zeros(p.shape); dvz = np.zeros(p.shape)
    dd = np.zeros((p.nt + 1, p.nrec, 3))
    hist = []
    for n in range(p.nt):
        hist.append(de)
        gx, gy, gz = grad_op(m * de + dm * e_of(n), h)
        dvx = dvx + dt * gx
        dvy = dvy + dt * gy
        dvz = dvz + dt * gz
        de = interior(de + dt * div_op(dvx, dvy, dvz, h))
        dd[n + 1] = _sample(p, dvx, dvy, dvz)
    return dd, hist


def hessvec_full(p: Problem, c: np.ndarray, d_obs: np.ndarray, dc: np.ndarray,
                 e_of: Callable[[int], np.ndarray],
                 de_of: Optional[Callable[[int], np.ndarray]] = None) -> np.ndarray:
    """Full Newton Hessian-vector product H dc of J(c) = 1/2 |F(c) - d_obs|^2 (Sec. 4's
    incremental forward and incremental adjoint problems with the second-order terms).

    Differentiating the gradient dJ/dm = sum_n dt e^n q^n (q^n = G^T lam^{n+1}, see
    adjoint) in the direction dm gives
        H_m dm = sum_n dt (de^n q^n + e^n dq^n),
    de^n the incremental forward strain and dq^n = G^T dlam^{n+1} from the second-order
    adjoint: the adjoint recursion driven by the residual B dv (dv the incremental
    forward velocity) plus the derivative of its own m-dependence, a source dt dm q^n
    in the mu update:
        dlam += B^T (B dv^{n+1});  dlam += dt D^T dmu;  dq = G^T dlam;
        dmu = interior(dmu + dt m dq + dt dm q).
    In c (m = c^2, dm = 2 c dc): H dc = 2 c H_m(2 c dc) + 2 dc (dJ/dm).
    Only the terms in q distinguish it from the Gauss-Newton product; at zero residual
    q = 0 and the two coincide.

    e_of(n) supplies the forward strain e^n; de_of(n) the incremental strain used in the
    de^n q^n term (None: the exact one from this incremental forward solve); the
    residual comes from an exact forward solve."""
    dt, h = p.dt, p.h
    m = c.astype(np.float64) ** 2
    dm = 2.0 * c * dc
    d, _, _ = forward(p, c)
    r = d - d_obs
    dd, de_hist = incremental_forward_states(p, c, dc, e_of)
    if de_of is None:
        de_of = lambda n: de_hist[n]
    lx = np.zeros(p.shape); ly = np.zeros(p.shape); lz = np.zeros(p.shape); mu = np.zeros(p.shape)
    hx = np.zeros(p.shape); hy = np.zeros(p.shape); hz = np.zeros(p.shape); hmu = np.zeros(p.shape)
    gm = np.zeros(p.shape)      # dJ/dm
    Hm = np.zeros(p.shape)      # H_m dm
    ri, rj, rk = p.rec[:, 0], p.rec[:, 1], p.rec[:, 2]
    for n in range(p.nt - 1, -1, -1):
        # first-order adjoint (as in adjoint)
        np.add.at(lx, (rk, rj, ri), r[n + 1][:, 0])
        np.add.at(ly, (rk, rj, ri), r[n + 1][:, 1])
        np.add.at(lz, (rk, rj, ri), r[n + 1][:, 2])
        ax, ay, az = div_op_T(mu, h)
        lx = lx + dt * ax; ly = ly + dt * ay; lz = lz + dt * az
        q = grad_op_T(lx, ly, lz, h)
        # second-order adjoint
        np.add.at(hx, (rk, rj, ri), dd[n + 1][:, 0])
        np.add.at(hy, (rk, rj, ri), dd[n + 1][:, 1])
        np.add.at(hz, (rk, rj, ri), dd[n + 1][:, 2])
        bx, by, bz = div_op_T(hmu, h)
        hx = hx + dt * bx; hy = hy + dt * by; hz = hz + dt * bz
        hq = grad_op_T(hx, hy, hz, h)
        e_n = e_of(n)
        gm += dt * e_n * q
        Hm += dt * (de_of(n) * q + e_n * hq)
        hmu = interior(hmu + dt * m * hq + dt * dm * q)
        mu = interior(mu + dt * m * q)
    return 2.0 * c * Hm + 2.0 * dc * gm


def forward_states(p: Problem, c: np.ndarray, wavelet=None):
    """Run the forward solve and keep every state; returns (d, states)."""
    d, _, states = forward(p, c, wavelet, keep_states=True)
    return d, states


# --------------------------------------------------------------------------------------
# Energy (used by the conservation pin)
# --------------------------------------------------------------------------------------
def energy(m, e_n, v_n: Sequence[np.ndarray], v_np1: Sequence[np.ndarray]) -> float:
    """E^n = 1/2 sum m (e^n)^2 + 1/2 sum v^n . v^{n+1} (conserved by the scheme)."""
    s = 0.5 * float(np.sum(m * e_n * e_n))
    for a, b in zip(v_n, v_np1):
        s += 0.5 * float(np.sum(a * b))
    return s
