"""FP64 oracle for compression in time: the strain of a small node block over 16 steps.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference legs may import this module; it shares no code with the CUDA
path.

Sec. 3.2 (compression on non-uniform meshes) treats each element as an independent
state and forms the autoencoder's input from that element's nodes over consecutive
time steps (64 nodes x 16 steps x 4 Runge-Kutta stages = 4096 values there).  On the
structured leapfrog grid the same construction reads (readings R24-R26):

* the element is a block of 2 (z) x 8 (y) x 8 (x) nodes; the time window is 16
  consecutive states e^n, n = 16*tb .. 16*tb + 15 (one leapfrog state per step, no
  stages).  Only the strain is stored: it is the only forward quantity the adjoint,
  incremental forward and incremental adjoint problems read (m enters only through
  G(m e)).  That gives 2 * 8 * 8 * 16 = 2048 values per vector, the input size of the
  space codec;
* order inside the vector: k = t*128 + z*64 + y*8 + x (t the step inside the window;
  z, y, x the node offsets inside the block); vector v = (bz*NBy + by)*NBx + bx with
  NBz = nz/2, NBy = ny/8, NBx = nx/8 (a layout definition shared with the GPU);
* states beyond the last one solved (n >= nt in the last, partial window) are 0;
* normalisation (Sec. 3.3: every vector scaled to O(1), scale kept at higher
  precision): the whole vector is divided by s_v = 2^max(e, -100), where its largest
  magnitude is m 2^e with m in [1/2, 1) (0 for a zero vector, which is fed as 0).

The autoencoder layers are the dense layers sigma(y W + b) of Eq. (5), encoded and
decoded by ``codec.encode`` / ``codec.decode`` (shape-generic).  ``pca_codec`` builds
the weights of the optimal rank-k linear code of a data set (Sec. 1: a linear
autoencoder learns the PCA subspace) inside a GELU network: with
GELU(a) - GELU(-a) = a, a hidden layer of 2k units carrying +a and -a passes k linear
components through the activation exactly.
"""
from __future__ import annotations

import numpy as np

from . import codec as C

TSTEPS = 16
BZ, BY, BX = 2, 8, 8
NODES = BZ * BY * BX          # 128
NIN = TSTEPS * NODES          # 2048
EXP_MIN = C.EXP_MIN


def grid_ok(shape) -> bool:
    nz, ny, nx = shape
    return nz % BZ == 0 and ny % BY == 0 and nx % BX == 0


def nvectors(shape) -> int:
    nz, ny, nx = shape
    return (nz // BZ) * (ny // BY) * (nx // BX)


def n_windows(nt: int) -> int:
    """Number of 16-step windows covering the states e^0 .. e^{nt-1}."""
    return (nt + TSTEPS - 1) // TSTEPS


# --------------------------------------------------------------------------------------
# Packing
# --------------------------------------------------------------------------------------
def pack(e_steps, shape) -> np.ndarray:
    """Strain fields of one window (up to 16 arrays [nz][ny][nx]; missing steps are 0)
    -> X [nvec][2048] in the order k = t*128 + z*64 + y*8 + x."""
    nz, ny, nx = shape
    NBz, NBy, NBx = nz // BZ, ny // BY, nx // BX
    X = np.zeros((NBz * NBy * NBx, NIN))
    for t, e in enumerate(e_steps):
        if t >= TSTEPS:
            raise ValueError("a window holds 16 steps")
        a = np.asarray(e, dtype=np.float64).reshape(NBz, BZ, NBy, BY, NBx, BX)
        a = a.transpose(0, 2, 4, 1, 3, 5).reshape(NBz * NBy * NBx, NODES)   # [v][z][y][x]
        X[:, t * NODES:(t + 1) * NODES] = a
    return X


def unpack(X: np.ndarray, shape) -> np.ndarray:
    """Inverse of pack: X [nvec][2048] -> [16][nz][ny][nx]."""
    nz, ny, nx = shape
    NBz, NBy, NBx = nz // BZ, ny // BY, nx // BX
    out = np.empty((TSTEPS, nz, ny, nx))
    for t in range(TSTEPS):
        a = X[:, t * NODES:(t + 1) * NODES].reshape(NBz, NBy, NBx, BZ, BY, BX)
        out[t] = a.transpose(0, 3, 1, 4, 2, 5).reshape(nz, ny, nx)
    return out


def vector_scales(X: np.ndarray) -> np.ndarray:
    """s_v = 2^max(e, -100) with max_k |X[v][k]| = m 2^e, m in [1/2, 1); 0 for a zero
    vector."""
    mx = np.abs(X).max(axis=1)
    _, e = np.frexp(mx)
    return np.where(mx > 0, np.ldexp(1.0, np.maximum(e, EXP_MIN)), 0.0)


def normalise(X: np.ndarray, s: np.ndarray) -> np.ndarray:
    """y = x / s_v (exact: s_v is a power of two); 0 where s_v = 0."""
    s = np.asarray(s, dtype=np.float64)[:, None]
    return np.where(s > 0, X / np.where(s > 0, s, 1.0), 0.0)


def encoder_inputs(X: np.ndarray, s: np.ndarray, emulate: bool = False) -> np.ndarray:
    """The encoder's input vectors.  Exact mode: x / s_v.  Emulated mode: as on the GPU,
    each state is stored in BF16 when it is written, before the window's scale is known,
    and divided by the power of two afterwards (exact), i.e. bf16(x) / s_v; this equals
    bf16(x / s_v) except for values below BF16's normal range (|x| < 2^-126)."""
    return normalise(C.round_bf16(X) if emulate else X, s)


BETA = 1e-7    # the paper's lower bound of the min-max range (Sec. 3.3)


def minmax_scales(X: np.ndarray, beta: float = BETA):
    """The paper's per-vector normalisation (Sec. 3.3): offset min(y_true) and range
    r = max(max(y_true) - min(y_true), beta), both kept in FP64."""
    mn = X.min(axis=1)
    r = np.maximum(X.max(axis=1) - mn, beta)
    return mn, r


def minmax_normalise(X: np.ndarray, mn: np.ndarray, r: np.ndarray) -> np.ndarray:
    """y = (y_true - min) / r, in [0, 1]."""
    return (X - mn[:, None]) / r[:, None]


def window_vectors(e_hist, shape, tb: int):
    """Raw vectors of window tb from the strain history e_hist[n], n = 0..nt-1."""
    nt = len(e_hist)
    steps = [e_hist[n] for n in range(TSTEPS * tb, min(TSTEPS * (tb + 1), nt))]
    return pack(steps, shape)


# --------------------------------------------------------------------------------------
# Compressed history
# --------------------------------------------------------------------------------------
def interior(f: np.ndarray) -> np.ndarray:
    out = np.zeros_like(f)
    out[1:-1, 1:-1, 1:-1] = f[1:-1, 1:-1, 1:-1]
    return out


def roundtrip_window(W: dict, e_hist, shape, tb: int, emulate: bool = False,
                     norm: str = "pow2", act: str = "gelu", beta: float = BETA) -> np.ndarray:
    """Encode and decode window tb: the decoded strain [16][nz][ny][nx] in physical
    units, 0 on boundary nodes (the boundary condition of Sec. 2 fixes e = 0 there; the
    stored forward strain is 0 there too).

    norm="pow2": each vector divided by its power-of-two scale s_v, decoded values
    times s_v.  norm="minmax": the paper's min-max normalisation (Sec. 3.3), inputs
    (bf16(x) - min) / r in emulated mode (the state is stored in BF16 when written, the
    FP32 normalisation follows once the window is complete, one more rounding to BF16),
    decoded values y r + min in FP64.  act: GELU or the paper's ELU."""
    X = window_vectors(e_hist, shape, tb)
    if norm == "minmax":
        Xs = C.round_bf16(X) if emulate else X
        mn, r = minmax_scales(Xs, beta)
        Y = minmax_normalise(Xs, mn, r)
        if emulate:
            Y = C.round_bf16(C.round_fp32(Y))
        Z = C.encode(W, Y, emulate, act)
        Xh = C.decode(W, Z, emulate, act=act) * r[:, None] + mn[:, None]
    else:
        s = vector_scales(X)
        Z = C.encode(W, encoder_inputs(X, s, emulate), emulate, act)
        Xh = C.decode(W, Z, emulate, act=act) * s[:, None]
    E = unpack(Xh, shape)
    return np.stack([interior(E[t]) for t in range(TSTEPS)])


def compressed_e_history(W: dict, e_hist, emulate: bool = False, norm: str = "pow2",
                         act: str = "gelu", beta: float = BETA):
    """Decoded strain history e-hat^n, n = 0..nt-1 (window by window).  The initial state
    e^0 is the zero initial condition of Eq. (2): it is known exactly and is not taken
    from the codec (window 0's scale is set by its later states, so decoding would turn
    the exact zero into small nonzero values)."""
    nt = len(e_hist)
    shape = np.asarray(e_hist[0]).shape
    out = []
    for tb in range(n_windows(nt)):
        E = roundtrip_window(W, e_hist, shape, tb, emulate, norm, act, beta)
        for t in range(TSTEPS):
            n = TSTEPS * tb + t
            if n < nt:
                out.append(np.zeros(shape) if n == 0 else E[t])
    return out


def bf16_history(e_hat):
    """A decoded strain history as the solves that read it (the gradient's adjoint, the
    Gauss-Newton and full-Newton HVPs' incremental forward and adjoints) see it (reading
    R34): the decoder's FP32 output rounded to BF16, round to nearest even."""
    return [C.round_bf16(C.round_fp32(e)) for e in e_hat]


# --------------------------------------------------------------------------------------
# Optimal linear code inside a GELU network
# --------------------------------------------------------------------------------------
def pca_codec(Y: np.ndarray, k: int, weights=None) -> dict:
    """Weights of a 2048 -> 2k (GELU) -> k -> 2k (GELU) -> 2048 autoencoder that
    computes the best rank-k affine code of the rows of Y in the weighted least-squares
    sense (Eckart-Young): with the weighted mean mu and the k leading eigenvectors V of
    the weighted scatter matrix sum_v w_v (y_v - mu)(y_v - mu)^T,

        encoder  a = y [V, -V] + [-mu V, mu V],  z = GELU(a) [I; -I]       = (y - mu) V
        decoder  a' = z [I, -I],                 y^ = GELU(a') [V^T; -V^T] + mu
                                                                          = z V^T + mu

    using GELU(a) - GELU(-a) = a.  weights: one per row (None: all ones)."""
    Y = np.asarray(Y, dtype=np.float64)
    w = np.ones(Y.shape[0]) if weights is None else np.asarray(weights, dtype=np.float64)
    mu = (w[:, None] * Y).sum(0) / w.sum()
    Yc = Y - mu
    G = (Yc * w[:, None]).T @ Yc
    _, V = np.linalg.eigh(G)
    V = V[:, ::-1][:, :k]                      # leading eigenvectors first
    I = np.eye(k)
    return {
        "W1": np.concatenate([V, -V], axis=1), "b1": np.concatenate([-mu @ V, mu @ V]),
        "W2": np.concatenate([I, -I], axis=0), "b2": np.zeros(k),
        "W3": np.concatenate([I, -I], axis=1), "b3": np.zeros(2 * k),
        "W4": np.concatenate([V.T, -V.T], axis=0), "b4": mu,
    }
