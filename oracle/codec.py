"""FP64 oracle for the per-block autoencoder codec and its training step.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference legs may import this module; it shares no code with the CUDA
path.

Compression in space (Sec. 3.1): the state of every 8x8x8-node block -- the four
fields e, vx, vy, vz -- is flattened into one vector of 2048 values.  The order
inside the vector is free as long as training and use agree (Sec. 3.1); the order
used here (and by the CUDA path, as a layout definition) is

    k = z*256 + f*64 + y*8 + x      (x, y, z the node offsets inside the block,
                                     f = 0:e, 1:vx, 2:vy, 3:vz)

Block b = (bz*NBy + by)*NBx + bx.  Normalisation (Sec. 3.3: every vector is scaled to
O(1) before encoding and its scale is kept at higher precision): each field of each
block is divided by s_{b,f} = 2^e, the power of two with max_x |f| in [s/2, s), so the
normalised values lie in (-1, 1) and scaling by s is exact in any binary format
(e >= -100, so that 1/s is finite in FP32).  A block-field that is identically zero has
s = 0 and is fed (and decoded) as 0.

Dense layers act as sigma(y W + b) (Sec. 3.3, Eq. (5)).  Shapes:
    encoder 2048 -> 512 (GELU) -> n_lat (linear),
    decoder n_lat -> 512 (GELU) -> 2048 (linear).
GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2.

Two modes.  ``emulate=False``: FP64 everywhere (exact math).  ``emulate=True``:
round exactly where the GPU rounds -- BF16 encoder inputs and weights, BF16 hidden
activations, FP16 latent, FP16 first decoder layer (latent and W3), BF16 second
decoder layer -- with FP64 accumulation, so the two differ only by accumulation
order.  Rounding is round-to-nearest-even, computed from the FP64 value directly.

Training (Sec. 3.3, Table 2): mean-squared reconstruction error on normalised
vectors, LAMB (You et al. 2019) per parameter tensor, FP16-rounded latent with a
straight-through derivative.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

BLK = 8
NFIELD = 4
NIN = BLK * BLK * BLK * NFIELD   # 2048


# --------------------------------------------------------------------------------------
# Round-to-nearest-even to narrow floating-point formats, from FP64
# --------------------------------------------------------------------------------------
def _round_mantissa(x, mant_bits: int, min_exp: int):
    """Round to a binary format with `mant_bits` fraction bits, minimum normal exponent
    `min_exp` (subnormals keep the spacing 2^(min_exp - mant_bits)); RNE via np.rint."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    with np.errstate(divide="ignore"):
        ex = np.floor(np.log2(np.where(ax > 0, ax, 1.0)))
    ex = np.maximum(ex, min_exp)
    q = np.exp2(ex - mant_bits)
    return np.rint(x / q) * q


def round_bf16(x):
    """RNE to bfloat16 (8 exponent bits, 7 fraction bits)."""
    return _round_mantissa(x, 7, -126)


def round_fp16(x):
    """RNE to IEEE binary16 (5 exponent bits, 10 fraction bits); overflow -> inf."""
    r = _round_mantissa(x, 10, -14)
    return np.where(np.abs(r) > 65504.0, np.copysign(np.inf, r), r)


def round_fp32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_prime(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def elu(x):
    """ELU of Sec. 3.3: e^y - 1 for y < 0, y otherwise."""
    x = np.asarray(x, dtype=np.float64)
    return np.where(x < 0, np.expm1(np.minimum(x, 0.0)), x)


def elu_prime(x):
    x = np.asarray(x, dtype=np.float64)
    return np.where(x < 0, np.exp(np.minimum(x, 0.0)), 1.0)


ACTIVATIONS = {"gelu": (gelu, gelu_prime), "elu": (elu, elu_prime),
               "linear": (lambda a: a, lambda a: np.ones_like(a))}


# --------------------------------------------------------------------------------------
# Block packing (Sec. 3.1 "compression data structure")
# --------------------------------------------------------------------------------------
def pack_blocks(fields) -> np.ndarray:
    """(e, vx, vy, vz) [nz][ny][nx] -> X [nblocks][2048] in the k-order above."""
    nz, ny, nx = fields[0].shape
    NBz, NBy, NBx = nz // BLK, ny // BLK, nx // BLK
    X = np.empty((NBz * NBy * NBx, NIN))
    for f in range(NFIELD):
        a = np.asarray(fields[f], dtype=np.float64).reshape(NBz, BLK, NBy, BLK, NBx, BLK)
        # -> [bz, by, bx, z, y, x]
        a = a.transpose(0, 2, 4, 1, 3, 5).reshape(NBz * NBy * NBx, BLK, BLK * BLK)
        for z in range(BLK):
            X[:, z * 256 + f * 64: z * 256 + f * 64 + 64] = a[:, z, :]
    return X


def unpack_field(X: np.ndarray, shape, f: int) -> np.ndarray:
    """Inverse of pack_blocks for one field f, from X [nblocks][2048]."""
    nz, ny, nx = shape
    NBz, NBy, NBx = nz // BLK, ny // BLK, nx // BLK
    a = np.empty((NBz * NBy * NBx, BLK, BLK * BLK))
    for z in range(BLK):
        a[:, z, :] = X[:, z * 256 + f * 64: z * 256 + f * 64 + 64]
    a = a.reshape(NBz, NBy, NBx, BLK, BLK, BLK).transpose(0, 3, 1, 4, 2, 5)
    return a.reshape(nz, ny, nx)


def field_columns(f: int) -> np.ndarray:
    """Indices k of field f inside the 2048-vector, in (z, y, x) order."""
    return np.concatenate([np.arange(z * 256 + f * 64, z * 256 + f * 64 + 64) for z in range(BLK)])


EXP_MIN = -100   # smallest scale exponent: 2^-e must stay finite in FP32


def block_scales(fields) -> np.ndarray:
    """s[b][f] = 2^max(e, EXP_MIN) with max_{x in block b} |f(x)| = m 2^e, m in [0.5, 1)
    (0 for a zero block-field); returns [nblocks][4].  The clamp only affects blocks
    whose largest magnitude is below 2^-101 (ahead of the numerical wavefront), which are
    then normalised to values far below 1 instead of overflowing the scale."""
    X = np.abs(pack_blocks(fields))
    s = np.zeros((X.shape[0], NFIELD))
    for f in range(NFIELD):
        mx = X[:, field_columns(f)].max(axis=1)
        _, e = np.frexp(mx)
        s[:, f] = np.where(mx > 0, np.ldexp(1.0, np.maximum(e, EXP_MIN)), 0.0)
    return s


def normalise(X: np.ndarray, s) -> np.ndarray:
    """y = x / s_{b,f}; s is [nblocks][4] (per block) or [4] (one scale per field);
    y = 0 where s = 0."""
    s = np.asarray(s, dtype=np.float64)
    if s.ndim == 1:
        s = np.broadcast_to(s, (X.shape[0], NFIELD))
    sv = np.empty_like(X)
    for f in range(NFIELD):
        sv[:, field_columns(f)] = s[:, f:f + 1]
    safe = np.where(sv > 0, sv, 1.0)
    return np.where(sv > 0, X / safe, 0.0)


# --------------------------------------------------------------------------------------
# Encoder / decoder
# --------------------------------------------------------------------------------------
def encode(W: dict, Y: np.ndarray, emulate: bool = False, act: str = "gelu") -> np.ndarray:
    """Normalised vectors Y [B][2048] -> latents [B][n_lat] (FP16-rounded if emulate);
    act: the hidden layer's activation (GELU, or the paper's ELU)."""
    sig = ACTIVATIONS[act][0]
    W1, b1, W2, b2 = (np.asarray(W[k], np.float64) for k in ("W1", "b1", "W2", "b2"))
    if emulate:
        Y = round_bf16(Y)
        W1, W2 = round_bf16(W1), round_bf16(W2)
        b1, b2 = round_fp32(b1), round_fp32(b2)
    h = sig(Y @ W1 + b1)
    if emulate:
        h = round_bf16(h)
    z = h @ W2 + b2
    if emulate:
        z = round_fp16(z)
    return z


def decode(W: dict, Z: np.ndarray, emulate: bool = False, cols=None,
           act: str = "gelu") -> np.ndarray:
    """Latents Z [B][n_lat] -> normalised reconstruction [B][2048] (or [B][len(cols)])."""
    sig = ACTIVATIONS[act][0]
    W3, b3, W4, b4 = (np.asarray(W[k], np.float64) for k in ("W3", "b3", "W4", "b4"))
    if cols is not None:
        W4, b4 = W4[:, cols], b4[cols]
    if emulate:
        Z = round_fp16(Z)
        W3 = round_fp16(W3)
        W4 = round_bf16(W4)
        b3, b4 = round_fp32(b3), round_fp32(b4)
    h = sig(Z @ W3 + b3)
    if emulate:
        h = round_bf16(h)
    return h @ W4 + b4


def roundtrip_e(W: dict, state, emulate: bool = False) -> np.ndarray:
    """Encode one state (per-block scales) and decode its strain field: e-hat, in physical
    units, set to 0 on boundary nodes, where the boundary condition of Sec. 2 fixes e = 0
    exactly (the stored forward strain is 0 there too)."""
    shape = state[0].shape
    s = block_scales(state)
    Y = normalise(pack_blocks(state), s)
    Z = encode(W, Y, emulate)
    cols = field_columns(0)
    E = decode(W, Z, emulate, cols=cols) * s[:, 0:1]
    Xe = np.zeros((E.shape[0], NIN))
    Xe[:, cols] = E
    e = unpack_field(Xe, shape, 0)
    inner = np.zeros_like(e)
    inner[1:-1, 1:-1, 1:-1] = e[1:-1, 1:-1, 1:-1]
    return inner


def compressed_e_history(W: dict, states, emulate: bool = False):
    """Decoded strain history e-hat^n, n = 0..nt-1."""
    return [roundtrip_e(W, st, emulate) for st in states]


# --------------------------------------------------------------------------------------
# Training step: MSE loss, backprop, LAMB
# --------------------------------------------------------------------------------------
PARAMS = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")


def loss_and_grad(W: dict, Y: np.ndarray, emulate: bool = False, act: str = "gelu",
                  weights: np.ndarray = None):
    """Mean squared error (1/(B*2048)) sum (decode(encode(Y)) - Y)^2 and its gradient.

    weights [B][4] (optional): every squared error of vector v in field f's columns is
    multiplied by weights[v][f] (None: all ones, the plain mean squared error of Table 2).

    The FP16 latent rounding (emulate) is treated as identity in the derivative
    (straight-through).  With emulate, GEMM operands are rounded as on the GPU:
    BF16 for all products except the decoder's first-layer forward product (FP16).
    act="linear" drops both activations (the linear autoencoder of Sec. 1, which
    learns the PCA subspace); act="elu" takes the paper's ELU (Sec. 3.3).
    """
    sig, sig_p = ACTIVATIONS[act]
    P = {k: np.asarray(W[k], np.float64) for k in PARAMS}
    rb = round_bf16 if emulate else (lambda a: a)
    rh = round_fp16 if emulate else (lambda a: a)
    B = Y.shape[0]
    Yin = rb(Y)
    a1 = Yin @ rb(P["W1"]) + P["b1"]
    h1 = rb(sig(a1))
    a2 = h1 @ rb(P["W2"]) + P["b2"]
    z = rh(a2)
    a3 = z @ rh(P["W3"]) + P["b3"]
    h3 = rb(sig(a3))
    a4 = h3 @ rb(P["W4"]) + P["b4"]
    diff = a4 - Y
    if weights is None:
        wfull = np.ones_like(diff)
    else:
        fcol = (np.arange(Y.shape[1]) >> 6) & 3          # field of each column
        wfull = np.asarray(weights, np.float64)[:, fcol]
    loss = float(np.mean(wfull * diff * diff))
    g = {}
    d4 = 2.0 * wfull * diff / diff.size
    g["W4"] = h3.T @ rb(d4)
    g["b4"] = d4.sum(0)
    dh3 = rb(d4) @ rb(P["W4"]).T
    d3 = dh3 * sig_p(a3)
    g["W3"] = rb(z).T @ rb(d3)
    g["b3"] = d3.sum(0)
    dz = rb(d3) @ rb(P["W3"]).T
    d2 = dz
    g["W2"] = h1.T @ rb(d2)
    g["b2"] = d2.sum(0)
    dh1 = rb(d2) @ rb(P["W2"]).T
    d1 = dh1 * sig_p(a1)
    g["W1"] = Yin.T @ rb(d1)
    g["b1"] = d1.sum(0)
    return loss, g


class Lamb:
    """LAMB optimiser (You et al. 2019), one trust ratio per parameter tensor.

    m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;  mh = m/(1-b1^t);  vh = v/(1-b2^t);
    u = mh / (sqrt(vh) + eps) + wd w;  r = |w| / |u| (1 if either norm is 0);
    w <- w - lr r u.
    """

    def __init__(self, W: dict, beta1=0.9, beta2=0.999, eps=1e-6, wd=0.0):
        self.b1, self.b2, self.eps, self.wd = beta1, beta2, eps, wd
        self.t = 0
        self.m = {k: np.zeros_like(np.asarray(W[k], np.float64)) for k in W}
        self.v = {k: np.zeros_like(np.asarray(W[k], np.float64)) for k in W}

    def step(self, W: dict, g: dict, lr: float) -> dict:
        self.t += 1
        out = {}
        for k in W:
            w = np.asarray(W[k], np.float64)
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * g[k]
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * g[k] * g[k]
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            u = mh / (np.sqrt(vh) + self.eps) + self.wd * w
            wn, un = float(np.linalg.norm(w)), float(np.linalg.norm(u))
            r = wn / un if (wn > 0 and un > 0) else 1.0
            out[k] = w - lr * r * u
        return out


def lr_schedule(epoch: int, lr0: float = 1e-3, halve_every: int = 5) -> float:
    """Table 2: lr = lr0, halved every 5 epochs."""
    return lr0 * 0.5 ** (epoch // halve_every)
