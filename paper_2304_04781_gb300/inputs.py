"""Seeded synthetic inputs for the wave-speed inverse problem.

This module holds no arithmetic of the method itself: it only draws the inputs that
both the CUDA path and the FP64 oracle are given (velocity models, perturbation
directions, receiver layouts, codec weight initialisation, random codec inputs).
Everything is generated on the host in FP64 from numpy's PCG64 generator
(``numpy.random.default_rng(seed)``), so the same seed gives the same array on any
machine.

Workload recipe (stand-in for the paper's box experiment of Sec. 4.1, whose meshes
and data are not available):

* wave speed c: a Gaussian random field with covariance exp(-r^2 / (2 l^2)),
  l = 80 m, made by FFT filtering of white noise, standardised to mean 0 / std 1 and
  mapped to 1500 + 1500 * Phi(z) m/s, i.e. into (1.5, 3.0) km/s;
* "true" model for synthetic observations: c * (1 + 0.05 * Gaussian bump);
* receivers: a regular grid on the top face (node plane k = 1), which records the
  velocity (Sec. 2, the parameter-to-observable map F = B A);
* source: a point force on the z-face of the centre node (Sec. 4.1 uses a Ricker
  wavelet in time with direction [0, 0, -1]);
* prior samples (MAP / DIAS): white noise w ~ N(0, I) per node, which the prior's
  elliptic operator maps to a sample A^{-1} w.
"""
from __future__ import annotations

import numpy as np
from scipy.special import ndtr

__all__ = [
    "gaussian_random_field",
    "velocity_model",
    "bump_model",
    "direction",
    "receiver_grid",
    "source_grid",
    "codec_init",
    "random_latents",
    "smooth_state",
    "white_noise",
    "orthonormal_rows",
]


def gaussian_random_field(shape, h: float, corr_len: float, seed: int) -> np.ndarray:
    """Standardised (mean 0, std 1) stationary Gaussian field on a [nz][ny][nx] grid.

    Covariance exp(-r^2/(2 corr_len^2)); its spectral density is proportional to
    exp(-k^2 corr_len^2 / 2), so white noise is filtered by exp(-k^2 corr_len^2 / 4).
    The FFT makes the field periodic, which is harmless for a synthetic input.
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape)
    nz, ny, nx = shape
    kz = 2.0 * np.pi * np.fft.fftfreq(nz, d=h)[:, None, None]
    ky = 2.0 * np.pi * np.fft.fftfreq(ny, d=h)[None, :, None]
    kx = 2.0 * np.pi * np.fft.rfftfreq(nx, d=h)[None, None, :]
    filt = np.exp(-(kz * kz + ky * ky + kx * kx) * corr_len * corr_len / 4.0)
    z = np.fft.irfftn(np.fft.rfftn(w) * filt, s=shape, axes=(0, 1, 2))
    z -= z.mean()
    sd = z.std()
    if sd > 0:
        z /= sd
    return z


def velocity_model(shape, h: float = 10.0, seed: int = 0, corr_len: float = 80.0,
                   cmin: float = 1500.0, cmax: float = 3000.0) -> np.ndarray:
    """Wave speed c(x) in m/s: cmin + (cmax - cmin) * Phi(GRF), float64 [nz][ny][nx]."""
    z = gaussian_random_field(shape, h, corr_len, seed)
    return cmin + (cmax - cmin) * ndtr(z)


def bump_model(c: np.ndarray, h: float = 10.0, amp: float = 0.05) -> np.ndarray:
    """c * (1 + amp * exp(-|x - x_b|^2 / (2 s^2))), x_b = (N/2, N/2, N/4) h, s = N h / 8.

    The bump sits between the centre source and the top-face receivers; N is the
    z extent.
    """
    nz, ny, nx = c.shape
    zc, yc, xc = nz / 4.0, ny / 2.0, nx / 2.0
    s = nz / 8.0
    k = np.arange(nz)[:, None, None]
    j = np.arange(ny)[None, :, None]
    i = np.arange(nx)[None, None, :]
    r2 = ((k - zc) ** 2 + (j - yc) ** 2 + (i - xc) ** 2) * h * h
    return c * (1.0 + amp * np.exp(-r2 / (2.0 * (s * h) ** 2)))


def direction(shape, h: float = 10.0, seed: int = 10, corr_len: float = 80.0) -> np.ndarray:
    """A smooth random perturbation direction dc (GRF, scaled to max |dc| = 1)."""
    z = gaussian_random_field(shape, h, corr_len, seed)
    return z / np.abs(z).max()


def receiver_grid(nx: int, ny: int, nrec: int) -> np.ndarray:
    """Receiver nodes (i, j, k=1) on a regular n_x x n_y grid over the top face.

    16 -> 4x4, 64 -> 8x8, 128 -> 16x8, 256 -> 16x16; other counts use the most
    square factorisation. Node i = floor((p + 1/2) nx / n_x + 1/2).
    Returns int32 [nrec][3] holding (i, j, k).
    """
    table = {16: (4, 4), 64: (8, 8), 128: (16, 8), 256: (16, 16)}
    if nrec in table:
        rx, ry = table[nrec]
    else:
        ry = int(np.floor(np.sqrt(nrec)))
        while nrec % ry:
            ry -= 1
        rx = nrec // ry
    out = np.zeros((rx * ry, 3), dtype=np.int32)
    r = 0
    for q in range(ry):
        for p in range(rx):
            i = int(np.floor((p + 0.5) * nx / rx + 0.5))
            j = int(np.floor((q + 0.5) * ny / ry + 0.5))
            out[r] = (min(max(i, 1), nx - 2), min(max(j, 1), ny - 2), 1)
            r += 1
    return out


def source_grid(nx: int, ny: int, nz: int, nshots: int):
    """Source nodes (i, j, k) of nshots shots: a regular grid over the horizontal plane
    at mid-depth k = nz // 2 (one shot: the centre node).  Returns a list of tuples."""
    ry = int(np.floor(np.sqrt(nshots)))
    while nshots % ry:
        ry -= 1
    rx = nshots // ry
    out = []
    for q in range(ry):
        for p in range(rx):
            i = int(np.floor((p + 0.5) * nx / rx))
            j = int(np.floor((q + 0.5) * ny / ry))
            out.append((min(max(i, 1), nx - 2), min(max(j, 1), ny - 2), nz // 2))
    return out


def codec_init(seed: int = 0, n_in: int = 2048, n_hid: int = 512, n_lat: int = 64) -> dict:
    """Glorot-uniform weights (zero biases) for the 4-layer codec, float32.

    Encoder: W1 [n_in, n_hid], b1, W2 [n_hid, n_lat], b2.
    Decoder: W3 [n_lat, n_hid], b3, W4 [n_hid, n_in], b4.  Layers act as y W + b.
    """
    rng = np.random.default_rng(seed)

    def glorot(fan_in, fan_out):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-a, a, size=(fan_in, fan_out)).astype(np.float32)

    return {
        "W1": glorot(n_in, n_hid), "b1": np.zeros(n_hid, np.float32),
        "W2": glorot(n_hid, n_lat), "b2": np.zeros(n_lat, np.float32),
        "W3": glorot(n_lat, n_hid), "b3": np.zeros(n_hid, np.float32),
        "W4": glorot(n_hid, n_in), "b4": np.zeros(n_in, np.float32),
    }


def random_latents(nblocks: int, n_lat: int, seed: int) -> np.ndarray:
    """Latent codes drawn N(0, 1), float32 [nblocks][n_lat]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nblocks, n_lat)).astype(np.float32)


def smooth_state(shape, h: float = 10.0, seed: int = 0, corr_len: float = 40.0) -> np.ndarray:
    """Four smooth random fields (e, vx, vy, vz), float64 [4][nz][ny][nx].

    Used as codec inputs and as initial conditions; each field gets its own scale
    (1, 2e-3, 5e-3, 1e-2) so the per-field normalisation is exercised.
    """
    scales = (1.0, 2e-3, 5e-3, 1e-2)
    out = np.empty((4,) + tuple(shape))
    for f in range(4):
        out[f] = scales[f] * gaussian_random_field(shape, h, corr_len, seed * 7 + f)
    return out


def white_noise(n: int, shape, seed: int) -> np.ndarray:
    """n white-noise fields N(0, 1), float32 [n][nz][ny][nx]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n,) + tuple(shape)).astype(np.float32)


def orthonormal_rows(r: int, n: int, seed: int) -> np.ndarray:
    """r orthonormal rows of length n (a random subspace), float64 [r][n]."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return np.ascontiguousarray(q.T)
