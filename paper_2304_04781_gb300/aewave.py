"""Python binding of the aewave C-ABI library (include/aewave.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels.  PyTorch supplies device memory (tensors' data pointers) and the current
CUDA stream.  There is no CPU fallback: if the library cannot be loaded or built,
every call raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_float, c_int, c_longlong, c_size_t, c_void_p
from typing import Optional

import numpy as np
import torch

from . import build as _build

AEW_FULL, AEW_REVOLVE, AEW_AE = 0, 1, 2
STORAGE = {"full": AEW_FULL, "revolve": AEW_REVOLVE, "ae": AEW_AE}
AEW_CODEC_SPACE, AEW_CODEC_TIME = 0, 1
CODEC = {"space": AEW_CODEC_SPACE, "time": AEW_CODEC_TIME}
WINDOW = 16   # steps per window of the time codec

_ERRORS = {
    -1: "AEW_E_CONFIG", -2: "AEW_E_CFL", -3: "AEW_E_NONFINITE", -4: "AEW_E_NOCODEC",
    -5: "AEW_E_NOGRADIENT", -6: "AEW_E_NOMEM", -7: "AEW_E_CUDA", -8: "AEW_E_OVERFLOW",
    -9: "AEW_E_ARG", -10: "AEW_E_IO", -11: "AEW_E_TIMEOUT", -12: "AEW_E_NOCONVERGE",
}


class AewError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class aew_config(ctypes.Structure):
    _fields_ = [
        ("nx", c_int), ("ny", c_int), ("nz", c_int),
        ("h", c_double), ("cfl", c_double), ("cmax", c_double),
        ("nt", c_int), ("src", c_int * 3), ("f0", c_double), ("t0", c_double),
        ("nrec", c_int), ("rec_ijk", POINTER(c_int)),
        ("storage", c_int), ("n_checkpoints", c_int), ("accum_window", c_int), ("n_lat", c_int),
        ("codec", c_int), ("norm", c_int), ("act", c_int), ("beta", c_double),
        ("src_sigma", c_double),
    ]


class aew_stats_t(ctypes.Structure):
    _fields_ = [
        ("device_bytes", c_size_t), ("latent_bytes", c_size_t), ("history_bytes", c_size_t),
        ("forward_steps", c_longlong), ("adjoint_steps", c_longlong),
        ("hvp_forward_steps", c_longlong), ("last_misfit", c_double), ("latent_overflow", c_int),
        ("kernel_launches", c_longlong), ("decoded_err_normalised", c_double),
        ("decoded_err_physical", c_double), ("last_gradient_ms", c_double),
        ("last_hessvec_ms", c_double),
    ]


class aew_train_cfg(ctypes.Structure):
    _fields_ = [
        ("epochs", c_int), ("batch", c_int), ("lr0", c_double), ("halve_every", c_int),
        ("loss", c_int), ("seed", ctypes.c_ulonglong),
    ]


LOSSES = {"state": 0, "strain": 1, "strain-amplitude": 2, "strain-energy": 3}


class aew_newton_cfg(ctypes.Structure):
    _fields_ = [
        ("alpha", c_double), ("theta", c_double), ("newton_iters", c_int), ("cg_max", c_int),
        ("full_hessian", c_int), ("c1", c_double), ("max_backtracks", c_int),
        ("eta_max", c_double), ("gtol", c_double),
    ]


class aew_newton_iter(ctypes.Structure):
    _fields_ = [
        ("cost", c_double), ("misfit", c_double), ("reg", c_double), ("gnorm", c_double),
        ("cg_iters", c_int), ("backtracks", c_int), ("step", c_double),
    ]


_LIB = None

# (name, restype, argtypes) of every exported entry point
_SIGS = [
    ("aew_create", c_int, [POINTER(aew_config), POINTER(c_void_p)]),
    ("aew_destroy", None, [c_void_p]),
    ("aew_last_error", ctypes.c_char_p, [c_void_p]),
    ("aew_stats", c_int, [c_void_p, POINTER(aew_stats_t)]),
    ("aew_codec_set", c_int, [c_void_p] + [c_void_p] * 8),
    ("aew_codec_get", c_int, [c_void_p] + [c_void_p] * 8),
    ("aew_codec_encode", c_int, [c_void_p, POINTER(c_void_p), c_void_p, c_void_p, c_void_p]),
    ("aew_codec_encode_vectors", c_int, [c_void_p, c_void_p, c_longlong, c_void_p, c_void_p]),
    ("aew_codec_decode", c_int, [c_void_p, c_void_p, c_longlong, c_void_p, c_void_p]),
    ("aew_codec_decode_e", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("aew_codec_encode_window", c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    ("aew_codec_decode_window", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("aew_sync_check", c_int, [c_void_p, c_void_p]),
    ("aew_test_wait_timeout", c_int, [c_void_p, ctypes.c_ulonglong, c_void_p]),
    ("aew_forward", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("aew_propagate", c_int, [c_void_p, c_void_p, POINTER(c_void_p), c_int, c_int, c_void_p,
                              c_void_p, c_void_p]),
    ("aew_gradient", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_double), c_void_p]),
    ("aew_hessvec", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("aew_hessvec_full", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("aew_jvp", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("aew_snapshots", c_int, [c_void_p, c_void_p, c_int, c_void_p, c_longlong, c_void_p,
                              POINTER(c_longlong), c_void_p]),
    ("aew_codec_train_step", c_int, [c_void_p, c_void_p, c_void_p, c_int, c_float,
                                     POINTER(c_float), c_void_p]),
    ("aew_dot", c_int, [c_void_p, c_void_p, c_size_t, POINTER(c_double), c_void_p]),
    ("aew_dot_noalloc", c_int, [c_void_p, c_void_p, c_size_t, c_void_p, c_void_p]),
    ("aew_test_gelu", c_int, [c_void_p, c_void_p, c_void_p, c_longlong, c_void_p]),
    ("aew_revolve_plan", c_int, [c_int, c_int, c_void_p, c_void_p, c_longlong,
                                 POINTER(c_longlong), POINTER(c_longlong)]),
    ("aew_codec_init_pca", c_int, [c_void_p, c_void_p, c_void_p, c_longlong, c_int, c_void_p,
                                   c_void_p]),
    ("aew_codec_train", c_int, [c_void_p, c_void_p, c_void_p, c_longlong, POINTER(aew_train_cfg),
                                c_void_p, c_void_p]),
    ("aew_codec_eval", c_int, [c_void_p, c_void_p, c_void_p, c_longlong, c_void_p, c_void_p]),
    ("aew_sym_eig", c_int, [c_int, c_void_p, c_void_p, c_void_p]),
    ("aew_profile_steps", c_int, [c_void_p, c_void_p, c_int, c_int, POINTER(c_double), c_void_p]),
    ("aew_prior_apply", c_int, [c_void_p, c_double, c_double, c_void_p, c_void_p, c_void_p]),
    ("aew_prior_solve", c_int, [c_void_p, c_double, c_double, c_void_p, c_void_p, c_double, c_int,
                                POINTER(c_int), c_void_p]),
    ("aew_newton_cg", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(aew_newton_cfg),
                              c_void_p, c_int, c_void_p, POINTER(c_int), c_void_p]),
    ("aew_dias_subspace", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_double,
                                  c_double, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
]


def library_path() -> str:
    return os.environ.get("AEW_LIBRARY") or _build.LIB


def lib():
    """Load libaewave.so (building it first if it is missing or stale).

    The environment variable AEW_LIBRARY may name another build of the same library
    (for A/B comparisons of build options); it is loaded as is."""
    global _LIB
    if _LIB is None:
        path = os.environ.get("AEW_LIBRARY")
        if not path:
            if not _build.up_to_date():
                _build.build()
            path = _build.LIB
        L = ctypes.CDLL(path)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return c_void_p(t.data_ptr())


def _stream():
    return c_void_p(torch.cuda.current_stream().cuda_stream)


def _host_f32(a) -> Optional[np.ndarray]:
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def dot(a: torch.Tensor, b: torch.Tensor) -> float:
    """FP64 inner product of two CUDA FP32 tensors (aew_dot)."""
    assert a.numel() == b.numel() and a.dtype == torch.float32 and b.dtype == torch.float32
    out = c_double(0.0)
    rc = lib().aew_dot(_ptr(a), _ptr(b), a.numel(), byref(out), _stream())
    if rc != 0:
        raise AewError(rc, "aew_dot failed")
    return out.value


def activation_probe(x: torch.Tensor):
    """(GELU(x) as the encoder/decoder kernels compute it, GELU'(x) as the training
    kernels compute it) for a CUDA FP32 tensor."""
    assert x.dtype == torch.float32 and x.is_cuda
    x = x.contiguous()
    y, dy = torch.empty_like(x), torch.empty_like(x)
    rc = lib().aew_test_gelu(_ptr(x), _ptr(y), _ptr(dy), x.numel(), _stream())
    if rc != 0:
        raise AewError(rc, "aew_test_gelu failed")
    return y, dy


def dot_noalloc(a: torch.Tensor, b: torch.Tensor, out: torch.Tensor) -> None:
    """aew_dot_noalloc: FP64 inner product into the CUDA FP64 scalar `out`, with no
    device allocation (asynchronous on the current stream)."""
    assert a.numel() == b.numel() and a.dtype == torch.float32 and b.dtype == torch.float32
    assert out.dtype == torch.float64 and out.numel() == 1
    rc = lib().aew_dot_noalloc(_ptr(a), _ptr(b), a.numel(), _ptr(out), _stream())
    if rc != 0:
        raise AewError(rc, "aew_dot_noalloc failed")


def revolve_plan(nt: int, s: int):
    """The library's checkpointing plan: (list of (op, arg), forward steps)."""
    L = lib()
    n = c_longlong(0)
    f = c_longlong(0)
    rc = L.aew_revolve_plan(nt, s, None, None, 0, byref(n), byref(f))
    if rc != 0:
        raise AewError(rc, "aew_revolve_plan failed")
    ops = (c_int * n.value)()
    args = (c_int * n.value)()
    L.aew_revolve_plan(nt, s, ops, args, n.value, byref(n), byref(f))
    names = {0: "advance", 1: "store", 2: "restore", 3: "final", 4: "reverse"}
    return [(names[ops[i]], args[i]) for i in range(n.value)], f.value


def sym_eig(A: np.ndarray):
    """Host eigensolver of the library (aew_sym_eig): (eigenvalues descending,
    eigenvectors as columns) of a symmetric FP64 matrix."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    n = A.shape[0]
    w = np.empty(n)
    V = np.empty((n, n))
    rc = lib().aew_sym_eig(n, A.ctypes.data, w.ctypes.data, V.ctypes.data)
    if rc != 0:
        raise AewError(rc, "aew_sym_eig failed")
    return w, V


class Solver:
    """Owns one aew_handle: grid, time stepping, receivers and history storage."""

    def __init__(self, shape, h: float, nt: int, rec, storage: str = "full",
                 n_checkpoints: int = 20, accum_window: int = 8, n_lat: Optional[int] = None,
                 cfl: float = 0.5, cmax: float = 3000.0, src=None, f0: float = 25.0,
                 t0: Optional[float] = None, codec: str = "space", norm: str = "pow2",
                 act: str = "gelu", beta: float = 0.0, src_sigma: float = 0.0):
        nz, ny, nx = shape
        self.shape = (nz, ny, nx)
        self.nt = nt
        rec = np.ascontiguousarray(np.asarray(rec, dtype=np.int32).reshape(-1, 3))
        self.nrec = rec.shape[0]
        self._rec = rec
        cfg = aew_config()
        cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
        cfg.h, cfg.cfl, cfg.cmax = h, cfl, cmax
        cfg.nt = nt
        s = src if src is not None else (nx // 2, ny // 2, nz // 2)
        cfg.src[0], cfg.src[1], cfg.src[2] = s
        cfg.f0 = f0
        cfg.t0 = t0 if t0 is not None else 1.0 / f0
        cfg.nrec = self.nrec
        cfg.rec_ijk = rec.ctypes.data_as(POINTER(c_int)) if self.nrec else None
        cfg.storage = STORAGE[storage]
        cfg.n_checkpoints = n_checkpoints
        cfg.accum_window = accum_window
        if n_lat is None:
            n_lat = 512 if codec == "time" else 64
        cfg.n_lat = n_lat
        cfg.codec = CODEC[codec]
        cfg.norm = {"pow2": 0, "minmax": 1}[norm]
        cfg.act = {"gelu": 0, "elu": 1}[act]
        cfg.beta = beta
        cfg.src_sigma = src_sigma
        self.norm = norm
        self.n_lat = n_lat
        self.codec = codec
        self.n_hid = 2 * n_lat if codec == "time" else 512
        self.dt = cfl * h / cmax
        self._h = c_void_p()
        L = lib()
        rc = L.aew_create(byref(cfg), byref(self._h))
        if rc != 0:
            raise AewError(rc, L.aew_last_error(None).decode())

    # ------------------------------------------------------------------ helpers
    def _check(self, rc: int):
        if rc != 0:
            raise AewError(rc, lib().aew_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().aew_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nblocks(self) -> int:
        nz, ny, nx = self.shape
        return (nz // 8) * (ny // 8) * (nx // 8)

    @property
    def nvec(self) -> int:
        """Vectors per window of the time codec (2 x 8 x 8-node blocks)."""
        nz, ny, nx = self.shape
        return (nz // 2) * (ny // 8) * (nx // 8)

    def _drec(self) -> torch.Tensor:
        return torch.empty((self.nt + 1, self.nrec, 3), device="cuda", dtype=torch.float32)

    # ------------------------------------------------------------------ solves
    def forward(self, c: torch.Tensor, wavelet=None) -> torch.Tensor:
        d = self._drec()
        w = _host_f32(wavelet)
        self._check(lib().aew_forward(self._h, _ptr(c), w.ctypes.data if w is not None else None,
                                      _ptr(d), _stream()))
        return d

    def propagate(self, c: torch.Tensor, state, n0: int, nsteps: int, wavelet=None,
                  record: bool = False):
        """Advance the (e, vx, vy, vz) CUDA tensors in place; returns receiver data or None."""
        arr = (c_void_p * 4)(*[t.data_ptr() for t in state])
        for t in state:
            _ptr(t)
        d = torch.empty((nsteps + 1, self.nrec, 3), device="cuda") if record else None
        w = _host_f32(wavelet)
        self._check(lib().aew_propagate(self._h, _ptr(c), arr, n0, nsteps,
                                        w.ctypes.data if w is not None else None, _ptr(d), _stream()))
        return d

    def gradient(self, c: torch.Tensor, d_obs: torch.Tensor, g: Optional[torch.Tensor] = None):
        """(J, dJ/dc) for J = 1/2 sum_{n>=1} |d^n - d_obs^n|^2."""
        if g is None:
            g = torch.empty_like(c)
        J = c_double(0.0)
        self._check(lib().aew_gradient(self._h, _ptr(c), _ptr(d_obs), _ptr(g), byref(J), _stream()))
        return J.value, g

    def hessvec(self, dc: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        if out is None:
            out = torch.empty_like(dc)
        self._check(lib().aew_hessvec(self._h, _ptr(dc), _ptr(out), _stream()))
        return out

    def hessvec_full(self, dc: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Full Newton Hessian-vector product (second-order terms included) at the c of
        the last gradient."""
        if out is None:
            out = torch.empty_like(dc)
        self._check(lib().aew_hessvec_full(self._h, _ptr(dc), _ptr(out), _stream()))
        return out

    # ------------------------------------------------------------------ MAP / DIAS
    def prior_apply(self, q: torch.Tensor, alpha: float, theta: float,
                    out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """A q = alpha (q - theta Lap_N q), the BiLaplacian prior's elliptic operator."""
        if out is None:
            out = torch.empty_like(q)
        self._check(lib().aew_prior_apply(self._h, alpha, theta, _ptr(q), _ptr(out), _stream()))
        return out

    def prior_solve(self, w: torch.Tensor, alpha: float, theta: float, rtol: float = 1e-6,
                    max_iter: int = 5000, out: Optional[torch.Tensor] = None):
        """(A^{-1} w, CG iterations)."""
        if out is None:
            out = torch.empty_like(w)
        it = c_int(0)
        self._check(lib().aew_prior_solve(self._h, alpha, theta, _ptr(w), _ptr(out), rtol,
                                          max_iter, byref(it), _stream()))
        return out, it.value

    def newton_cg(self, c: torch.Tensor, d_obs: torch.Tensor, c0: torch.Tensor, alpha: float,
                  theta: float, newton_iters: int = 5, cg_max: int = 20, full_hessian: bool = False,
                  c1: float = 1e-4, max_backtracks: int = 10, eta_max: float = 0.5,
                  gtol: float = 0.0, W1: Optional[torch.Tensor] = None):
        """Inexact Newton-CG for the MAP point (or, with the active subspace W1 [r][n],
        the DIAS-F point).  c is updated in place; returns the per-iteration history as
        a list of dicts."""
        cfg = aew_newton_cfg(alpha, theta, newton_iters, cg_max, int(full_hessian), c1,
                             max_backtracks, eta_max, gtol)
        hist = (aew_newton_iter * newton_iters)()
        n = c_int(0)
        r = 0 if W1 is None else W1.shape[0]
        self._check(lib().aew_newton_cg(self._h, _ptr(c), _ptr(d_obs), _ptr(c0), byref(cfg),
                                        _ptr(W1), r, hist, byref(n), _stream()))
        return [{k: getattr(hist[i], k) for k, _ in aew_newton_iter._fields_}
                for i in range(n.value)]

    def dias_subspace(self, c: torch.Tensor, d_obs: torch.Tensor, noise: torch.Tensor,
                      alpha: float, theta: float, r: int, G: Optional[torch.Tensor] = None):
        """DIAS active subspace at c from the gradients at the prior samples
        c + A^{-1} noise[i]: (eigenvalues [N], W1 [r][n], sample gradients G [N][n])."""
        N = noise.shape[0]
        n = c.numel()
        if G is None:
            G = torch.empty((N, n), device="cuda", dtype=torch.float32)
        W1 = torch.empty((r, n), device="cuda", dtype=torch.float32)
        lam = np.empty(N)
        self._check(lib().aew_dias_subspace(self._h, _ptr(c), _ptr(d_obs), _ptr(noise), N, alpha,
                                            theta, r, _ptr(G), _ptr(W1), lam.ctypes.data,
                                            _stream()))
        return lam, W1, G

    def jvp(self, dc: torch.Tensor) -> torch.Tensor:
        dd = self._drec()
        self._check(lib().aew_jvp(self._h, _ptr(dc), _ptr(dd), _stream()))
        return dd

    def sync_check(self):
        """Synchronise the current stream; raise AewError if a kernel of this handle gave
        up a bounded device wait since the last check."""
        self._check(lib().aew_sync_check(self._h, _stream()))

    def test_wait_timeout(self, wait_ns: int = 1_000_000):
        """Enqueue a kernel whose bounded wait runs out (failure-path test hook)."""
        self._check(lib().aew_test_wait_timeout(self._h, int(wait_ns), _stream()))

    PROFILE_KINDS = {"forward": 0, "forward_pack": 1, "adjoint": 2, "incremental": 3,
                     "encode_window": 4, "decode_window": 5, "adjoint_bf16": 6,
                     "decode_window_bf16": 7, "incremental_bf16": 8, "decode_state": 9}

    def profile(self, c: torch.Tensor, kind: str, nsteps: int) -> float:
        """aew_profile_steps: mean device ms per launch of one hot-path kernel."""
        ms = c_double(0.0)
        self._check(lib().aew_profile_steps(self._h, _ptr(c), self.PROFILE_KINDS[kind], nsteps,
                                            byref(ms), _stream()))
        return ms.value

    def stats(self) -> dict:
        s = aew_stats_t()
        self._check(lib().aew_stats(self._h, byref(s)))
        return {k: getattr(s, k) for k, _ in aew_stats_t._fields_}

    # ------------------------------------------------------------------ codec
    def codec_set(self, W: dict):
        arrs = [_host_f32(W[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")]
        self._codec_host = arrs
        self._check(lib().aew_codec_set(self._h, *[a.ctypes.data for a in arrs]))

    def codec_get(self) -> dict:
        nl, nh = self.n_lat, self.n_hid
        shapes = {"W1": (2048, nh), "b1": (nh,), "W2": (nh, nl), "b2": (nl,),
                  "W3": (nl, nh), "b3": (nh,), "W4": (nh, 2048), "b4": (2048,)}
        out = {k: np.empty(v, np.float32) for k, v in shapes.items()}
        self._check(lib().aew_codec_get(self._h, *[out[k].ctypes.data for k in shapes]))
        return out

    def codec_encode(self, fields):
        """Encode one state (e, vx, vy, vz CUDA tensors): returns (FP16 latents
        [nblocks][n_lat], FP32 block maxima [nblocks][4] that fix the scales)."""
        lat = torch.empty((self.nblocks, self.n_lat), device="cuda", dtype=torch.float16)
        bmax = torch.empty((self.nblocks, 4), device="cuda", dtype=torch.float32)
        arr = (c_void_p * 4)(*[f.data_ptr() for f in fields])
        for f in fields:
            _ptr(f)
        self._check(lib().aew_codec_encode(self._h, arr, _ptr(lat), _ptr(bmax), _stream()))
        return lat, bmax

    def codec_encode_vectors(self, vec: torch.Tensor) -> torch.Tensor:
        """BF16 normalised block vectors [n][2048] -> FP16 latents [n][n_lat]."""
        assert vec.dtype == torch.bfloat16 and vec.shape[-1] == 2048
        lat = torch.empty((vec.shape[0], self.n_lat), device="cuda", dtype=torch.float16)
        self._check(lib().aew_codec_encode_vectors(self._h, _ptr(vec), vec.shape[0], _ptr(lat),
                                                   _stream()))
        return lat

    def codec_decode(self, lat: torch.Tensor) -> torch.Tensor:
        out = torch.empty((lat.shape[0], 2048), device="cuda", dtype=torch.float32)
        self._check(lib().aew_codec_decode(self._h, _ptr(lat), lat.shape[0], _ptr(out), _stream()))
        return out

    def codec_decode_e(self, lat: torch.Tensor, block_max: torch.Tensor) -> torch.Tensor:
        """Strain field decoded from latents with the blocks' scales (from block maxima)."""
        e = torch.empty(self.shape, device="cuda", dtype=torch.float32)
        self._check(lib().aew_codec_decode_e(self._h, _ptr(lat), _ptr(block_max.contiguous()),
                                             _ptr(e), _stream()))
        return e

    def codec_encode_window(self, e: torch.Tensor):
        """Time codec: encode one window of strain fields e [nsteps <= 16][nz][ny][nx]
        (CUDA FP32): returns (FP16 latents [nvec][n_lat], the scales: FP32 vector maxima
        [nvec], or with min-max normalisation FP64 [2][nvec] offsets and ranges)."""
        e = e.contiguous()
        lat = torch.empty((self.nvec, self.n_lat), device="cuda", dtype=torch.float16)
        if self.norm == "minmax":      # offsets then ranges, FP64
            vmax = torch.empty((2, self.nvec), device="cuda", dtype=torch.float64)
        else:
            vmax = torch.empty((self.nvec,), device="cuda", dtype=torch.float32)
        self._check(lib().aew_codec_encode_window(self._h, _ptr(e), e.shape[0], _ptr(lat),
                                                  _ptr(vmax), _stream()))
        return lat, vmax

    def codec_decode_window(self, lat: torch.Tensor, vmax: torch.Tensor) -> torch.Tensor:
        """Time codec: the 16 decoded strain fields [16][nz][ny][nx] of one window."""
        e = torch.empty((WINDOW,) + self.shape, device="cuda", dtype=torch.float32)
        self._check(lib().aew_codec_decode_window(self._h, _ptr(lat), _ptr(vmax.contiguous()),
                                                  _ptr(e), _stream()))
        return e

    def snapshots(self, c: torch.Tensor, every: int, max_vectors: int,
                  out: Optional[torch.Tensor] = None, with_scales: bool = False):
        """Algorithm 1: normalised BF16 vectors of every `every`-th state (space codec)
        or window (time codec).

        Returns the [n][2048] bfloat16 tensor (and the maxima that fix the scales:
        [n][4] block maxima, or [n] vector maxima with the time codec)."""
        if out is None:
            out = torch.empty((max_vectors, 2048), device="cuda", dtype=torch.bfloat16)
        mshape = ((max_vectors, 2) if self.norm == "minmax" else (max_vectors,)) \
            if self.codec == "time" else (max_vectors, 4)
        bm = torch.zeros(mshape, device="cuda") if with_scales else None
        n = c_longlong(0)
        self._check(lib().aew_snapshots(self._h, _ptr(c), every, _ptr(out), max_vectors, _ptr(bm),
                                        byref(n), _stream()))
        if with_scales:
            return out[: n.value], bm[: n.value]
        return out[: n.value]

    def codec_init_pca(self, vectors: torch.Tensor, maxima: Optional[torch.Tensor] = None,
                       loss: str = "state"):
        """aew_codec_init_pca: set the codec to the optimal rank-n_lat code of the BF16
        vectors [n][2048] under `loss` (weights from the vectors' maxima on the device);
        returns the covariance's eigenvalues (descending, FP64 numpy array of 2048)."""
        assert vectors.dtype == torch.bfloat16 and vectors.shape[-1] == 2048
        ev = np.empty(2048)
        m = None if maxima is None else maxima.contiguous().float()
        self._check(lib().aew_codec_init_pca(self._h, _ptr(vectors.contiguous()), _ptr(m),
                                             vectors.shape[0], LOSSES[loss], ev.ctypes.data,
                                             _stream()))
        return ev

    def codec_train(self, vectors: torch.Tensor, maxima: Optional[torch.Tensor] = None,
                    epochs: int = 20, batch: int = 512, lr0: float = 1e-3, halve_every: int = 5,
                    loss: str = "state", seed: int = 0):
        """aew_codec_train: Table 2's epochs on the device; returns each epoch's mean loss."""
        cfg = aew_train_cfg()
        cfg.epochs, cfg.batch, cfg.lr0, cfg.halve_every = epochs, batch, lr0, halve_every
        cfg.loss, cfg.seed = LOSSES[loss], seed
        out = np.zeros(max(epochs, 1))
        m = None if maxima is None else maxima.contiguous().float()
        self._check(lib().aew_codec_train(self._h, _ptr(vectors.contiguous()), _ptr(m),
                                          vectors.shape[0], byref(cfg), out.ctypes.data, _stream()))
        return out[:epochs].tolist()

    def codec_eval(self, vectors: torch.Tensor, maxima: torch.Tensor) -> dict:
        """aew_codec_eval: decoded rel-L2 errors, normalised and physical units."""
        out = np.zeros(10)
        self._check(lib().aew_codec_eval(self._h, _ptr(vectors.contiguous()),
                                         _ptr(maxima.contiguous().float()), vectors.shape[0],
                                         out.ctypes.data, _stream()))
        names = ["e", "vx", "vy", "vz", "all"]
        return {"normalised": dict(zip(names, out[:5].tolist())),
                "physical": dict(zip(names, out[5:].tolist())), "vectors": int(vectors.shape[0])}

    def train_step(self, batch: torch.Tensor, lr: float, want_loss: bool = True,
                   weights: Optional[torch.Tensor] = None) -> Optional[float]:
        """One LAMB step on a BF16 minibatch [B][2048]; weights (FP32 [B][4], optional)
        weigh each vector's fields in the squared error."""
        loss = c_float(0.0)
        w = None if weights is None else weights.contiguous().float()
        self._check(lib().aew_codec_train_step(self._h, _ptr(batch), _ptr(w), batch.shape[0],
                                               c_float(lr), byref(loss) if want_loss else None,
                                               _stream()))
        return loss.value if want_loss else None


class Misfit(torch.autograd.Function):
    """J(c) = 1/2 |F(c) - d_obs|^2 with dJ/dc from the library's adjoint solve."""

    @staticmethod
    def forward(ctx, c: torch.Tensor, d_obs: torch.Tensor, solver: Solver):
        J, g = solver.gradient(c.contiguous(), d_obs.contiguous())
        ctx.save_for_backward(g)
        return torch.tensor(J, dtype=torch.float64, device=c.device)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return (gJ.to(g.dtype) * g, None, None)


class ForwardMap(torch.autograd.Function):
    """d = F(c) with the vector-Jacobian product J_F^T r from the adjoint solve."""

    @staticmethod
    def forward(ctx, c: torch.Tensor, solver: Solver):
        d = solver.forward(c.contiguous())
        ctx.solver = solver
        ctx.save_for_backward(c, d)
        return d

    @staticmethod
    def backward(ctx, r):
        c, d = ctx.saved_tensors
        # the gradient of 1/2 |F(c) - (d - r)|^2 is J_F^T r
        _, g = ctx.solver.gradient(c, (d - r).contiguous())
        return g, None
