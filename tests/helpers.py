"""Shared fixtures for the GPU parity tests: problem setups built identically for the
CUDA path (aewave.Solver) and the FP64 oracle (oracle.wave.Problem)."""
import numpy as np
import torch

from oracle import wave as W
from paper_2304_04781_gb300 import inputs


def relerr(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def setup(shape, nt, nrec, seed=0, h=10.0):
    """(oracle Problem, c as float64 rounded through float32, receivers)."""
    nz, ny, nx = shape
    rec = inputs.receiver_grid(nx, ny, nrec)
    prob = W.Problem(shape=tuple(shape), h=h, nt=nt, rec=rec)
    c = inputs.velocity_model(shape, h, seed=seed).astype(np.float32).astype(np.float64)
    return prob, c, rec


def solver(prob, storage="full", **kw):
    from paper_2304_04781_gb300 import aewave
    return aewave.Solver(prob.shape, prob.h, prob.nt, prob.rec, storage=storage, src=prob.src,
                         f0=prob.f0, t0=prob.t0, cfl=prob.cfl, cmax=prob.cmax,
                         src_sigma=prob.src_sigma, **kw)


def cuda(a) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.float32))).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().astype(np.float64)
