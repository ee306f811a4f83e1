"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
entry point include/aewave.h declares, rejects invalid configurations before touching
the device, and its checkpointing planner is optimal and valid against the oracle."""
import ctypes
import os
import re

import pytest

from oracle import revolve as R
from paper_2304_04781_gb300 import aewave

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "aewave.h")).read()
    return re.findall(r"^\s*(?:int|void|const char\*)\s+(aew_\w+)\s*\(", hdr, re.M)


def test_library_exports_every_declared_symbol():
    L = aewave.lib()
    names = declared_symbols()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n
    # the binding and the header list the same entry points: nothing the binding calls
    # is undeclared, and every declared call is reachable from Python
    bound = {n for n, _, _ in aewave._SIGS}
    assert bound == set(names), (sorted(set(names) - bound), sorted(bound - set(names)))


def _cfg(**kw):
    c = aewave.aew_config()
    c.nx = c.ny = c.nz = 16
    c.h, c.cfl, c.cmax, c.nt = 10.0, 0.5, 3000.0, 10
    c.src[0] = c.src[1] = c.src[2] = 8
    c.f0, c.t0 = 25.0, 0.04
    c.nrec, c.rec_ijk = 0, None
    c.storage, c.n_checkpoints, c.accum_window, c.n_lat = 0, 4, 8, 64
    for k, v in kw.items():
        setattr(c, k, v)
    return c


@pytest.mark.parametrize("kw,frag", [
    (dict(nx=18), "multiples of 4"),
    (dict(nt=0), "nt"),
    (dict(cfl=0.7), "cfl"),
    (dict(h=-1.0), "> 0"),
    (dict(storage=7), "storage"),
    (dict(accum_window=0), "accum_window"),
    (dict(storage=2, nx=20), "multiples of 8"),
    (dict(n_lat=48), "n_lat"),
    (dict(codec=2), "codec"),
    (dict(codec=1, n_lat=64), "n_lat"),
    (dict(codec=1, storage=2, n_lat=512, nx=20), "multiples of 8"),
    (dict(codec=1, storage=2, n_lat=512, nz=12, ny=20), "multiples of 8"),
    (dict(src_sigma=-1.0), "src_sigma"),
    (dict(src_sigma=30.0), "smoothed source's box"),
])
def test_create_rejects_bad_configs(kw, frag):
    L = aewave.lib()
    h = ctypes.c_void_p()
    rc = L.aew_create(ctypes.byref(_cfg(**kw)), ctypes.byref(h))
    assert rc == -1
    assert h.value is None
    assert frag in L.aew_last_error(None).decode()


def test_receivers_must_share_one_plane():
    L = aewave.lib()
    rec = (ctypes.c_int * 6)(2, 2, 1, 3, 3, 2)
    c = _cfg(nrec=2, rec_ijk=ctypes.cast(rec, ctypes.POINTER(ctypes.c_int)))
    h = ctypes.c_void_p()
    assert L.aew_create(ctypes.byref(c), ctypes.byref(h)) == -1
    assert "one node plane" in L.aew_last_error(None).decode()


@pytest.mark.parametrize("nt", [1, 2, 3, 7, 30, 101, 1000, 2000])
@pytest.mark.parametrize("s", [0, 1, 2, 3, 5, 20, 31])
def test_revolve_plan_is_valid_and_optimal(nt, s):
    if s == 0 and nt > 200:
        pytest.skip("quadratic plan, large")
    plan, fwd = aewave.revolve_plan(nt, s)
    assert R.simulate(plan, nt, s) == fwd
    assert fwd == R.gradient_forward_steps(nt, s)


def test_revolve_plan_matches_brute_force_small():
    for nt in range(1, 25):
        for s in range(0, 4):
            _, fwd = aewave.revolve_plan(nt, s)
            assert fwd == R.brute_force(nt, s) + 1


@pytest.mark.parametrize("n", [1, 2, 7, 64, 257])
def test_host_eigensolver_matches_the_definition(n):
    """aew_sym_eig (the PCA initialisation's solver) on random symmetric matrices, one
    with clustered eigenvalues: A V = V diag(w), V orthonormal, w descending and equal to
    numpy's eigenvalues."""
    import numpy as np
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    A = B + B.T
    if n == 257:   # repeated eigenvalues in clusters of 8
        Q, _ = np.linalg.qr(B)
        lam = np.repeat(np.linspace(3.0, -1.0, 33), 8)[:n]
        A = (Q * lam) @ Q.T
    w, V = aewave.sym_eig(A)
    scale = max(1.0, float(np.abs(w).max()))
    assert np.all(np.diff(w) <= 1e-12 * scale)
    np.testing.assert_allclose(w, np.sort(np.linalg.eigvalsh(A))[::-1], atol=1e-12 * scale)
    assert np.abs(A @ V - V * w).max() < 1e-12 * scale
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-12
