"""Parity at the benchmark's full size: 256^3 nodes (32,768 blocks), 128 receivers, the
kernels and launch shapes the benchmark times (codec kernels capped at 76 CTAs, as they
run beside a stencil step).  The FP64 oracle cannot follow 2000 steps at this size, so
the checks take outputs it computes one by one or properties that hold at any size:

- two stencil steps from a smooth state that fills the grid, whole fields;
- the encoder (layer 1 on SM pairs) and the fused strain decoder on sampled blocks of a
  full-grid state;
- the packing forward step's block vectors and maxima after 400 steps, on sampled
  blocks against the host packing of the same state;
- the adjoint identity <J dc, r> = <dc, J^T r> over 400 steps (the wave reaches the
  receivers on the top plane)."""
import numpy as np
import pytest
import torch

from oracle import codec as C
from oracle import wave as W
from paper_2304_04781_gb300 import inputs

from .helpers import cuda, host, relerr, setup, solver

pytestmark = pytest.mark.gpu

SHAPE = (256, 256, 256)
NREC = 128
CODEC_TOL = 2e-3


def _valid_state(seed):
    """Smooth (e, vx, vy, vz) over the whole grid, FP32-representable, with e = 0 on the
    boundary and the unused last faces of vx, vy, vz at 0 (the storage convention)."""
    st = [a.astype(np.float32).astype(np.float64) for a in inputs.smooth_state(SHAPE, 10.0, seed=seed)]
    st[0] = W.interior(st[0])
    st[1][:, :, -1] = 0.0
    st[2][:, -1, :] = 0.0
    st[3][-1, :, :] = 0.0
    return st


def _sample_blocks(nb, seed, n=200):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, nb - 1], rng.integers(0, nb, n)]))


def _block_slices(b):
    NBy, NBx = SHAPE[1] // 8, SHAPE[2] // 8
    bz, rem = divmod(int(b), NBy * NBx)
    by, bx = divmod(rem, NBx)
    return bz, by, bx, (slice(8 * bz, 8 * bz + 8), slice(8 * by, 8 * by + 8),
                        slice(8 * bx, 8 * bx + 8))


def _packed_rows(fields, rows):
    """The oracle's packing and block scales of the sampled blocks, each applied to the
    block's own 8^3 nodes (the same functions as on the whole grid, block by block)."""
    X, S = [], []
    for b in rows:
        sub = [f[_block_slices(b)[3]] for f in fields]
        X.append(C.pack_blocks(sub)[0])
        S.append(C.block_scales(sub)[0])
    return np.array(X), np.array(S)


@pytest.fixture(scope="module")
def grid():
    """Velocity model of the benchmark (seed 2), receivers, and a smooth full-grid state."""
    prob, c, rec = setup(SHAPE, 2, NREC, seed=2)
    return prob, c, rec, _valid_state(8)


def _problem(rec, nt):
    return W.Problem(shape=SHAPE, h=10.0, nt=nt, rec=rec)


def test_stencil_steps_match_oracle_at_full_size(grid):
    prob, c, _, st0 = grid
    s = solver(prob)
    st = [cuda(a) for a in st0]
    wav = W.default_wavelet(prob)
    d = s.propagate(cuda(c), st, 0, 2, wavelet=wav[:2], record=True)
    d_ref, fin, _ = W.forward(prob, c, state0=st0)
    for got, ref in zip(st, fin):
        assert relerr(host(got), ref) < 1e-5
    assert relerr(host(d)[1:], d_ref[1:]) < 1e-5   # row 0 of a propagate record is left 0


def test_codec_at_full_size_on_sampled_blocks(grid, monkeypatch):
    monkeypatch.setenv("AEW_GEMM_CTAS", "76")   # read when the handle's codec is made
    prob, _, _, st = grid
    s = solver(prob, storage="ae")
    Wt = inputs.codec_init(seed=1, n_lat=64)
    s.codec_set(Wt)
    lat, bm = s.codec_encode([cuda(a) for a in st])
    nb = s.nblocks
    assert lat.shape == (nb, 64)
    rows = _sample_blocks(nb, 4)
    X, sc = _packed_rows(st, rows)
    z_ref = C.encode(Wt, C.normalise(X, sc), emulate=True)
    z = lat[torch.from_numpy(rows).cuda()].float().cpu().numpy().astype(np.float64)
    assert relerr(z, z_ref) < CODEC_TOL
    # the fused strain decoder on the GPU's own latents, block by block
    e = host(s.codec_decode_e(lat, bm))
    Zr = C.round_fp16(z)
    dec = C.decode(Wt, Zr, emulate=True, cols=C.field_columns(0))
    bmr = host(bm)[rows, 0]
    _, ex = np.frexp(bmr)
    sb = np.where(bmr > 0, np.ldexp(1.0, np.maximum(ex, C.EXP_MIN)), 0.0)
    worst = 0.0
    for i, b in enumerate(rows):
        bz, by, bx, sl = _block_slices(b)
        want = dec[i].reshape(8, 8, 8) * sb[i]
        kk, jj, ii = np.meshgrid(np.arange(8 * bz, 8 * bz + 8), np.arange(8 * by, 8 * by + 8),
                                 np.arange(8 * bx, 8 * bx + 8), indexing="ij")
        edge = ((kk == 0) | (kk == SHAPE[0] - 1) | (jj == 0) | (jj == SHAPE[1] - 1) |
                (ii == 0) | (ii == SHAPE[2] - 1))
        want = np.where(edge, 0.0, want)
        got = e[sl]
        assert np.all(got[edge] == 0.0)
        nrm = np.linalg.norm(want)
        if nrm > 0:
            worst = max(worst, np.linalg.norm(got - want) / nrm)
    assert worst < 5 * CODEC_TOL, worst


def test_packing_step_at_full_size_on_sampled_blocks(grid):
    """State 400 packed by the forward step that reads it (normalised by the maxima the
    step before stored), against the oracle's packing and normalisation of the same
    state advanced by the plain step, rounded once to BF16: maxima to a few FP32 ulps,
    BF16 codes bit for bit except rarely one ulp."""
    _, c, rec, _ = grid
    prob = _problem(rec, 401)
    s = solver(prob, storage="ae")
    nb = s.nblocks
    snaps, bm = s.snapshots(cuda(c), every=400, max_vectors=nb, with_scales=True)
    assert snaps.shape == (nb, 2048)
    st = [torch.zeros(SHAPE, device="cuda") for _ in range(4)]
    s.propagate(cuda(c), st, 0, 400, wavelet=W.default_wavelet(prob)[:400])
    hs = [host(t) for t in st]
    rows = _sample_blocks(nb, 5)
    X, sc = _packed_rows(hs, rows)
    Xa = np.abs(X)
    bm_ref = np.stack([Xa[:, C.field_columns(f)].max(1) for f in range(4)], 1)
    assert np.count_nonzero(bm_ref) > 0
    np.testing.assert_allclose(host(bm)[rows], bm_ref, rtol=1e-6, atol=0)
    want = torch.from_numpy(C.normalise(X, sc)).to(torch.bfloat16).view(torch.int16).numpy()
    got = snaps[torch.from_numpy(rows).cuda()].view(torch.int16).cpu().numpy()
    assert np.mean(got == want) > 0.999
    gv = torch.from_numpy(got).view(torch.bfloat16).double().numpy()
    wv = torch.from_numpy(want).view(torch.bfloat16).double().numpy()
    assert np.all(np.abs(gv - wv) <= 2.0 ** -7 * np.maximum(np.abs(gv), np.abs(wv)))


def test_adjoint_identity_at_full_size(grid):
    from paper_2304_04781_gb300 import aewave
    _, c, rec, _ = grid
    prob = _problem(rec, 400)
    s = solver(prob)
    cc = cuda(c)
    d = s.forward(cc)
    assert float(d.abs().max()) > 0   # the wave has reached the receivers
    gen = torch.Generator(device="cuda").manual_seed(6)
    white = torch.randn(d.shape, device="cuda", generator=gen)
    w = white.permute(1, 2, 0).reshape(-1, 1, d.shape[0])
    r = torch.nn.functional.conv1d(w, torch.full((1, 1, 9), 1.0 / 9, device="cuda"), padding=4)
    r = r.reshape(d.shape[1], d.shape[2], d.shape[0]).permute(2, 0, 1) * d.abs().max()
    r = r.contiguous()
    r[0] = 0
    _, JTr = s.gradient(cc, (d - r).contiguous())
    dc = cuda(inputs.direction(SHAPE, 10.0, seed=21))
    Jdc = s.jvp(dc)
    lhs = aewave.dot(Jdc, r)
    rhs = aewave.dot(dc, JTr)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)
