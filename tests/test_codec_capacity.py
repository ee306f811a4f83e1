"""How far a rank-k linear code can compress the solver's own block vectors.

The codec sees 2048-vectors (8^3 blocks x 4 fields, every field of every block divided
by its power-of-two scale; Algorithm 1 packing).  A linear autoencoder reaches exactly
the truncated-PCA error (Sec. 1, pinned in test_oracle_codec.py), so the singular
values of the centred vectors say how much a rank-k linear code keeps.  On the states
of a point-source forward solve in a Gaussian-random-field medium the spectrum decays
slowly: at k = 64 (the 32x latent size) about half the energy of all four fields and a
quarter of the strain's is lost, and even k = 256 loses ~20%.  This is why the trained
2048-512-64 codec, a mildly nonlinear code of the same latent size, cannot bring the
decoded states, and hence the compressed gradient, anywhere near 1e-2 on this
workload.  CPU only (FP64 oracle forward, 48^3 x 300 steps, a few seconds)."""
import numpy as np

from oracle import codec as C
from oracle import wave as W
from paper_2304_04781_gb300 import inputs


def _block_vectors(n=48, nt=300, every=10, seed=100):
    rec = inputs.receiver_grid(n, n, 16)
    prob = W.Problem(shape=(n, n, n), h=10.0, nt=nt, rec=rec)
    c = inputs.velocity_model(prob.shape, 10.0, seed=seed)
    vecs = []

    def keep(k, e, vx, vy, vz):
        if k % every == 0 and k > 0:
            st = [e, vx, vy, vz]
            s = C.block_scales(st)
            X = C.normalise(C.pack_blocks(st), s)
            vecs.append(X[s.max(1) > 0])

    W.forward(prob, c, on_state=keep)
    return np.concatenate(vecs)


def _truncation_error(X, k):
    """Relative L2 error of the best rank-k affine code (centred truncated SVD)."""
    S = np.linalg.svd(X - X.mean(0), compute_uv=False)
    return float(np.sqrt((S[k:] ** 2).sum() / (X ** 2).sum()))


def test_rank_64_linear_code_keeps_only_about_half_of_the_state():
    X = _block_vectors()
    assert X.shape[1] == 2048 and X.shape[0] > 2048
    err = {k: _truncation_error(X, k) for k in (16, 64, 256, 2048)}
    assert err[2048] < 1e-12                       # full rank reproduces the data
    assert err[16] > err[64] > err[256] > 0.1      # slow decay, far from 1e-2 at 256
    assert 0.35 < err[64] < 0.65
    E = X[:, C.field_columns(0)]
    E = E[np.abs(E).max(1) > 0]
    e64 = _truncation_error(E, 64)
    assert 0.15 < e64 < 0.4                        # strain alone, rank 64 of 512
