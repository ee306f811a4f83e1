"""Codec training pipeline: data generation by Algorithm 1 and training per Table 2.

Data (Algorithm 1): for each prior draw of the wave speed (a seeded Gaussian random
field), run the forward solve and keep every `every`-th state, cut into 8x8x8-node
blocks of the four fields (2048 values each, every field of every block divided by its
power-of-two scale, the per-vector normalisation of Sec. 3.3), as BF16 vectors resident
in HBM.  Training (Table 2): mean-squared
reconstruction error, LAMB, learning rate 1e-3 halved every 5 epochs, batch 512, a
fresh seeded shuffle per epoch.  All arithmetic runs in the library's kernels
(aew_snapshots, aew_codec_train_step, aew_codec_encode_vectors, aew_codec_decode);
this module only schedules the calls and gathers minibatches.

    python -m paper_2304_04781_gb300.train --epochs 20 --out weights.npz
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import aewave, inputs


def field_columns(f: int) -> torch.Tensor:
    """Positions of field f (0:e, 1:vx, 2:vy, 3:vz) inside the 2048-vector (k = z*256 + f*64 + y*8 + x)."""
    return torch.cat([torch.arange(z * 256 + f * 64, z * 256 + f * 64 + 64) for z in range(8)])


def make_handle(shape, h=10.0, nt=1000, n_lat=64, nrec=64, f0=25.0) -> aewave.Solver:
    nz, ny, nx = shape
    rec = inputs.receiver_grid(nx, ny, nrec)
    # no history storage is needed for data generation / training
    return aewave.Solver(shape, h, nt, rec, storage="revolve", n_checkpoints=0, n_lat=n_lat,
                         f0=f0)


def block_scale(bmax: torch.Tensor) -> torch.Tensor:
    """Power-of-two scales s = 2^max(e, -100) of block maxima m 2^e, m in [0.5, 1)
    (0 for 0), as the library applies them."""
    _, e = torch.frexp(bmax)
    e = torch.clamp(e, min=-100)
    return torch.where(bmax > 0, torch.ldexp(torch.ones_like(bmax), e), torch.zeros_like(bmax))


def generate(solver: aewave.Solver, seeds, every: int = 10, h: float = 10.0,
             drop_zero: bool = True):
    """Algorithm 1 over several prior draws.  Returns (BF16 [N][2048] normalised vectors,
    FP32 [N][4] block maxima).  Vectors of blocks that are still entirely at rest (all four
    fields zero) encode and decode to zero whatever the weights, and are dropped."""
    per_seed = solver.nblocks * ((solver.nt - 1) // every)
    data = torch.empty((per_seed * len(seeds), 2048), device="cuda", dtype=torch.bfloat16)
    bmax = torch.empty((per_seed * len(seeds), 4), device="cuda")
    n = 0
    for s in seeds:
        c = torch.from_numpy(inputs.velocity_model(solver.shape, h, seed=s).astype(np.float32)).cuda()
        v, bm = solver.snapshots(c, every, per_seed, out=data[n:n + per_seed], with_scales=True)
        bmax[n:n + v.shape[0]] = bm
        n += v.shape[0]
    data, bmax = data[:n], bmax[:n]
    if drop_zero:
        keep = torch.nonzero(bmax.amax(dim=1) > 0).squeeze(1)
        data, bmax = data.index_select(0, keep), bmax.index_select(0, keep)
    return data, bmax


LOSSES = ("state", "strain", "strain-amplitude", "strain-energy")


def loss_weights(bmax: torch.Tensor, kind: str):
    """Per-vector, per-field weights [N][4] of the squared error (None for "state").

    state             every field of every vector alike (Table 2's plain error)
    strain            the strain outputs only (the adjoint decodes nothing else)
    strain-amplitude  strain only, each vector weighted by its block scale s_e
    strain-energy     strain only, weighted by s_e^2: the physical squared error
    Amplitude weights are divided by their mean over the data set."""
    if kind == "state":
        return None
    w = torch.zeros(bmax.shape, device=bmax.device, dtype=torch.float32)
    if kind == "strain":
        w[:, 0] = 1.0
        return w
    se = block_scale(bmax[:, 0].contiguous()).double()
    a = se if kind == "strain-amplitude" else se * se
    w[:, 0] = (a / a.mean()).float()
    return w


def train(solver: aewave.Solver, data: torch.Tensor, epochs: int = 20, batch: int = 512,
          lr0: float = 1e-3, halve_every: int = 5, seed: int = 0, log_every: int = 0,
          weights: torch.Tensor = None):
    """Train the handle's codec in place on `data` (weights: optional [N][4], see
    loss_weights); returns per-epoch mean losses (over about 16 sampled minibatches per
    epoch, each loss taken before its update)."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    N = data.shape[0]
    nb = N // batch
    hist = []
    for ep in range(epochs):
        lr = lr0 * 0.5 ** (ep // halve_every)
        perm = torch.randperm(N, device="cuda", generator=g)
        tot = 0.0
        cnt = 0
        every = log_every or max(1, nb // 16)
        for i in range(nb):
            idx = perm[i * batch:(i + 1) * batch]
            mb = data.index_select(0, idx)
            wb = None if weights is None else weights.index_select(0, idx)
            loss = solver.train_step(mb, lr, want_loss=(i % every == 0) or i == nb - 1,
                                     weights=wb)
            if loss is not None:
                tot += loss
                cnt += 1
        hist.append(tot / max(cnt, 1))
    return hist


def decoded_error(solver: aewave.Solver, data: torch.Tensor, bmax: torch.Tensor, chunk: int = 65536):
    """Relative L2 error of decode(encode(y)) over all vectors, per field and overall, in
    normalised units and in physical units (x = y * s_{b,f})."""
    num = torch.zeros(4, dtype=torch.float64, device="cuda")
    den = torch.zeros(4, dtype=torch.float64, device="cuda")
    pnum = torch.zeros(4, dtype=torch.float64, device="cuda")
    pden = torch.zeros(4, dtype=torch.float64, device="cuda")
    cols = [field_columns(f).cuda() for f in range(4)]
    scale = block_scale(bmax)
    for i in range(0, data.shape[0], chunk):
        y = data[i:i + chunk]
        yh = solver.codec_decode(solver.codec_encode_vectors(y))
        yf = y.float()
        for f in range(4):
            d = (yh[:, cols[f]] - yf[:, cols[f]]).double().pow(2).sum(1)
            r = yf[:, cols[f]].double().pow(2).sum(1)
            s2 = scale[i:i + chunk, f].double() ** 2
            num[f] += d.sum(); den[f] += r.sum()
            pnum[f] += (d * s2).sum(); pden[f] += (r * s2).sum()
    names = ["e", "vx", "vy", "vz"]
    out = {"normalised": {names[f]: float((num[f] / den[f]).sqrt()) for f in range(4)},
           "physical": {names[f]: float((pnum[f] / pden[f]).sqrt()) for f in range(4)}}
    out["normalised"]["all"] = float((num.sum() / den.sum()).sqrt())
    out["vectors"] = int(data.shape[0])
    return out


def weights_finite(W: dict) -> bool:
    return all(np.isfinite(np.asarray(v)).all() for v in W.values())


def save(W: dict, path: str):
    np.savez(path, **{k: np.asarray(v, np.float32) for k, v in W.items()})


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--shape", type=int, nargs=3, default=[128, 128, 128])
    p.add_argument("--nt", type=int, default=1000)
    p.add_argument("--every", type=int, default=10)
    p.add_argument("--seeds", type=int, nargs="*", default=list(range(100, 108)))
    p.add_argument("--holdout", type=int, default=200)
    p.add_argument("--epochs", type=int, default=20)
    p.add_argument("--batch", type=int, default=512)
    p.add_argument("--n-lat", type=int, default=64)
    p.add_argument("--init-seed", type=int, default=0)
    p.add_argument("--f0", type=float, default=25.0, help="Ricker peak frequency [Hz]")
    p.add_argument("--loss", default="state", choices=LOSSES,
                   help="weights of the squared error (see loss_weights)")
    p.add_argument("--out", default="")
    a = p.parse_args()
    shape = tuple(a.shape)
    solver = make_handle(shape, nt=a.nt, n_lat=a.n_lat, f0=a.f0)
    solver.codec_set(inputs.codec_init(seed=a.init_seed, n_lat=a.n_lat))
    t0 = time.time()
    data, bmax = generate(solver, a.seeds, a.every)
    nvec = data.shape[0]
    weights = loss_weights(bmax, a.loss)
    torch.cuda.synchronize()
    t1 = time.time()
    hist = train(solver, data, a.epochs, a.batch, weights=weights)
    torch.cuda.synchronize()
    t2 = time.time()
    del data
    hold, hsc = generate(solver, [a.holdout], a.every)
    err = decoded_error(solver, hold, hsc)
    W = solver.codec_get()
    res = {"vectors": int(nvec), "loss_kind": a.loss, "gen_s": t1 - t0, "train_s": t2 - t1, "epochs": a.epochs,
           "loss": hist, "holdout_decoded_error": err, "weights_finite": weights_finite(W)}
    print(json.dumps(res))
    if a.out:
        save(W, a.out)


if __name__ == "__main__":
    main()
