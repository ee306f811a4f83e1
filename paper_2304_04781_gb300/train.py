"""Codec training pipeline: data generation by Algorithm 1 and training per Table 2.

Every step runs in the library; this module only schedules the calls:

1. data (aew_snapshots): for each prior draw of the wave speed (a seeded Gaussian
   random field), the forward solve's snapshots as normalised BF16 vectors resident in
   HBM, with the maxima that fix their scales.  Space codec: every `every`-th state,
   cut into 8x8x8-node blocks of the four fields (each field of each block divided by
   its power-of-two scale).  Time codec: every `every`-th complete 16-step window of
   the strain of 2x8x8-node blocks (each vector divided by its power-of-two scale);
2. initialisation: Glorot-uniform weights (seeded), or (aew_codec_init_pca) the optimal
   rank-n_lat code of the data under the chosen loss (Sec. 1: a linear autoencoder
   learns the principal subspace), written into the GELU layers;
3. training (aew_codec_train): Table 2 -- LAMB, learning rate 1e-3 halved every 5
   epochs, batch 512, a fresh seeded shuffle per epoch -- for --epochs passes;
4. evaluation (aew_codec_eval): decoded error on a held-out draw.

    python -m paper_2304_04781_gb300.train --codec time --init pca --epochs 0 \\
        --loss strain-energy --out weights/codec_time_512.npz
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import aewave, inputs

LOSSES = tuple(aewave.LOSSES)


def make_handle(shape, codec="space", n_lat=None, h=10.0, nt=1000, nrec=64,
                f0=25.0, norm="pow2", act="gelu", beta=0.0) -> aewave.Solver:
    nz, ny, nx = shape
    rec = inputs.receiver_grid(nx, ny, nrec)
    # no history storage is needed for data generation / training
    return aewave.Solver(shape, h, nt, rec, storage="revolve", n_checkpoints=0, n_lat=n_lat,
                         f0=f0, codec=codec, norm=norm, act=act, beta=beta)


def per_draw(solver: aewave.Solver, every: int) -> int:
    """Vectors one forward solve contributes to the data set."""
    if solver.codec == "time":
        complete = solver.nt // aewave.WINDOW
        return solver.nvec * ((complete - 1) // every + 1 if complete > 0 else 0)
    return solver.nblocks * ((solver.nt - 1) // every)


def generate(solver: aewave.Solver, seeds, every: int, h: float = 10.0,
             drop_zero: bool = True):
    """Algorithm 1 over several prior draws.  Returns (BF16 [N][2048] normalised vectors,
    FP32 maxima: [N][4] block maxima (space codec), [N] vector maxima (time codec), or
    [N][2] offsets and ranges (min-max normalisation)).  With the power-of-two scales,
    vectors that are still entirely at rest (maxima 0) encode and decode to zero whatever
    the weights, and are dropped."""
    k = per_draw(solver, every)
    data = torch.empty((k * len(seeds), 2048), device="cuda", dtype=torch.bfloat16)
    if solver.codec == "time":
        mshape = (k * len(seeds), 2) if solver.norm == "minmax" else (k * len(seeds),)
    else:
        mshape = (k * len(seeds), 4)
    maxima = torch.empty(mshape, device="cuda")
    n = 0
    for s in seeds:
        c = torch.from_numpy(inputs.velocity_model(solver.shape, h, seed=s).astype(np.float32)).cuda()
        v, m = solver.snapshots(c, every, k, out=data[n:n + k], with_scales=True)
        maxima[n:n + v.shape[0]] = m
        n += v.shape[0]
    data, maxima = data[:n], maxima[:n]
    if drop_zero and solver.norm != "minmax":
        live = maxima if maxima.dim() == 1 else maxima.amax(dim=1)
        keep = torch.nonzero(live > 0).squeeze(1)
        data, maxima = data.index_select(0, keep), maxima.index_select(0, keep)
    return data, maxima


def weights_finite(W: dict) -> bool:
    return all(np.isfinite(np.asarray(v)).all() for v in W.values())


def save(W: dict, path: str, meta: dict):
    np.savez(path, meta=np.array(json.dumps(meta)),
             **{k: np.asarray(v, np.float32) for k, v in W.items()})


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--codec", default="space", choices=("space", "time"))
    p.add_argument("--shape", type=int, nargs=3, default=[128, 128, 128])
    p.add_argument("--nt", type=int, default=1000)
    p.add_argument("--every", type=int, default=0,
                   help="states (space codec, default 10) or windows (time codec, default 1)")
    p.add_argument("--seeds", type=int, nargs="*", default=list(range(100, 108)))
    p.add_argument("--holdout", type=int, default=200)
    p.add_argument("--init", default="glorot", choices=("glorot", "pca"))
    p.add_argument("--epochs", type=int, default=20)
    p.add_argument("--batch", type=int, default=512)
    p.add_argument("--lr0", type=float, default=1e-3)
    p.add_argument("--halve-every", type=int, default=5)
    p.add_argument("--n-lat", type=int, default=0)
    p.add_argument("--init-seed", type=int, default=0)
    p.add_argument("--seed", type=int, default=0, help="shuffle seed")
    p.add_argument("--f0", type=float, default=25.0, help="Ricker peak frequency [Hz]")
    p.add_argument("--loss", default="state", choices=LOSSES)
    p.add_argument("--norm", default="pow2", choices=("pow2", "minmax"),
                   help="time codec: power-of-two vector scales, or the paper's min-max")
    p.add_argument("--act", default="gelu", choices=("gelu", "elu"))
    p.add_argument("--beta", type=float, default=0.0, help="min-max range floor (0: 1e-7)")
    p.add_argument("--out", default="")
    a = p.parse_args()
    shape = tuple(a.shape)
    n_lat = a.n_lat or (512 if a.codec == "time" else 64)
    every = a.every or (1 if a.codec == "time" else 10)
    solver = make_handle(shape, a.codec, n_lat, nt=a.nt, f0=a.f0, norm=a.norm, act=a.act,
                         beta=a.beta)
    solver.codec_set(inputs.codec_init(seed=a.init_seed, n_hid=solver.n_hid, n_lat=n_lat))
    t0 = time.time()
    data, maxima = generate(solver, a.seeds, every)
    torch.cuda.synchronize()
    t1 = time.time()
    res = {"codec": a.codec, "norm": a.norm, "act": a.act, "beta": a.beta,
           "n_lat": n_lat, "n_hid": solver.n_hid, "vectors": int(data.shape[0]),
           "loss_kind": a.loss, "init": a.init, "f0_hz": a.f0, "every": every,
           "train_shape": list(shape), "train_nt": a.nt, "seeds": list(a.seeds)}
    if a.init == "pca":
        ev = solver.codec_init_pca(data, maxima, a.loss)
        res["pca_tail_rel"] = float(np.sqrt(max(ev[n_lat:].sum(), 0.0) / max(ev.sum(), 1e-300)))
    t2 = time.time()
    res["train_loss"] = solver.codec_train(data, maxima, a.epochs, a.batch, a.lr0, a.halve_every,
                                           a.loss, a.seed) if a.epochs > 0 else []
    torch.cuda.synchronize()
    t3 = time.time()
    res["train_decoded_error"] = solver.codec_eval(data, maxima)
    del data, maxima
    hold, hm = generate(solver, [a.holdout], every)
    res["holdout_decoded_error"] = solver.codec_eval(hold, hm)
    W = solver.codec_get()
    res.update({"gen_s": t1 - t0, "init_s": t2 - t1, "train_s": t3 - t2, "epochs": a.epochs,
                "weights_finite": weights_finite(W)})
    print(json.dumps(res))
    if a.out:
        save(W, a.out, res)


if __name__ == "__main__":
    main()
