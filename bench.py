"""Benchmark: autoencoder-compressed adjoint gradients per hour at 256^3 x 2000 steps
(128 receivers, codec 2048 -> 512 -> 64, FP16 latents held in HBM), against binomial
recompute-checkpointing on the same GPU, plus the forward stencil's HBM bandwidth.

One step = one gradient of the misfit (forward solve with per-step encoding into the
latent store, residual and misfit, adjoint solve with per-step decoding and FP64
gradient accumulation).  Inputs: synthetic Gaussian-random-field velocity model, data
from a +5% bump model; the working set (~1 GB of fields per step) is far larger than
L2, so no explicit flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank computes its own independent gradient (its own velocity
model): weak scaling, no data-path collective; the timed region is bracketed by a
barrier and the maximum time over ranks is used.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gradients/hour at 256^3x2000 steps: AE vs checkpointing; stencil HBM GB/s"
# DRAM bytes (read + write) of one forward-step launch at 256^3, from an ncu capture of
# the current kernel (dram__bytes_read.sum + dram__bytes_write.sum); None once the
# kernel changes until it is captured again
FWD_TRAFFIC_256 = 586.19e6
SHAPE = (256, 256, 256)
NT = 2000
NREC = 128
H = 10.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--revolve-runs", type=int, default=2)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--shape", type=int, nargs=3, default=list(SHAPE))
    p.add_argument("--nt", type=int, default=NT)
    p.add_argument("--nrec", type=int, default=NREC)
    p.add_argument("--n-lat", type=int, default=64)
    p.add_argument("--weights", default="")
    p.add_argument("--accuracy", action="store_true",
                   help="instead of timing: AE gradient / GN-HVP errors against full storage "
                        "(or checkpointing with --ref revolve), decoded-state error")
    p.add_argument("--ref", default="full", choices=["full", "revolve"])
    p.add_argument("--hvps", type=int, default=1)
    p.add_argument("--f0", type=float, default=25.0,
                   help="accuracy mode: Ricker peak frequency [Hz] of the workload")
    p.add_argument("--err-hvps", type=int, default=0,
                   help="compare only the first k HVPs with the reference (0: all)")
    return p.parse_args()


def workload(shape, nt, nrec=NREC, n_lat=64):
    return {
        "workload": f"{shape[2]}x{shape[1]}x{shape[0]} grid, {nt} steps, {nrec} receivers; "
                    f"AE storage (8^3-node blocks x 4 fields = 2048 -> 512 -> {n_lat}, FP16 latents)",
        "grid": list(shape), "nt": nt, "receivers": nrec, "codec": f"2048-512(GELU)-{n_lat}, bf16 x bf16 -> f32",
        "l2": "inputs larger than L2 (per-step working set ~1 GB)",
        "storage": "AE latents in HBM; baseline binomial checkpointing with 20 state slots",
    }


# --------------------------------------------------------------------------- distributed
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, world: int, device=None) -> float:
    """Maximum of a float over all ranks (identity for one rank)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- CPU oracle
def cpu_sample(shape, nt, steps_in_sample=1):
    """Time the FP64 oracle on a bounded sample of the same workload: `steps_in_sample`
    forward steps (with the codec encode of each state), then as many adjoint steps
    (with the decode); scaled to gradients/hour for nt steps."""
    from oracle import codec as C
    from oracle import wave as W
    from paper_2304_04781_gb300 import inputs
    rec = inputs.receiver_grid(shape[2], shape[1], NREC)
    prob = W.Problem(shape=tuple(shape), h=H, nt=steps_in_sample, rec=rec)
    c = inputs.velocity_model(shape, H, seed=2)
    Wt = inputs.codec_init(seed=0)
    m = c * c
    z = np.zeros(shape)
    t0 = time.perf_counter()
    st = (z, z.copy(), z.copy(), z.copy())
    states = []
    for n in range(steps_in_sample):
        st = W.forward_step(prob, m, *st, -1.0)
        states.append(st)
    ehat = [C.roundtrip_e(Wt, s) for s in states]
    resid = np.zeros((steps_in_sample + 1, prob.nrec, 3))
    W.adjoint(prob, c, lambda n: ehat[n], resid)
    dt = time.perf_counter() - t0
    per_step = dt / steps_in_sample
    return 3600.0 / (per_step * nt), dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    shape, nt = tuple(args.shape), args.nt
    vals = []
    for i in range(args.warmup + args.steps):
        v, _ = cpu_sample(shape, nt)
        if i >= args.warmup:
            vals.append(v)
    v = float(np.mean(vals))
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "gradients/hour",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 3600e3 / v, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload(shape, nt),
        "cpu_baseline": {"value": v, "unit": "gradients/hour", "cores": cores, "kind": "oracle",
                         "sample": "per step: one FP64 forward step + encode/decode of its state + one adjoint step "
                                   "at the full grid, scaled to nt steps"},
        "e2e": {"value": v, "unit": "gradients/hour", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# --------------------------------------------------------------------------- GPU arm
def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def run_ours(args):
    import torch
    from paper_2304_04781_gb300 import aewave, inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    shape, nt = tuple(args.shape), args.nt
    nz, ny, nx = shape
    rec = inputs.receiver_grid(nx, ny, NREC)
    C = nx * ny * nz
    seed = 2 + rank
    c_np = inputs.velocity_model(shape, H, seed=seed).astype(np.float32)
    ctrue = inputs.bump_model(c_np.astype(np.float64), H).astype(np.float32)
    c = torch.from_numpy(c_np).cuda()
    Wt, trained = load_weights(args.weights or default_weights(64), 64)

    ae = aewave.Solver(shape, H, nt, rec, storage="ae")
    ae.codec_set(Wt)
    d_obs = ae.forward(torch.from_numpy(ctrue).cuda())
    g = torch.empty_like(c)
    stream = torch.cuda.current_stream()

    # ---- warm-up and timed AE gradients
    for _ in range(args.warmup):
        ae.gradient(c, d_obs, g)
    torch.cuda.synchronize()
    l0 = ae.stats()["kernel_launches"]
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            ae.gradient(c, d_obs, g)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1) / args.steps
    launches = ae.stats()["kernel_launches"] - l0
    ms_max = reduce_max(ms, world, torch.device("cuda", local))
    value = world * 3600e3 / ms_max

    # ---- Gauss-Newton Hessian-vector products reusing this gradient's latents
    dc = torch.from_numpy(inputs.direction(shape, H, seed=20).astype(np.float32)).cuda()
    hv = torch.empty_like(c)
    ae.hessvec(dc, hv)
    torch.cuda.synchronize()
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    for _ in range(args.steps):
        ae.hessvec(dc, hv)
    h1.record(stream)
    torch.cuda.synchronize()
    ae_hvp_ms = h0.elapsed_time(h1) / args.steps

    # ---- end to end through the public API with host buffers
    c_host = torch.from_numpy(c_np).pin_memory()
    d_host = d_obs.cpu().pin_memory()
    g_host = torch.empty(shape, dtype=torch.float32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        cd = c_host.cuda(non_blocking=True)
        dd = d_host.cuda(non_blocking=True)
        J, gg = ae.gradient(cd, dd)
        g_host.copy_(gg, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = reduce_max(e2e_s, world, torch.device("cuda", local))
    h2d = c_host.numel() * 4 + d_host.numel() * 4
    d2h = g_host.numel() * 4 + 8

    # ---- forward stencil kernel alone (nt back-to-back launches)
    aefwd = ae
    aefwd.forward(c)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    aefwd.forward(c)
    f1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = f0.elapsed_time(f1)
    step_s = fwd_ms / 1e3 / nt
    bytes_step = 36.0 * C
    stencil_gbs = bytes_step / step_s / 1e9
    peak, peak_kind = load_peaks()
    latent_bytes = int(ae.stats()["latent_bytes"])
    del ae
    torch.cuda.empty_cache()

    # ---- binomial checkpointing baseline (20 slots) on the same GPU
    rev = aewave.Solver(shape, H, nt, rec, storage="revolve", n_checkpoints=20)
    rev.gradient(c, d_obs, g)
    torch.cuda.synchronize()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(args.revolve_runs):
        rev.gradient(c, d_obs, g)
    r1.record(stream)
    torch.cuda.synchronize()
    rev_ms = r0.elapsed_time(r1) / args.revolve_runs
    rev_fwd = rev.stats()["forward_steps"]
    rev.hessvec(dc, hv)
    torch.cuda.synchronize()
    r0.record(stream)
    for _ in range(args.revolve_runs):
        rev.hessvec(dc, hv)
    r1.record(stream)
    torch.cuda.synchronize()
    rev_hvp_ms = r0.elapsed_time(r1) / args.revolve_runs
    rev_hvp_fwd = rev.stats()["hvp_forward_steps"]
    del rev
    torch.cuda.empty_cache()

    def time_gradient(solver):
        solver.gradient(c, d_obs, g)
        torch.cuda.synchronize()
        t0_, t1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0_.record(stream)
        for _ in range(args.revolve_runs):
            solver.gradient(c, d_obs, g)
        t1_.record(stream)
        torch.cuda.synchronize()
        return t0_.elapsed_time(t1_) / args.revolve_runs

    # ---- checkpointing with as many state slots as the latent store's bytes (4 FP32
    # fields per slot), and full storage of e^n where it fits: references, not the headline
    slots_eq = max(1, latent_bytes // (16 * C))
    req = aewave.Solver(shape, H, nt, rec, storage="revolve", n_checkpoints=slots_eq)
    req_ms = time_gradient(req)
    req_fwd = req.stats()["forward_steps"]
    del req
    torch.cuda.empty_cache()
    full = None
    hist = nt * C * 4
    if torch.cuda.mem_get_info()[0] > hist + 16 * C * 8:
        try:
            fs = aewave.Solver(shape, H, nt, rec, storage="full")
        except aewave.AewError as err:
            full = {"unavailable": str(err)}
        else:
            full_ms = time_gradient(fs)
            full = {"ms_per_gradient": full_ms, "gradients_per_hour": 3600e3 / full_ms,
                    "history_bytes": hist,
                    "note": "e^n of every step kept in HBM (no recomputation, no compression)"}
            del fs
            torch.cuda.empty_cache()
    else:
        full = {"unavailable": f"e^n history of {hist / 1e9:.1f} GB does not fit beside the rest"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, secs = cpu_sample(shape, nt)
        cpu = {"value": v, "unit": "gradients/hour", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one FP64 forward step + encode/decode + one adjoint step at the full grid "
                         f"({secs:.1f} s), scaled to {nt} steps"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "gradients/hour", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 stencil, bf16 codec", "data": "synthetic (GRF velocity, bump-model observations)",
            "config": dict(workload(shape, nt), codec_weights="trained" if trained else "random-init"),
            "roofline": {"kernel": "forward leapfrog step", "bound": "hbm", "achieved": stencil_gbs,
                         "peak": peak, "unit": "GB/s", "frac": stencil_gbs / peak,
                         "peak_kind": f"{peak_kind} copy bandwidth",
                         "traffic": FWD_TRAFFIC_256 if tuple(shape) == SHAPE else None,
                         "bytes_per_launch": bytes_step},
            "stencil": {"cell_updates_per_s": C / step_s, "gbs": stencil_gbs,
                        "frac_of_8tbs": stencil_gbs / 8000.0},
            "revolve": {"gradients_per_hour": 3600e3 / rev_ms, "ms_per_gradient": rev_ms,
                        "forward_steps": rev_fwd, "slots": 20},
            "speedup_vs_revolve": rev_ms / ms_max,
            "revolve_equal_memory": {"slots": slots_eq, "ms_per_gradient": req_ms,
                                     "gradients_per_hour": 3600e3 / req_ms, "forward_steps": req_fwd,
                                     "latent_bytes": latent_bytes},
            "full_storage": full,
            "hvp": {"ae_ms": ae_hvp_ms, "revolve_ms": rev_hvp_ms, "speedup_vs_revolve": rev_hvp_ms / ae_hvp_ms,
                    "ae_hvps_per_hour": 3600e3 / ae_hvp_ms, "revolve_forward_steps": rev_hvp_fwd,
                    "note": "Gauss-Newton HVP reusing the gradient's latents (AE) vs recomputing "
                            "states from 20 checkpoint slots"},
            "e2e": {"value": world * 3600.0 / e2e_s, "unit": "gradients/hour",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def default_weights(n_lat: int) -> str:
    return os.path.join(ROOT, "paper_2304_04781_gb300", "weights", f"codec_{n_lat}.npz")


def load_weights(path: str, n_lat: int):
    from paper_2304_04781_gb300 import inputs
    W = inputs.codec_init(seed=0, n_lat=n_lat)
    if path and os.path.exists(path):
        z = np.load(path)
        return {k: z[k] for k in W}, True
    return W, False


def run_accuracy(args):
    """Errors of the compressed gradient / GN-HVP against an uncompressed reference on
    the same GPU, decoded-state error, adjoint identity and checkpointing equality at the
    full size.  Prints one JSON line."""
    import torch
    from paper_2304_04781_gb300 import aewave, inputs, train
    shape, nt = tuple(args.shape), args.nt
    nz, ny, nx = shape
    rec = inputs.receiver_grid(nx, ny, args.nrec)
    W, trained = load_weights(args.weights or default_weights(args.n_lat), args.n_lat)
    c_np = inputs.velocity_model(shape, H, seed=2).astype(np.float32)
    c = torch.from_numpy(c_np).cuda()
    ctrue = torch.from_numpy(inputs.bump_model(c_np.astype(np.float64), H).astype(np.float32)).cuda()
    dirs = [torch.from_numpy(inputs.direction(shape, H, seed=(20 if args.hvps == 1 else 30) + k)
                             .astype(np.float32)).cuda() for k in range(args.hvps)]
    out = {"config": dict(workload(shape, nt, args.nrec, args.n_lat), f0_hz=args.f0), "codec_weights": "trained" if trained else "random-init",
           "n_lat": args.n_lat, "reference": args.ref}
    def ev():
        return torch.cuda.Event(enable_timing=True)

    ae = aewave.Solver(shape, H, nt, rec, storage="ae", n_lat=args.n_lat, f0=args.f0)
    ae.codec_set(W)
    d_obs = ae.forward(ctrue)
    a, b = ev(), ev(); a.record()
    J_ae, g_ae = ae.gradient(c, d_obs)
    b.record(); torch.cuda.synchronize()
    out["ae_gradient_ms"] = a.elapsed_time(b)
    H_ae, t_hvp = [], []
    for dc in dirs:
        a, b = ev(), ev(); a.record()
        H_ae.append(ae.hessvec(dc).cpu())
        b.record(); torch.cuda.synchronize()
        t_hvp.append(a.elapsed_time(b))
    out["ae_hvp_ms"] = float(np.mean(t_hvp))
    st = ae.stats()
    free, total = torch.cuda.mem_get_info()
    out["ae_memory"] = {"device_bytes": st["device_bytes"], "latent_bytes": st["latent_bytes"],
                        "torch_peak_bytes": int(torch.cuda.max_memory_allocated()),
                        "device_used_bytes": int(total - free)}
    g_ae = g_ae.cpu()
    del ae
    torch.cuda.empty_cache()

    if args.ref == "full":
        ref = aewave.Solver(shape, H, nt, rec, storage="full", f0=args.f0)
    else:
        ref = aewave.Solver(shape, H, nt, rec, storage="revolve", n_checkpoints=20, f0=args.f0)
    a, b = ev(), ev(); a.record()
    J_ref, g_ref = ref.gradient(c, d_obs)
    b.record(); torch.cuda.synchronize()
    out["ref_gradient_ms"] = a.elapsed_time(b)
    rel = lambda x, y: float(torch.linalg.vector_norm((x - y).double()) / torch.linalg.vector_norm(y.double()))
    out["misfit"] = {"ae": J_ae, "ref": J_ref}
    out["gradient_rel_err"] = rel(g_ae, g_ref.cpu())
    errs, t_ref = [], []
    ncmp = args.err_hvps if args.err_hvps > 0 else len(dirs)
    for k, dc in enumerate(dirs[:ncmp]):
        a, b = ev(), ev(); a.record()
        Hr = ref.hessvec(dc).cpu()
        b.record(); torch.cuda.synchronize()
        t_ref.append(a.elapsed_time(b))
        errs.append(rel(H_ae[k], Hr))
    out["hvp_rel_err"] = errs
    out["hvps_timed"] = len(dirs)
    out["hvps_compared"] = ncmp
    out["ref_hvp_ms"] = float(np.mean(t_ref))
    # adjoint identity at the full size: <J dc, r> = <dc, J^T r>, for a random residual
    # (|<J dc, r>| is then small against |J dc| |r|: the cancellation is reported) and
    # for the smooth residual r = J dc2 of a second direction
    d = ref.forward(c)
    ref.gradient(c, d_obs)      # a forward history at c for the Jacobian-vector products
    Jdc = ref.jvp(dirs[0])
    dc2 = torch.from_numpy(inputs.direction(shape, H, seed=99).astype(np.float32)).cuda()
    Jdc2 = ref.jvp(dc2)
    ident = {}
    for name, r in [("random", None), ("smooth", Jdc2)]:
        if r is None:
            r = torch.randn(d.shape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(5)) * d.abs().max()
            r[0] = 0
        _, JTr = ref.gradient(c, (d - r).contiguous())
        lhs, rhs = aewave.dot(Jdc, r), aewave.dot(dirs[0], JTr)
        nrm = float(torch.linalg.vector_norm(Jdc.double()) * torch.linalg.vector_norm(r.double()))
        ident[name] = {"lhs": lhs, "rhs": rhs, "rel": abs(lhs - rhs) / abs(lhs),
                       "cos": abs(lhs) / nrm, "rel_to_norms": abs(lhs - rhs) / nrm}
    out["adjoint_identity"] = ident
    out["adjoint_identity_rel"] = ident["smooth"]["rel"]
    out["ref_memory_bytes"] = ref.stats()["device_bytes"]
    del ref
    torch.cuda.empty_cache()

    # decoded-state error on states of this run (every 50th step)
    tr = train.make_handle(shape, nt=nt, n_lat=args.n_lat, f0=args.f0)
    tr.codec_set(W)
    every = max(1, nt // 40)
    snaps, sc = train.generate(tr, [2], every)
    out["decoded_state_error"] = train.decoded_error(tr, snaps, sc)
    out["decoded_state_sample"] = f"states n = {every}, {2 * every}, ... of this run, all blocks"
    print(json.dumps(out))


def main():
    args = parse()
    if args.accuracy:
        run_accuracy(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
