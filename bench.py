"""Benchmark: autoencoder-compressed adjoint gradients per hour at 256^3 x 2000 steps
(128 receivers, FP16 latents held in HBM), against binomial recompute-checkpointing and
full storage on the same GPU, with the accuracy of the compressed gradient and GN-HVP
and the hot-path kernels' rooflines.

One step = one gradient of the misfit (forward solve with the history compressed into
the latent store, residual and misfit, adjoint solve decoding it, FP64 gradient
accumulation).  The default codec compresses in time (Sec. 3.2): the strain of each
2x8x8-node block over 16 steps, 2048 -> 1024 (GELU) -> 512 FP16 latents, 16.8 GB at
256^3 x 2000 (--codec space: the 8x8x8-node, 4-field codec 2048 -> 512 -> 64).
Inputs: synthetic Gaussian-random-field velocity model, data from a +5% bump model;
the working set (~1 GB of fields per step) is far larger than L2, so no explicit flush
is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own shot (source position) of the same model and
one all-reduce sums the gradients (and the HVPs): the multi-shot gradient, weak scaling
(one shot per GPU); the timed region is bracketed by a barrier and the maximum time over
ranks is used.  At one GPU the single shot is the centre source.
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
# DRAM bytes (read + write) of one adjoint-step launch at 256^3, from an ncu capture of
# the current kernel (dram__bytes_read.sum + dram__bytes_write.sum, a window-middle step
# without the FP64 flush); to be set to None when the kernel changes until it is
# captured again
ADJ_TRAFFIC_256 = 701.6e6     # FP32 e^n (full storage / checkpointing)
ADJ16_TRAFFIC_256 = 665.5e6   # BF16 e^n (the time codec's adjoint sweeps)
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
    p.add_argument("--codec", default="time", choices=["time", "space"])
    p.add_argument("--n-lat", type=int, default=0, help="latent width (default 512 time, 64 space)")
    p.add_argument("--weights", default="")
    p.add_argument("--no-accuracy", action="store_true",
                   help="skip the accuracy block of the timed run (errors against full storage)")
    p.add_argument("--norm", default="pow2", choices=["pow2", "minmax"],
                   help="time codec normalisation (accuracy / kernel modes): power of two, or "
                        "the paper's min-max")
    p.add_argument("--act", default="gelu", choices=["gelu", "elu"])
    p.add_argument("--beta", type=float, default=0.0, help="min-max range floor (0: 1e-7)")
    p.add_argument("--accuracy", action="store_true",
                   help="instead of timing: AE gradient / GN-HVP errors against full storage "
                        "(or checkpointing with --ref revolve), decoded-state error")
    p.add_argument("--ref", default="full", choices=["full", "revolve"])
    p.add_argument("--hvps", type=int, default=1)
    p.add_argument("--f0", type=float, default=25.0,
                   help="accuracy mode: Ricker peak frequency [Hz] of the workload")
    p.add_argument("--err-hvps", type=int, default=0,
                   help="compare only the first k HVPs with the reference (0: all)")
    p.add_argument("--kernel", default="",
                   choices=["", "forward", "forward_pack", "adjoint", "incremental",
                            "encode_window", "decode_window", "adjoint_bf16",
                            "decode_window_bf16", "incremental_bf16", "decode_state"],
                   help="instead of the benchmark: time one hot-path kernel alone "
                        "(aew_profile_steps) on an AE handle of --shape, for profiling")
    p.add_argument("--launches", type=int, default=16)
    p.add_argument("--map", action="store_true",
                   help="MAP estimation (Newton-CG, BiLaplacian prior) and DIAS at the workload "
                        "size with the compressed history against full storage")
    p.add_argument("--theta", type=float, default=6400.0, help="prior theta [m^2]")
    p.add_argument("--prior-std", type=float, default=30.0, help="prior sample std [m/s]")
    p.add_argument("--noise-rel", type=float, default=0.01,
                   help="noise std relative to the rms of the observed data")
    p.add_argument("--newton-iters", type=int, default=3)
    p.add_argument("--cg-max", type=int, default=10)
    p.add_argument("--dias-samples", type=int, default=30)
    p.add_argument("--dias-rank", type=int, default=5)
    p.add_argument("--dias-iters", type=int, default=2)
    p.add_argument("--map-ref", default="full", choices=["full", "revolve", "none"],
                   help="MAP reference: full storage, 20-slot checkpointing (exact states "
                        "where full storage does not fit) or none")
    p.add_argument("--map-cmax", type=float, default=3000.0,
                   help="MAP / DIAS: the speed that sets dt (stability bound 1.155 x this)")
    p.add_argument("--src-sigma", type=float, default=50.0,
                   help="MAP / DIAS: source smoothing in space [m] (Sec. 4.1's box problem: 50 m)")
    p.add_argument("--train-step", action="store_true",
                   help="time codec training steps (Table 2's batch) alone")
    p.add_argument("--batch", type=int, default=512)
    return p.parse_args()


def codec_desc(codec: str, n_lat: int):
    if codec == "time":
        return (f"compression in time: strain of 2x8x8-node blocks x 16 steps = 2048 -> "
                f"{2 * n_lat} (GELU) -> {n_lat} FP16 latents", f"2048-{2 * n_lat}(GELU)-{n_lat}")
    return (f"compression in space: 8^3-node blocks x 4 fields = 2048 -> 512 (GELU) -> {n_lat} "
            f"FP16 latents", f"2048-512(GELU)-{n_lat}")


def workload(shape, nt, nrec=NREC, n_lat=512, codec="time"):
    desc, arch = codec_desc(codec, n_lat)
    return {
        "workload": f"{shape[2]}x{shape[1]}x{shape[0]} grid, {nt} steps, {nrec} receivers; "
                    f"AE storage ({desc})",
        "grid": list(shape), "nt": nt, "receivers": nrec,
        "codec": f"{arch}, bf16 x bf16 -> f32", "codec_kind": codec,
        "l2": "inputs larger than L2 (per-step working set ~1 GB)",
        "storage": "AE latents in HBM; baseline binomial checkpointing with 20 state slots",
    }


def nlat_of(args):
    return args.n_lat or (512 if args.codec == "time" else 64)


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
        """Median SM clock, the largest maximum clock reported, and the throttle reasons
        seen Active; a row counts only if every column it is read for parses."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                clk, cmax = float(r[1]), float(r[2])
                act = [r[5 + k].lower().startswith("active") for k in range(len(names))]
            except Exception:
                continue
            sm.append(clk)
            mx.append(cmax)
            reasons.update(nm for nm, a in zip(names, act) if a)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- CPU oracle
def cpu_sample(shape, nt, codec="time"):
    """Time the FP64 oracle on a bounded sample of the same workload, one step's share:
    one forward step, the codec work of one step, one adjoint step; scaled to
    gradients/hour for nt steps.  The codec work of a step is, for the time codec, the
    encode and decode of a sixteenth of a window's vectors (one window holds 16 steps),
    and for the space codec the encode and decode of the step's state.  Returns
    (gradients/hour, seconds, description)."""
    from oracle import codec as C
    from oracle import wave as W
    from paper_2304_04781_gb300 import inputs
    nz, ny, nx = shape
    rec = inputs.receiver_grid(nx, ny, NREC)
    prob = W.Problem(shape=tuple(shape), h=H, nt=1, rec=rec)
    c = inputs.velocity_model(shape, H, seed=2)
    m = c * c
    z = np.zeros(shape)
    if codec == "time":
        Wt = inputs.codec_init(seed=0, n_hid=1024, n_lat=512)
        nvec = (nx // 8) * (ny // 8) * (nz // 2)
        Y = np.random.default_rng(0).uniform(-1.0, 1.0, (max(nvec // 16, 1), 2048))
    else:
        Wt = inputs.codec_init(seed=0)
    t0 = time.perf_counter()
    st = W.forward_step(prob, m, z, z.copy(), z.copy(), z.copy(), -1.0)
    if codec == "time":
        C.decode(Wt, C.encode(Wt, Y))
        e_hat = st[0]
    else:
        e_hat = C.roundtrip_e(Wt, st)
    W.adjoint(prob, c, lambda n: e_hat, np.zeros((2, prob.nrec, 3)))
    dt = time.perf_counter() - t0
    what = ("one FP64 forward step + encode/decode of 1/16 of a window's vectors + one adjoint "
            "step" if codec == "time" else
            "one FP64 forward step + encode/decode of its state + one adjoint step")
    return 3600.0 / (dt * nt), dt, f"{what} at the full grid ({dt:.1f} s), scaled to {nt} steps"


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    shape, nt = tuple(args.shape), args.nt
    vals = []
    for i in range(args.warmup + args.steps):
        v, _, what = cpu_sample(shape, nt, args.codec)
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
                         "sample": what},
        "e2e": {"value": v, "unit": "gradients/hour", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# --------------------------------------------------------------------------- GPU arm
def load_peaks():
    """(HBM copy GB/s, BF16 TFLOP/s burst, sustained, kind) from MEASURED_PEAKS.json."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return (float(p["hbm_gbs"]), float(p["bf16_tflops"]), float(p["bf16_tflops_sustained"]),
                "measured")
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


# algorithmic bytes per node of the stencil kernels (FP32 fields; W = 8 steps per FP64
# flush of the gradient accumulator)
BYTES_PER_NODE = {
    "forward": 36.0,        # read e, m, vx, vy, vz; write e, vx, vy, vz
    "forward_pack": 38.0,   # + the output strain as BF16 into its window slot
    "adjoint": 50.0,        # read mu, lam (3), m, e^n, FP32 window acc; write mu, lam, acc;
                            # + 16 B FP64 read-modify-write / 8
    "adjoint_bf16": 48.0,   # the same with e^n read as BF16 (the time codec's sweeps)
    "incremental": 44.0,    # forward + dm, e^n
    "incremental_bf16": 42.0,   # the same with e^n read as BF16 (the time codec's GN-HVP)
}


def codec_flops_per_window(nvec: int, n_lat: int, n_hid: int) -> dict:
    """Dense flops of one window's encoder (2048 -> n_hid -> n_lat) and decoder."""
    enc = 2.0 * nvec * (2048 * n_hid + n_hid * n_lat)
    dec = 2.0 * nvec * (n_lat * n_hid + n_hid * 2048)
    return {"encode_window": enc, "decode_window": dec}


def run_ours(args):
    import torch
    from paper_2304_04781_gb300 import aewave, inputs, multishot

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    shape, nt = tuple(args.shape), args.nt
    nz, ny, nx = shape
    n_lat = nlat_of(args)
    rec = inputs.receiver_grid(nx, ny, NREC)
    src = inputs.source_grid(nx, ny, nz, world)[rank]
    C = nx * ny * nz
    seed = 2
    c_np = inputs.velocity_model(shape, H, seed=seed).astype(np.float32)
    ctrue = inputs.bump_model(c_np.astype(np.float64), H).astype(np.float32)
    c = torch.from_numpy(c_np).cuda()
    wpath = args.weights or default_weights(args.codec, n_lat)
    Wt, trained = load_weights(wpath, args.codec, n_lat)
    hbm_peak, tf_peak, tf_sust, peak_kind = load_peaks()

    ae = aewave.Solver(shape, H, nt, rec, storage="ae", codec=args.codec, n_lat=n_lat, src=src)
    ae.codec_set(Wt)
    d_obs = ae.forward(torch.from_numpy(ctrue).cuda())
    g = torch.empty_like(c)
    stream = torch.cuda.current_stream()

    def shots(solver):      # this rank's shot, summed over the ranks' shots
        return multishot.multishot_gradient(lambda: solver.gradient(c, d_obs, g))

    # ---- warm-up and timed AE gradients
    for _ in range(args.warmup):
        shots(ae)
    torch.cuda.synchronize()
    l0 = ae.stats()["kernel_launches"]
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            shots(ae)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1) / args.steps
    launches = ae.stats()["kernel_launches"] - l0
    ms_max = reduce_max(ms, world, torch.device("cuda", local))
    value = world * 3600e3 / ms_max
    g_ae = g.clone()

    # ---- Gauss-Newton Hessian-vector products reusing this gradient's latents
    dc = torch.from_numpy(inputs.direction(shape, H, seed=20).astype(np.float32)).cuda()
    hv = torch.empty_like(c)

    def hv_shots(solver):
        return multishot.multishot_hessvec(lambda: solver.hessvec(dc, hv))

    hv_shots(ae)
    torch.cuda.synchronize()
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    for _ in range(args.steps):
        hv_shots(ae)
    h1.record(stream)
    torch.cuda.synchronize()
    ae_hvp_ms = h0.elapsed_time(h1) / args.steps
    hv_ae = hv.clone()

    # ---- full Newton HVPs (second-order terms; the incremental strain compressed too)
    hvf_ae, ae_hvpf_ms = None, None
    if args.codec == "time":
        hvf = torch.empty_like(c)
        multishot.multishot_hessvec(lambda: ae.hessvec_full(dc, hvf))
        torch.cuda.synchronize()
        h0.record(stream)
        for _ in range(max(1, args.steps // 2)):
            multishot.multishot_hessvec(lambda: ae.hessvec_full(dc, hvf))
        h1.record(stream)
        torch.cuda.synchronize()
        ae_hvpf_ms = h0.elapsed_time(h1) / max(1, args.steps // 2)
        hvf_ae = hvf.clone()

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
        J, gg = multishot.multishot_gradient(lambda: ae.gradient(cd, dd))
        g_host.copy_(gg, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = reduce_max(e2e_s, world, torch.device("cuda", local))
    h2d = c_host.numel() * 4 + d_host.numel() * 4
    d2h = g_host.numel() * 4 + 8
    latent_bytes = int(ae.stats()["latent_bytes"])

    # ---- decoded-state error of this run's windows / states (the codec as trained)
    decoded = None
    if not args.no_accuracy:
        every = 8 if args.codec == "time" else max(1, nt // 40)
        complete = nt // aewave.WINDOW
        k = (ae.nvec * ((complete - 1) // every + 1) if complete > 0 else 0) \
            if args.codec == "time" else ae.nblocks * ((nt - 1) // every)
        if k > 0:    # (a run shorter than one window has no complete window to sample)
            vec, mx = ae.snapshots(c, every, k, with_scales=True)
            decoded = ae.codec_eval(vec, mx)
            decoded["sample"] = (f"every {every}th {'16-step window' if args.codec == 'time' else 'state'} "
                                 f"of this run, all vectors")
            del vec, mx
            torch.cuda.empty_cache()

    # ---- the hot-path kernels alone (CUDA events around back-to-back launches)
    nprof = min(nt, 200)
    kernels = {}
    kinds = ["forward", "adjoint", "incremental"] + (["forward_pack", "adjoint_bf16",
                                                      "incremental_bf16"]
                                                     if args.codec == "time" else [])
    for kind in kinds:
        kms = ae.profile(c, kind, nprof)
        b = BYTES_PER_NODE[kind] * C
        kernels[kind] = {"ms_per_launch": kms, "bytes_per_launch": b, "bytes_per_node": BYTES_PER_NODE[kind],
                         "achieved_gbs": b / kms / 1e6, "frac_of_hbm": b / kms / 1e6 / hbm_peak}
    if args.codec == "time":
        fl = codec_flops_per_window(ae.nvec, n_lat, ae.n_hid)
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        share = (sms // 2) / sms      # the codec GEMMs' CTA cap beside a stencil step
        for kind, prof in (("encode_window", "encode_window"), ("decode_window", "decode_window_bf16")):
            kms = ae.profile(c, prof, 8)
            tf = fl[kind] / kms / 1e9
            kernels[kind] = {"ms_per_launch": kms, "flops_per_launch": fl[kind],
                             "achieved_tflops": tf, "ctas": sms // 2,
                             "frac_of_bf16_burst_share": tf / (tf_peak * share),
                             "note": f"both layers of one window (two tcgen05 GEMMs on SM pairs) "
                                     f"on {sms // 2} CTAs, the cap they run with beside the "
                                     f"stencil; frac against that share of the measured peak"
                                     + ("; the decoder writes BF16 strain, as for the adjoint "
                                        "sweeps" if kind == "decode_window" else "")}
    del ae
    torch.cuda.empty_cache()

    # ---- binomial checkpointing baseline (20 slots) on the same GPU
    rev = aewave.Solver(shape, H, nt, rec, storage="revolve", n_checkpoints=20, src=src)
    shots(rev)
    torch.cuda.synchronize()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(args.revolve_runs):
        shots(rev)
    r1.record(stream)
    torch.cuda.synchronize()
    rev_ms = r0.elapsed_time(r1) / args.revolve_runs
    rev_fwd = rev.stats()["forward_steps"]
    g_exact = g.clone()        # checkpointing recomputes the exact states (= full storage)
    hv_shots(rev)
    torch.cuda.synchronize()
    r0.record(stream)
    for _ in range(args.revolve_runs):
        hv_shots(rev)
    r1.record(stream)
    torch.cuda.synchronize()
    rev_hvp_ms = r0.elapsed_time(r1) / args.revolve_runs
    rev_hvp_fwd = rev.stats()["hvp_forward_steps"]
    hv_exact = hv.clone()
    del rev
    torch.cuda.empty_cache()

    def time_gradient(solver):
        shots(solver)
        torch.cuda.synchronize()
        t0_, t1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0_.record(stream)
        for _ in range(args.revolve_runs):
            shots(solver)
        t1_.record(stream)
        torch.cuda.synchronize()
        return t0_.elapsed_time(t1_) / args.revolve_runs

    # ---- checkpointing with as many state slots as the latent store's bytes (4 FP32
    # fields per slot), and full storage of e^n where it fits: references, not the headline
    slots_eq = max(1, latent_bytes // (16 * C))
    req = aewave.Solver(shape, H, nt, rec, storage="revolve", n_checkpoints=slots_eq, src=src)
    req_ms = time_gradient(req)
    req_fwd = req.stats()["forward_steps"]
    del req
    torch.cuda.empty_cache()
    full = None
    hvf_exact = "full storage unavailable"
    hist = nt * C * 4
    if torch.cuda.mem_get_info()[0] > hist + 16 * C * 8:
        try:
            fs = aewave.Solver(shape, H, nt, rec, storage="full", src=src)
        except aewave.AewError as err:
            full = {"unavailable": str(err)}
        else:
            full_ms = time_gradient(fs)
            full = {"ms_per_gradient": full_ms, "gradients_per_hour": 3600e3 / full_ms,
                    "history_bytes": hist,
                    "note": "e^n of every step kept in HBM (no recomputation, no compression)"}
            g_exact = g.clone()
            hv_shots(fs)
            hv_exact = hv.clone()
            if hvf_ae is not None:
                try:      # needs a second e^n-sized history (the incremental strain)
                    multishot.multishot_hessvec(lambda: fs.hessvec_full(dc, hv))
                    hvf_exact = hv.clone()
                except aewave.AewError as err:
                    hvf_exact = str(err)
            del fs
            torch.cuda.empty_cache()
    else:
        full = {"unavailable": f"e^n history of {hist / 1e9:.1f} GB does not fit beside the rest"}

    rel = lambda x, y: float(torch.linalg.vector_norm((x - y).double()) / torch.linalg.vector_norm(y.double()))
    accuracy = {
        "gradient_rel_err": rel(g_ae, g_exact), "hvp_rel_err": rel(hv_ae, hv_exact),
        "reference": "full storage of e^n" if "ms_per_gradient" in (full or {}) else
                     "20-slot checkpointing (bitwise equal to full storage)",
        "decoded_strain_rel_err": None if decoded is None else
            {"normalised": decoded["normalised"]["e"], "physical": decoded["physical"]["e"],
             "vectors": decoded["vectors"], "sample": decoded["sample"]},
        "codec_weights": os.path.relpath(wpath, ROOT) if trained else "random-init",
        "target": "<= 1e-2 relative to the full-storage gradient / HVP",
    }
    if hvf_ae is not None:
        accuracy["hvp_full_newton_rel_err"] = (rel(hvf_ae, hvf_exact) if torch.is_tensor(hvf_exact)
                                              else f"no full-storage reference: {hvf_exact}")

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, secs, what = cpu_sample(shape, nt, args.codec)
        cpu = {"value": v, "unit": "gradients/hour", "cores": os.cpu_count(), "kind": "oracle",
               "sample": what}

    if rank == 0:
        dom = kernels["adjoint_bf16" if args.codec == "time" else "adjoint"]
        line = {
            "metric": METRIC, "value": value, "unit": "gradients/hour", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 stencil, bf16 codec", "data": "synthetic (GRF velocity, bump-model observations)",
            "config": dict(workload(shape, nt, NREC, n_lat, args.codec),
                           codec_weights="trained" if trained else "random-init",
                           shots=world, parallelism=(f"{world} shots, one per GPU, gradients "
                                                     f"summed by one all-reduce") if world > 1
                           else "one shot on one GPU"),
            "accuracy": accuracy,
            "roofline": {"kernel": "adjoint step (adj_tma_kernel), the longest per-step kernel "
                                   "of the AE gradient" + (", reading its decoded strain as BF16 "
                                                           "(48 B/node)" if args.codec == "time"
                                                           else ""), "bound": "hbm",
                         "achieved": dom["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
                         "frac": dom["achieved_gbs"] / hbm_peak,
                         "peak_kind": f"{peak_kind} copy bandwidth (burst: kernel timed alone)",
                         "traffic": ((ADJ16_TRAFFIC_256 if args.codec == "time" else ADJ_TRAFFIC_256)
                                     if shape == SHAPE else None),
                         "traffic_source": "ncu capture of a window-middle adjoint step at 256^3 "
                                           + ("(profiles/adj_tma_kernel_bf16_256cubed.md)"
                                              if args.codec == "time" else
                                              "(profiles/adj_tma_kernel_256cubed.md)"),
                         "bytes_per_launch": dom["bytes_per_launch"],
                         "timing": f"CUDA events around {nprof} back-to-back launches"},
            "kernels": kernels,
            "stencil": {"cell_updates_per_s": C / (kernels["forward"]["ms_per_launch"] / 1e3),
                        "gbs": kernels["forward"]["achieved_gbs"],
                        "frac_of_8tbs": kernels["forward"]["achieved_gbs"] / 8000.0},
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
            "hvp_full_newton": None if ae_hvpf_ms is None else
                {"ae_ms": ae_hvpf_ms, "ae_hvps_per_hour": 3600e3 / ae_hvpf_ms,
                 "note": "full Newton HVP: incremental forward with its strain compressed by the "
                         "time codec, then first- and second-order adjoints in lockstep"},
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


def default_weights(codec: str, n_lat: int) -> str:
    name = f"codec_time_{n_lat}.npz" if codec == "time" else f"codec_{n_lat}.npz"
    return os.path.join(ROOT, "paper_2304_04781_gb300", "weights", name)


def load_weights(path: str, codec: str, n_lat: int):
    """(weights, trained): the file's weights, or Glorot-uniform ones if it is missing."""
    from paper_2304_04781_gb300 import inputs
    W = inputs.codec_init(seed=0, n_hid=2 * n_lat if codec == "time" else 512, n_lat=n_lat)
    if path and os.path.exists(path):
        z = np.load(path)
        return {k: z[k] for k in W}, True
    return W, False


def run_accuracy(args):
    """Errors of the compressed gradient / GN-HVP against an uncompressed reference on
    the same GPU, decoded-state error, adjoint identity and checkpointing equality at the
    full size.  Prints one JSON line."""
    import torch
    from paper_2304_04781_gb300 import aewave, inputs
    shape, nt = tuple(args.shape), args.nt
    nz, ny, nx = shape
    n_lat = nlat_of(args)
    rec = inputs.receiver_grid(nx, ny, args.nrec)
    W, trained = load_weights(args.weights or default_weights(args.codec, n_lat), args.codec, n_lat)
    c_np = inputs.velocity_model(shape, H, seed=2).astype(np.float32)
    c = torch.from_numpy(c_np).cuda()
    ctrue = torch.from_numpy(inputs.bump_model(c_np.astype(np.float64), H).astype(np.float32)).cuda()
    dirs = [torch.from_numpy(inputs.direction(shape, H, seed=(20 if args.hvps == 1 else 30) + k)
                             .astype(np.float32)).cuda() for k in range(args.hvps)]
    out = {"config": dict(workload(shape, nt, args.nrec, n_lat, args.codec), f0_hz=args.f0,
                          norm=args.norm, act=args.act, beta=args.beta),
           "codec_weights": "trained" if trained else "random-init", "n_lat": n_lat,
           "reference": args.ref}
    def ev():
        return torch.cuda.Event(enable_timing=True)

    ae = aewave.Solver(shape, H, nt, rec, storage="ae", codec=args.codec, n_lat=n_lat, f0=args.f0,
                       norm=args.norm, act=args.act, beta=args.beta)
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

    # decoded-state error on this run's states (every 8th window / every nt/40-th state)
    from paper_2304_04781_gb300 import train
    tr = train.make_handle(shape, args.codec, n_lat, nt=nt, f0=args.f0, norm=args.norm,
                           act=args.act, beta=args.beta)
    tr.codec_set(W)
    every = 8 if args.codec == "time" else max(1, nt // 40)
    snaps, mx = train.generate(tr, [2], every)
    out["decoded_state_error"] = tr.codec_eval(snaps, mx)
    out["decoded_state_sample"] = f"every {every}th {'window' if args.codec == 'time' else 'state'} of this run"
    print(json.dumps(out))


def run_map(args):
    """MAP estimation and DIAS (Sec. 2, Sec. 4.3) at the workload size: Newton-CG with
    the BiLaplacian prior on the compressed history and on full storage from the same
    start, then the DIAS active subspace at the compressed MAP point and the DIAS-F
    solve from it.  Prints one JSON line.

    The misfit is unweighted, 1/2 |d - d_obs|^2; noise of std sigma_n (noise-rel x the
    rms of the data) and a prior with sample std prior-std [m/s] make the objective, times
    sigma_n^2, 1/2 |d - d_obs|^2 + 1/2 |alpha_reg A_1 (c - c0)|^2 with
    alpha_reg = sigma_n alpha_s (A_1: the operator at alpha = 1).  alpha_s is measured:
    the std of a sample A_1^{-1} w scales as 1 / alpha.  The source is smoothed by a
    Gaussian of --src-sigma (50 m, as in Sec. 4.1's box problem): a point source makes
    the misfit's sensitivity singular at its node, where Newton steps then grow the
    speed up to the stability bound.  Errors against the true model are reported over
    all nodes (the paper's average relative error), inside the bump and outside it."""
    import torch
    from paper_2304_04781_gb300 import aewave, inputs
    shape, nt = tuple(args.shape), args.nt
    nz, ny, nx = shape
    n_lat = nlat_of(args)
    rec = inputs.receiver_grid(nx, ny, args.nrec)
    W, trained = load_weights(args.weights or default_weights(args.codec, n_lat), args.codec, n_lat)
    c0_np = inputs.velocity_model(shape, H, seed=2).astype(np.float32)
    c0 = torch.from_numpy(c0_np).cuda()
    ctrue = torch.from_numpy(inputs.bump_model(c0_np.astype(np.float64), H).astype(np.float32)).cuda()
    theta = args.theta

    def ev():
        return torch.cuda.Event(enable_timing=True)

    bump = (ctrue - c0).abs() / c0 > 0.005      # where the true model differs by > 0.5%

    def mean_rel(c):
        e = ((c - ctrue).abs() / ctrue).double()
        return {"all": float(e.mean()), "bump": float(e[bump].mean()), "rest": float(e[~bump].mean())}

    ae = aewave.Solver(shape, H, nt, rec, storage="ae", codec=args.codec, n_lat=n_lat, f0=args.f0,
                       norm=args.norm, act=args.act, beta=args.beta, cmax=args.map_cmax,
                       src_sigma=args.src_sigma)
    ae.codec_set(W)
    d_obs = ae.forward(ctrue)
    w = torch.from_numpy(inputs.white_noise(1, shape, seed=77)[0]).cuda()
    ae.prior_solve(w, 1.0, theta)      # warm-up (first-call allocations)
    a, b = ev(), ev(); a.record()
    x1, its = ae.prior_solve(w, 1.0, theta)
    b.record(); torch.cuda.synchronize()
    solve_ms = a.elapsed_time(b)
    alpha_s = float(x1.double().std()) / args.prior_std
    # the prior's HBM-bound kernels alone: A q (8 B per node: read q, write A q) and one
    # CG iteration (apply 8 + update 24 + direction 12 = 44 B per node)
    peaks = load_peaks()
    y1 = torch.empty_like(w)
    for _ in range(3):
        ae.prior_apply(w, 1.0, theta, out=y1)
    a, b = ev(), ev(); a.record()
    for _ in range(20):
        ae.prior_apply(w, 1.0, theta, out=y1)
    b.record(); torch.cuda.synchronize()
    apply_ms = a.elapsed_time(b) / 20
    del y1
    sigma_n = args.noise_rel * float(d_obs[1:].double().pow(2).mean().sqrt())
    if not sigma_n > 0:
        raise SystemExit("the observed data are zero: the wave does not reach the receivers "
                         "within nt steps (raise --nt)")
    alpha = alpha_s * sigma_n
    out = {"config": dict(workload(shape, nt, args.nrec, n_lat, args.codec), f0_hz=args.f0,
                          norm=args.norm, act=args.act, dt_cmax=args.map_cmax, dt_s=ae.dt,
                          src_sigma_m=args.src_sigma),
           "codec_weights": "trained" if trained else "random-init",
           "prior": {"theta_m2": theta, "sample_std": args.prior_std, "alpha_s": alpha_s,
                     "noise_rel": args.noise_rel, "sigma_n": sigma_n, "alpha_reg": alpha,
                     "solve_ms": solve_ms, "solve_cg_iters": its,
                     "apply_ms": apply_ms,
                     "apply_gbs": 8.0 * c0.numel() / (apply_ms * 1e-3) / 1e9,
                     "cg_iter_gbs": 44.0 * c0.numel() * its / (solve_ms * 1e-3) / 1e9,
                     "hbm_peak_gbs": peaks[0]},
           "initial_mean_rel_err": mean_rel(c0)}
    del x1, w
    kw = dict(alpha=alpha, theta=theta, newton_iters=args.newton_iters, cg_max=args.cg_max)

    def solve(s, W1=None, c_start=None, iters=None):
        c = (c_start if c_start is not None else c0).clone()
        k = dict(kw) if iters is None else dict(kw, newton_iters=iters)
        a, b = ev(), ev(); a.record()
        hist = s.newton_cg(c, d_obs, c0, W1=W1, **k)
        b.record(); torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        hvps = sum(h["cg_iters"] for h in hist)
        grads = 1 + sum(h["backtracks"] + 1 for h in hist)
        return c, {"ms": ms, "ms_per_iter": ms / max(len(hist), 1), "hvps": hvps,
                   "gradients": grads, "mean_rel_err": mean_rel(c), "history": hist}

    c_ae, out["map_ae"] = solve(ae)
    out["map_ae"]["max_c"] = float(c_ae.max())
    # DIAS: active subspace at the compressed MAP point, then the DIAS-F solve from it
    noise = torch.from_numpy(inputs.white_noise(args.dias_samples, shape, seed=500)).cuda()
    try:
        a, b = ev(), ev(); a.record()
        lam, W1, G = ae.dias_subspace(c_ae, d_obs, noise, alpha_s, theta, args.dias_rank)
        b.record(); torch.cuda.synchronize()
        del G
        torch.cuda.empty_cache()
        c_dias, dias = solve(ae, W1=W1, c_start=c_ae, iters=args.dias_iters)
        # the same iterations from the MAP point with the full prior: what the projection
        # alone changes
        c_cont, cont = solve(ae, c_start=c_ae, iters=args.dias_iters)
        nrm = lambda x: float(torch.linalg.vector_norm(x.double()))
        out["dias"] = {"samples": args.dias_samples, "rank": args.dias_rank,
                       "subspace_ms": a.elapsed_time(b),
                       "ms_per_sample": a.elapsed_time(b) / args.dias_samples,
                       "eigenvalues": [float(v) for v in lam[:max(args.dias_rank + 3, 8)]],
                       "solve": dias, "map_continued": cont,
                       "dias_vs_map_continued_rel_diff": (nrm(c_dias - c_cont) / nrm(c_cont - c0)
                                                          if nrm(c_cont - c0) > 0 else None)}
        del W1, c_dias, c_cont
    except aewave.AewError as err:
        out["dias"] = {"error": str(err)}
    del noise
    out["ae_device_bytes"] = ae.stats()["device_bytes"]
    c_ae_h = c_ae.cpu()
    del ae
    torch.cuda.empty_cache()
    if args.map_ref != "none":
        kw_ref = {"storage": "full"} if args.map_ref == "full" else {"storage": "revolve",
                                                                     "n_checkpoints": 20}
        full = aewave.Solver(shape, H, nt, rec, f0=args.f0, cmax=args.map_cmax,
                             src_sigma=args.src_sigma, **kw_ref)
        c_full, out["map_full"] = solve(full)
        out["map_full"]["storage"] = args.map_ref
        du_ref = (c_full.cpu() - c0.cpu()).double()
        out["map_update_rel_diff"] = float(torch.linalg.vector_norm(c_ae_h.double() - c0.cpu().double() - du_ref)
                                           / torch.linalg.vector_norm(du_ref))
        del full
    print(json.dumps(out))


def run_train_step(args):
    """Codec training steps alone (aew_codec_train_step: forward, back-propagation and
    LAMB over one BF16 minibatch, Table 2's batch 512): 10 warm-up steps, then --launches
    timed steps with CUDA events on the current stream.  Prints one JSON line."""
    import torch
    from paper_2304_04781_gb300 import aewave, inputs
    n_lat = nlat_of(args)
    shape = (16, 16, 16)
    s = aewave.Solver(shape, H, 4, inputs.receiver_grid(16, 16, 4), storage="ae", codec=args.codec,
                      n_lat=n_lat, norm=args.norm, act=args.act)
    s.codec_set(inputs.codec_init(seed=0, n_hid=s.n_hid, n_lat=n_lat))
    g = torch.Generator(device="cuda").manual_seed(3)
    pool = (torch.rand((8 * args.batch, 2048), device="cuda", generator=g) * 2 - 1).to(torch.bfloat16)
    batches = [pool[k * args.batch:(k + 1) * args.batch] for k in range(8)]
    for k in range(10):
        s.train_step(batches[k % 8], 1e-4, want_loss=False)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for k in range(args.launches):
        s.train_step(batches[k % 8], 1e-4, want_loss=False)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.launches
    I, Hh, L, B = 2048, s.n_hid, n_lat, args.batch
    flop = 3 * 2 * B * (I * Hh + Hh * L + L * Hh + Hh * I)   # forward + two backward products
    print(json.dumps({"train_step_ms": ms, "batch": B, "codec": args.codec, "n_hid": Hh,
                      "n_lat": L, "tflops": flop / (ms * 1e-3) / 1e12, "steps": args.launches}))


def run_kernel(args):
    """One hot-path kernel alone: 2 warm-up launches, then --launches timed ones (CUDA
    events on the launching stream); prints one JSON line."""
    import torch
    from paper_2304_04781_gb300 import aewave, inputs
    shape, nt = tuple(args.shape), args.nt
    nz, ny, nx = shape
    n_lat = nlat_of(args)
    W, trained = load_weights(args.weights or default_weights(args.codec, n_lat), args.codec, n_lat)
    s = aewave.Solver(shape, H, nt, inputs.receiver_grid(nx, ny, args.nrec), storage="ae",
                      codec=args.codec, n_lat=n_lat, norm=args.norm, act=args.act, beta=args.beta)
    s.codec_set(W)
    c = torch.from_numpy(inputs.velocity_model(shape, H, seed=2).astype(np.float32)).cuda()
    s.profile(c, args.kernel, 2)
    ms = s.profile(c, args.kernel, args.launches)
    print(json.dumps({"kernel": args.kernel, "shape": list(shape), "ms_per_launch": ms,
                      "launches": args.launches, "codec_weights": "trained" if trained else "random-init"}))


def main():
    args = parse()
    if args.kernel:
        run_kernel(args)
    elif args.map:
        run_map(args)
    elif args.train_step:
        run_train_step(args)
    elif args.accuracy:
        run_accuracy(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
