#!/usr/bin/env python
"""Benchmark of the ESI hot path on one GB300 (or N, one process per GPU).

One step = the inner problem of Algorithm 2 for a batch of shots on the 801 x 241,
nt = 3000, 16-shot FP32 workload (seeded dipping layers + anomalies, 8 Hz Ricker data):
  set-up of c = v^2 dt^2 for the current model;
  b = S^T d and CG on (S^T S + beta B^T B) q = S^T d to ||r|| < 1e-3 ||r_0|| with the
  diagonal preconditioner z = r / (beta B^2) (the learned network, measured beside it,
  does not reach the tolerance faster);
  the saddle-point gradient of Algorithm 2 (u = A^{-1} q, lambda = beta B^H B q);
  the on-the-fly DTFT of u = A^{-1} q at 2, 4, 6, 8 Hz into FP16.
The metric is FD cell-updates per second over every forward and adjoint propagation of
the step (Gcell/s).  Beside it, outside the timed steps: the CG time to 1e-3 of the same
system with each preconditioner -- none (plain Algorithm 1, capped at --plain-iter
iterations; the residual it reaches is given when the cap comes first), the diagonal
z = r / (beta B^2), and the learned network (when its weights are present) -- and in its
data-space form, with the device time split into the product, the vector updates and the
preconditioner.

Multi-GPU: shots are independent systems, so each rank solves its own 16 shots (weak
scaling) with no collective on the data path; ranks meet only at the timing barriers.

--impl reference times the FP64 CPU oracle on the host cores (a bounded sample of the
same workload: one shot's forward + adjoint over nt_sample steps per bench step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FD Gcell-updates/s fwd+adj; ESI CG time to 1e-3 residual, plain vs learned PC"
UNIT = "Gcell-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--ns", type=int, default=16, help="shots per GPU")
    ap.add_argument("--nt", type=int, default=3000)
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--max-iter", type=int, default=60)
    ap.add_argument("--plain-iter", type=int, default=60)
    ap.add_argument("--beta-factor", type=float, default=10.0)
    ap.add_argument("--precond", default="diag", choices=["auto", "none", "diag", "learned"],
                    help="preconditioner of the timed solve; auto: the learned one when its "
                         "weights are present")
    ap.add_argument("--pc-weights", default=os.path.join(ROOT, "paper_2211_06300_gb300",
                                                         "pc_weights.npy"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the untimed CG comparison (none / diag / data space / frequency "
                         "domain / learned)")
    ap.add_argument("--ref-nt", type=int, default=1500, help="oracle sample: steps per bench step")
    ap.add_argument("--workload", default="esi2d",
                    choices=["esi2d", "dft3d", "wri2d", "invert2d", "grad2d"],
                    help="dft3d: forward modelling with the on-the-fly DTFT (5 frequencies, FP16 "
                         "output) on the 400^3, nt 2000 volume instead of the ESI step; wri2d: "
                         "the WRI solve (B = I) and its gradient on the ESI step's workload; "
                         "invert2d: the ESI outer loop (esi_invert) on that workload; grad2d: "
                         "the adjoint-state gradient with BF16 checkpoints on 64 shots of "
                         "1201 x 301")
    ap.add_argument("--outer", type=int, default=2, help="invert2d: outer iterations per step")
    ap.add_argument("--wri-factor", type=float, default=1e-2,
                    help="WRI penalty: beta = factor * lambda_max(S^T S)")
    ap.add_argument("--groups", type=int, default=1,
                    help="esi2d, wri2d, invert2d, grad2d: run the shots as this many concurrent groups "
                         "(esi_set_shot_groups) in the timed steps")
    ap.add_argument("--n3d", type=int, default=400)
    ap.add_argument("--nt3d", type=int, default=2000)
    return ap.parse_args()


def workload_name(ns, nt):
    return f"esi2d-801x241-nt{nt}-{ns}shots-fp32"


# ----------------------------------------------------------------------------- DRAM traffic
# ncu dram__bytes_read.sum + dram__bytes_write.sum per cell update of a step-kernel variant,
# from an ncu capture of the 2D step kernel on 16 shots of 801 x 241 (one launch =
# 3,088,656 cell updates), valid only for the kernel it was taken on: the
# SHA-256 below of its template source and the header's argument struct (_sources_sha).
_SHA = "5e1d3b4d18ef73966c665b764822e8bfd92c3349c58d284ccc6d45b8206ddf0a"
MEASURED_TRAFFIC = {
    "fd2_step[PT|AP]": ((52.655616e6 + 1.062656e6) / 3088656, _SHA),
    "fd2_step[CGP|SMP]": ((65.971712e6 + 1.078528e6) / 3088656, _SHA),
    "fd2_step[EXT|SAD]": ((51.677952e6 + 0.215296e6) / 3088656, _SHA),
    "fd2_step[EXT|SMP|DFT]": ((39.824896e6 + 0.086016e6) / 3088656, _SHA),
}
TRAFFIC_SOURCES = ("paper_2211_06300_gb300/csrc/fd2d.cu", "paper_2211_06300_gb300/csrc/esi_internal.h")


def _sources_sha():
    """Hash of what the 2D step kernel variants are compiled from: the kernel template (its
    source up to the dispatch list) and the shared header up to the end of the kernel
    argument struct (later declarations do not reach the kernel)."""
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            text = fh.read()
        if f.endswith(".h"):
            i = text.find(b"struct StepArgs {")
            j = text.find(b"\n};", i)
            if i >= 0 and j >= 0:
                text = text[:j + 3]
        else:   # the kernel template; the dispatch list after it picks variants only
            i = text.find(b"#define ESI_CASE")
            if i >= 0:
                text = text[:i]
        h.update(text)
    return h.hexdigest()


def traffic_per_launch(entry):
    """DRAM bytes of one launch of the profiled variant, scaled from the capture by the cell
    updates the launch performs; None when not captured or the kernel changed since."""
    m = MEASURED_TRAFFIC.get(entry["name"])
    if m is None or m[1] != _sources_sha():
        return None
    return m[0] * entry["cells"] / max(entry["launches"], 1)


def pinned_like(t):
    """A page-locked host buffer of t's shape and type, made (and its pages touched, by the
    zero fill) before a timed loop: copies from the device into it run at the link's speed
    (a pageable target goes through a staging buffer)."""
    import torch
    return torch.zeros(t.shape, dtype=t.dtype, pin_memory=True)


# ----------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2211_06300_gb300 import synth
    w = synth.workload_esi_2d(nt=args.ref_nt, ns=1)
    o = oracle.Oracle(w.v_start, w.dx, w.dt, w.nt, w.nb, vref=float(w.v_true.max()))
    sh = o.shot(w.geom.src_xyz[0], w.geom.receivers(0))
    wav = w.wavelets()[0]

    def step():
        d = o.forward(sh, wavelet=wav)["traces"]
        o.adjoint(sh, d)
        return 2 * w.ncell * w.nt
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    cells = sum(step() for _ in range(args.steps))
    dt = time.perf_counter() - t0
    val = cells / dt / 1e9
    sample = f"1 shot x {w.nt} steps forward + adjoint on the 801x241 grid, FP64 oracle"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args.ns, args.nt), "reference_sample": sample},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline(nt_sample=3000, shots=8):
    """The oracle as it stands on the host cores: `shots` shots of the same workload, one
    forward + one adjoint modelling each over nt_sample steps (about 15 s on 16 cores)."""
    import oracle
    from paper_2211_06300_gb300 import synth
    w = synth.workload_esi_2d(nt=nt_sample, ns=shots)
    o = oracle.Oracle(w.v_start, w.dx, w.dt, w.nt, w.nb, vref=float(w.v_true.max()))
    wav = w.wavelets()
    t0 = time.perf_counter()
    for s in range(shots):
        sh = o.shot(w.geom.src_xyz[s], w.geom.receivers(s))
        d = o.forward(sh, wavelet=wav[s])["traces"]
        o.adjoint(sh, d)
    dt = time.perf_counter() - t0
    return {"value": 2 * shots * w.ncell * w.nt / dt / 1e9, "unit": UNIT,
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{shots} shots x {nt_sample} steps forward + adjoint (801x241, FP64), "
                      f"{dt:.1f} s"}


# ----------------------------------------------------------------------------- 3D DTFT arm
def roofline_of(prof, peaks, groups=1, step_ms=None, steps=1):
    """The dominant kernel's algorithmic bytes per launch over its average launch duration on
    the stream it runs on.  With G concurrent shot groups every group's launches are in the
    profile, each timed while the other groups' launches run beside it, so this per-launch
    rate is a group's share; `step` then gives the whole step's algorithmic bytes (every
    kernel) over its device time, which holds for any G."""
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    single = [k for k in prof if k["name"] != "pc_net"]
    if not single:
        return None
    top = max(single, key=lambda k: k["ms"])
    per_launch_ms = top["ms"] / max(top["launches"], 1)
    bytes_per_launch = top["cells"] * top["bytes_per_cell"] / max(top["launches"], 1)
    achieved = bytes_per_launch / (per_launch_ms * 1e-3) / 1e9
    out = {"bound": "hbm", "kernel": top["name"], "achieved": achieved, "peak": hbm,
           "unit": "GB/s", "frac": achieved / hbm,
           "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
           "traffic": traffic_per_launch(top) if groups == 1 else None,
           "per_launch_us": 1e3 * per_launch_ms, "bytes_per_launch": bytes_per_launch,
           "share": top["ms"] / sum(k["ms"] for k in prof)}
    if groups > 1:
        out["groups"] = groups
        out["note"] = "per-launch rate of one of the concurrent shot groups"
    if step_ms:
        total = sum(k["cells"] * k["bytes_per_cell"] for k in prof) / max(steps, 1)
        out["step"] = {"achieved": total / (step_ms * 1e-3) / 1e9,
                       "frac": total / (step_ms * 1e-3) / 1e9 / hbm,
                       "bytes_per_step": total}
    return out


def run_dft3d(args, rank, world, local):
    """One step = forward modelling of the 400^3 volume over nt 2000 steps with the DTFT at
    4, 6, 8, 10, 12 Hz into FP16 and the 160 x 160 receiver traces; every rank runs its own
    copy of the shot (replicas: the volume is not split)."""
    import torch
    from paper_2211_06300_gb300 import esi, shard, synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    w = synth.workload_3d(n=args.n3d, nt=args.nt3d)
    ctx = esi.Context(torch.tensor(w.v_true, dtype=torch.float32, device=dev), w.dx, w.dt,
                      w.nt, w.nb, w.geom, vref=float(w.v_true.max()))
    wav = torch.tensor(w.wavelets(), dtype=torch.float32, device=dev)
    tr = torch.empty(w.nt * int(w.geom.rec_offset[-1]), dtype=torch.float32, device=dev)
    freqs = [4.0, 6.0, 8.0, 10.0, 12.0]

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
    for _ in range(args.warmup):
        ctx.dft_extract(freqs, wavelet=wav, half=True, traces=tr)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    l0 = ctx.launches
    ctx.set_profiling(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        U, _ = ctx.dft_extract(freqs, wavelet=wav, half=True, traces=tr)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile()
    ctx.set_profiling(False)
    launches = ctx.launches - l0
    clk = clocks.stop()
    cells = args.steps * w.ncell * w.nt
    t_max = shard.max_over_ranks(ms, dist, dev)
    cells_all = shard.sum_over_ranks(cells, dist, dev)
    # the blocked DTFT's bytes per cell update and block length, from the library's profile
    # entry of the step + fold (FP32: 24 + 16 nf / K bytes)
    bpc_blk = next(k["bytes_per_cell"] for k in prof if k["name"].endswith("+dft_block"))
    kblk = int(round(16 * len(freqs) / (bpc_blk - 24)))
    # end to end: the wavelet from pinned host memory in, traces and the FP16 wavefields out
    wav_h = wav.cpu().pin_memory()
    tr_h, U_h = pinned_like(tr), pinned_like(U)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        wav.copy_(wav_h, non_blocking=True)
        U, _ = ctx.dft_extract(freqs, wavelet=wav, half=True, traces=tr)
        tr_h.copy_(tr, non_blocking=True)
        U_h.copy_(U, non_blocking=True)
        torch.cuda.synchronize()
    te = shard.max_over_ranks(time.perf_counter() - t0, dist, dev)
    if rank == 0:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        print(json.dumps({
            "metric": "FD Gcell-updates/s (forward modelling with on-the-fly DTFT)",
            "value": cells_all / (t_max * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"dft3d-{args.n3d}^3-nt{args.nt3d}-5freqs-fp16",
                       "freqs_hz": freqs,
                       "l2": "inputs larger than L2 (states 2 x %.0f MB, DTFT stash %.1f GB)"
                             % (4 * w.ncell / 1e6, kblk * 4 * w.ncell / 1e9)},
            # algorithmic bytes per cell update: accumulating every state into the nf complex
            # FP32 accumulators directly costs 16 + 16 nf; the blocked DTFT stashes the states
            # of a block of K steps and folds them once (16 + 4 stash write + 4 stash read +
            # 16 nf / K), K chosen by the library for the context's memory (from its profile)
            "bytes_per_cell": {"per_step_accumulation": 16 + 16 * len(freqs),
                               "blocked": bpc_blk, "block_steps": kblk},
            "roofline": roofline_of(prof, peaks), "kernels": prof,
            "e2e": {"value": cells_all / te / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": int(wav_h.numel() * 4),
                    "d2h_bytes_per_step": int(tr_h.numel() * 4 + U_h.numel() * 2)},
            "gpu_launches": launches, "clocks": clk}), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- WRI arm
def run_wri2d(args, rank, world, local):
    """One step = WRI on the 801 x 241, nt 3000, 16-shot workload: the data residual of the
    point sources, CG on (S^T S + beta I) q = S^T (d - S f) to 1e-3 (the CG section: the
    ESI CG with the identity as annihilator and its own right-hand side), and the saddle-point gradient with
    u = A^{-1}(f + q), lambda = beta q.  Shots are sharded over ranks as in the ESI step."""
    import numpy as np
    import torch
    from paper_2211_06300_gb300 import esi, pc_train, shard, synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    ns, nt = args.ns, args.nt
    wl = synth.workload_esi_2d(nt=nt, ns=ns * world)
    geom = wl.geom.select(range(*shard.shot_range(ns * world, rank, world)))
    vref = float(wl.v_true.max())
    f32 = torch.float32
    v0 = torch.tensor(wl.v_start, dtype=f32, device=dev)
    wav = torch.tensor(wl.wavelets()[rank * ns:(rank + 1) * ns], dtype=f32, device=dev).contiguous()
    ct = esi.Context(torch.tensor(wl.v_true, dtype=f32, device=dev), wl.dx, wl.dt, nt, wl.nb,
                     geom, vref=vref)
    dobs = ct.forward(wavelet=wav)
    ct.close()
    ctx = esi.Context(v0, wl.dx, wl.dt, nt, wl.nb, geom, vref=vref)
    c1 = esi.Context(v0, wl.dx, wl.dt, nt, wl.nb, geom.select([0]), vref=vref)
    # beta = factor * lambda_max(S^T S): pc_train.penalty divides by (max B)^2, undone here
    nz, nx = wl.shape
    far = max(math.hypot(x, z) for x in (0.0, (nx - 1) * wl.dx) for z in (0.0, (nz - 1) * wl.dx))
    beta = pc_train.penalty(c1, wl.shape, wl.dx, nt, dev, factor=args.wri_factor) * (far + wl.dx) ** 2
    c1.close()
    q = ctx.empty_field()
    N = wl.ncell
    if args.groups > 1:
        ctx.set_shot_groups(args.groups)

    def step():
        ctx.set_velocity(v0)
        _, rep = ctx.cg_solve(dobs, lam=beta, tol=args.tol, max_iter=args.max_iter, out=q,
                              wri_wavelet=wav)
        g, _ = ctx.gradient(wavelet=wav, ext=q, mode="wri", beta=beta, param="v")
        props = sum(1 + 1 + 2 * int(k) + 1 for k in rep["iters"])   # S f, b, products, gradient
        return g, rep, props * N * nt

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
    for _ in range(args.warmup):
        step()
    barrier()
    clocks = Clocks(local)
    clocks.start()
    l0 = ctx.launches
    ctx.set_profiling(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    barrier()
    e0.record(stream)
    cells, reps = 0, []
    for _ in range(args.steps):
        _, rep, c = step()
        cells += c
        reps.append(rep)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile()
    ctx.set_profiling(False)
    launches = ctx.launches - l0
    clk = clocks.stop()
    t_max = shard.max_over_ranks(ms, dist, dev)
    cells_all = shard.sum_over_ranks(cells, dist, dev)
    d_host = dobs.cpu().pin_memory()
    d_dev = torch.empty_like(dobs)
    g_host = pinned_like(v0)
    barrier()
    t0 = time.perf_counter()
    ce = 0
    for _ in range(args.steps):
        d_dev.copy_(d_host, non_blocking=True)
        ctx.set_velocity(v0)
        _, rep = ctx.cg_solve(d_dev, lam=beta, tol=args.tol, max_iter=args.max_iter, out=q,
                              wri_wavelet=wav)
        g, _ = ctx.gradient(wavelet=wav, ext=q, mode="wri", beta=beta, param="v")
        g_host.copy_(g, non_blocking=True)
        torch.cuda.synchronize()
        ce += sum(3 + 2 * int(k) for k in rep["iters"]) * N * nt
    te = shard.max_over_ranks(time.perf_counter() - t0, dist, dev)
    ce = shard.sum_over_ranks(ce, dist, dev)
    if rank == 0:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        print(json.dumps({
            "metric": "FD Gcell-updates/s fwd+adj; WRI CG time to 1e-3 residual",
            "value": cells_all / (t_max * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "wri2d-801x241-nt%d-%dshots-fp32" % (nt, ns), "beta": beta,
                       "wri_factor": args.wri_factor, "tol": args.tol, "shot_groups": args.groups,
                       "l2": "inputs larger than L2 (CG vectors 4 x %.2f GB per GPU)"
                             % (4 * ns * nt * N / 1e9)},
            "cg": {"iters_max_per_step": [int(max(r["iters"])) for r in reps],
                   "time_to_tol_ms": [r["ms_total"] for r in reps],
                   "converged": [bool(r["converged"]) for r in reps]},
            "roofline": roofline_of(prof, peaks, args.groups, t_max / args.steps, args.steps),
            "kernels": prof,
            "e2e": {"value": ce / te / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": int(d_host.numel() * d_host.element_size()),
                    "d2h_bytes_per_step": int(g_host.numel() * g_host.element_size())},
            "gpu_launches": launches, "clocks": clk}), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- outer loop
def run_invert2d(args, rank, world, local):
    """One step = the outer loop (Algorithm "nestedloop", esi_invert) on the 801 x 241, nt 3000,
    16-shot workload from the smoothed starting model: args.outer L-BFGS iterations, each
    evaluation 10 diagonally preconditioned CG iterations (the paper's numerical tests use 10)
    plus the objective and saddle-point gradient from one forward run.  Shots are sharded over
    ranks; J and the gradient are summed through the reduce callback."""
    import torch
    from paper_2211_06300_gb300 import esi, pc_train, shard, synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    ns, nt = args.ns, args.nt
    wl = synth.workload_esi_2d(nt=nt, ns=ns * world)
    geom = wl.geom.select(range(*shard.shot_range(ns * world, rank, world)))
    vref = float(wl.v_true.max())
    f32 = torch.float32
    v0 = torch.tensor(wl.v_start, dtype=f32, device=dev)
    wav = torch.tensor(wl.wavelets()[rank * ns:(rank + 1) * ns], dtype=f32, device=dev).contiguous()
    ct = esi.Context(torch.tensor(wl.v_true, dtype=f32, device=dev), wl.dx, wl.dt, nt, wl.nb,
                     geom, vref=vref)
    dobs = ct.forward(wavelet=wav)
    ct.close()
    ctx = esi.Context(v0, wl.dx, wl.dt, nt, wl.nb, geom, vref=vref)
    c1 = esi.Context(v0, wl.dx, wl.dt, nt, wl.nb, geom.select([0]), vref=vref)
    beta = pc_train.penalty(c1, wl.shape, wl.dx, nt, dev, factor=args.beta_factor)
    c1.close()
    vel = v0.clone()
    grad = torch.empty_like(v0)
    N = wl.ncell
    if args.groups > 1:
        ctx.set_shot_groups(args.groups)
    red = (lambda J, g: shard.reduce_objective(J, g, dist)) if dist is not None else None
    kw = dict(n_outer=args.outer, n_cg=10, precond="diag", beta0=beta, vmin=1400.0,
              vmax=4700.0, reduce=red)

    def step(d):
        vel.copy_(v0)
        _, rep = ctx.invert(d, vel, grad=grad, **kw)
        props = 2 * rep["evaluations"] + 2 * rep["cg_iters_total"]   # S^T d, forward; products
        return rep, props * N * nt * ns

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
    for _ in range(args.warmup):
        step(dobs)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    l0 = ctx.launches
    ctx.set_profiling(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    barrier()
    e0.record(stream)
    cells, reps = 0, []
    for _ in range(args.steps):
        rep, c = step(dobs)
        cells += c
        reps.append(rep)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile()
    ctx.set_profiling(False)
    launches = ctx.launches - l0
    clk = clocks.stop()
    t_max = shard.max_over_ranks(ms, dist, dev)
    cells_all = shard.sum_over_ranks(cells, dist, dev)
    d_host = dobs.cpu().pin_memory()
    d_dev = torch.empty_like(dobs)
    v_host = pinned_like(vel)
    barrier()
    t0 = time.perf_counter()
    ce = 0
    for _ in range(args.steps):
        d_dev.copy_(d_host, non_blocking=True)
        _, c = step(d_dev)
        v_host.copy_(vel, non_blocking=True)
        torch.cuda.synchronize()
        ce += c
    te = shard.max_over_ranks(time.perf_counter() - t0, dist, dev)
    ce = shard.sum_over_ranks(ce, dist, dev)
    if rank == 0:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        print(json.dumps({
            "metric": "FD Gcell-updates/s fwd+adj; ESI outer loop (nestedloop)",
            "value": cells_all / (t_max * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "invert2d-801x241-nt%d-%dshots-fp32" % (nt, ns),
                       "outer_iterations": args.outer, "inner_cg": 10, "precond": "diag",
                       "beta": beta, "shot_groups": args.groups,
                       "l2": "inputs larger than L2 (q %.2f GB per GPU)" % (4 * ns * nt * N / 1e9)},
            "outer": [{"J_start": r["J_start"], "J_end": r["J_end"], "trials": r["trials"],
                       "evaluations": r["evaluations"], "stop": r["stop"],
                       "ms": r["ms_total"]} for r in reps],
            "roofline": roofline_of(prof, peaks, args.groups, t_max / args.steps, args.steps),
            "kernels": prof,
            "e2e": {"value": ce / te / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": int(d_host.numel() * d_host.element_size()),
                    "d2h_bytes_per_step": int(v_host.numel() * v_host.element_size())},
            "gpu_launches": launches, "clocks": clk}), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- gradient arm
def run_grad2d(args, rank, world, local):
    """One step = the adjoint-state gradient (Eq. "gradient", "FWI_lambda") of the misfit on
    the 1201 x 301, nt 3000, 64-shot workload of uneven apertures (201-801 receivers): the
    forward modelling storing BF16 (u_n, u_{n-1}) checkpoints every 20 steps, then per
    segment the recompute with the stash of Lap u_n + q_n and the adjoint with the
    correlation.  Shots are sharded over ranks; the gradient is summed in rank order."""
    import torch
    from paper_2211_06300_gb300 import esi, shard, synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    nt = args.nt
    ns_all = 64 * world
    wl = synth.workload_batched_2d(nt=nt, ns=ns_all)
    lo, hi = shard.shot_range(ns_all, rank, world)
    geom = wl.geom.select(range(lo, hi))
    ns = hi - lo
    vref = float(wl.v_true.max())
    f32 = torch.float32
    wav = torch.tensor(wl.wavelets()[lo:hi], dtype=f32, device=dev).contiguous()
    ct = esi.Context(torch.tensor(wl.v_true, dtype=f32, device=dev), wl.dx, wl.dt, nt, wl.nb,
                     geom, vref=vref)
    dobs = ct.forward(wavelet=wav)
    ct.close()
    v0 = torch.tensor(wl.v_start, dtype=f32, device=dev)
    ctx = esi.Context(v0, wl.dx, wl.dt, nt, wl.nb, geom, vref=vref)
    N = wl.ncell
    cells_step = 3 * ns * N * nt      # forward, recompute, adjoint
    if args.groups > 1:
        ctx.set_shot_groups(args.groups)

    def step(d):
        g, J = ctx.gradient(wavelet=wav, dobs=d, param="v", ckpt_every=20, ckpt="bf16")
        if dist is not None:
            J = shard.reduce_objective(J, g, dist)
        return g, J

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
    for _ in range(args.warmup):
        step(dobs)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    l0 = ctx.launches
    ctx.set_profiling(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step(dobs)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile()
    ctx.set_profiling(False)
    launches = ctx.launches - l0
    clk = clocks.stop()
    t_max = shard.max_over_ranks(ms, dist, dev)
    cells_all = shard.sum_over_ranks(cells_step * args.steps, dist, dev)
    d_host = dobs.cpu().pin_memory()
    d_dev = torch.empty_like(dobs)
    g_host = pinned_like(v0)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        d_dev.copy_(d_host, non_blocking=True)
        g, J = step(d_dev)
        g_host.copy_(g, non_blocking=True)
        torch.cuda.synchronize()
    te = shard.max_over_ranks(time.perf_counter() - t0, dist, dev)
    if rank == 0:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        print(json.dumps({
            "metric": "FD Gcell-updates/s fwd+adj; adjoint-state gradient",
            "value": cells_all / (t_max * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "grad2d-1201x301-nt%d-%dshots-fp32-bf16ckpt" % (nt, ns),
                       "checkpoint_every": 20, "checkpoints": "bf16", "shot_groups": args.groups,
                       "checkpoint_codec": "u_n and u_n - u_{n-1}, each as BF16 even-index "
                                           "cells plus the BF16 residual against their "
                                           "bilinear interpolation, unscaled "
                                           "(5 bytes per cell per checkpoint)",
                       "l2": "inputs larger than L2 (states 2 x %.1f MB, checkpoints %.1f GB)"
                             % (4 * ns * N / 1e6, 5 * ns * N * ((nt + 19) // 20) / 1e9)},
            "misfit": J,
            "roofline": roofline_of(prof, peaks, args.groups, t_max / args.steps, args.steps),
            "kernels": prof,
            "e2e": {"value": cells_all / te / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": int(d_host.numel() * d_host.element_size()),
                    "d2h_bytes_per_step": int(g_host.numel() * g_host.element_size())},
            "gpu_launches": launches, "clocks": clk}), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- CUDA arm
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "dft3d":
        run_dft3d(args, rank, world, local)
        return
    if args.workload == "wri2d":
        run_wri2d(args, rank, world, local)
        return
    if args.workload == "invert2d":
        run_invert2d(args, rank, world, local)
        return
    if args.workload == "grad2d":
        run_grad2d(args, rank, world, local)
        return
    import numpy as np
    import torch
    from paper_2211_06300_gb300 import esi, pc_train, shard, synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ns, nt = args.ns, args.nt
    wl = synth.workload_esi_2d(nt=nt, ns=ns * world)
    geom = wl.geom.select(range(*shard.shot_range(ns * world, rank, world)))
    vref = float(wl.v_true.max())
    f32 = torch.float32
    v_true = torch.tensor(wl.v_true, dtype=f32, device=dev)
    v0 = torch.tensor(wl.v_start, dtype=f32, device=dev)
    wav = torch.tensor(wl.wavelets()[:ns], dtype=f32, device=dev)
    # observed data: forward modelling on the true model (untimed set-up)
    ctx_t = esi.Context(v_true, wl.dx, wl.dt, nt, wl.nb, geom, vref=vref)
    dobs = ctx_t.forward(wavelet=wav)
    ctx_t.close()
    del ctx_t
    ctx = esi.Context(v0, wl.dx, wl.dt, nt, wl.nb, geom, vref=vref)
    # penalty: beta = factor * lambda_max(S^T S) / max B^2 (power iterations on the first shot)
    c1 = esi.Context(v0, wl.dx, wl.dt, nt, wl.nb, geom.select([0]), vref=vref)
    beta = pc_train.penalty(c1, wl.shape, wl.dx, nt, dev, factor=args.beta_factor)
    c1.close()
    del c1
    have_pc = os.path.exists(args.pc_weights)
    if have_pc:
        ctx.pc_load(torch.tensor(np.load(args.pc_weights), dtype=f32, device=dev))
    precond = args.precond
    if precond == "auto":
        precond = "learned" if have_pc else "diag"
    if args.groups > 1:
        ctx.set_shot_groups(args.groups)   # the learned solve would run ungrouped
    if precond == "learned" and not have_pc:
        raise SystemExit(f"--precond learned needs {args.pc_weights}")
    freqs = [2.0, 4.0, 6.0, 8.0]
    q = torch.empty((ns, nt) + wl.shape, dtype=f32, device=dev)
    N = wl.ncell

    def step(d_obs, precond=precond, max_iter=args.max_iter):
        ctx.set_velocity(v0)
        _, rep = ctx.cg_solve(d_obs, lam=beta, tol=args.tol, max_iter=max_iter, out=q,
                              precond=precond)
        g, _ = ctx.gradient(ext=q, mode="saddle", beta=beta, param="v")
        U, sc = ctx.dft_extract(freqs, ext=q, half=True)
        props = sum(1 + 2 * int(k) + 2 for k in rep["iters"])   # b, CG products, grad, DTFT
        return g, rep, props * N * nt, U, sc

    for _ in range(args.warmup):
        step(dobs)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    l0 = ctx.launches
    ctx.set_profiling(True)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    cells, reps = 0, []
    for _ in range(args.steps):
        g, rep, c, U, sc = step(dobs)
        cells += c
        reps.append(rep)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile()
    ctx.set_profiling(False)
    launches = ctx.launches - l0
    clk = clocks.stop()
    t_max = shard.max_over_ranks(ms, dist, dev)
    cells_all = shard.sum_over_ranks(cells, dist, dev)
    value = cells_all / (t_max * 1e-3) / 1e9

    # end to end through the public API with host buffers: pinned d_obs in; the gradient and
    # the FP16 DTFT fields with their scales out (the CG solution q stays on the device: it
    # is the step's intermediate, consumed by the gradient and the DTFT)
    e2e = None
    if not args.no_e2e:
        d_host = dobs.cpu().pin_memory()
        d_dev = torch.empty_like(dobs)
        g_host, U_host = pinned_like(g), pinned_like(U)
        # one untimed step on the end-to-end buffers (the loops' graphs are keyed by them)
        d_dev.copy_(d_host, non_blocking=True)
        step(d_dev)
        barrier()
        t0 = time.perf_counter()
        ce = 0
        for _ in range(args.steps):
            d_dev.copy_(d_host, non_blocking=True)
            g, rep, c, U, sc = step(d_dev)   # the call returns the scales on the host
            g_host.copy_(g, non_blocking=True)
            U_host.copy_(U, non_blocking=True)
            torch.cuda.synchronize()
            ce += c
        barrier()
        te = shard.max_over_ranks(time.perf_counter() - t0, dist, dev)
        ce = shard.sum_over_ranks(ce, dist, dev)
        e2e = {"value": ce / te / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(d_host.numel() * d_host.element_size()),
               "d2h_bytes_per_step": int(g_host.numel() * g_host.element_size() +
                                         U_host.numel() * U_host.element_size() + sc.nbytes),
               "outputs_copied": "gradient (FP32), DTFT fields (FP16) and their scales"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    # dominant kernel = largest accumulated device time among single-kernel entries
    # ("pc_net" groups the preconditioner network's 13 launches per batch)
    roof = roofline_of(prof, peaks, args.groups, t_max / args.steps, args.steps) if prof else None
    iters = [int(max(r["iters"])) for r in reps]
    cg_ms = [r["ms_total"] for r in reps]

    def run_compare():
        # the comparison runs on the context itself (the groups' scratch freed first)
        if args.groups > 1:
            ctx.set_shot_groups(1)
        # CG alone on the same system with each preconditioner (untimed by the steps above)
        # the true residual ||S^T d - (S^T S + beta B^2) q|| / ||S^T d|| of each solution, on the
        # first and last shot (a two-shot context keeps the extra memory to a few GB)
        sel = [0, ns - 1]
        ctx2 = esi.Context(v0, wl.dx, wl.dt, nt, wl.nb, geom.select(sel), vref=vref)
        d2 = torch.cat([ctx.traces_of(dobs, s).reshape(-1) for s in sel]).contiguous()
        b_rhs, _ = ctx2.adjoint(d2)

        def true_rel_res():
            q2 = q[sel].contiguous()
            res = ctx2.normal_apply(q2, beta)
            torch.sub(b_rhs, res, out=res)
            num = res.reshape(len(sel), -1).norm(dim=1)
            den = b_rhs.reshape(len(sel), -1).norm(dim=1)
            del res, q2
            return float((num / den).max())

        def cg_only(pc, cap, data_space=False):
            torch.cuda.synchronize()
            ctx.set_velocity(v0)
            _, r = ctx.cg_solve(dobs, lam=beta, tol=args.tol, max_iter=cap, out=q, precond=pc,
                                data_space=data_space)
            return {"iters_max": int(max(r["iters"])), "time_ms": r["ms_total"],
                    "true_rel_res_first_last_shot": true_rel_res(),
                    "reached_tol": bool(r["converged"]),
                    "rel_res_max_over_shots": float(max(x[-1] for x in r["rel_res"] if x.size)),
                    "device_ms": {"product": r["ms_matvec"], "vector": r["ms_vector"],
                                  "precond": r["ms_precond"]}}
        compare = {}
        if args.plain_iter > 0:
            compare["none"] = cg_only("none", args.plain_iter)
        compare["diag"] = cg_only("diag", args.max_iter)
        # the same ESI system in data space (section "Switching from the wavefield to data space");
        # its stopping test is on the data-space residual, so it is also run to tol / 10 to
        # compare at a matching true residual
        compare["data_space"] = cg_only("none", args.max_iter, data_space=True)
        tol0 = args.tol
        args.tol = tol0 / 10
        compare["data_space_tol_div10"] = cg_only("none", args.max_iter, data_space=True)
        args.tol = tol0
        # frequency-domain ESI by time-domain modelling (section "Frequency domain inversion by
        # time domain modelling"): CG on F A F^H qbar / nt = F S^T d at the DTFT frequencies, its
        # vectors nf complex fields per shot instead of nt real ones (the residual is that of the
        # frequency-domain system)
        torch.cuda.synchronize()
        ctx.set_velocity(v0)
        qb, r = ctx.cg_solve(dobs, lam=beta, tol=args.tol, max_iter=args.max_iter, freqs=freqs,
                             precond="diag")
        compare["frequency_domain"] = {
            "precond": "diag", "freqs_hz": freqs, "iters_max": int(max(r["iters"])), "time_ms": r["ms_total"],
            "reached_tol": bool(r["converged"]),
            "rel_res_max_over_shots": float(max(x[-1] for x in r["rel_res"] if x.size)),
            "device_ms": {"product": r["ms_matvec"], "vector": r["ms_vector"]},
            "cg_vector_bytes_per_shot": int(qb[0].numel() * qb.element_size()),
            "time_domain_cg_vector_bytes_per_shot": int(q[0].numel() * q.element_size())}
        del qb
        if have_pc:
            compare["learned"] = cg_only("learned", args.max_iter)
            compare["learned"]["fallbacks"] = ctx.pc_fallbacks
        del b_rhs
        ctx2.close()
        return compare
    compare = None if args.no_compare else run_compare()
    cb = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cb = cpu_baseline()
        except Exception as ex:  # the baseline is a report, never a blocker
            cb = {"error": str(ex)}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(ns, nt), "grid": "801x241 (z 241, x 801)",
                   "nt": nt, "shots_per_gpu": ns, "tol": args.tol, "beta": beta,
                   "freqs_hz": freqs, "precond": precond, "beta_factor": args.beta_factor,
                   "shot_groups": args.groups,
                   "l2": "inputs larger than L2 (CG vectors 4 x %.2f GB per GPU)"
                         % (4 * ns * nt * N / 1e9)},
        "cg": {"precond": precond, "iters_max_per_step": iters, "time_to_tol_ms": cg_ms,
               "converged": [bool(r["converged"]) for r in reps],
               "rel_res_max_over_shots": float(max(r[-1] for r in reps[-1]["rel_res"] if r.size)),
               "compare": compare},
        "roofline": roof, "kernels": prof, "cpu_baseline": cb, "e2e": e2e,
        "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
