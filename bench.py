"""Benchmark: MLFMA matvec throughput (points/s) on the 2^20-point sphere of radius 32.

Workload: N = 1,048,576 points uniform on a sphere of diameter 64 wavelengths
(k = 2 pi), complex-normal charges, level-uniform tree with quarter-wavelength
leaves (9 levels), 3 digits, FP32 complex path, one right-hand side.  A step is
one apply (near field + C2M, M2M, M2L, L2L, L2O + permutations); the tree and
operators are built once by mlfma_plan_create (timed separately, reported as
setup_ms).

Prints ONE JSON line.  ``--impl reference`` times the CPU oracle (FP64 direct
sum on a bounded sample of targets) instead.  Under torchrun every rank runs an
independent replica (the path has no exchange step); value = points of all
ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "sphere1m"
DIGITS = 3
SAMPLE_TARGETS = 2000


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def work_model(info):
    """Algorithmic work per apply and per stage (roofline section)."""
    nl, top = info["nlev"], info["top"]
    cb = 8  # complex64 bytes
    m2l_flops = sum(8.0 * info["nv"][l] * info["K"][l] for l in range(top, nl + 1))
    m2l_bytes = sum(info["nbox"][l] * info["K"][l] * 2 * cb + 316 * info["K"][l] * cb for l in range(top, nl + 1))
    interp_flops = 0.0
    for l in range(top, nl):
        Lc, Lp = info["L"][l + 1], info["L"][l]
        nc = info["nbox"][l + 1]
        nthc, nphc, nthp, nphp, nm = Lc + 1, 2 * Lc + 2, Lp + 1, 2 * Lp + 2, 2 * Lc + 1
        # dense phi-DFT on the children, real theta map per mode, inverse DFT per (parent, xy-pair)
        dft_c = 8.0 * nc * nthc * nphc * nm
        theta = 4.0 * nc * nm * nthc * nthp
        inv_p = 8.0 * (nc / 2.0) * nthp * nphp * nm
        interp_flops += dft_c + theta + inv_p
    return {"M2L": {"flops": m2l_flops, "bytes": m2l_bytes}, "M2M": {"flops": interp_flops},
            "L2L": {"flops": interp_flops}}


def run_reference(args, ws, rank):
    """CPU oracle: FP64 direct sum at a bounded sample of targets per step."""
    if rank != 0:
        return 0
    import synth
    from oracle import direct
    pts, q, prm = synth.workload(WORKLOAD)
    n = pts.shape[0]
    per_step = 256
    rng = np.random.default_rng(123)
    cores = direct.max_threads()
    for _ in range(args.warmup):
        direct.direct(pts, q[0], prm["k"], targets=rng.choice(n, 16, replace=False))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        direct.direct(pts, q[0], prm["k"], targets=np.sort(rng.choice(n, per_step, replace=False)))
    dt = (time.perf_counter() - t0) / args.steps
    v = per_step / dt
    line = {"impl": "reference", "metric": "MLFMA matvec points/s (rel. err vs FP64 direct)", "value": v,
            "unit": "points/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "sphere N=1048576 r=32 wavelengths, k=2pi, 3 digits", "n": n},
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": cores, "kind": "oracle",
                             "sample": f"FP64 direct sum over all {n} sources at {per_step} random targets per step"},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu", action="store_true",
                    help="profile-region mode: warm up, then run one apply between cudaProfilerStart/Stop and exit")
    ap.add_argument("--workload", default=WORKLOAD, help="synthetic workload name (synth.workload)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    import paper_2006_15367_gb300 as mf
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    pts, q, prm = synth.workload(args.workload)
    n = pts.shape[0]
    ptd = torch.as_tensor(pts, device=dev)
    cdt = np.complex64 if args.precision == "fp32" else np.complex128
    qd = torch.as_tensor(q[0].astype(cdt), device=dev)
    out = torch.empty_like(qd)
    plan = mf.Plan(ptd, prm["k"], prm["digits"], precision=args.precision)
    if args.ncu:
        for _ in range(2):
            plan.apply(qd, out)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        plan.apply(qd, out)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        plan.close()
        return 0
    info = plan.info()
    stream = plan.stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # ---- warm-up
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            plan.apply(qd, out)
    torch.cuda.synchronize()

    # ---- launches per apply (profiling pass, outside the timed region)
    plan.profile(True)
    plan.apply(qd, out)
    tm = plan.timings(reset=True)
    plan.profile(False)
    launches_per_apply = int(sum(tm["launches"].values()))

    # ---- timed region: K applies, L2 flushed between steps, device time by CUDA events
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.fill_(float(i))
                evs[i][0].record(stream)
                plan.apply(qd, out)
                evs[i][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = n * ws / (ms / 1e3)

    # ---- per-stage times (CUDA events on the plan stream), same workload
    plan.profile(True)
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i))
            plan.apply(qd, out)
    tm = plan.timings(reset=True)
    plan.profile(False)
    napp = max(tm["applies"], 1)
    stage_ms = {k: v / napp for k, v in tm["ms"].items()}

    # ---- end to end through the C call with pinned host buffers
    qh = torch.empty(n, dtype=torch.complex64, pin_memory=True)
    qh.copy_(torch.as_tensor(q[0].astype(np.complex64)))
    ph = torch.empty(n, dtype=torch.complex64, pin_memory=True)
    for _ in range(2):
        mf.mlfma_apply(plan.handle, qh, ph, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        mf.mlfma_apply(plan.handle, qh, ph, 1)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e = {"value": n * ws / e2e_s, "unit": "points/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n}

    # ---- accuracy: GPU FP64 direct sum at sampled targets
    rng = np.random.default_rng(2001)
    tg = np.sort(rng.choice(n, SAMPLE_TARGETS, replace=False))
    dref = mf.direct_fp64(ptd, torch.as_tensor(q[0], device=dev), prm["k"], torch.as_tensor(tg, device=dev))
    got = out.to(torch.complex128)[torch.as_tensor(tg, device=dev)]
    rel_err = float(torch.linalg.norm(got - dref) / torch.linalg.norm(dref))

    # ---- roofline of the dominant stage
    pk, pk_kind = peaks()
    wm = work_model(info)
    dom = max((s for s in ("M2L", "M2M", "L2L", "P2P", "C2M", "L2O")), key=lambda s: stage_ms.get(s, 0.0))
    sm_max = pk.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s, FMA = 2 flops
    roof = {"kernel": dom}
    if dom in wm:
        fl = wm[dom]["flops"]
        ach = fl / (stage_ms[dom] / 1e3) / 1e12
        roof.update({"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                     "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (clock from MEASURED_PEAKS.json)",
                     "traffic": None})
    else:
        roof.update({"bound": "alu", "achieved": None, "peak": fp32_peak, "unit": "TFLOP/s", "frac": None,
                     "traffic": None})
    m2l = {"ms": stage_ms["M2L"], "flops": wm["M2L"]["flops"], "unique_bytes": wm["M2L"]["bytes"],
           "tflops": wm["M2L"]["flops"] / (stage_ms["M2L"] / 1e3) / 1e12,
           "hbm_frac_unique_bytes": wm["M2L"]["bytes"] / (stage_ms["M2L"] / 1e3) / 1e9 / pk["hbm_gbs"]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import direct
        ct = tg[:512]
        t0 = time.perf_counter()
        cref = direct.direct(pts, q[0], prm["k"], targets=ct)
        cdt = time.perf_counter() - t0
        cpu = {"value": ct.shape[0] / cdt, "unit": "points/s", "cores": direct.max_threads(), "kind": "oracle",
               "sample": f"FP64 direct sum (oracle, C/OpenMP) at {ct.shape[0]} of the {SAMPLE_TARGETS} sampled "
                         f"targets over all {n} sources",
               "rel_err_gpu_vs_oracle_direct": float(np.linalg.norm(out.cpu().numpy()[ct] - cref) /
                                                     np.linalg.norm(cref))}

    line = {
        "metric": "MLFMA matvec points/s at stated rel. err vs FP64 direct; % HBM roofline",
        "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64 (fp32)",
        "data": "synthetic",
        "config": {"workload": "sphere N=1048576 r=32 wavelengths (k=2pi), leaf 0.25 wavelength, 9 levels, "
                               "3 digits, FP32 complex, nrhs=1", "n": n, "digits": DIGITS, "nrhs": 1,
                   "levels": info["nlev"], "L": info["L"], "parallelism": f"replicas x{ws}",
                   "l2": "flushed between steps (256 MiB write outside the timed events)"},
        "accuracy": {"rel_err_vs_fp64_direct": rel_err, "targets": SAMPLE_TARGETS, "reference": "GPU FP64 direct sum"},
        "stage_ms": stage_ms, "setup_ms": info["setup_ms"], "m2l": m2l,
        "roofline": roof, "peaks_source": pk_kind, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches_per_apply * args.steps,
    }
    line["clocks"] = clk.summary()
    if rank == 0:
        print(json.dumps(line))
    plan.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
