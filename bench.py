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
CPU_BASELINE_TARGETS = 6144          # about 10 s of FP64 direct sum on 16 host cores at N = 2^20
METRIC = "MLFMA matvec points/s at stated rel. err vs FP64 direct; % HBM roofline"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_time_and_value(ms, points_per_rank, ws, dist=None, device="cpu"):
    """Replicas: the step time is the slowest rank's (max over ranks) and the value is the
    whole job's points per second, ws x points_per_rank / that time."""
    if dist is not None and ws > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, points_per_rank * ws / (ms / 1e3)


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


def work_model(info, cb=8):
    """Algorithmic work per apply and per stage (cb = bytes per complex number).

    M2L: 8 flops per complex MAC over the V pairs; unique bytes = F read + G write per box and
    sample + the 316 K operators of each level.  M2M: one read of every child signature F_c and
    one write of every parent signature F_p per level pair; L2L: one read of every parent G_p and
    a read-modify-write of every child G_c (the HBM bytes a fused interpolation must move)."""
    nl, top = info["nlev"], info["top"]
    m2l_flops = sum(8.0 * info["nv"][l] * info["K"][l] for l in range(top, nl + 1))
    m2l_bytes = sum(info["nbox"][l] * info["K"][l] * 2 * cb + 316 * info["K"][l] * cb for l in range(top, nl + 1))
    m2m_bytes = l2l_bytes = 0.0
    for l in range(top, nl):
        fc = info["nbox"][l + 1] * info["K"][l + 1] * cb
        fp = info["nbox"][l] * info["K"][l] * cb
        m2m_bytes += fc + fp
        l2l_bytes += fp + 2 * fc
    return {"M2L": {"flops": m2l_flops, "bytes": m2l_bytes}, "M2M": {"bytes": m2m_bytes},
            "L2L": {"bytes": l2l_bytes}}


def fp32_alu_peak(dev, sm_mhz):
    """FP32 FMA peak derived from the device: SMs (read at run time) x 128 FP32 lanes per SM
    (Blackwell) x 2 flops x the maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12, sms


KERNEL_SOURCES = ("paper_2006_15367_gb300/csrc/far.cu", "paper_2006_15367_gb300/csrc/common.cuh")


def source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(workload, precision, nrhs, mode):
    """DRAM bytes (read + write) of k_m2l per step from a committed ncu summary, or None.

    The summary records the hash of the kernel sources it was taken on; a different hash
    (the kernel changed since) gives None.
    """
    if (workload, precision, nrhs, mode) != ("sphere1m", "fp32", 1, "apply"):
        return None
    p = os.path.join(ROOT, "profiles", "k_m2l_sphere1m.md")
    if not os.path.exists(p):
        return None
    vals = {}
    for ln in open(p):
        if ln.startswith("- ") and ":" in ln:
            k, v = ln[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha256_16") != source_hash() or "dram_bytes_per_step" not in vals:
        return None
    return {"bytes_per_step": float(vals["dram_bytes_per_step"]), "source": "profiles/k_m2l_sphere1m.md"}


def oracle_mlfma_rate(name="sphere256k"):
    """The oracle's plain FP64 MLFMA (numpy) on a sphere of the bench workload's family (same point
    density, quarter-wavelength leaves, 3 digits; 2^18 points on radius 16 by default): points/s
    of one apply (setup excluded), the CPU rate of the same fast algorithm beside the direct sum.
    A failure is reported, not fatal."""
    try:
        import synth
        from oracle import mlfma as om
        pts, q, prm = synth.workload(name)
        t0 = time.perf_counter()
        o = om.OracleMLFMA(pts, prm["k"], prm["digits"])
        setup = time.perf_counter() - t0
        t0 = time.perf_counter()
        o.apply(q[0])
        dt = time.perf_counter() - t0
        return {"kind": "oracle MLFMA (numpy, FP64)", "workload": WORKLOADS[name], "n": int(pts.shape[0]),
                "value": pts.shape[0] / dt, "unit": "points/s", "apply_s": dt, "setup_s": setup,
                "cores": os.cpu_count(), "threads": "numpy: BLAS calls may use every core, the stage loops one"}
    except Exception as e:                                # pragma: no cover - reported in the line
        return {"error": f"{type(e).__name__}: {e}"[:200]}


def run_reference(args, ws, rank):
    """CPU oracle: FP64 direct sum at a bounded sample of targets per step."""
    if rank != 0:
        return 0
    import synth
    from oracle import direct
    pts, q, prm, _ = load_case(args.workload)
    if args.digits:
        prm = dict(prm, digits=args.digits)
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
    line = {"impl": "reference", "metric": METRIC, "value": v,
            "unit": "points/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, n, prm),
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": cores, "kind": "oracle",
                             "sample": f"FP64 direct sum over all {n} sources at {per_step} random targets per step"},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


WORKLOADS = {
    "sphere1m": "sphere N=1048576 r=32 wavelengths (k=2pi), leaf 0.25 wavelength, 9 levels, 3 digits",
    "sphere256k": "sphere N=262144 r=16 wavelengths (k=2pi), leaf 0.25 wavelength, 8 levels, 3 digits",
    "sphere4k": "sphere N=4096 r=2 wavelengths (k=2pi), leaf 0.25 wavelength, 5 levels, 3 digits",
    "cubeclusters4m": "cube surface 32 wavelengths (70%) + 64 Gaussian clusters sigma 0.05 (30%), N=4194304, "
                      "adaptive leaf_max=64, far field down to 0.25-wavelength boxes, 4 digits",
    "cubeclusters512k": "cube surface 32 wavelengths (70%) + 64 Gaussian clusters sigma 0.05 (30%), N=524288, "
                        "adaptive leaf_max=64, far field down to 0.25-wavelength boxes, 4 digits",
    "ellipsoid256k": "ellipsoid (8,4,2) wavelengths N=262144, leaf 0.25 wavelength, 3 digits",
    "batch256": "256 random ellipsoids (semi-axes U(2,16) wavelengths, N log-uniform 1000..65536) in one batched "
                "plan, leaf 0.25 wavelength, 3 digits",
}


def _time_ms(fn, stream, steps, warmup=2):
    """Mean CUDA-event time of fn() on stream (after warm-up)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def _rel_err(mf, torch, ptd, q0, k, out, n, ntg=500, seed=7):
    rng = np.random.default_rng(seed)
    tg = np.sort(rng.choice(n, min(ntg, n), replace=False))
    dev = ptd.device
    dref = mf.direct_fp64(ptd, torch.as_tensor(q0, device=dev), k, torch.as_tensor(tg, device=dev))
    got = out.to(torch.complex128)[torch.as_tensor(tg, device=dev)]
    return float(torch.linalg.norm(got - dref) / torch.linalg.norm(dref))


def measure_forms(dev, pts, q, prm, fp32_ms):
    """The precision, batching and adjoint forms against the plain paths, same geometry and digits.

    precision: the plain FP64 path vs the FP32 (and split-TF32 tensor-core) paths at the same
    digits; batching: 64 right-hand sides per apply vs one, and one plan over 64 ellipsoids vs
    64 separate plans; adjoint: forward + backward (charges and positions) vs one apply;
    solve: restarted GMRES around the matvec, time per matvec against one apply.
    """
    import torch
    import paper_2006_15367_gb300 as mf
    import synth
    out = {}
    n = pts.shape[0]
    ptd = torch.as_tensor(pts, device=dev)

    def guarded(name, fn):
        try:
            out[name] = fn()
        except Exception as e:                    # a form that fails is reported, not fatal
            out[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
        torch.cuda.empty_cache()

    def precision(prec, sampled=0):
        cdt = np.complex128 if prec == "fp64" else np.complex64
        qd = torch.as_tensor(q[0].astype(cdt), device=dev)
        res = torch.empty_like(qd)
        plan = mf.Plan(ptd, prm["k"], prm["digits"], precision=prec, sampled_operators=sampled)
        t = _time_ms(lambda: plan.apply(qd, res), plan.stream, 3)
        err = _rel_err(mf, torch, ptd, q[0], prm["k"], res, n)
        info = plan.info()
        plan.close()
        return {"ms": t, "rel_err_vs_fp64_direct": err, "device_bytes": info["device_bytes"],
                "setup_ms": info["setup_ms"], "sampled_levels": [l for l, v in enumerate(info["sampled"]) if v]}

    guarded("fp64", lambda: precision("fp64"))
    guarded("tf32x3", lambda: precision("tf32x3"))
    guarded("bf16x3", lambda: precision("bf16x3"))
    if "ms" in out.get("fp64", {}):
        out["fp64"]["note"] = "plain FP64 path, same digits"
        out["fp32_speedup_vs_fp64"] = out["fp64"]["ms"] / fp32_ms
        if "ms" in out.get("tf32x3", {}):
            out["tf32x3_speedup_vs_fp64"] = out["fp64"]["ms"] / out["tf32x3"]["ms"]
            out["tf32x3_speedup_vs_fp32"] = fp32_ms / out["tf32x3"]["ms"]
        if "ms" in out.get("bf16x3", {}):
            out["bf16x3_speedup_vs_fp32"] = fp32_ms / out["bf16x3"]["ms"]

    # sampled translation operators (Sec. 3.2.3) at the levels with boxes of a wavelength or
    # more, against the full operator tables: time, accuracy, plan memory and creation time
    def sampled(prec, s):
        full = out["fp64"] if prec == "fp64" else precision(prec)
        smp = precision(prec, s)
        if "ms" not in full:
            return smp
        smp.update({"oversampling": s, "full_ms": full["ms"], "full_rel_err": full["rel_err_vs_fp64_direct"],
                    "full_device_bytes": full["device_bytes"], "full_setup_ms": full["setup_ms"],
                    "bytes_saved": full["device_bytes"] - smp["device_bytes"], "time_ratio": smp["ms"] / full["ms"]})
        return smp

    guarded("sampled_operators_fp32", lambda: sampled("fp32", 6))
    guarded("sampled_operators_fp64", lambda: sampled("fp64", 8))

    def nrhs64():
        Q = synth.complex_normal(2003, n, nrhs=64).astype(np.complex64)
        qd = torch.as_tensor(Q, device=dev)
        res = torch.empty_like(qd)
        plan = mf.Plan(ptd, prm["k"], prm["digits"], precision="fp32")
        t = _time_ms(lambda: plan.apply(qd, res), plan.stream, 2, warmup=1)
        err = _rel_err(mf, torch, ptd, Q[5], prm["k"], res[5], n)
        plan.close()
        return {"ms": t, "ms_per_rhs": t / 64, "speedup_per_rhs_vs_single": fp32_ms / (t / 64),
                "rel_err_rhs5": err}

    guarded("nrhs64", nrhs64)

    def geometries():
        geoms, sizes, _ = synth.ellipsoid_batch(64, seed=4001)
        allp = np.concatenate(geoms)
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        Q = synth.complex_normal(4002, allp.shape[0])[0].astype(np.complex64)
        ap = torch.as_tensor(allp, device=dev)
        qd = torch.as_tensor(Q, device=dev)
        res = torch.empty_like(qd)
        plan = mf.Plan(ap, prm["k"], prm["digits"], precision="fp32", offsets=off)
        tb = _time_ms(lambda: plan.apply(qd, res), plan.stream, 3)
        plan.close()
        ts = 0.0
        for g in range(64):
            a, b = int(off[g]), int(off[g + 1])
            pg = mf.Plan(ap[a:b].contiguous(), prm["k"], prm["digits"], precision="fp32")
            qg = qd[a:b].contiguous()
            rg = torch.empty_like(qg)
            ts += _time_ms(lambda: pg.apply(qg, rg), pg.stream, 3)
            pg.close()
        return {"geometries": 64, "points": int(allp.shape[0]), "batched_ms": tb, "separate_plans_ms": ts,
                "speedup": ts / tb}

    guarded("geometries64", geometries)

    def adjoint():
        pe, qe, pre = synth.workload("ellipsoid256k")
        pdev = torch.as_tensor(pe, device=dev)
        qd = torch.as_tensor(qe[0].astype(np.complex64), device=dev)
        tgt = torch.as_tensor(synth.complex_normal(5003, pe.shape[0])[0].astype(np.complex64), device=dev)
        plan = mf.Plan(pdev, pre["k"], pre["digits"], precision="fp32")
        res = torch.empty_like(qd)
        ta = _time_ms(lambda: plan.apply(qd, res), plan.stream, 3)
        rt = pdev.clone().requires_grad_(True)

        def fb():
            qv = qd.detach().requires_grad_(True)
            phi = mf.mlfma(qv, rt, plan)
            torch.sum(torch.abs(phi - tgt) ** 2).backward()
        tg = _time_ms(fb, plan.stream, 3)
        plan.close()
        return {"workload": "ellipsoid (8,4,2) N=262144", "apply_ms": ta, "forward_backward_ms": tg,
                "ratio": tg / ta}

    guarded("adjoint", adjoint)

    def gmres():
        # the iterative solve the matvec serves (Sec. 1): (sigma I + A) x = b on the same sphere.
        # At fixed point density the propagating part of the spectrum of A grows like the
        # radius R, so the shift scales with R: sigma = 50 i R keeps the system as well
        # conditioned as sigma = 100 i on the 2-wavelength-radius sphere (kappa 8.6).
        R = float(np.max(np.linalg.norm(pts - pts.mean(axis=0), axis=1)))
        sigma = 50j * R
        b = torch.as_tensor(synth.complex_normal(2004, n)[0].astype(np.complex64), device=dev)
        plan = mf.Plan(ptd, prm["k"], prm["digits"], precision="fp32")
        plan.apply(b)                              # captures the apply graph outside the timing
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, info = plan.solve(b, sigma=sigma, tol=1e-3, restart=30, max_iter=200)
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0)
        plan.close()
        rng = np.random.default_rng(11)
        tg = torch.as_tensor(np.sort(rng.choice(n, 2000, replace=False)), device=dev)
        ax = mf.direct_fp64(ptd, x.to(torch.complex128), prm["k"], tg)
        bs, xs = b.to(torch.complex128)[tg], x.to(torch.complex128)[tg]
        true_res = float(torch.linalg.norm(bs - sigma * xs - ax) / torch.linalg.norm(bs))
        return {"system": f"({sigma.imag:.0f}i I + A) x = b, b complex normal, GMRES(30), tol 1e-3, FP32 plan",
                "iterations": info["iterations"], "matvecs": info["matvecs"], "converged": info["converged"],
                "ms": ms, "ms_per_matvec": ms / info["matvecs"], "apply_ms": fp32_ms,
                "krylov_overhead": (ms - info["matvecs"] * fp32_ms) / ms, "rel_residual": info["rel_residual"],
                "true_residual_2000_targets_vs_fp64_direct": true_res}

    guarded("solve", gmres)
    return out


def config_dict(args, n, prm):
    """The workload description shared by both arms of the benchmark."""
    import re
    wl = re.sub(r"\d+ digits", f"{prm['digits']} digits", WORKLOADS[args.workload])
    if args.digits:
        wl += " (digits set on the command line; leaf edge and level count as in the plan object)"
    return {"workload": wl + f", {args.precision.upper()} complex, nrhs={args.nrhs}"
                        + (", forward+backward (charges and positions)" if args.mode == "grad" else "")
                        + (f", sampled operators (oversampling {args.sampled_operators})"
                           if getattr(args, "sampled_operators", 0) else ""),
            "n": n, "digits": prm["digits"], "nrhs": args.nrhs, "mode": args.mode,
            "parallelism": f"replicas x{_dist()[0]}",
            "l2": "flushed between steps (256 MiB write outside the timed events)"}


def load_case(name):
    """(points, charges [1][n], params, offsets or None)."""
    import synth
    if name == "batch256":
        geoms, sizes, axes = synth.ellipsoid_batch(256, seed=4001)
        pts = np.concatenate(geoms)
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        q = synth.complex_normal(4002, pts.shape[0])
        return pts, q, dict(k=synth.K_WAVE, digits=3, leaf_max=0), off
    pts, q, prm = synth.workload(name)
    return pts, q, prm, None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu", action="store_true",
                    help="profile-region mode: warm up, then run one step between cudaProfilerStart/Stop and exit")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "tf32x3", "bf16x3"])
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--digits", type=int, default=0, help="override the workload's digits (0: keep)")
    ap.add_argument("--sampled-operators", type=int, default=0,
                    help="oversampling of sampled translation operators at the wavelength-sized levels (0: full tables)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the default interpolation tile budgets instead of the plan-time autotuner "
                         "(--ncu always does: kernels outside the capture run slower under the profiler)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the precision / batching / adjoint form comparisons added to the JSON line")
    ap.add_argument("--mode", default="apply", choices=["apply", "grad"],
                    help="apply: phi = A q; grad: forward + backward of sum |phi - t|^2 for q and the positions")
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

    pts, q, prm, offsets = load_case(args.workload)
    if args.digits:
        prm = dict(prm, digits=args.digits)
    n = pts.shape[0]
    nrhs = args.nrhs
    ptd = torch.as_tensor(pts, device=dev)
    cdt = np.complex128 if args.precision == "fp64" else np.complex64
    Q = q[0] if nrhs == 1 else synth.complex_normal(2003, n, nrhs=nrhs)
    qd = torch.as_tensor(Q.astype(cdt), device=dev)
    out = torch.empty_like(qd)
    plan = mf.Plan(ptd, prm["k"], prm["digits"], leaf_max=prm.get("leaf_max", 0), precision=args.precision,
                   offsets=offsets, autotune=not (args.no_autotune or args.ncu), sampled_operators=args.sampled_operators)
    info = plan.info()
    stream = plan.stream

    if args.mode == "grad":
        tgt = torch.as_tensor(synth.complex_normal(5003, n)[0].astype(cdt), device=dev)
        rt = ptd.clone().requires_grad_(True)

        def step():
            qv = qd.detach().requires_grad_(True)
            phi = mf.mlfma(qv, rt, plan)
            loss = torch.sum(torch.abs(phi - tgt) ** 2)
            loss.backward()
            out.copy_(phi.detach())
            return qv.grad
    else:
        def step():
            plan.apply(qd, out)

    if args.ncu:
        for _ in range(2):
            step()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        plan.close()
        return 0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # ---- warm-up
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            step()
    torch.cuda.synchronize()

    # ---- launches per step (profiling pass, outside the timed region)
    plan.profile(True)
    step()
    tm = plan.timings(reset=True)
    plan.profile(False)
    launches_per_step = int(sum(tm["launches"].values()))
    m2l_launches = int(tm["launches"]["M2L"])

    # ---- timed region: K steps, L2 flushed between steps, device time by CUDA events
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.fill_(float(i))
                evs[i][0].record(stream)
                step()
                evs[i][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    ms, value = job_time_and_value(ms, n * nrhs, ws, dist, dev)

    # ---- per-stage times (CUDA events on the plan stream), same workload
    plan.profile(True)
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i))
            step()
    tm = plan.timings(reset=True)
    plan.profile(False)
    steps_done = max(args.steps, 1)
    stage_ms = {k: v / steps_done for k, v in tm["ms"].items()}

    # ---- end to end: inputs from pinned host memory, result read back, inside the timed region
    qh = torch.empty(tuple(qd.shape), dtype=qd.dtype, pin_memory=True)
    qh.copy_(qd.cpu())
    ph = torch.empty(tuple(qd.shape), dtype=qd.dtype, pin_memory=True)
    if args.mode == "apply":
        def e2e_step():
            mf.mlfma_apply(plan.handle, qh, ph, nrhs)
        h2d, d2h = qh.numel() * qh.element_size(), ph.numel() * ph.element_size()
    else:
        gh = torch.empty(tuple(qd.shape), dtype=qd.dtype, pin_memory=True)

        def e2e_step():
            qd.copy_(qh, non_blocking=True)
            gq = step()
            gh.copy_(gq, non_blocking=True)
            torch.cuda.current_stream().synchronize()
        h2d, d2h = qh.numel() * qh.element_size(), gh.numel() * gh.element_size()
    for _ in range(2):
        e2e_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e = {"value": n * nrhs * ws / e2e_s, "unit": "points/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h)}

    # ---- accuracy: GPU FP64 direct sum at sampled targets (first right-hand side)
    rng = np.random.default_rng(2001)
    q0 = Q if nrhs == 1 else Q[0]
    o0 = out if nrhs == 1 else out[0]
    if offsets is None:
        tg = np.sort(rng.choice(n, SAMPLE_TARGETS, replace=False))
        dref = mf.direct_fp64(ptd, torch.as_tensor(q0, device=dev), prm["k"], torch.as_tensor(tg, device=dev))
        got = o0.to(torch.complex128)[torch.as_tensor(tg, device=dev)]
        groups = [(0, n, tg)]
    else:
        gsel = np.sort(rng.choice(len(offsets) - 1, 8, replace=False))
        groups, drefs, gots = [], [], []
        for g in gsel:
            a, b = int(offsets[g]), int(offsets[g + 1])
            tgl = np.sort(rng.choice(b - a, min(250, b - a), replace=False))
            drefs.append(mf.direct_fp64(ptd[a:b].contiguous(), torch.as_tensor(q0[a:b], device=dev), prm["k"],
                                        torch.as_tensor(tgl, device=dev)))
            gots.append(o0[a:b].to(torch.complex128)[torch.as_tensor(tgl, device=dev)])
            groups.append((a, b, tgl))
        dref, got = torch.cat(drefs), torch.cat(gots)
    rel_err = float(torch.linalg.norm(got - dref) / torch.linalg.norm(dref))

    # ---- roofline of the dominant kernel: k_m2l (one launch per far level, timed by the M2L stage events)
    pk, pk_kind = peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0)
    fp32_peak, nsm = fp32_alu_peak(dev, sm_max)               # TFLOP/s, FMA = 2 flops
    roof = {"kernel": "k_m2l", "bound": "alu", "peak": fp32_peak, "unit": "TFLOP/s", "achieved": None, "frac": None,
            "traffic": None,
            "peak_source": f"derived: {nsm} SMs (device query) x 128 FP32 lanes x 2 flops x {sm_max:.0f} MHz "
                           f"(maximum SM clock from MEASURED_PEAKS.json)"}
    m2l = None
    stages = None
    if offsets is None and info["top"]:
        wm = work_model(info, 16 if args.precision == "fp64" else 8)
        reps = nrhs * (2 if args.mode == "grad" else 1)
        ach = wm["M2L"]["flops"] * reps / (stage_ms["M2L"] / 1e3) / 1e12
        roof.update({"achieved": ach, "frac": ach / fp32_peak, "launches_per_step": int(m2l_launches),
                     "work": "8 flops per complex MAC x sum over levels of nv_l K_l (per step, all launches of "
                             "k_m2l and k_m2l_tail)"})
        tr = None if args.sampled_operators else measured_traffic(args.workload, args.precision, nrhs, args.mode)
        if tr is not None:
            roof["traffic"] = tr["bytes_per_step"]
            roof["traffic_source"] = tr["source"]
        m2l = {"ms": stage_ms["M2L"], "flops": wm["M2L"]["flops"] * reps, "unique_bytes": wm["M2L"]["bytes"] * reps,
               "tflops": ach,
               "hbm_frac_unique_bytes": wm["M2L"]["bytes"] * reps / (stage_ms["M2L"] / 1e3) / 1e9 / pk["hbm_gbs"]}
        stages = {}
        for s in ("M2M", "L2L"):
            b = wm[s]["bytes"] * reps
            gbs = b / (stage_ms[s] / 1e3) / 1e9
            stages[s] = {"ms": stage_ms[s], "algorithmic_bytes": b, "achieved_gbs": gbs,
                         "hbm_frac": gbs / pk["hbm_gbs"],
                         "bytes_model": "M2M: F_c read + F_p write; L2L: G_p read + G_c read and write (per level pair)"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import direct
        a, b, tgl = groups[0]
        ct = tgl if offsets is not None else np.sort(
            np.random.default_rng(77).choice(b - a, min(CPU_BASELINE_TARGETS, b - a), replace=False))
        t0 = time.perf_counter()
        cref = direct.direct(pts[a:b], q0[a:b], prm["k"], targets=ct)
        cdt_s = time.perf_counter() - t0
        o0h = o0.cpu().numpy()[a:b]
        cpu = {"value": ct.shape[0] / cdt_s, "unit": "points/s", "cores": direct.max_threads(), "kind": "oracle",
               "sample": f"FP64 direct sum (oracle, C/OpenMP) at {ct.shape[0]} sampled targets over all {b - a} "
                         f"sources of their geometry",
               "rel_err_gpu_vs_oracle_direct": float(np.linalg.norm(o0h[ct] - cref) / np.linalg.norm(cref)),
               "oracle_mlfma": oracle_mlfma_rate()}

    cfg = config_dict(args, n, prm)
    line = {
        "metric": METRIC,
        "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "c64 (fp32)", "fp64": "c128 (fp64)", "tf32x3": "c64 (fp32; theta maps split-tf32 x3 on "
                  "tensor cores)", "bf16x3": "c64 (fp32; theta maps split-bf16 x3 on tensor cores)"}[args.precision], "data": "synthetic", "config": cfg,
        "accuracy": {"rel_err_vs_fp64_direct": rel_err, "targets": int(sum(len(g[2]) for g in groups)),
                     "reference": "GPU FP64 direct sum"},
        "plan": {"levels": info["nlev"], "top": info["top"], "L": info["L"], "n_geom": info["n_geom"],
                 "device_bytes": info["device_bytes"], "autotune": not args.no_autotune,
                 "tile_bytes": info["tile_bytes"]},
        "stage_ms": stage_ms, "setup_ms": info["setup_ms"], "m2l": m2l, "interp_rates": stages,
        "roofline": roof, "peaks_source": pk_kind, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
    }
    line["clocks"] = clk.summary()
    plan.close()
    if rank == 0 and not args.no_forms and args.workload == WORKLOAD and args.precision == "fp32" and nrhs == 1 \
            and args.mode == "apply":
        line["forms"] = measure_forms(dev, pts, q, prm, ms)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
