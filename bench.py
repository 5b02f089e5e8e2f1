#!/usr/bin/env python
"""Benchmark of the theta-method hot path (plain Cholesky form vs modal form).

One bench step = one pass of the whole hot path over the workload: constraint
elimination, plain setup (Cholesky of Z) and T plain theta-steps, modal setup
(Cholesky of R_i, reduction, tridiagonalisation, tridiagonal eigensolver,
back-transform, projections) and T modal theta-steps, with probe outputs every
step and current snapshots.  Inputs are resident in HBM before timing.

Prints ONE JSON line.  `value` is the modal form's transient throughput in
theta-steps/s; setup seconds and the plain form's numbers ride along.
`--impl reference` times the FP64 CPU oracle (the deliberately slow plain
definition) on the host cores instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (builder kwargs, description)
    "n8192_electrodes": dict(kind="config2", T=20000, snap=100,
                             desc="N=8192 plate (32x32x8), 2 electrodes with a 1 A step, 16 pickups, "
                                  "dt=0.5us, theta=1/2, T=20000, snapshots every 100 steps, FP64"),
    "n65536_coil": dict(kind="config4", T=100000, snap=1000,
                        desc="N=65536 plate (64x64x16), one coil sin 10 kHz, 4 pickups, dt=0.1us, "
                             "theta=1/2, T=100000, snapshots every 1000 steps, FP64"),
    "n512_coil": dict(kind="config1", T=2000, snap=0,
                      desc="N=512 plate (16x8x4), one coil sin 10 kHz, coil self-pickup, dt=1us, "
                           "theta=1/2, T=2000, FP64"),
}
DEFAULT_WORKLOAD = "n8192_electrodes"
METRIC = "modal theta-steps/s (setup s alongside), modal vs Cholesky theta-method"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 2 DFMA/clk/SM x 152 SMs x 2070 MHz


def build_problem(name: str, T: int | None):
    from workloads import synth
    w = WORKLOADS[name]
    T = w["T"] if T is None else T
    if w["kind"] == "config2":
        return synth.config2(T=T, snap_stride=w["snap"])
    if w["kind"] == "config4":
        return synth.config4(T=T, snap_stride=w["snap"])
    return synth.config1(T=T)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines) -> dict:
        """Median SM clock under load, the maximum clock, and every throttle reason seen
        active, from nvidia-smi csv lines (noheader, nounits) in FIELDS order."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_subprocess(workload: str, T_sample: int, threads: int, steps: int, warmup: int) -> dict:
    """Run the oracle timing in a fresh interpreter (spawned, BLAS threads pinned)."""
    code = f"""
import json, os, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
from oracle import theta as orc
import bench
p = bench.build_problem({workload!r}, {T_sample} * ({steps} + {warmup}))
t0 = time.perf_counter()
red = orc.eliminate(p.L, p.R, p.E, p.M, p.MD, p.C)
t1 = time.perf_counter()
Ts = {T_sample}
times = []
Ii = None
k0 = 0
import scipy.linalg as sla
Z = red.Li + p.dt * p.theta * red.Ri
Cz = np.linalg.cholesky(Z)
t2 = time.perf_counter()
for rep in range({steps} + {warmup}):
    a = time.perf_counter()
    tr = orc.theta_plain(red, p.theta, p.dt, p.src[:, k0:k0 + Ts + 1], p.iD[:, k0:k0 + Ts + 1], Ts,
                         None, 0)
    b = time.perf_counter()
    if rep >= {warmup}:
        times.append(b - a)
    k0 += Ts
print(json.dumps({{"elim_s": t1 - t0, "chol_s": t2 - t1, "times": times, "T_sample": Ts}}))
"""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle subprocess failed:\n" + r.stderr[-4000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def reference_arm(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    T_sample = args.oracle_steps
    res = oracle_subprocess(args.workload, T_sample, threads, args.steps, args.warmup)
    per = statistics.mean(res["times"])
    value = T_sample / per
    w = WORKLOADS[args.workload]
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": w["desc"],
                   "bench_step": f"{T_sample} theta-steps of the oracle (plain Cholesky form)"},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": threads, "kind": "oracle",
                         "sample": f"{T_sample} plain-form theta-steps per bench step at the full "
                                   f"workload size; elimination {res['elim_s']:.1f} s and "
                                   f"Cholesky {res['chol_s']:.1f} s untimed"},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def our_arm(args) -> None:
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_11993_gb300 import eddy

    p = build_problem(args.workload, args.T)
    T = p.T
    n, m, S, P = p.n, p.E.shape[0], p.M.shape[1], p.C.shape[0]
    stride = p.snap_stride
    nsnap = T // stride if stride else 0

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)

    Ld, Rd = to_dev(p.L), to_dev(p.R)
    Ed = to_dev(p.E) if m else None
    Md = to_dev(p.M) if S else None
    MDd = to_dev(p.MD) if m else None
    Cd = to_dev(p.C)
    srcd = to_dev(p.src) if S else None
    iDd = to_dev(p.iD) if m else None
    probes_p = torch.empty((T, P), dtype=torch.float64, device=dev)
    probes_m = torch.empty((T, P), dtype=torch.float64, device=dev)
    snaps_p = torch.empty((nsnap, n), dtype=torch.float64, device=dev)
    snaps_m = torch.empty((nsnap, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    DEV = eddy.EC_MEM_DEVICE
    plain = eddy.ThetaMethod("plain", p.theta, p.dt, device=local, stream=stream.cuda_stream,
                             profile=True)
    modal = eddy.ThetaMethod("modal", p.theta, p.dt, device=local, stream=stream.cuda_stream,
                             profile=True)

    def one_step(record):
        plain.setup(Ld, Rd, Ed, Md, MDd, Cd, mem=DEV)
        plain.run(T, srcd, iDd, stride, mem=DEV, probes_out=probes_p, snaps_out=snaps_p)
        tp = plain.timings()
        modal.setup(Ld, Rd, Ed, Md, MDd, Cd, mem=DEV)
        modal.run(T, srcd, iDd, stride, mem=DEV, probes_out=probes_m, snaps_out=snaps_m)
        tm = modal.timings()
        if record is not None:
            record.append((tp, tm))

    for _ in range(args.warmup):
        one_step(None)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_id = vis.split(",")[local] if vis else str(local)
    clocks = ClockSampler(smi_id)
    clocks.start()
    rec = []
    launches0 = eddy.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(args.steps):
        one_step(rec)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    launches = eddy.launch_count() - launches0
    clk = clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
        dist.barrier()

    def mean(key, form):
        return statistics.mean(r[0 if form == "plain" else 1][key] for r in rec)

    modal_run_s = mean("run_ms", "modal") / 1e3
    plain_run_s = mean("run_ms", "plain") / 1e3
    modal_setup_s = mean("setup_ms", "modal") / 1e3
    plain_setup_s = mean("setup_ms", "plain") / 1e3
    value = world * T / modal_run_s

    # dominant kernel: whichever timed family holds the most device time per bench step
    n0 = n - m
    fwd_ms = mean("fwd_ms", "plain") / max(1.0, mean("fwd_launches", "plain"))
    bwd_ms = mean("bwd_ms", "plain") / max(1.0, mean("bwd_launches", "plain"))
    fam = {
        "plain forward solve (tile_trmv_kernel<false>)": fwd_ms * T,
        "plain backward solve (tile_trmv_kernel<true>)": bwd_ms * T,
        "modal setup (FP64 eigensolver pipeline)": mean("setup_ms", "modal"),
    }
    dominant = max(fam, key=fam.get)
    # roofline of the plain step's forward solve y = C^{-1} b (FP64-pipe bound on GB300)
    flops_fwd = float(n0) * float(n0)          # n0(n0+1)/2 multiply-adds
    bytes_fwd = 8.0 * n0 * (n0 + 1) / 2.0
    achieved = flops_fwd / (fwd_ms * 1e-3) / 1e12
    pk, pk_kind = peaks()
    roofline = {"kernel": "tile_trmv_kernel<false>", "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": None, "algorithmic_bytes": bytes_fwd,
                "achieved_gbs": bytes_fwd / (fwd_ms * 1e-3) / 1e9,
                "hbm_peak_gbs": pk.get("hbm_gbs"), "hbm_frac": bytes_fwd / (fwd_ms * 1e-3) / 1e9 / pk.get("hbm_gbs", 1.0),
                "peak_note": "FP64 peak derived from unit counts: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz "
                             f"(HBM peak {pk_kind})",
                "avg_launch_ms": fwd_ms, "dominant_family": dominant}
    # DRAM traffic from the committed ncu summary of this kernel, scaled by N0^2
    traffic_path = os.path.join(ROOT, "profiles", "tile_trmv_n8192.md")
    try:
        tv = {}
        with open(traffic_path) as f:
            for ln in f:
                if ln.startswith("traffic_"):
                    k, v = ln.split(":", 1)
                    tv[k.strip()] = float(v)
        if tv.get("traffic_bytes_per_launch") and tv.get("traffic_n0"):
            roofline["traffic"] = tv["traffic_bytes_per_launch"] * (n0 * n0) / tv["traffic_n0"] ** 2
            roofline["traffic_note"] = "ncu DRAM read+write of one launch (profiles/tile_trmv_n8192.md)"
    except (OSError, ValueError):
        pass

    # FP64-pipe rooflines of the modal setup's dominant phases, from their event-timed
    # durations and the algorithmic flops of the algorithms used: reduction N^3 + N^3/3
    # (left solve, lower-triangle right solve), tridiagonalisation 2 x (2/3) N^3 FMA
    # (symmetric product + lower-triangle rank-2 update), back-transformation 2N^3 + N^3
    # (blocked Householder application + triangular solve)
    nf = float(n0)
    setup_rooflines = {}
    for ph, fl in (("reduce_ms", 4.0 / 3.0 * nf ** 3), ("tridiag_ms", 4.0 / 3.0 * nf ** 3),
                   ("backtransform_ms", 3.0 * nf ** 3)):
        ms_ph = mean(ph, "modal")
        if ms_ph > 0:
            tf = fl / (ms_ph * 1e-3) / 1e12
            setup_rooflines[ph[:-3]] = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS,
                                        "unit": "TFLOP/s", "frac": tf / FP64_PEAK_TFLOPS,
                                        "algorithmic_flop": fl}

    # end to end through the public API with host buffers (modal form)
    e2e = None
    if True:
        hm = eddy.ThetaMethod("modal", p.theta, p.dt, device=local, stream=stream.cuda_stream)
        src_h = p.src if S else None
        iD_h = p.iD if m else None
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        hm.setup(p.L, p.R, p.E if m else None, p.M if S else None, p.MD if m else None, p.C)
        t1 = time.perf_counter()
        pr, sn = hm.run(T, src_h, iD_h, stride)
        t2 = time.perf_counter()
        hm.close()
        e2e = {"value": world * T / (t2 - t1), "unit": "steps/s",
               "h2d_bytes_per_step": 8 * (S + m) * (T + 1),
               "d2h_bytes_per_step": 8 * (T * P + nsnap * n),
               "setup_s": t1 - t0,
               "setup_h2d_bytes": 8 * (2 * n * n + (m + S + m + P) * n),
               "note": "modal form via ThetaMethod with numpy host arrays; run H2D/D2H inside"}

    # precision variants of the modal form on the same workload, error stated against the
    # FP64 run just above (one run each, outside the timed region)
    variants = None
    if rank == 0 and e2e is not None:
        def rel(a, b):
            nb = float(np.linalg.norm(b))
            return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0))
        try:
            variants = {}
            for prec in ("bf16x3", "bf16"):
                hv = eddy.ThetaMethod("modal", p.theta, p.dt, device=local,
                                      stream=stream.cuda_stream, precision=prec)
                hv.setup(p.L, p.R, p.E if m else None, p.M if S else None, p.MD if m else None, p.C)
                pv, sv = hv.run(T, src_h, iD_h, stride)
                tv = hv.timings()
                hv.close()
                variants["modal_" + prec] = {
                    "steps_per_s": T / (tv["run_ms"] / 1e3), "setup_s": tv["setup_ms"] / 1e3,
                    "probe_rel_err_vs_fp64": rel(pv, pr),
                    "snapshot_rel_err_vs_fp64": rel(sv, sn) if nsnap else None}
        except Exception as ex:  # noqa: BLE001 - the main line must still be printed
            variants = {"error": str(ex)[:300]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        res = oracle_subprocess(args.workload, args.oracle_steps, threads, 1, 0)
        per = res["times"][0]
        cpu = {"value": args.oracle_steps / per, "unit": "steps/s", "cores": threads,
               "kind": "oracle",
               "sample": f"{args.oracle_steps} plain-form theta-steps of the FP64 oracle at the "
                         f"full workload size (elimination {res['elim_s']:.1f} s, Cholesky "
                         f"{res['chol_s']:.1f} s untimed)"}

    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    line = {
        "metric": METRIC,
        "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": w["desc"], "N": n, "T": T,
                   "l2": "inputs larger than L2 (L, R: %.0f MB each)" % (8 * n * n / 1e6),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "modal": {"steps_per_s": T / modal_run_s, "setup_s": modal_setup_s,
                  "total_s": modal_setup_s + modal_run_s,
                  "phases_ms": {k: mean(k, "modal") for k in
                                ("elim_ms", "factor_ms", "reduce_ms", "tridiag_ms", "eig_ms",
                                 "backtransform_ms", "project_ms")},
                  "scan_ms_per_launch": mean("scan_ms", "modal") / max(1.0, mean("scan_launches", "modal"))},
        "plain": {"steps_per_s": T / plain_run_s, "setup_s": plain_setup_s,
                  "total_s": plain_setup_s + plain_run_s,
                  "phases_ms": {k: mean(k, "plain") for k in ("elim_ms", "factor_ms")},
                  "fwd_solve_ms": fwd_ms, "bwd_solve_ms": bwd_ms},
        "roofline": roofline,
        "setup_rooflines": setup_rooflines,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "precision_variants": variants,
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--T", type=int, default=None, help="override the workload's step count")
    ap.add_argument("--oracle-steps", type=int, default=40,
                    help="theta-steps per oracle sample (CPU baseline / reference arm)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
