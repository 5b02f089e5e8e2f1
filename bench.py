#!/usr/bin/env python
"""Benchmark of the theta-method hot path: modal form vs plain (Cholesky) form.

Default workload: the N = 65,536 plate with one coil, 4 pickups, dt = 0.1 us,
theta = 1/2, a 10^5-step transient with snapshots every 1,000 steps, FP64.

Each form is set up ONCE before the timed loop (setup seconds, per phase, the
tridiagonal eigensolver on its own, are reported alongside).  One bench step is
one chunk of theta-steps of BOTH forms continuing the transient: `plain_chunk`
plain steps (two triangular products with the inverse factor each) and
`modal_chunk` modal steps (time-chunked per-mode scan, probe contraction,
snapshot reconstruction).  With the default 5 + 20 steps the modal form covers
the paper's whole 10^5-step transient.  Inputs are resident in HBM before
timing (the factors exceed L2 many times over).

Prints ONE JSON line.  `value` is the modal form's theta-steps/s over the timed
steps; the plain form's rate, both setups, the end-to-end time of 10^5 steps for
each form, the errors (modal vs plain per probe trace and snapshot, the plain
step's equation residual and the modal eigen residuals at full size, computed on
the host from the GPU results) ride along.  `--impl reference` times the FP64
CPU oracle (the deliberately slow plain definition of the method) instead.
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
    # the oracle cannot hold the larger sizes' dense projections in host memory: it is
    # timed on the same recipe at `oracle_n` and scaled by its N^2 per-step cost
    "n65536_coil": dict(kind="config4", n=65536, T=100000, snap=1000, plain_chunk=100,
                        modal_chunk=4000, err_steps=1000, oracle_n=4096, oracle_steps=60,
                        desc="N=65536 plate (64x64x16), one coil sin 10 kHz, 4 pickups, "
                             "dt=0.1us, theta=1/2, T=100000, snapshots every 1000 steps, FP64"),
    "n8192_electrodes": dict(kind="config2", n=8192, T=20000, snap=100, plain_chunk=400,
                             modal_chunk=800, err_steps=400, oracle_n=8192, oracle_steps=10,
                             desc="N=8192 plate (32x32x8), 2 electrodes with a 1 A step, 16 "
                                  "pickups, dt=0.5us, theta=1/2, T=20000, snapshots every 100 "
                                  "steps, FP64"),
    "n512_coil": dict(kind="config1", n=512, T=2000, snap=0, plain_chunk=80, modal_chunk=80,
                      err_steps=80, oracle_n=512, oracle_steps=40,
                      desc="N=512 plate (16x8x4), one coil sin 10 kHz, coil self-pickup, "
                           "dt=1us, theta=1/2, T=2000, FP64"),
}
DEFAULT_WORKLOAD = "n65536_coil"
METRIC = "time steps/s + setup s, modal vs Cholesky θ-method, N=65536, 1 GB300, at stated err"
TOL = 1e-10


def build_problem(name: str, T: int | None = None, n: int | None = None):
    from workloads import synth
    w = WORKLOADS[name]
    T = w["T"] if T is None else T
    n = w["n"] if n is None else n
    if w["kind"] == "config2":
        return synth.config2(T=T, n=n, snap_stride=w["snap"])
    if w["kind"] == "config4":
        return synth.config4(T=T, n=n, snap_stride=w["snap"])
    return synth.config1(T=T, n=n)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


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


def oracle_subprocess(workload: str, n: int, T_sample: int, threads: int, reps: int,
                      form: str) -> dict:
    """Time the oracle (as it stands) in a fresh interpreter with BLAS threads pinned:
    elimination and the form's setup untimed, then `reps` timed samples of T_sample
    theta-steps each, continuing the transient."""
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
from oracle import theta as orc
import bench
p = bench.build_problem({workload!r}, T={T_sample} * {reps}, n={n})
t0 = time.perf_counter()
red = orc.eliminate(p.L, p.R, p.E, p.M, p.MD, p.C)
modes = orc.modal_setup(red.Li, red.Ri) if {form!r} == "modal" else None
t1 = time.perf_counter()
times = []
k0 = 0
I0 = None
for rep in range({reps}):
    src = p.src[:, k0:k0 + {T_sample} + 1]
    iD = p.iD[:, k0:k0 + {T_sample} + 1]
    a = time.perf_counter()
    if {form!r} == "modal":
        tr = orc.theta_modal(red, modes, p.theta, p.dt, src, iD, {T_sample}, I0, 0)
    else:
        tr = orc.theta_plain(red, p.theta, p.dt, src, iD, {T_sample}, I0, 0)
    times.append(time.perf_counter() - a)
    I0 = tr.I_final
    k0 += {T_sample}
print(json.dumps({{"setup_s": t1 - t0, "times": times}}))
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


def oracle_rate(workload: str, T_sample: int, reps: int, form: str) -> dict:
    """Oracle theta-steps/s at the workload's size: measured at the oracle sample size and,
    when that is smaller, scaled by (n_sample / n)^2 -- each oracle step is a few dense
    N^2 products (plain: R_i I and two triangular solves; modal: U^T g and the snapshot
    U x), so its time grows as N^2."""
    w = WORKLOADS[workload]
    threads = os.cpu_count() or 1
    ns = w["oracle_n"]
    res = oracle_subprocess(workload, ns, T_sample, threads, reps, form)
    per = statistics.mean(res["times"]) / T_sample
    scale = (ns / w["n"]) ** 2
    rate = scale / per
    sample = (f"{reps} x {T_sample} {form}-form theta-steps of the FP64 oracle on the same recipe "
              f"at N={ns}" + ("" if ns == w["n"] else
                              f", scaled by (N_sample/N)^2 = {scale:.3g} to N={w['n']} (the "
                              f"oracle cannot hold the N={w['n']} projections in host memory)")
              + f"; elimination and setup {res['setup_s']:.1f} s untimed")
    return {"value": rate, "measured_steps_per_s": 1.0 / per, "sample_n": ns, "cores": threads,
            "sample": sample, "times": res["times"]}


def reference_arm(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    T_sample = args.oracle_steps or w["oracle_steps"]
    r = oracle_rate(args.workload, T_sample, args.steps + args.warmup, "modal")
    timed = r["times"][args.warmup:] or r["times"]
    per_step_s = statistics.mean(timed)
    scale = (r["sample_n"] / w["n"]) ** 2
    r["value"] = scale * T_sample / per_step_s           # the timed samples only
    line = {
        "impl": "reference", "metric": METRIC, "value": r["value"],
        "unit": "steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": w["desc"],
                   "bench_step": f"{T_sample} theta-steps of the oracle (modal form) at "
                                 f"N={r['sample_n']}"},
        "cpu_baseline": {"value": r["value"], "unit": "steps/s", "cores": r["cores"],
                         "kind": "oracle", "sample": r["sample"]},
        "e2e": {"value": r["value"], "unit": "steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def _per_trace(a, b):
    import numpy as np
    num = np.linalg.norm(a - b, axis=1)
    den = np.linalg.norm(b, axis=1)
    den = np.where(den > 0, den, max(float(den.max()), 1e-300))
    return float((num / den).max())


def _per_snapshot(a, b):
    import numpy as np
    if a.size == 0:
        return None
    num = np.linalg.norm(a - b, axis=0)
    den = np.linalg.norm(b, axis=0)
    den = np.where(den > 0, den, max(float(den.max()), 1e-300))
    return float((num / den).max())


def _functional(a, b, C, snaps):
    """Max over probes of max_k |a - b| / (||C_p|| max_j ||I_j||)."""
    import numpy as np
    Inorm = float(np.linalg.norm(snaps, axis=0).max()) if snaps.size else 1.0
    cn = np.linalg.norm(C, axis=1)
    return float((np.abs(a - b).max(axis=1) / (cn * Inorm)).max())


def _snapshot_view(run_ms, scan_ms, chunks, n0, nsnap, hbm_gbs):
    """The modal chunk's time outside the scan against the bytes of U's kept slices.

    From N_0 = 4096 on, an FP64 modal run reconstructs its nsnap snapshots per chunk from
    U's kept tensor-core slices (16 B per entry of U, read once per group of up to 32
    columns).  Everything of the chunk that is not the scan (the product, its operand split
    and zeroing, the probe reduction) is charged to it, so the rate is a lower bound on the
    product's own."""
    if nsnap <= 0 or chunks <= 0 or n0 < 4096:
        return None
    ms = (run_ms - scan_ms) / chunks
    if ms <= 0:
        return None
    groups = -(-nsnap // 32)
    nbytes = 16.0 * n0 * n0 * groups
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"kernel": "oz_narrow_kernel (snapshots from U's kept slices)",
            "snapshots_per_chunk": int(nsnap), "bytes_per_chunk": float(nbytes),
            "ms_per_chunk_outside_scan": float(ms), "achieved_lower_bound": float(gbs),
            "peak": float(hbm_gbs), "unit": "GB/s", "frac_lower_bound": float(gbs / hbm_gbs),
            "note": "modal run time minus scan time per chunk (library CUDA events), "
                    "against 16 n0^2 bytes per group of <= 32 snapshot columns"}


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
    from paper_2407_11993_gb300 import eddy, peaks as peak_probe

    w = WORKLOADS[args.workload]
    cp, cm = args.plain_chunk or w["plain_chunk"], args.modal_chunk or w["modal_chunk"]
    nsteps = args.warmup + args.steps
    T_src = max(w["T"], cm * nsteps, cp * nsteps) + w["err_steps"] + 2
    t_gen = time.perf_counter()
    p = build_problem(args.workload, T=T_src)
    t_gen = time.perf_counter() - t_gen
    n, m, S, P = p.n, p.E.shape[0], p.M.shape[1], p.C.shape[0]
    n0 = n - m
    stride = p.snap_stride
    if stride and cm % stride:
        raise SystemExit("modal_chunk must be a multiple of the snapshot stride")

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)

    srcd = to_dev(p.src) if S else None
    iDd = to_dev(p.iD) if m else None
    stream = torch.cuda.current_stream(dev)
    E = p.E if m else None
    MD = p.MD if m else None
    M = p.M if S else None

    fp = peak_probe.measure(reps=3)                       # FP64 / FP32 pipes, live
    # setups, once each (library CUDA events per phase; wall clock around the call)
    def setup(form):
        tm = eddy.ThetaMethod(form, p.theta, p.dt, device=local, stream=stream.cuda_stream,
                              profile=True, release_inputs=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        tm.setup(p.L, p.R, E, M, MD, p.C)
        torch.cuda.synchronize(dev)
        return tm, time.perf_counter() - t0, tm.timings()

    modal, modal_setup_wall, tms = setup("modal")       # largest footprint first
    plain, plain_setup_wall, tps = setup("plain")

    # ---- plain-step precision variant (FP32 hi/lo pair inverse factor), run before
    # the timed loop so that its setup's transient memory comes before the modal
    # form's kept slices of U; its errors are filled in after the FP64 runs below
    px_out, px_err = None, None
    if rank == 0 and not args.no_variants:
        try:
            px = eddy.ThetaMethod("plain", p.theta, p.dt, device=local,
                                  stream=stream.cuda_stream, profile=True,
                                  precision="fp32x2", release_inputs=True)
            t0 = time.perf_counter()
            px.setup(p.L, p.R, E, M, MD, p.C)
            setup_x = time.perf_counter() - t0
            Te = w["err_steps"]
            prx, snx = px.run(Te, p.src[:, :Te + 1] if S else None,
                              p.iD[:, :Te + 1] if m else None, 500 if Te % 500 == 0 else Te // 2)
            tx = px.timings()
            px.close()
            fx = tx["fwd_ms"] / max(1.0, tx["fwd_launches"])
            bytes_fx = 8.0 * n0 * (n0 + 1) / 2.0
            pk_, _ = peaks()
            gbs = bytes_fx / (fx * 1e-3) / 1e9
            px_out = (np.asarray(prx), np.asarray(snx), {
                "steps_per_s": Te / (tx["run_ms"] / 1e3), "setup_s": setup_x,
                "fwd_product_ms": fx, "fwd_product_gbs": gbs,
                "fwd_product_hbm_frac": gbs / float(pk_.get("hbm_gbs", 6800.0)),
                "note": "inverse factor as FP32 hi/lo pairs (8 B per entry), compensated FP32 "
                        "products; errors against the FP64 plain form over the same first steps"})
        except Exception as ex:  # noqa: BLE001 - the main line must still be printed
            px_err = str(ex)[:300]

    probes_p = torch.empty((cp, P), dtype=torch.float64, device=dev)
    probes_m = torch.empty((cm, P), dtype=torch.float64, device=dev)
    nsn = cm // stride if stride else 0
    snaps_m = torch.empty((max(nsn, 1), n), dtype=torch.float64, device=dev)

    def window(k0, T):
        s = srcd[:, k0:k0 + T + 1].contiguous() if S else None
        d = iDd[:, k0:k0 + T + 1].contiguous() if m else None
        return s, d

    state = {"kp": 0, "km": 0}

    def one_step(record):
        s, d = window(state["kp"], cp)
        plain.run(cp, s, d, 0, mem=eddy.EC_MEM_DEVICE, probes_out=probes_p)
        tp = plain.timings()
        s, d = window(state["km"], cm)
        modal.run(cm, s, d, stride if nsn else 0, mem=eddy.EC_MEM_DEVICE, probes_out=probes_m,
                  snaps_out=snaps_m if nsn else None)
        tmm = modal.timings()
        state["kp"] += cp
        state["km"] += cm
        if record is not None:
            record.append((tp, tmm))

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

    def total(key, form):
        return sum(r[0 if form == "plain" else 1][key] for r in rec)

    modal_run_s = total("run_ms", "modal") / 1e3
    plain_run_s = total("run_ms", "plain") / 1e3
    modal_rate = args.steps * cm / modal_run_s
    plain_rate = args.steps * cp / plain_run_s
    value = world * modal_rate

    # roofline of the plain step's forward product y = C^{-1} b (the kernel holding the
    # most device time in the timed region): its algorithmic bytes are the packed lower
    # inverse factor, 8 n0 (n0 + 1) / 2 per launch
    fwd_ms = total("fwd_ms", "plain") / max(1.0, total("fwd_launches", "plain"))
    bwd_ms = total("bwd_ms", "plain") / max(1.0, total("bwd_launches", "plain"))
    scan_ms = total("scan_ms", "modal") / max(1.0, total("scan_launches", "modal"))
    fam_ms = {"tile_trmv_kernel<false> (plain forward product)": fwd_ms * cp * args.steps,
              "tile_trmv_kernel<true> (plain transposed product)": bwd_ms * cp * args.steps,
              "modal_scan_kernel (modal replay)": total("scan_ms", "modal")}
    dominant = max(fam_ms, key=fam_ms.get)
    bytes_fwd = 8.0 * n0 * (n0 + 1) / 2.0
    pk, pk_kind = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    achieved_gbs = bytes_fwd / (fwd_ms * 1e-3) / 1e9
    roofline = {"kernel": "tile_trmv_kernel<false>", "bound": "hbm", "achieved": achieved_gbs,
                "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm, "traffic": None,
                "algorithmic_bytes": bytes_fwd, "avg_launch_ms": fwd_ms,
                "peak_note": f"HBM copy bandwidth of MEASURED_PEAKS.json ({pk_kind})",
                "dominant_family": dominant,
                "fp64_view": {"achieved_tflops": float(n0) * n0 / (fwd_ms * 1e-3) / 1e12,
                              "peak_tflops": fp["fp64_fma_tflops"],
                              "frac": float(n0) * n0 / (fwd_ms * 1e-3) / 1e12 /
                                      fp["fp64_fma_tflops"],
                              "peak_note": "FP64 FMA loop over all SMs, measured in this run "
                                           "(paper_2407_11993_gb300.peaks)"}}
    sv = _snapshot_view(total("run_ms", "modal"), total("scan_ms", "modal"), args.steps, n0,
                        nsn, hbm)
    if sv is not None:
        roofline["modal_snapshot_view"] = sv
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
            roofline["traffic_note"] = ("ncu DRAM read+write of one launch at N0=8191 "
                                        "(profiles/tile_trmv_n8192.md), scaled by N0^2")
    except (OSError, ValueError):
        pass

    # setup phases and their achieved arithmetic (FP64-equivalent TFLOP/s of the
    # algorithms' flops; the large products run as FP64 emulation on the tensor cores)
    nf = float(n0)
    phase_flop = {"factor_ms": nf ** 3 / 3.0, "reduce_ms": 4.0 / 3.0 * nf ** 3,
                  "tridiag_ms": 4.0 / 3.0 * nf ** 3, "backtransform_ms": 3.0 * nf ** 3}
    setup_rates = {}
    for ph, fl in phase_flop.items():
        ms_ph = tms.get(ph, 0.0)
        if ms_ph > 0:
            tf = fl / (ms_ph * 1e-3) / 1e12
            setup_rates[ph[:-3]] = {"fp64_equiv_tflops": tf, "algorithmic_flop": fl,
                                    "x_fp64_pipe": tf / fp["fp64_fma_tflops"]}

    # ---- stated errors (outside the timed region) ------------------------------
    err = {}
    outs = {}
    if rank == 0:
        Te = w["err_steps"]
        se = 500 if (Te % 500 == 0 and Te >= 500) else max(1, Te // 2)
        for name, tm in (("plain", plain), ("modal", modal)):
            tm.set_state(np.zeros(tm.state_size()))
            pr, sn = tm.run(Te, p.src[:, :Te + 1] if S else None, p.iD[:, :Te + 1] if m else None,
                            se)
            outs[name] = (np.asarray(pr), np.asarray(sn))
        (pp, sp), (pm, sm) = outs["plain"], outs["modal"]
        err["modal_vs_plain"] = {
            "steps": Te, "probe_rel_per_trace": _per_trace(pm, pp),
            "probe_rel_functional": _functional(pm, pp, p.C, sp),
            "snapshot_rel_per_snapshot": _per_snapshot(sm, sp),
            "note": "both GPU forms from I=0 over the first steps; functional = max |dy| / "
                    "(||C_p|| max ||I||)"}
        if m == 0:
            # the plain step's equation (Eq. time_integration) at full size, on the host:
            # Z (I^{k+1} - I^k) = -dt R I^k - M (s^{k+1} - s^k) for k = 0, 1
            plain.set_state(np.zeros(plain.state_size()))
            _, I12 = plain.run(2, p.src[:, :3] if S else None, None, 1)
            I12 = np.asarray(I12)
            Ik = [np.zeros(n), I12[:, 0], I12[:, 1]]
            res = []
            for k in range(2):
                dI = Ik[k + 1] - Ik[k]
                lhs = p.L @ dI + (p.theta * p.dt) * (p.R @ dI)
                rhs = -p.dt * (p.R @ Ik[k])
                if S:
                    rhs = rhs - p.M @ (p.src[:, k + 1] - p.src[:, k])
                res.append(float(np.linalg.norm(lhs - rhs) /
                                 (np.linalg.norm(lhs) + np.linalg.norm(rhs))))
            err["plain_step_residual"] = {"max": max(res), "steps": 2,
                                          "note": "||Z dI - rhs|| / (||Z dI|| + ||rhs||) with "
                                                  "host products by the inputs L, R"}
            # sampled eigenpairs of the modal setup (Eq. generalized_eigenvalues_discrete)
            tau, U = modal.modes()
            idx = np.unique(np.linspace(0, n0 - 1, 16).astype(int))
            Us = np.ascontiguousarray(U[:, idx])
            del U
            LU, RU = p.L @ Us, p.R @ Us
            eres = np.linalg.norm(LU - RU * tau[idx], axis=0) / (
                np.linalg.norm(LU, axis=0) + tau[idx] * np.linalg.norm(RU, axis=0))
            gram = Us.T @ RU
            err["modal_eigen"] = {"modes_sampled": int(idx.size),
                                  "residual_max": float(eres.max()),
                                  "r_orthonormality_max": float(np.abs(gram - np.eye(idx.size)).max()),
                                  "tau_max": float(tau[0]), "tau_min": float(tau[-1]),
                                  "note": "||L u - tau R u|| / (||L u|| + tau ||R u||) and "
                                          "|U_s^T R U_s - 1| over 16 modes spread over the "
                                          "spectrum, host products by L, R"}
        if args.workload != "n65536_coil" or args.oracle_check:
            from oracle import theta as orc
            q = build_problem(args.workload, T=min(40, Te))
            ref = orc.run_problem(q, "plain")
            To = ref.probes.shape[1]
            err["vs_oracle_first_steps"] = {"steps": To,
                                            "plain_probe_rel_per_trace": _per_trace(pp[:, :To], ref.probes),
                                            "modal_probe_rel_per_trace": _per_trace(pm[:, :To], ref.probes)}

    # ---- precision variants ----------------------------------------------------
    variants = {}
    if rank == 0 and not args.no_variants:
        if px_out is not None:
            prx, snx, stats = px_out
            pp_, sp_ = outs.get("plain", (None, None))
            stats["probe_rel_per_trace_vs_fp64_plain"] = (_per_trace(prx, pp_)
                                                          if pp_ is not None else None)
            stats["snapshot_rel_vs_fp64_plain"] = (_per_snapshot(snx, sp_)
                                                   if sp_ is not None else None)
            variants["plain_fp32x2"] = stats
        elif px_err is not None:
            variants["plain_fp32x2"] = {"error": px_err}
        # modal form: the same modes with the products by U in reduced arithmetic
        pm_, sm_ = outs.get("modal", (None, None))
        Te = w["err_steps"]
        se = 500 if (Te % 500 == 0 and Te >= 500) else max(1, Te // 2)
        for prec in ("fp32x2", "fp32", "bf16x3", "bf16"):
            key = "modal_" + prec
            try:
                t0 = time.perf_counter()
                modal.set_precision(prec)
                switch_s = time.perf_counter() - t0
                modal.set_state(np.zeros(modal.state_size()))
                prv, snv = modal.run(Te, p.src[:, :Te + 1] if S else None,
                                     p.iD[:, :Te + 1] if m else None, se)
                prv, snv = np.asarray(prv), np.asarray(snv)
                rates = []
                for i in range(3):                 # one warm-up chunk, two timed
                    s_, d_ = window(i * cm, cm)
                    modal.run(cm, s_, d_, stride if nsn else 0, mem=eddy.EC_MEM_DEVICE,
                              probes_out=probes_m, snaps_out=snaps_m if nsn else None)
                    if i:
                        rates.append(cm / (modal.timings()["run_ms"] / 1e3))
                variants[key] = {
                    "steps_per_s": statistics.mean(rates), "switch_s": switch_s,
                    "probe_rel_per_trace_vs_fp64_modal": _per_trace(prv, pm_),
                    "probe_rel_functional_vs_fp64_modal": _functional(prv, pm_, p.C, sm_),
                    "snapshot_rel_vs_fp64_modal": _per_snapshot(snv, sm_),
                    "note": "same modes (one eigensolve), products by U in " + prec +
                            "; errors against the FP64 modal run over the same first steps"}
            except Exception as ex:  # noqa: BLE001
                variants[key] = {"error": str(ex)[:300]}
        try:
            modal.set_precision("fp64")
        except Exception:  # noqa: BLE001
            pass

    # ---- end to end through the public API with host buffers (modal form) --------
    e2e = None
    if rank == 0:
        modal.set_state(np.zeros(modal.state_size()))
        host_src = [np.ascontiguousarray(p.src[:, i * cm:i * cm + cm + 1]) if S else None
                    for i in range(args.steps)]
        host_iD = [np.ascontiguousarray(p.iD[:, i * cm:i * cm + cm + 1]) if m else None
                   for i in range(args.steps)]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for i in range(args.steps):
            modal.run(cm, host_src[i], host_iD[i], stride if nsn else 0)
        t1 = time.perf_counter()
        e2e = {"value": world * args.steps * cm / (t1 - t0), "unit": "steps/s",
               "h2d_bytes_per_step": 8 * (S + m) * (cm + 1),
               "d2h_bytes_per_step": 8 * (cm * P + nsn * n),
               "note": "modal form through ThetaMethod.run with numpy host arrays: the chunk's "
                       "sources copied in, probes and snapshots copied out, inside the timing"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        r = oracle_rate(args.workload, args.oracle_steps or w["oracle_steps"], 1, "modal")
        cpu = {"value": r["value"], "unit": "steps/s", "cores": r["cores"], "kind": "oracle",
               "sample": r["sample"], "measured_steps_per_s_at_sample": r["measured_steps_per_s"]}

    modal.close()
    plain.close()

    # ---- setup variant: the tridiagonalisation's symmetric products in compensated FP32
    # (its own modal setup, after the main contexts are gone); errors of its first steps
    # against the FP64 modal and plain runs above
    setup_variant = None
    if rank == 0 and not args.no_variants and args.setup_variant:
        try:
            tv = eddy.ThetaMethod("modal", p.theta, p.dt, device=local, stream=stream.cuda_stream,
                                  profile=True, release_inputs=True,
                                  setup_gemm="tensor_pairsymv")
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            tv.setup(p.L, p.R, E, M, MD, p.C)
            torch.cuda.synchronize(dev)
            wall = time.perf_counter() - t0
            tvs = tv.timings()
            Te = w["err_steps"]
            se = 500 if (Te % 500 == 0 and Te >= 500) else max(1, Te // 2)
            prv, snv = tv.run(Te, p.src[:, :Te + 1] if S else None, p.iD[:, :Te + 1] if m else None,
                              se)
            tv.close()
            prv, snv = np.asarray(prv), np.asarray(snv)
            (pp_, sp_), (pm_, sm_) = outs["plain"], outs["modal"]
            setup_variant = {
                "setup_gemm": "tensor_pairsymv", "setup_s": tvs["setup_ms"] / 1e3,
                "setup_wall_s": wall,
                "phases_ms": {k: tvs[k] for k in ("factor_ms", "reduce_ms", "tridiag_ms",
                                                   "eig_ms", "backtransform_ms", "project_ms")},
                "end_to_end_s_for_T": tvs["setup_ms"] / 1e3 + w["T"] / modal_rate,
                "vs_plain": {"probe_rel_per_trace": _per_trace(prv, pp_),
                             "probe_rel_functional": _functional(prv, pp_, p.C, sp_),
                             "snapshot_rel_per_snapshot": _per_snapshot(snv, sp_)},
                "vs_fp64_modal": {"probe_rel_per_trace": _per_trace(prv, pm_),
                                  "snapshot_rel_per_snapshot": _per_snapshot(snv, sm_)},
                "note": "modal setup with the tridiagonalisation's symmetric products in "
                        "compensated FP32 (entries as FP32 hi/lo pairs); stepping as the FP64 "
                        "modal form (end to end uses the measured modal rate); errors over "
                        "the first steps against the GPU plain and FP64-setup modal runs"}
        except Exception as ex:  # noqa: BLE001 - the main line must still be printed
            setup_variant = {"error": str(ex)[:300]}
    if rank != 0:
        return
    T_paper = w["T"]
    mod_setup_s = tms["setup_ms"] / 1e3
    pla_setup_s = tps["setup_ms"] / 1e3
    line = {
        "metric": METRIC,
        "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": w["desc"], "N": n, "T": T_paper,
                   "bench_step": f"{cp} plain + {cm} modal theta-steps continuing the transient "
                                 f"(setups once, before the timed steps)",
                   "l2": "inputs larger than L2 (factor %.1f GB, modes %.1f GB)" %
                         (4.0 * n0 * (n0 + 1) / 1e9, 8.0 * n0 * n0 / 1e9),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "modal": {"steps_per_s": modal_rate, "setup_s": mod_setup_s,
                  "setup_wall_s": modal_setup_wall,
                  "phases_ms": {k: tms[k] for k in ("elim_ms", "factor_ms", "reduce_ms",
                                                    "tridiag_ms", "eig_ms", "backtransform_ms",
                                                    "project_ms")},
                  "eigensolver_s": tms["eig_ms"] / 1e3,
                  "end_to_end_s_for_T": mod_setup_s + T_paper / modal_rate,
                  "scan_ms_per_launch": scan_ms},
        "plain": {"steps_per_s": plain_rate, "setup_s": pla_setup_s,
                  "setup_wall_s": plain_setup_wall,
                  "end_to_end_s_for_T": pla_setup_s + T_paper / plain_rate,
                  "fwd_product_ms": fwd_ms, "bwd_product_ms": bwd_ms},
        "modal_over_plain_end_to_end": (pla_setup_s + T_paper / plain_rate) /
                                       (mod_setup_s + T_paper / modal_rate),
        "err": err,
        "roofline": roofline,
        "setup_rates": setup_rates,
        "measured_peaks": {"fp64_fma_tflops": fp["fp64_fma_tflops"],
                           "fp64_mma_tflops": fp["fp64_mma_tflops"],
                           "fp32_fma_tflops": fp["fp32_fma_tflops"],
                           "hbm_gbs": hbm, "bf16_tflops": pk.get("bf16_tflops")},
        "precision_variants": variants,
        "setup_variant": setup_variant,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "input_generation_s": t_gen,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--plain-chunk", type=int, default=0, help="plain theta-steps per bench step")
    ap.add_argument("--modal-chunk", type=int, default=0, help="modal theta-steps per bench step")
    ap.add_argument("--oracle-steps", type=int, default=0,
                    help="theta-steps per oracle sample (CPU baseline / reference arm)")
    ap.add_argument("--oracle-check", action="store_true",
                    help="also run the oracle's first steps at the full size")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--setup-variant", action="store_true",
                    help="also run a second modal setup with the tridiagonalisation's symmetric "
                         "products in compensated FP32 and report its time and errors "
                         "(about 4.5 more minutes at N=65536)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the precision variants (plain FP32-pair factor; modal FP32 pair, "
                         "FP32, split BF16 and BF16 products)")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
