"""Single-case drivers of the library, for profiling one form at one size.

    python -m paper_2407_11993_gb300.profile_cases --form plain --n 8192 --T 5
    python -m paper_2407_11993_gb300.profile_cases --form modal --n 4096 --T 100
    python -m paper_2407_11993_gb300.profile_cases --batch 64 --nmin 1024 --nmax 12288 --T 200

Builds a seeded synthetic problem (plate grid, one electrode row, one coil,
16 pickups), runs setup and T steps through the C ABI on cuda:0 and prints the
library's phase timings as one JSON line.  Used as the workload of ncu
captures so that each capture holds only the kernels of one form.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def batch_case(args) -> dict:
    """Uneven plain-form instances (N uniform in [nmin, nmax], seeds 0..batch-1, one coil,
    4 pickups): total setup, T steps of all instances through ec_batch_run, and the same T
    steps run instance by instance through ec_run for comparison."""
    import time

    import numpy as np

    from paper_2407_11993_gb300 import eddy
    from workloads import synth

    rng = np.random.default_rng(12345)
    sizes = [int(x) for x in rng.integers(args.nmin, args.nmax + 1, size=args.batch)]
    models, srcs = [], []
    t_setup = 0.0
    for i, n in enumerate(sizes):
        p = synth.small(n, T=args.T, seed=i, electrodes=False, coil=True, probes=4, dt=1e-6)
        tm = eddy.ThetaMethod("plain", p.theta, p.dt)
        t0 = time.perf_counter()
        tm.setup(p.L, p.R, None, p.M, None, p.C)
        t_setup += time.perf_counter() - t0
        models.append(tm)
        srcs.append(p.src)
        del p
    state0 = [m.get_state() for m in models]
    eddy.batch_run(models, 3, srcs, None)                  # warm-up (graph, autotune paths)
    for m, s0 in zip(models, state0):
        m.set_state(s0)
    t0 = time.perf_counter()
    outs = eddy.batch_run(models, args.T, srcs, None)
    t_batch = time.perf_counter() - t0
    batch_ms = models[0].timings()["run_ms"]
    for m, s0 in zip(models, state0):
        m.set_state(s0)
    t0 = time.perf_counter()
    single = [m.run(args.T, s, None, 0)[0] for m, s in zip(models, srcs)]
    t_single = time.perf_counter() - t0
    same = all(np.array_equal(a[0], b) for a, b in zip(outs, single))
    fma_per_step = float(sum(n * (n + 1) for n in sizes))  # two triangular products per instance
    return {"batch": args.batch, "sizes": sizes, "T": args.T, "setup_s_total": t_setup,
            "batch_run_ms_device": batch_ms, "batch_run_s_wall": t_batch,
            "sequential_run_s_wall": t_single,
            "instance_steps_per_s_batch": args.batch * args.T / (batch_ms / 1e3),
            "instance_steps_per_s_sequential": args.batch * args.T / t_single,
            "batch_fp64_tflops": 2.0 * fma_per_step * args.T / (batch_ms / 1e3) / 1e12,
            "batch_equals_sequential_bitwise": bool(same), "launches": eddy.launch_count()}


def coil_scan_case(args) -> dict:
    """Independent coil excitations (paired read-out: each coil's own pickup) on one
    setup: plain and modal forms, T steps each (plain: --plain-T steps)."""
    import time

    from paper_2407_11993_gb300 import eddy
    from workloads import synth

    T = max(args.T, args.plain_T)
    p = synth.coil_scan(args.n, T, n_side=args.coil_side, dt=1e-6)
    S = p.M.shape[1]
    out = {"n": args.n, "rhs": S, "T_modal": args.T, "T_plain": args.plain_T}
    for form, steps in (("plain", args.plain_T), ("modal", args.T)):
        tm = eddy.ThetaMethod(form, p.theta, p.dt, rhs="paired")
        t0 = time.perf_counter()
        tm.setup(p.L, p.R, None, p.M, None, p.C)
        t1 = time.perf_counter()
        probes, _ = tm.run(steps, p.src[:, :steps + 1], None, 0)
        tim = tm.timings()
        tm.close()
        out[form] = {"setup_s": t1 - t0, "run_ms": tim["run_ms"],
                     "steps_per_s": steps / (tim["run_ms"] / 1e3),
                     "rhs_steps_per_s": S * steps / (tim["run_ms"] / 1e3)}
        out[form + "_probes_head"] = probes[:2, :, :3].tolist()
    return out


def dt_sweep_case(args) -> dict:
    """Sec. 5: the eigenmode analysis does not depend on dt, the Cholesky factor does.
    One modal setup followed by k runs at k different dt (ec_set_step: O(N) per dt)
    against the plain form, which re-forms and re-factors Z for every dt (ec_set_step
    re-factors); T steps per run.  Reports the cumulative seconds after each dt."""
    import time

    import numpy as np
    import torch

    from paper_2407_11993_gb300 import eddy
    from workloads import synth

    p = synth.config4(T=args.T, n=args.n) if args.config4 else synth.small(
        args.n, T=args.T, seed=1, electrodes=False, coil=True, probes=4, dt=1e-7)
    dts = [p.dt * (1.0 + 0.5 * i) for i in range(args.dt_sweep)]
    out = {"n": args.n, "T": args.T, "dts": dts}
    for form in ("modal", "plain"):
        tm = eddy.ThetaMethod(form, p.theta, dts[0], setup_gemm=args.setup_gemm)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tm.setup(p.L, p.R, None, p.M, None, p.C)
        cum = []
        for i, dt in enumerate(dts):
            if i > 0:
                tm.set_step(p.theta, dt)
            tm.set_state(np.zeros(tm.state_size()))
            tm.run(args.T, p.src, None, 0)
            cum.append(time.perf_counter() - t0)
        tm.close()
        out[form] = {"cumulative_s": cum}
    out["plain_over_modal_after_k"] = [a / b for a, b in zip(out["plain"]["cumulative_s"],
                                                            out["modal"]["cumulative_s"])]
    return out


def grad_config5_case(args) -> dict:
    """The differentiation workload: N = 4096, T = 5000, checkpoints every 250 steps,
    targets from a 3x3x2 block at twice the resistivity plus seeded 1 % noise; the GPU
    adjoint gradient (ec_grad) timed, and compared with the FP64 oracle's gradient
    (all states kept, no checkpoints), timed on the host cores."""
    import time

    import numpy as np
    import torch

    from oracle import adjoint as adj
    from paper_2407_11993_gb300 import eddy
    from workloads import synth

    n, T, ck = args.n, args.T, 250
    p = synth.small(n, T=T, seed=0, electrodes=False, coil=True, probes=16, dt=1e-6)
    g2 = synth.geometry(n, 0)
    nx, ny, nz = g2.grid
    ijk = g2.ijk
    block = ((ijk[:, 0] >= nx // 2 - 1) & (ijk[:, 0] <= nx // 2 + 1) &
             (ijk[:, 1] >= ny // 2 - 1) & (ijk[:, 1] <= ny // 2 + 1) & (ijk[:, 2] <= 1))
    g2.rho = g2.rho.copy()
    g2.rho[block] *= 2.0
    tm = eddy.ThetaMethod("plain", p.theta, p.dt)
    tm.setup(p.L, synth.resistance(g2), None, p.M, None, p.C)
    v, _ = tm.run(T, p.src, None, 0)
    tm.close()
    v = v + 1e-2 * np.std(v) * np.random.default_rng(1000).standard_normal(v.shape)
    tm = eddy.ThetaMethod("plain", p.theta, p.dt)
    tm.setup(p.L, p.R, None, p.M, None, p.C)
    tm.grad(50, p.src[:, :51], v[:, :50], 25)               # warm-up
    tm.set_state(np.zeros(tm.state_size()))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, gR, gs = tm.grad(T, p.src, v, ck)
    t_gpu = time.perf_counter() - t0
    tm.close()
    t0 = time.perf_counter()
    ref = adj.misfit_and_gradient(p.L, p.R, p.M, p.C, p.theta, p.dt, p.src, v)
    t_cpu = time.perf_counter() - t0
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return {"n": n, "T": T, "ckpt_every": ck, "gpu_grad_s": t_gpu, "oracle_grad_s": t_cpu,
            "J_rel_err": abs(J - ref.J) / ref.J, "dJ_dR_rel_err": rel(gR, ref.dJ_dRdiag),
            "dJ_dsrc_rel_err": rel(gs, ref.dJ_dsrc), "host_cores": __import__("os").cpu_count()}


def gemm_case(args) -> dict:
    """One FP64-accurate tensor-core product C = A B (M x K times K x N, seeded normal
    entries) through ec_gemm_f64_emulated: wall time of the call (split, products,
    workspace) over `reps` calls after one warm-up, FP64-equivalent TFLOP/s, and the
    largest error relative to |A||B| against torch's FP64 product."""
    import time
    from ctypes import c_void_p

    import torch

    from paper_2407_11993_gb300 import eddy

    M, N, K = args.gemm
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randn(K, M, dtype=torch.float64, device="cuda", generator=g)   # column-major M x K
    B = torch.randn(N, K, dtype=torch.float64, device="cuda", generator=g)   # column-major K x N
    C = torch.zeros(N, M, dtype=torch.float64, device="cuda")

    def call():
        rc = eddy.lib().ec_gemm_f64_emulated(0, 0, M, N, K, 1.0, c_void_p(A.data_ptr()), M,
                                             c_void_p(B.data_ptr()), K, 0.0,
                                             c_void_p(C.data_ptr()), M,
                                             2 if args.kept else 0, None)
        if rc != 0:
            raise RuntimeError(f"ec_gemm_f64_emulated: {rc}")

    call()
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(max(1, args.reps)):
        t0 = time.perf_counter()
        call()
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    ref = A.t() @ B.t()
    err = float(((C.t() - ref).abs() / (A.t().abs() @ B.t().abs())).max())
    return {"M": M, "N": N, "K": K, "kept": bool(args.kept), "best_call_s": best,
            "fp64_equiv_tflops": 2.0 * M * N * K / best / 1e12, "max_err_rel_absAB": err}


def compare_setup_case(args) -> dict:
    """The modal setup with the tridiagonalisation's symmetric products in FP64 (tensor
    path) and in compensated FP32 (tensor_pairsymv) on the headline recipe at size --n:
    setup seconds per phase, tau and the first T steps' outputs of the two, and sampled
    eigen-residuals ||L u - tau R u|| / (||L u|| + tau ||R u||) of each (host products)."""
    import numpy as np

    from paper_2407_11993_gb300 import eddy
    from workloads import synth

    p = synth.config4(T=args.T, n=args.n)
    out = {"n": args.n, "T": args.T}
    res = {}
    idx = None
    for g in ("tensor", "tensor_pairsymv"):
        tm = eddy.ThetaMethod("modal", p.theta, p.dt, profile=True, setup_gemm=g,
                              release_inputs=True)
        tm.setup(p.L, p.R, None, p.M, None, p.C)
        tms = tm.timings()
        pr, sn = tm.run(p.T, p.src, None, p.snap_stride)
        tau, U = tm.modes()
        tm.close()
        n0 = tau.size
        if idx is None:
            idx = np.unique(np.linspace(0, n0 - 1, 16).astype(int))
        Us = np.ascontiguousarray(U[:, idx])
        del U
        LU, RU = p.L @ Us, p.R @ Us
        eres = np.linalg.norm(LU - RU * tau[idx], axis=0) / (
            np.linalg.norm(LU, axis=0) + tau[idx] * np.linalg.norm(RU, axis=0))
        gram = Us.T @ RU
        res[g] = (tau, np.asarray(pr), np.asarray(sn))
        out[g] = {k: tms[k] for k in ("factor_ms", "reduce_ms", "tridiag_ms", "eig_ms",
                                       "backtransform_ms", "setup_ms")}
        out[g].update(eigen_residual_max=float(eres.max()),
                      r_orthonormality_max=float(np.abs(gram - np.eye(idx.size)).max()))
    # the plain form on the same recipe as the common reference of both
    tp = eddy.ThetaMethod("plain", p.theta, p.dt, release_inputs=True)
    tp.setup(p.L, p.R, None, p.M, None, p.C)
    pp, sp = (np.asarray(x) for x in tp.run(p.T, p.src, None, p.snap_stride))
    tp.close()

    def rel_cols(a, b, axis):
        num = np.linalg.norm(a - b, axis=axis)
        den = np.linalg.norm(b, axis=axis)
        return float((num / np.where(den > 0, den, 1.0)).max()) if a.size else None

    for g in ("tensor", "tensor_pairsymv"):
        out[g]["vs_plain_probe_rel_per_trace"] = rel_cols(res[g][1], pp, 1)
        out[g]["vs_plain_snapshot_rel"] = rel_cols(res[g][2], sp, 0)
    (t0, p0, s0), (t1, p1, s1) = res["tensor"], res["tensor_pairsymv"]
    out["tau_rel_max"] = float(np.max(np.abs(t1 - t0)) / np.max(np.abs(t0)))
    out["probe_rel_per_trace"] = float((np.linalg.norm(p1 - p0, axis=1) /
                                        np.linalg.norm(p0, axis=1)).max())
    out["snapshot_rel_per_snapshot"] = float((np.linalg.norm(s1 - s0, axis=0) /
                                              np.linalg.norm(s0, axis=0)).max()) if s0.size else None
    return out


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--form", choices=["plain", "modal"], default="plain")
    ap.add_argument("--solver", choices=["inverse", "substitution"], default="inverse")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--T", type=int, default=10)
    ap.add_argument("--no-electrodes", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "fp32x2", "bf16", "bf16x3"])
    ap.add_argument("--refine", type=int, default=0, help="plain fp32: refinement sweeps per step")
    ap.add_argument("--setup-gemm", default="tensor", choices=["tensor", "fp64", "tensor_pairsymv"],
                    help="arithmetic units of the setup's large dense products")
    ap.add_argument("--config4", action="store_true",
                    help="the N=65,536 headline recipe (one coil, 4 pickups, dt = 0.1 us, no "
                         "electrodes, snapshots every 1000 steps) at size --n")
    ap.add_argument("--config2", action="store_true",
                    help="the N=8,192 electrode recipe (2 electrodes, 1 A step, 16 pickups, "
                         "dt = 0.5 us, snapshots every 100 steps) at size --n")
    ap.add_argument("--batch", type=int, default=0, help="uneven plain-form instances (ec_batch_run)")
    ap.add_argument("--coil-scan", action="store_true",
                    help="coil_side^2 independent coil excitations on one setup, both forms")
    ap.add_argument("--coil-side", type=int, default=16)
    ap.add_argument("--plain-T", type=int, default=20)
    ap.add_argument("--nmin", type=int, default=1024)
    ap.add_argument("--nmax", type=int, default=12288)
    ap.add_argument("--dt-sweep", type=int, default=0,
                    help="k runs at k different dt on one setup (modal) vs k re-factorisations "
                         "(plain)")
    ap.add_argument("--gemm", type=int, nargs=3, metavar=("M", "N", "K"),
                    help="one FP64-accurate tensor-core product of this shape")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--kept", action="store_true",
                    help="--gemm through the kept-slice path (A cut once per call, stream-K)")
    ap.add_argument("--compare-setup", action="store_true",
                    help="modal setup with FP64 vs compensated-FP32 symmetric products")
    ap.add_argument("--grad-config5", action="store_true",
                    help="the differentiation workload (N=4096, T=5000, checkpoints every 250)")
    args = ap.parse_args()

    from paper_2407_11993_gb300 import build, eddy
    from workloads import synth

    build.build()
    if args.batch:
        print(json.dumps(batch_case(args)))
        return
    if args.coil_scan:
        print(json.dumps(coil_scan_case(args)))
        return
    if args.dt_sweep:
        print(json.dumps(dt_sweep_case(args)))
        return
    if args.grad_config5:
        print(json.dumps(grad_config5_case(args)))
        return
    if args.compare_setup:
        print(json.dumps(compare_setup_case(args)))
        return
    if args.gemm:
        print(json.dumps(gemm_case(args)))
        return
    if args.config4:
        p = synth.config4(T=args.T, n=args.n)
    elif args.config2:
        p = synth.config2(T=args.T, n=args.n)
    else:
        p = synth.small(args.n, T=args.T, seed=1, electrodes=not args.no_electrodes, coil=True,
                        probes=16, dt=0.5e-6)
    tm = eddy.ThetaMethod(args.form, p.theta, p.dt, solver=args.solver, profile=True,
                          precision=args.precision, refine_steps=args.refine,
                          setup_gemm=args.setup_gemm)
    m = p.E.shape[0]
    import time
    t0 = time.perf_counter()
    tm.setup(p.L, p.R, p.E if m else None, p.M if p.M.shape[1] else None, p.MD if m else None,
             p.C)
    t1 = time.perf_counter()
    setup_launches = eddy.launch_count()
    tm.run(p.T, p.src if p.M.shape[1] else None, p.iD if m else None,
           p.snap_stride if (args.config4 or args.config2) else 0)
    t2 = time.perf_counter()
    out = tm.timings()
    out.update(setup_wall_s=t1 - t0, run_wall_s=t2 - t1,
               steps_per_s=p.T / (out["run_ms"] / 1e3) if out["run_ms"] > 0 else None)
    out.update(form=args.form, n=args.n, T=args.T, precision=args.precision, refine=args.refine,
               setup_gemm=args.setup_gemm, setup_launches=setup_launches,
               launches=eddy.launch_count())
    print(json.dumps(out))


if __name__ == "__main__":
    main()
