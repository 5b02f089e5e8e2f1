"""Single-case drivers of the library, for profiling one form at one size.

    python -m paper_2407_11993_gb300.profile_cases --form plain --n 8192 --T 5
    python -m paper_2407_11993_gb300.profile_cases --form modal --n 4096 --T 100

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


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--form", choices=["plain", "modal"], default="plain")
    ap.add_argument("--solver", choices=["inverse", "substitution"], default="inverse")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--T", type=int, default=10)
    ap.add_argument("--no-electrodes", action="store_true")
    args = ap.parse_args()

    from paper_2407_11993_gb300 import build, eddy
    from workloads import synth

    build.build()
    p = synth.small(args.n, T=args.T, seed=1, electrodes=not args.no_electrodes, coil=True,
                    probes=16, dt=0.5e-6)
    tm = eddy.ThetaMethod(args.form, p.theta, p.dt, solver=args.solver, profile=True)
    m = p.E.shape[0]
    tm.setup(p.L, p.R, p.E if m else None, p.M, p.MD if m else None, p.C)
    tm.run(p.T, p.src, p.iD if m else None, 0)
    out = tm.timings()
    out.update(form=args.form, n=args.n, T=args.T, launches=eddy.launch_count())
    print(json.dumps(out))


if __name__ == "__main__":
    main()
