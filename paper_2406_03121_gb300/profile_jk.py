"""Profiling driver for the J/K build: repeated host-buffer builds of one water-cluster workload
through the C ABI, without PyTorch, so that a kernel profiler sees only this library's launches.

  python -m paper_2406_03121_gb300.profile_jk [--workload water8|water32] [--steps K] [--warmup W]
                                              [--prec mixed|fp64|fp32] [--no-df32] [--no-autotune]
                                              [--tuning FILE]

The workloads and options are those of the J/K benchmark: (H2O)_8 (seed 2002, 12-bohr cube) or
(H2O)_32 (seed 2006, 19-bohr cube), 6-31G*, Schwarz threshold 1e-10, split quartets in
double-float unless --no-df32, kernel choice autotuned unless --no-autotune, or read from a file
written by ``bench.py --save-tuning`` (a profiler slows every launch and would skew the autotuner's
own timings).  The density is a
seeded symmetric positive semidefinite matrix: screening uses only the Schwarz factors, so the
launches (classes, parts, grid sizes) are those of any density.  The timed steps are bracketed by a
profiler range (ncu --profile-from-start off records only them, not the autotuning and warm-up).
Prints one line per step with the host wall time of the call.
"""
from __future__ import annotations

import argparse
import time

WORKLOADS = {"water8": (8, 12.0, 2002), "water32": (32, 19.0, 2006)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="water8", choices=sorted(WORKLOADS))
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64", "fp32"])
    ap.add_argument("--no-df32", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuning", default=None,
                    help="kernel choice saved by bench.py --save-tuning (used instead of autotuning here)")
    args = ap.parse_args(argv)

    import mess_inputs as mi
    import paper_2406_03121_gb300 as mess

    nw, box, seed = WORKLOADS[args.workload]
    mol = mi.water_cluster(nw, box, seed)
    g = mess.Basis.from_molecule(mol, mi.basis_path("6-31gs"))
    D = mi.random_symmetric_density(g.nbf, seed, nocc=g.nelectron // 2)
    kw = dict(prec=args.prec, schwarz_tau=1e-10, split_df32=not args.no_df32)
    if args.tuning:
        import json
        saved = json.load(open(args.tuning))
        if saved.get("workload") != args.workload:
            raise SystemExit(f"{args.tuning} holds the tuning of {saved.get('workload')}, not {args.workload}")
        g.jk_set_tuning(saved["table"], **kw)
        print(f"tuning: {len(saved['table'])} parts from {args.tuning}", flush=True)
    elif not args.no_autotune:
        changed = g.jk_autotune(D, reps=3, **kw)
        print(f"autotune: {changed} parts changed", flush=True)
    for _ in range(args.warmup):
        g.jk(D, **kw)
    mess.profiler_range(True)          # a profiler started with --profile-from-start off records from here
    for k in range(args.steps):
        t0 = time.perf_counter()
        _, _, info = g.jk(D, **kw)
        print(f"step {k}: {1e3 * (time.perf_counter() - t0):.3f} ms, {info['kernel_launches']} launches, "
              f"{info['function_quartets']} function quartets", flush=True)
    mess.profiler_range(False)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
