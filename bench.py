#!/usr/bin/env python3
"""Benchmark of the integral-direct, Schwarz-screened J/K build (the hot path of the Hartree-Fock
energy functional H(P)) on synthetic water clusters.

Also reported (one run each, outside the timed J/K steps): batched SCF molecules/s over seeded alkane
conformers in the reduced-precision and plain FP64 forms, and the learned SCF guess against the
core-Hamiltonian and SAD guesses.

One step = one J/K build of the workload's density: every unique shell quartet that passes
Schwarz screening (tau = 1e-10) is evaluated (Boys, Obara-Saika VRR, contraction, HGP HRR) and
digested into J and K, then J and K are symmetrised.  Metric: unique Cartesian function quartets
per second (after screening) in the reduced-precision mode, whose energy error against the FP64
path is reported beside it (bar: <= 1e-6 Ha); the plain FP64 path is timed on the same input.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload water32|water8]

N > 1 runs under torchrun: independent replicas of the workload, one per GPU (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "water8": dict(nwater=8, box=12.0, seed=2002, basis="6-31gs",
                   desc="(H2O)_8 cluster, seed 2002, O uniform in a 12-bohr cube, O-O >= 5 bohr, 6-31G* (152 functions)"),
    "water32": dict(nwater=32, box=19.0, seed=2006, basis="6-31gs",
                    desc="(H2O)_32 cluster, seed 2006, 19-bohr cube, O-O >= 5 bohr, 6-31G* (608 functions)"),
}
METRIC = "Schwarz-screened ERI quartets/s and SCF molecules/s vs plain FP64, at <=1e-6 Ha"
UNIT = "unique function quartets/s"
SCHWARZ_TAU = 1e-10
L2_FLUSH_BYTES = 512 << 20
MODE_NAMES = {0: "FP64", 1: "FP32 + FP64 Boys", 2: "FP32", 3: "double-float"}


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _build_library():
    import __graft_entry__ as ge
    ge.build()


def max_over_ranks(dist, value, device):
    """The largest of every rank's value (the slowest replica sets the job's time); dist may be None."""
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_step, steps, max_ms):
    """Units processed by all ranks (each runs its own replica of the workload) per second."""
    return world * units_per_step * steps / (max_ms * 1e-3)


def _workload(name):
    import mess_inputs as mi
    w = WORKLOADS[name]
    mol = mi.water_cluster(w["nwater"], w["box"], w["seed"])
    return mol, mi.basis_path(w["basis"]), w


def _scf_density(g, iters=60):
    """Input preparation: a converged closed-shell density from Roothaan iterations whose J/K come
    from the library's FP64 path (not timed)."""
    import numpy as np
    S, H = g.overlap(), g.kinetic() + g.nuclear()
    s, U = np.linalg.eigh(S)
    X = U @ np.diag(s ** -0.5) @ U.T
    nocc = g.nelectron // 2

    def dens(F):
        _, C = np.linalg.eigh(X.T @ F @ X)
        C = X @ C
        return 2.0 * C[:, :nocc] @ C[:, :nocc].T

    D, Fs, es, E_old = dens(H), [], [], 0.0
    for _ in range(iters):
        J, K, _ = g.jk(D, prec="fp64", schwarz_tau=SCHWARZ_TAU)
        F = H + J - 0.5 * K
        E = 0.5 * float(np.sum(D * (H + F)))
        err = F @ D @ S - S @ D @ F
        if abs(E - E_old) < 1e-9 and np.abs(err).max() < 1e-7:
            break
        E_old = E
        Fs, es = (Fs + [F])[-8:], (es + [err])[-8:]
        if len(Fs) >= 2:
            k = len(Fs)
            B = -np.ones((k + 1, k + 1))
            B[-1, -1] = 0.0
            for i in range(k):
                for j in range(k):
                    B[i, j] = float(np.sum(es[i] * es[j]))
            c = np.linalg.solve(B, np.r_[np.zeros(k), -1.0])[:k]
            F = sum(ci * Fi for ci, Fi in zip(c, Fs))
        D = dens(F)
    return D


class ClockSampler:
    """nvidia-smi samples of SM clock / throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.device_index = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.device_index is not None:
                cmd += ["-i", str(self.device_index)]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def _nvsmi_index(torch, local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",")]
        if local_rank < len(ids):
            return ids[local_rank]
    try:
        u = str(torch.cuda.get_device_properties(local_rank).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return local_rank


def _oracle_counts(o, Q, rows, cols, tau):
    """Integrals the oracle's defining sums evaluate for the elements (rows, cols): for J_mn every
    (l, s) with Q_mn Q_ls >= tau, for K_mn every (l, s) with Q_ml Q_ns >= tau (the screening rule of
    both sides; Q per function from its shell's Schwarz factor)."""
    import numpy as np
    sh = np.asarray(o.shell)
    Qf = np.asarray(Q)[np.ix_(sh, sh)]
    total = 0
    for m, a in zip(rows, cols):
        if tau <= 0.0:
            total += 2 * o.nfn * o.nfn
            continue
        total += int(np.count_nonzero(Qf[m, a] * Qf >= tau))
        total += int(np.count_nonzero(np.multiply.outer(Qf[m, :], Qf[a, :]) >= tau))
    return total


def _oracle_rate(mol, basis_path, D, nelem, seed=7, tau=SCHWARZ_TAU):
    """The FP64 CPU oracle as it stands on a bounded sample of the workload: nelem seeded J/K
    elements of the workload's density, each by its defining sum over all (l, s) with the same
    Schwarz screening as the GPU build.  Each evaluation is one function-quartet integral (the
    oracle's unit of work in its full symmetric build as well).  Returns (evaluations per second,
    threads, seconds, evaluations)."""
    import numpy as np
    import oracle
    oracle.build()
    o = oracle.basis_for(mol, basis_path)
    Q = oracle.schwarz(o)
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, o.nfn, nelem)
    cols = rng.integers(0, o.nfn, nelem)
    t0 = time.perf_counter()
    oracle.jk_elements(o, D, rows, cols, tau=tau, Q=Q)
    dt = time.perf_counter() - t0
    evals = _oracle_counts(o, Q, rows, cols, tau)
    return evals / dt, oracle.num_threads(), dt, evals


def _oracle_full_h2o():
    """The oracle's full J/K build of one water in STO-3G (7 functions, 406 unique function quartets,
    its symmetric loop) on a seeded density, with one thread and with every processor: seconds and
    unique function quartets per second (best of 20 calls each)."""
    import mess_inputs as mi
    import oracle
    oracle.build()
    o = oracle.basis_for(mi.h2o(), mi.basis_path("sto-3g"))
    D = mi.random_symmetric_density(o.nfn, 1)
    nq = (o.nfn * (o.nfn + 1) // 2) * (o.nfn * (o.nfn + 1) // 2 + 1) // 2
    out = {"workload": "H2O / STO-3G (7 functions), full J/K by the oracle's 8-fold symmetric loop",
           "unique_function_quartets": nq}
    for name, threads in (("one_thread", 1), ("all_threads", 0)):
        oracle.set_num_threads(threads)
        best = 1e30
        for _ in range(20):
            t0 = time.perf_counter()
            oracle.jk(o, D)
            best = min(best, time.perf_counter() - t0)
        out[name] = {"threads": oracle.num_threads(), "seconds": best, "unique_function_quartets_per_s": nq / best}
    oracle.set_num_threads(0)
    return out


JK_KERNEL_SOURCES = ("gen_eri.py", "eri_common.cuh", "eri_launch.h", "mess_device.h", "df32.cuh")


def _source_digest():
    """Digest of the sources the J/K kernels are generated and compiled from (the counters of a
    profile taken with other kernel sources no longer describe these kernels)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2406_03121_gb300", "csrc")
    for f in JK_KERNEL_SOURCES:
        h.update(f.encode())
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(workload, key, launches):
    """DRAM bytes per launch of a kernel function of the build, from the ncu capture summarised in
    profiles/jk_dram_traffic.txt, if that capture was taken with the current sources; else None."""
    path = os.path.join(ROOT, "profiles", "jk_dram_traffic.txt")
    if not os.path.exists(path):
        return None
    try:
        body = "".join(line for line in open(path) if not line.lstrip().startswith("#"))
        tj = json.loads(body)
    except Exception:
        return None
    if tj.get("source_digest") != _source_digest():
        return None
    rec = tj.get("workloads", {}).get(workload, {}).get(key)
    if not rec or rec.get("launches") != launches:
        return None
    return rec["dram_bytes_total"] / rec["launches"]


def _kernel_label(p):
    tag = f"{p['la']}{p['lb']}{p['lc']}{p['ld']}"
    if p["team"]:
        shape = f"{32 if p['team'] == 1 else 128} threads per quartet"
        return f"k_jk_team_{tag} ({MODE_NAMES[p['mode']]}, {shape})"
    return f"k_jk_{tag} ({MODE_NAMES[p['mode']]}, {p['G']} lanes per quartet)"


def _scf_section(mess, args):
    """SCF molecules/s: one batched SCF (every molecule in the same launches, one CUDA graph per
    iteration) over seeded linear-alkane conformers, C_nH_2n+2 with n uniform on 1..12 (seed 2003),
    STO-3G, SAD guess, Schwarz screening at 1e-10, wall time of the whole call.  The reduced-precision form runs the
    whole batch; the plain FP64 form (64x slower arithmetic on this GPU) runs its first
    args.scf_fp64_molecules molecules, the energies compared on those."""
    import mess_inputs as mi
    mols = mi.alkane_batch(args.scf_molecules, 1, 12, 2003)
    bases = [mess.Basis.from_molecule(m, mi.basis_path("sto-3g")) for m in mols]
    n64 = min(len(bases), args.scf_fp64_molecules)
    out = {"workload": f"{len(mols)} alkane conformers C_nH_2n+2, n uniform 1..12, seed 2003, STO-3G "
                       f"({min(b.nbf for b in bases)}-{max(b.nbf for b in bases)} functions), batched SCF",
           "fp64_subset": f"the first {n64} molecules of the batch"}
    energies = {}
    common = dict(guess=mess.MESS_GUESS_SAD, schwarz_tau=SCHWARZ_TAU)
    out["options"] = "SAD initial guess; Schwarz screening at tau = 1e-10"
    for name, sub, kw in (("mixed", bases, dict(prec="mixed", split_df32=True, **common)),
                          ("fp64", bases[:n64], dict(prec="fp64", **common))):
        mess.scf_batch(sub[:4], **kw)                         # warm-up: kernels loaded, pools created
        t0 = time.perf_counter()
        res, st = mess.scf_batch(sub, **kw)
        dt = time.perf_counter() - t0
        energies[name] = [r["E_total"] for r in res]
        energies[name + "_iter"] = [r["E_iter"] for r in res]
        out[name] = {"molecules": len(sub), "molecules_per_s": len(sub) / dt, "seconds": dt,
                     "converged": sum(int(r["converged"]) for r in res),
                     "mean_iterations": sum(r["iterations"] for r in res) / len(res)}
    out["max_abs_dE_mixed_vs_fp64_Ha"] = max(abs(a - b) for a, b in zip(energies["mixed"], energies["fp64"]))
    # the reduced-precision iterations' own energy (before the final full-precision evaluation)
    out["max_abs_dE_mixed_iterations_vs_fp64_Ha"] = max(abs(a - b) for a, b in
                                                         zip(energies["mixed_iter"], energies["fp64"]))
    out["speedup_of_reduced_precision"] = out["mixed"]["molecules_per_s"] / out["fp64"]["molecules_per_s"]
    return out


def _mlp_section(mess, args):
    """Learned SCF guess: the MLP trained by the library's own kernels on converged densities of
    seeded alkane conformers with n = 1..8 (seed 2004), then the SCF of unseen conformers with
    n = 9..12 (seed 2005) from the core-Hamiltonian, SAD and learned guesses: the energy error after
    one diagonalisation of the guess's Fock matrix (FP64, the SCF stopped after its second energy),
    iterations to convergence and wall time of the batched reduced-precision SCF, and the spread of
    the final energies across guesses."""
    import tempfile
    import mess_inputs as mi
    sto = mi.basis_path("sto-3g")
    train = [mess.Basis.from_molecule(m, sto) for m in mi.alkane_batch(args.mlp_molecules, 1, 8, 2004)]
    test = [mess.Basis.from_molecule(m, sto) for m in mi.alkane_batch(args.mlp_test_molecules, 9, 12, 2005)]
    kw = dict(prec="mixed", split_df32=True)
    net = mess.MLP(seed=3)
    t0 = time.perf_counter()
    losses = net.train(train, epochs=40, batch_rows=2048, lr=5e-3, **kw)
    t_train = time.perf_counter() - t0
    out = {"workload": f"train: {len(train)} alkanes n = 1..8 (seed 2004, labels = converged densities of the "
                       f"library's own SCF); test: {len(test)} alkanes n = 9..12 (seed 2005); STO-3G",
           "train_seconds": t_train, "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1]}
    with tempfile.TemporaryDirectory() as d:
        w = os.path.join(d, "guess.bin")
        net.save(w)
        energies = {}
        for name, guess in (("core", mess.MESS_GUESS_CORE), ("sad", mess.MESS_GUESS_SAD), ("mlp", mess.MESS_GUESS_MLP)):
            extra = dict(mlp_weights=w) if name == "mlp" else {}
            mess.scf_batch(test[:2], guess=guess, **kw, **extra)
            t0 = time.perf_counter()
            res, st = mess.scf_batch(test, guess=guess, **kw, **extra)
            dt = time.perf_counter() - t0
            energies[name] = [r["E_total"] for r in res]
            first, _ = mess.scf_batch(test, guess=guess, prec="fp64", max_iter=2, **extra)
            de1 = [f["E_total"] - r["E_total"] for f, r in zip(first, res)]
            out[name] = {"mean_iterations": sum(r["iterations"] for r in res) / len(res),
                         "converged": sum(int(r["converged"]) for r in res), "molecules_per_s": len(res) / dt,
                         "mean_dE_after_one_diagonalisation_Ha": sum(de1) / len(de1),
                         "max_dE_after_one_diagonalisation_Ha": max(de1)}
    out["max_abs_dE_between_guesses_Ha"] = max(abs(a - b) for k in ("sad", "mlp")
                                               for a, b in zip(energies[k], energies["core"]))
    return out


def run_reference(args):
    """The oracle as it stands, on the host cores, over the same workload: each step one bounded
    sample of it (per_step seeded J/K elements of the workload's converged-density stand-in, each by
    its screened defining sum).  Rate = function-quartet integrals evaluated per second."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    import mess_inputs as mi
    mol, bpath, w = _workload(args.workload)
    per_step = 8
    import oracle
    oracle.build()
    nfn = oracle.basis_for(mol, bpath).nfn
    D = mi.random_symmetric_density(nfn, w["seed"], nocc=sum(int(z) for z in mol.Z) // 2)
    for _ in range(args.warmup):
        _oracle_rate(mol, bpath, D, 1)
    rates, total, evals = [], 0.0, 0
    threads = 0
    for k in range(args.steps):
        r, threads, dt, ev = _oracle_rate(mol, bpath, D, per_step, seed=100 + k)
        rates.append(r)
        total += dt
        evals += ev
    value = evals / total
    unit = "function-quartet integrals/s"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": w["desc"], "schwarz_tau": SCHWARZ_TAU,
                   "l2": "host CPU run"},
        "cpu_baseline": {"value": value, "unit": unit, "cores": threads, "kind": "oracle",
                         "sample": f"{per_step} seeded J/K elements per step, each by its defining sum over all "
                                   f"(l, s) with the same Schwarz screening (tau = {SCHWARZ_TAU:g}); every "
                                   f"evaluation is one function-quartet integral, the unit of work of the "
                                   f"GPU metric's unique function quartets"},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local_rank = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    if rank == 0:
        _build_library()
    if dist:
        dist.barrier(device_ids=[local_rank])
    import paper_2406_03121_gb300 as mess

    mol, bpath, w = _workload(args.workload)
    g = mess.Basis.from_molecule(mol, bpath)
    n = g.nbf
    D = _scf_density(g)
    dev = torch.device("cuda", local_rank)
    dD = torch.from_numpy(D).to(dev)
    dJ, dK = torch.empty_like(dD), torch.empty_like(dD)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    kw = dict(prec=args.prec, schwarz_tau=SCHWARZ_TAU, fp64_tau=args.fp64_tau, stream=stream,
              split_df32=not args.no_df32)

    def timed(nsteps, **over):
        opts = dict(kw, **over)
        tot, info = 0.0, None
        for _ in range(nsteps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = g.jk_device(dD, dJ, dK, **opts)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot, info

    # kernel choice per bin part by timing the candidates (untimed set-up, like the warm-up)
    tune_kw = dict(prec=args.prec, schwarz_tau=SCHWARZ_TAU, fp64_tau=args.fp64_tau, split_df32=not args.no_df32)
    torch.cuda.synchronize(dev)
    tuned = None if args.no_autotune else g.jk_autotune(D, reps=3, **tune_kw)
    if args.save_tuning and rank == 0:
        with open(args.save_tuning, "w") as fh:
            json.dump({"workload": args.workload, "options": tune_kw, "table": g.jk_tuning(**tune_kw)}, fh)
    for _ in range(args.warmup):
        g.jk_device(dD, dJ, dK, **kw)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(_nvsmi_index(torch, local_rank))
    clocks.start()
    if dist:
        dist.barrier(device_ids=[local_rank])
    torch.cuda.synchronize(dev)
    total_ms, info = timed(args.steps)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier(device_ids=[local_rank])
    clk = clocks.stop()
    max_ms = max_over_ranks(dist, total_ms, dev)
    fnq = info["function_quartets"]
    value = whole_job_rate(world, fnq, args.steps, max_ms)
    J_mix, K_mix = dJ.cpu().numpy(), dK.cpu().numpy()

    # roofline of the dominant kernel: per-launch CUDA events on the launching stream
    prof = None
    for _ in range(3):
        parts = g.jk_profile(dD, dJ, dK, **kw)
        if prof is None:
            prof = [dict(p, ms=[p["ms"]]) for p in parts]
        else:
            for acc, p in zip(prof, parts):
                acc["ms"].append(p["ms"])
    for p in prof:
        p["ms"] = statistics.mean(p["ms"])
    # the dominant kernel: the kernel function (class x variant) with the largest total time over its
    # launches in one build; its achieved rate = its launches' algorithmic flops / their total time
    groups = {}
    for p in prof:
        key = (p["la"], p["lb"], p["lc"], p["ld"], p["G"], p["team"], p["mode"])
        g_ = groups.setdefault(key, {"la": p["la"], "lb": p["lb"], "lc": p["lc"], "ld": p["ld"], "G": p["G"],
                                     "team": p["team"], "mode": p["mode"], "fp64": p["fp64"], "ms": 0.0,
                                     "flops": 0.0, "launches": 0})
        g_["ms"] += p["ms"]
        g_["flops"] += p["flops"]
        g_["launches"] += 1
    dom = max(groups.values(), key=lambda x: x["ms"])
    fp32_peak, fp64_peak = mess.fma_peak(stream)
    dom_fp64_pipe = dom["mode"] == 0
    peak = fp64_peak if dom_fp64_pipe else fp32_peak
    achieved = dom["flops"] / (dom["ms"] * 1e-3) / 1e12
    tot_flops = sum(p["flops"] for p in prof)
    tot_ms = sum(p["ms"] for p in prof)
    dom_key = f"{dom['la']}{dom['lb']}{dom['lc']}{dom['ld']}_{MODE_NAMES[dom['mode']]}_G{dom['G']}_t{dom['team']}"
    traffic = _profiled_traffic(args.workload, dom_key, dom["launches"])

    # end to end through the public host-buffer call: H2D of D, the build, D2H of J and K
    # (D, J and K in page-locked host memory: the copies run at full link speed)
    D_pin = torch.from_numpy(D).pin_memory()
    J_pin, K_pin = torch.empty_like(D_pin).pin_memory(), torch.empty_like(D_pin).pin_memory()
    D_h, J_h, K_h = D_pin.numpy(), J_pin.numpy(), K_pin.numpy()
    e2e_t = []
    for _ in range(max(2, min(args.steps, 5))):
        t0 = time.perf_counter()
        g.jk(D_h, J=J_h, K=K_h, **tune_kw)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = statistics.mean(e2e_t)

    # plain FP64 path on the same input (its own bins, also autotuned), and the energy error of the
    # reduced-precision path
    fp64_steps = max(2, min(args.steps, 5))
    torch.cuda.synchronize(dev)
    if not args.no_autotune:
        g.jk_autotune(D, prec="fp64", schwarz_tau=SCHWARZ_TAU, reps=2)
    for _ in range(2):
        g.jk_device(dD, dJ, dK, **dict(kw, prec="fp64", split_df32=False))
    ms64, info64 = timed(fp64_steps, prec="fp64", split_df32=False)
    J64, K64 = dJ.cpu().numpy(), dK.cpu().numpy()
    e2 = lambda J, K: 0.5 * float(np.sum(D * (J - 0.5 * K)))  # noqa: E731
    dE = e2(J_mix, K_mix) - e2(J64, K64)
    fp64_rate = info64["function_quartets"] * fp64_steps / (ms64 * 1e-3)
    # the benchmark spec's recipe keeps the Boys function of the FP32 quartets in FP64: the same build
    # with that option (its own bins), timed and compared on the same density
    g.jk_autotune(D, reps=2, **dict(tune_kw, boys_fp64=True))
    for _ in range(2):
        g.jk_device(dD, dJ, dK, **dict(kw, boys_fp64=True))
    msb, infob = timed(fp64_steps, boys_fp64=True)
    dE_boys = e2(dJ.cpu().numpy(), dK.cpu().numpy()) - e2(J64, K64)

    scf = _scf_section(mess, args) if args.scf_molecules > 0 else None
    mlp = None
    if args.mlp_molecules > 0:
        try:
            mlp = _mlp_section(mess, args)
        except Exception as exc:          # reported in the line; the J/K numbers stand on their own
            mlp = {"error": f"{type(exc).__name__}: {exc}"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, threads, dt, ev = _oracle_rate(mol, bpath, D, args.cpu_elements)
        cpu = {"value": r, "unit": "function-quartet integrals/s", "cores": threads, "kind": "oracle",
               "sample": f"{args.cpu_elements} seeded J/K elements of the same workload and density, each by its "
                         f"defining sum over all (l, s) with the same Schwarz screening: {ev} function-quartet "
                         f"integrals in {dt:.1f} s (one evaluation per integral, the unit of work of the GPU "
                         f"metric's unique function quartets)",
               "full_build_h2o_sto3g": _oracle_full_h2o()}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.prec != "fp64" else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": w["desc"], "nbf": n, "precision": args.prec,
                   "schwarz_tau": SCHWARZ_TAU, "fp64_tau": args.fp64_tau if args.fp64_tau else 3e-2,
                   "split_arithmetic": "FP64" if args.no_df32 else "double-float (FP32 pairs)",
                   "density": "converged RHF density of the workload", "l2": "flushed (512 MiB write) before every timed step",
                   "kernel_choice": "autotuned per bin part" if tuned is not None else "fixed rules",
                   "parallelism": f"replicas x{world}"},
        "shell_quartets_per_step": info["shell_quartets"], "function_quartets_per_step": fnq,
        "shell_quartets_fp64_per_step": info["shell_quartets_fp64"],
        "shell_quartets_per_s": world * info["shell_quartets"] * args.steps / (max_ms * 1e-3),
        "energy_error_vs_fp64_Ha": dE,
        "boys_fp64_variant": {"energy_error_vs_fp64_Ha": dE_boys, "ms_per_step": msb / fp64_steps,
                              "value": infob["function_quartets"] * fp64_steps / (msb * 1e-3), "unit": UNIT,
                              "note": "the same reduced-precision build with the Boys function of its FP32 "
                                      "quartets evaluated in FP64 for T < 36"},
        "fp64_path": {"value": fp64_rate, "unit": UNIT, "ms_per_step": ms64 / fp64_steps,
                      "speedup_of_reduced_precision": fp64_rate and value / world / fp64_rate},
        "gpu_launches": int(info["kernel_launches"]) * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": _kernel_label(dom),
                     "kernel_launches": dom["launches"], "kernel_ms": dom["ms"],
                     "kernel_share": dom["ms"] / tot_ms,
                     "peak_source": f"measured FMA-chain peak of this GPU ({'FP64' if dom_fp64_pipe else 'FP32'})",
                     "traffic_source": "ncu capture summarised in profiles/jk_dram_traffic.txt (null unless "
                                       "taken with the current sources)",
                     "whole_build": {"flops_per_step": tot_flops,
                                     "achieved_serialised": tot_flops / (tot_ms * 1e-3) / 1e12,
                                     "ms_serialised": tot_ms,
                                     "achieved_concurrent": tot_flops / (max_ms / args.steps * 1e-3) / 1e12,
                                     "frac_concurrent_of_fp32_peak":
                                         tot_flops / (max_ms / args.steps * 1e-3) / 1e12 / fp32_peak}},
        "peaks_measured_tflops": {"fp32": fp32_peak, "fp64": fp64_peak},
        "e2e": {"value": fnq / e2e_s, "unit": UNIT, "h2d_bytes_per_step": n * n * 8, "d2h_bytes_per_step": 2 * n * n * 8,
                "call": "mess_jk_build on page-locked host D, J, K (copies and synchronisation inside the timing)"},
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
    }
    if cpu:
        line["cpu_baseline"] = cpu
    if scf:
        line["scf"] = scf
    if mlp:
        line["learned_guess"] = mlp
    if args.breakdown:
        line["kernels"] = [{k: p[k] for k in ("la", "lb", "lc", "ld", "fp64", "G", "team", "mode", "shell_quartets",
                                             "primitive_quartets", "flops", "ms")} for p in prof]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier(device_ids=[local_rank])
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="water32", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp32", "fp64"])
    ap.add_argument("--fp64-tau", dest="fp64_tau", type=float, default=0.0)
    ap.add_argument("--cpu-elements", dest="cpu_elements", type=int, default=48)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-df32", action="store_true", help="evaluate the split quartets in FP64 instead of double-float")
    ap.add_argument("--breakdown", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the fixed kernel-choice rules")
    ap.add_argument("--save-tuning", dest="save_tuning", default=None,
                    help="write the kernel choice of the timed J/K build to this JSON file")
    ap.add_argument("--scf-molecules", dest="scf_molecules", type=int, default=2048,
                    help="alkane conformers of the batched-SCF section (0: skip it)")
    ap.add_argument("--scf-fp64-molecules", dest="scf_fp64_molecules", type=int, default=256,
                    help="molecules of that batch also run in plain FP64")
    ap.add_argument("--mlp-molecules", dest="mlp_molecules", type=int, default=20000,
                    help="training conformers of the learned-guess section (0: skip it)")
    ap.add_argument("--mlp-test-molecules", dest="mlp_test_molecules", type=int, default=512,
                    help="held-out conformers (n = 9..12) of the learned-guess section")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
