"""AIMD throughput benchmark: RI-HF energy + analytic gradient per velocity-Verlet step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed] [--impl reference]

One step = move the nuclei (Verlet), rebuild the geometry-dependent integrals and
fit (rihf_update_geometry), converge the SCF from the previous step's orbitals
(rihf_scf), evaluate the analytic gradient (rihf_gradient), update velocities.
Workload: (H2O)8 (seed = rank), 192 primary / 848 auxiliary spherical functions,
dt = 0.5 fs, Maxwell-Boltzmann 300 K start.  The fitted tensor B (250 MB) exceeds
the 129 MB L2, so no explicit L2 flush is needed between steps.

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica on its own GPU (the path has no data exchange between geometries):
weak scaling, value = sum of steps over ranks / max elapsed time.
"""
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

METRIC = "RI-HF AIMD steps/s (E+grad), mixed vs FP64 at |dE|<=1e-6 Eh; % of roofline"
UNIT = "AIMD steps/s"
DT_FS = 0.5
CONV = dict(conv_e=1e-8, conv_diis=1e-7, max_iter=60)
# FP64 peak from unit counts and clock: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz
FP64_PEAK_GFLOPS = 152 * 4 * 2.07
FALLBACK = dict(hbm_gbs=6800.0, bf16_tflops=1900.0)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def allreduce_max(pg, x, local):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda:%d" % local if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg):
    if pg is not None:
        pg.barrier()


class Trajectory:
    """Velocity-Verlet driver over one context (host-side integrator, 3*natoms doubles)."""

    def __init__(self, ctx, mol, seed, R):
        from paper_2407_19614_gb300 import workloads as W
        self.ctx, self.R = ctx, R
        self.m = W.masses_au(mol.Z)[:, None]
        self.x = mol.xyz.copy()
        self.v = W.maxwell_boltzmann(mol.Z, 300.0, seed)
        self.dt = DT_FS * W.FS_TO_AU
        out = ctx.scf(guess=0, outputs=False)
        self.E = out["energy"]
        self.g = ctx.gradient()
        self.iters = [out["iterations"]]

    def step(self):
        a = -self.g / self.m
        self.x = self.x + self.v * self.dt + 0.5 * a * self.dt ** 2
        self.ctx.update_geometry(self.x)
        out = self.ctx.scf(guess=2, outputs=False)
        self.E = out["energy"]
        self.iters.append(out["iterations"])
        g_new = self.ctx.gradient()
        self.v = self.v + 0.5 * (a - g_new / self.m) * self.dt
        self.g = g_new

    def total_energy(self):
        return self.E + 0.5 * float(np.sum(self.m * self.v ** 2))


def cpu_oracle_sample(n_iter):
    """Time the CPU oracle on a bounded sample of one (H2O)8 AIMD step and scale
    to a full step: integrals + fit, 2 SCF iterations (scaled to n_iter), the
    gradient terms of 1 of 24 atoms (scaled to all atoms)."""
    import scipy.linalg as sla
    from oracle import integrals as OI
    from oracle import rihf as O
    from paper_2407_19614_gb300 import workloads as W
    mol = W.water8(0)
    t0 = time.perf_counter()
    s = O.System(mol)
    L, B = O.cholesky_fit(s.A, s.T3)
    t1 = time.perf_counter()
    X = O.canonical_orthogonaliser(s.S)
    e, Cp = np.linalg.eigh(X.T @ s.h @ X)
    C = X @ Cp
    for _ in range(2):
        Co = C[:, : s.nocc]
        D = 2 * Co @ Co.T
        F = s.h + O.coulomb_ri(B, D) + O.exchange_ri(B, Co)
        e, Cp = np.linalg.eigh(X.T @ F @ X)
        C = X @ Cp
    t2 = time.perf_counter()
    # gradient: shared prep, then one atom's derivative integrals
    Ct = np.sqrt(2.0) * C[:, : s.nocc]
    cho = sla.cho_factor(s.A, lower=True)
    Tij = np.einsum("mi,pmn,nj->pij", Ct, s.T3, Ct, optimize=True)
    Xf = sla.cho_solve(cho, Tij.reshape(s.naux, -1))
    t3 = time.perf_counter()
    for d in range(3):
        s.eri3_ao(datom=0, ddim=d)
        OI.eri2(s.aux.cb, datom=0, ddim=d)
        OI.one_electron(2, s.bas.cb, s.Z, s.xyz, datom=0, ddim=d)
    t4 = time.perf_counter()
    del Xf
    step_s = (t1 - t0) + (t2 - t1) / 2 * n_iter + (t3 - t2) + (t4 - t3) * mol.natoms
    return {"step_s": step_s, "sample_s": t4 - t0,
            "sample": "(H2O)8 oracle: integrals+fit, 2 SCF iterations (scaled to %.1f), gradient terms of 1/24 atoms "
                      "(scaled to 24)" % n_iter}


def run_reference(args):
    world, rank, local, pg = dist_setup()
    if rank != 0:
        return 0
    ncore = os.cpu_count()
    for _ in range(args.warmup):
        cpu_oracle_sample(12.0)
    times = []
    samples = []
    for _ in range(args.steps):
        r = cpu_oracle_sample(12.0)
        times.append(r["step_s"])
        samples.append(r["sample_s"])
    step_s = statistics.median(times)
    value = 1.0 / step_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "(H2O)8 RI-HF E+grad AIMD step, N=192, Naux=848, spherical, dt 0.5 fs, "
                               "previous-orbital guess",
                   "precision": "fp64 (CPU oracle)", "scf_iters_assumed": 12},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncore, "kind": "oracle",
                         "sample": r["sample"] + "; per step %.1f s of CPU work" % statistics.median(samples)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_batch(args):
    """Batched AIMD: K independent water clusters (3..batch_max molecules, the
    config-1 basis), one velocity-Verlet step per cluster per batch step through
    rihf_batch_step (concurrent contexts, CUDA-graph SCF iterations).  Reports
    molecule-steps per second; device time is the wall clock of the batch
    steps (they synchronise)."""
    from paper_2407_19614_gb300 import rihf as R
    from paper_2407_19614_gb300 import workloads as W
    R.load()
    prec = R.PRECISION_MIXED if args.precision == "mixed" else R.PRECISION_FP64
    sizes = W.batch_sizes(args.batch, seed=0, lo=3, hi=args.batch_max)
    mols = [W.water_n(int(n), seed=k) for k, n in enumerate(sizes)]
    ctxs = [R.Context(m, precision=prec, **CONV) for m in mols]
    ms = [W.masses_au(m.Z)[:, None] for m in mols]
    xs = [m.xyz.copy() for m in mols]
    vs = [W.maxwell_boltzmann(m.Z, 300.0, k) for k, m in enumerate(mols)]
    dt = DT_FS * W.FS_TO_AU
    E, G, it = R.batch_step(ctxs, None, guess=0)

    def step():
        nonlocal E, G
        acc = [-g / m for g, m in zip(G, ms)]
        for i in range(len(xs)):
            xs[i] = xs[i] + vs[i] * dt + 0.5 * acc[i] * dt * dt
        E, Gn, its = R.batch_step(ctxs, xs, guess=2)
        for i in range(len(xs)):
            vs[i] = vs[i] + 0.5 * (acc[i] - Gn[i] / ms[i]) * dt
        G = Gn
        return its

    for _ in range(max(args.warmup, 1)):
        step()
    iters = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        iters.append(step())
    wall = time.perf_counter() - t0
    line = {"metric": "batched RI-HF AIMD molecule-steps/s (E+grad)", "value": len(ctxs) * args.steps / wall,
            "unit": "molecule-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "bf16 digit planes (RI-K, fit, gradient products) + f64", "data": "synthetic",
            "config": {"workload": "%d water clusters, 3..%d molecules (sizes %s), config-1 basis, dt 0.5 fs"
                                   % (len(ctxs), args.batch_max, np.bincount(sizes).tolist()),
                       "precision": args.precision, "scf_iters_avg": float(np.mean(iters))}}
    print(json.dumps(line))
    for c in ctxs:
        c.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64-path comparison run (mixed only)")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=0,
                    help="batched mode: this many independent clusters of 3..--batch-max waters per AIMD step")
    ap.add_argument("--batch-max", type=int, default=8)
    ap.add_argument("--profile-step", action="store_true",
                    help="untimed: setup, one SCF and one gradient of the workload (for ncu captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.batch > 0:
        return run_batch(args)
    if args.profile_step:
        from paper_2407_19614_gb300 import rihf as R
        from paper_2407_19614_gb300 import workloads as W
        R.load()
        prec = R.PRECISION_MIXED if args.precision == "mixed" else R.PRECISION_FP64
        ctx = R.Context(W.water8(0), precision=prec, **CONV)
        out = ctx.scf(outputs=False)
        g = ctx.gradient()
        print(json.dumps({"energy": out["energy"], "iterations": out["iterations"], "grad_max": float(abs(g).max())}))
        ctx.close()
        return 0

    world, rank, local, pg = dist_setup()
    import torch
    from paper_2407_19614_gb300 import rihf as R
    from paper_2407_19614_gb300 import workloads as W

    torch.cuda.set_device(local)
    R.load()
    main_prec = args.precision
    res = measure_path(R, W, torch, main_prec, args, rank, local, pg, trace=True)
    cmp = None
    if main_prec == "mixed" and not args.no_compare:
        # the FP64 path on the same trajectory: its throughput, and the largest
        # per-step energy difference of the two paths (the |dE| of the metric)
        cmp = measure_path(R, W, torch, "fp64", args, rank, local, pg, trace=False)
    if rank != 0:
        return 0
    world = res["world"]
    value = world * args.steps / (res["ms_max"] / 1e3)
    stats = res["stats"]
    pk, pk_src = peaks()
    roof = None
    kernels = [s for s in stats if not s["name"].startswith("SCF iteration graph")]
    if kernels:
        dom = max(kernels, key=lambda s: s["ms"])
        timed = [s for s in kernels if s["work"] > 0]
        roof_k = dom if dom["work"] > 0 else max(timed, key=lambda s: s["ms"])
        per_launch_s = roof_k["ms"] / roof_k["launches"] / 1e3
        work = roof_k["work"] / roof_k["launches"]
        if roof_k["kind"] == "hbm_bytes":
            achieved, peak, unit, bound = work / per_launch_s / 1e9, pk["hbm_gbs"], "GB/s", "hbm"
            src = "hbm_gbs of %s" % pk_src
        elif roof_k["kind"] == "fp64_flops":
            achieved, peak, unit, bound = work / per_launch_s / 1e12, FP64_PEAK_GFLOPS / 1e3, "TFLOP/s", "alu"
            src = "FP64 DFMA peak derived from unit counts (152 SMs x 2 DFMA/clk x 2.07 GHz)"
        elif roof_k["kind"] == "bf16_tensor_flops":
            # BF16 MMA flops issued (digit-pair products included); the kernel runs
            # inside a long step, so the sustained cuBLAS figure is the peak
            key = "bf16_tflops_sustained" if "bf16_tflops_sustained" in pk else "bf16_tflops"
            achieved, peak, unit, bound = work / per_launch_s / 1e12, pk[key], "TFLOP/s", "tensor"
            src = "%s of %s" % (key, pk_src)
        else:
            achieved, peak, unit, bound = work / per_launch_s / 1e12, pk["bf16_tflops"] / 2, "TFLOP/s", "alu"
            src = "FP32 SIMT: half the bf16 tensor figure of %s (fallback)" % pk_src
        traffic = None
        tpath = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tpath):
            with open(tpath) as f:
                traffic = json.load(f).get(roof_k["name"])
        roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": traffic, "kernel": roof_k["name"], "peak_source": src,
                "dominant_kernel": dom["name"], "dominant_share": dom["ms"] / sum(s["ms"] for s in stats)}
    cpu = None
    if not args.no_cpu_baseline:
        r = cpu_oracle_sample(float(np.mean(res["iters"])))
        cpu = {"value": 1.0 / r["step_s"], "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": r["sample"]}
    grad_bytes = res["natoms"] * 3 * 8
    config = {"workload": "(H2O)8 RI-HF E+grad AIMD step, N=192, Naux=848, spherical, dt 0.5 fs, "
                          "previous-orbital guess",
              "precision": main_prec, "parallelism": "replicas" if world > 1 else "1 GPU",
              "l2": "inputs larger than L2 (B = 250 MB)", "scf_conv": CONV,
              "scf_iters_avg": float(np.mean(res["iters"])), "energy_drift_eh": res["drift"],
              "kernel_times": "CUDA events per launch on the library stream during the timed steps; SCF "
                              "iterations replay as CUDA graphs and are timed as a unit"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": res["ms_max"] / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if main_prec == "fp64" else "bf16 digit planes (RI-K, fit, gradient products) + f64", "data": "synthetic",
        "config": config,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": world * args.steps / res["e2e_s"], "unit": UNIT, "h2d_bytes_per_step": grad_bytes,
                "d2h_bytes_per_step": grad_bytes + 8 + int(np.mean(res["iters"])) * 16},
        "clocks": res["clocks"],
        "gpu_launches": int(res["launches"]),
        "kernels": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in s.items()} for s in
                    sorted(stats, key=lambda s: -s["ms"])],
    }
    if cmp is not None:
        dE = float(np.max(np.abs(np.array(res["energies"]) - np.array(cmp["energies"]))))
        line["fp64_path"] = {"value": world * args.steps / (cmp["ms_max"] / 1e3), "unit": UNIT,
                             "ms_per_step": cmp["ms_max"] / args.steps,
                             "scf_iters_avg": float(np.mean(cmp["iters"])),
                             "gpu_launches": int(cmp["launches"])}
        config["max_abs_dE_vs_fp64_path_eh"] = dE
    print(json.dumps(line))
    return 0


def measure_path(R, W, torch, precision, args, rank, local, pg, trace):
    """Warm-up and timed AIMD steps of one context (device time by CUDA events on
    the library stream, then the end-to-end pass through the public API)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    prec = R.PRECISION_MIXED if precision == "mixed" else R.PRECISION_FP64
    mol = W.water8(rank)
    ctx = R.Context(mol, precision=prec, device=local, **CONV)
    traj = Trajectory(ctx, mol, rank, R)
    stream = torch.cuda.ExternalStream(ctx.stream(), device=local)
    for _ in range(max(args.warmup, 0)):
        traj.step()
    # ---- timed region 1: device time (CUDA events on the library stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = ctx.timings()["launches"]
    it0 = len(traj.iters)
    Etot0 = traj.total_energy()
    energies = []
    ctx.trace(bool(trace))
    barrier(pg)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            traj.step()
            energies.append(traj.E)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(pg)
    ms = e0.elapsed_time(e1)
    ms_max = allreduce_max(pg, ms, local)
    launches = ctx.timings()["launches"] - launches0
    stats = ctx.trace_stats() if trace else []
    ctx.trace(False)
    iters = traj.iters[it0:]
    drift = traj.total_energy() - Etot0

    # ---- timed region 2: end to end through the public API, host buffers
    xyz_pinned = torch.empty(mol.natoms * 3, dtype=torch.float64, pin_memory=True).numpy()
    barrier(pg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        a = -traj.g / traj.m
        traj.x = traj.x + traj.v * traj.dt + 0.5 * a * traj.dt ** 2
        xyz_pinned[:] = traj.x.reshape(-1)
        ctx.update_geometry(xyz_pinned.reshape(-1, 3))
        out = ctx.scf(guess=2, outputs=False)
        g_new = ctx.gradient()
        traj.v = traj.v + 0.5 * (a - g_new / traj.m) * traj.dt
        traj.g, traj.E = g_new, out["energy"]
    torch.cuda.synchronize()
    e2e_s = allreduce_max(pg, time.perf_counter() - t0, local)
    barrier(pg)
    out = dict(world=world, ms_max=ms_max, launches=launches, stats=stats, iters=iters, drift=drift,
               e2e_s=e2e_s, clocks=clk.summary(), energies=energies, natoms=mol.natoms)
    ctx.close()
    return out


if __name__ == "__main__":
    sys.exit(main())
