#!/usr/bin/env python
"""Benchmark of the smoothed-circulant-embedding MLMC hot path.

One step = one MLMC sweep of the oscillatory workload (workloads.OSCILLATORY):
for every level l = 0..5 (n = 16..512), N_l samples of Algorithm 2 --
Philox normals -> sqrt(Lambda~)-scaled spectrum -> 2D FFT -> Hartley -> exp,
the fine and the coarse Darcy solve (multigrid-preconditioned CG with FP64
iterative refinement), the QoI and the level differences Y_l -- and the level
sums, through mlmc_level_estimate of the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision 32|64]
    python bench.py --impl reference ...      # the FP64 CPU oracle, bounded sample

Prints one JSON line (rank 0).  value = MLMC level-samples per second over all
levels and ranks (each a Y_l sample: field + fine and coarse solve + QoI); the
finest-level rate (the n = 512 samples of a sweep per second) and each level's
rate are reported beside it.
"""
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

import workloads  # noqa: E402

METRIC = ("MLMC level-samples/s, all levels of one sweep (each sample: field + fine and "
          "coarse Darcy solves + QoI + Y_l)")
UNIT = "level-samples/s"
DTYPE_MIXED = "f32+ff(fp32x2)+f64 eig/QoI"
L2_BYTES = 129 * 1024 * 1024
# DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum) per algorithmic byte of
# a kernel family, from one capture of its n = 512 x 32 launch (profiles/ summary named
# below); scaled to the bench's launches by their algorithmic bytes for the roofline
# family, and reported only while the kernel source is the one that was captured
# (sha256 below).
TRAFFIC_PER_ALG = {
    # fused CG pass, n = 512 x 32 samples (profiles/cg_pass_n512x32.md)
    "cg_spmv_dot": ((168.580608 + 63.755776) / 269.485056,
                    "paper_2306_13493_gb300/csrc/darcy.cu", "pspmv_kernel",
                    "9a76b841323f6d80ce7b0bc9ee4c5a1f56e55f9e4fc43749a2e76bd639234e5b"),
    # n = 512 launch of the tile kernel, 48-row windows (profiles/mg_up_n512x32.md)
    "mg_up": ((143.223296 + 20.216576) / 176.882432,
              "paper_2306_13493_gb300/csrc/mg_tiles.cuh", "mg_up_kernel",
              "1e6c3d6b2ae324929df37ce45854077b49df36df7edd57bdbf3e5778ac9dd6b9"),
}


def kernel_source_digest(path, name):
    """sha256 of the source text of kernel `name` in `path` (from its template
    line to the closing brace at column 0): a traffic ratio is reported only
    while the kernel's own code is the one that was captured."""
    import hashlib
    lines = open(os.path.join(ROOT, path)).read().split("\n")
    for i, ln in enumerate(lines):
        if name + "(" in ln and ("__global__" in ln or "__global__" in lines[i - 1]):
            start = i - 1 if lines[i - 1].startswith("template") else i
            if "__global__" in lines[i - 1] and lines[i - 2].startswith("template"):
                start = i - 2
            end = next(j for j in range(i, len(lines)) if lines[j] == "}")
            return hashlib.sha256("\n".join(lines[start:end + 1]).encode()).hexdigest()
    return None
# oracle sample sizes per level for the CPU baseline (bounded: ~10-30 s of CPU work)
CPU_SAMPLES = [24, 12, 8, 4, 2, 1]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--concurrency", type=int, default=8,
                    help="levels in flight at once (each on its own streams); 1 = one after another")
    ap.add_argument("--study", default=None,
                    choices=[None, "precision", "smoothing", "qmc", "3d"],
                    help="run a study instead of the benchmark (prints its own JSON line)")
    ap.add_argument("--study-count", type=int, default=None)
    ap.add_argument("--study-oracle", type=int, default=None)
    ap.add_argument("--serve-seconds", type=float, default=12.0,
                    help="open-loop window of the served-requests measurement (0: skip)")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-slice-vertices", type=int, default=0,
                    help="server slice size in fine vertices (0: 2^24, <0: no slicing)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default FFT launch shapes (no tuning before the timed steps)")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-level launch measurement")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the FP32 FMA issue rate and the L2 read bandwidth and exit")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-path", action="store_true")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="multiply the per-level sample counts (tests only)")
    ap.add_argument("--case", default=None, choices=[None, "darcy", "field", "darcy3", "field3"],
                    help="time one kernel family on one batch (profiling driver)")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--count", type=int, default=64)
    return ap.parse_args()


def run_case3(args):
    """One batch of the three-dimensional workload's field at n cells per side,
    then one Darcy solve (a small launch sequence for kernel captures)."""
    import numpy as np
    import torch
    from paper_2306_13493_gb300 import build, sce
    build.build_library()
    sce.load()
    wl = workloads.THREE_D
    n, count = args.n, args.count
    emb = sce.ce3_setup_embedding(0, wl.nu, wl.lam, wl.sigma2, n, pad_mode=sce.CE_PAD_SMOOTH)
    k = torch.empty(count, n + 1, n + 1, n + 1, dtype=torch.float32, device="cuda")
    qoi = torch.empty(count, 3, dtype=torch.float64, device="cuda")
    iters = torch.empty(count, dtype=torch.int32, device="cuda")
    times = []
    for rep in range(1 + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if args.case == "field3" or rep == 0:
            sce.ce3_sample_batch(emb, wl.seed, 0, rep * count, count, k)
        if args.case == "darcy3":
            sce.darcy3_solve_batch(n, k, count, qoi, f=wl.f, rtol=wl.rtol, iters=iters,
                                   allow_not_converged=True)
        e1.record()
        torch.cuda.synchronize()
        if rep > 0:
            times.append(e0.elapsed_time(e1))
    it = iters.cpu().numpy() if args.case == "darcy3" else np.zeros(1)
    print(json.dumps({"case": args.case, "n": n, "count": count,
                      "ms": statistics.mean(times) if times else None,
                      "iters_mean": float(it.mean()), "iters_max": int(it.max())}), flush=True)
    emb.close()
    return 0


def run_case(args):
    """One batch of the oscillatory field at n cells: fields, then one Darcy
    solve (the small, fixed launch sequence used for kernel captures)."""
    if args.case in ("darcy3", "field3"):
        return run_case3(args)
    import torch
    from paper_2306_13493_gb300 import build, sce
    build.build_library()
    sce.load()
    wl = workloads.OSCILLATORY
    n, count, prec = args.n, args.count, args.precision
    emb = sce.ce_setup_embedding(wl.kind, wl.nu, wl.lam, wl.sigma2, n, pad_mode=wl.pad_mode)
    dt = torch.float32 if prec == 32 else torch.float64
    k = torch.empty(count, n + 1, n + 1, dtype=dt, device="cuda")
    qoi = torch.empty(count, 3, dtype=torch.float64, device="cuda")
    iters = torch.empty(count, dtype=torch.int32, device="cuda")
    times = []
    for rep in range(1 + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if args.case == "field":
            sce.ce_sample_batch(emb, wl.seed, 0, rep * count, count, prec, k)
        else:
            if rep == 0:
                sce.ce_sample_batch(emb, wl.seed, 0, 0, count, prec, k)
            sce.darcy_solve_batch(n, k, count, qoi, f=wl.f, rtol=wl.rtol, precision=prec,
                                  iters=iters, allow_not_converged=True)
        e1.record()
        torch.cuda.synchronize()
        if rep > 0:
            times.append(e0.elapsed_time(e1))
    it = iters.cpu().numpy()
    print(json.dumps({"case": args.case, "n": n, "count": count, "precision": prec,
                      "ms": statistics.mean(times) if times else None,
                      "iters_mean": float(it.mean()), "iters_max": int(it.max())}), flush=True)
    emb.close()
    return 0


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks/throttle sampling every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.idx), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ------------------------------------------------------------------ CPU oracle (baseline)
_ORACLE_LEVELS = None


def _oracle_init(wl):
    global _ORACLE_LEVELS
    try:
        from oracle import embedding as oem
        levels = {}
        L = len(wl.N) - 1
        for (l, n, _) in wl.levels:
            e = oem.setup_embedding(wl.kind, wl.nu, wl.lam, wl.sigma2, n, wl.pad_mode)
            kf, kc = workloads.keep_counts(e.P, l == L, wl.smoothing)
            mf = oem.smoothing_mask(e.Lam, kf)
            mc = oem.smoothing_mask(e.Lam, kc)
            levels[l] = (e, mf, mc)
        _ORACLE_LEVELS = (wl, levels)
    except Exception as exc:  # reported by the first task instead of respawning workers
        _ORACLE_LEVELS = exc


def _oracle_task(task):
    from oracle import mlmc as omlmc
    if isinstance(_ORACLE_LEVELS, Exception):
        raise RuntimeError(f"oracle worker set-up failed: {_ORACLE_LEVELS!r}")
    wl, levels = _ORACLE_LEVELS
    l, sample = task
    e, mf, mc = levels[l]
    t0 = time.perf_counter()
    omlmc.level_estimate(e, mf, mc, wl.seed, l, sample, 1, qoi_index=wl.qoi, f=wl.f,
                         precision=64)
    return l, time.perf_counter() - t0


def _oracle_ready(_):
    time.sleep(0.2)
    return isinstance(_ORACLE_LEVELS, Exception)


def oracle_pool(wl):
    """Spawned worker pool with the oracle set-up done in every worker (the
    set-up finishes here, so it never overlaps a timed GPU region)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    env_threads = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}
    os.environ.update(env_threads)
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(cores, initializer=_oracle_init, initargs=(wl,))
    pool.map(_oracle_ready, range(2 * cores), chunksize=1)
    return pool, cores


def oracle_measure(pool, cores, wl, step):
    """Times one bounded sample of the workload on the oracle (all cores, one
    sample per task, single-threaded BLAS).  Returns (samples/s of the N_l mix,
    wall seconds, per-level mean seconds)."""
    tasks = [(l, 10_000_000 + step * 1000 + i) for (l, n, N) in wl.levels
             for i in range(CPU_SAMPLES[l])]
    t0 = time.perf_counter()
    res = pool.map(_oracle_task, tasks, chunksize=1)
    wall = time.perf_counter() - t0
    per = {}
    for l, t in res:
        per.setdefault(l, []).append(t)
    mean = {l: sum(v) / len(v) for l, v in per.items()}
    Ntot = sum(N for (_, _, N) in wl.levels)
    sec_per_sample = sum(N * mean[l] for (l, _, N) in wl.levels) / Ntot
    return cores / sec_per_sample, wall, mean


def cpu_sample_text(wl, cores):
    return (f"oracle (numpy/scipy FP64) on {cores} host cores, one sample per task with "
            f"single-threaded BLAS; {'/'.join(map(str, CPU_SAMPLES))} samples on levels 0..5, "
            f"per-sample times scaled to the N_l mix {'/'.join(map(str, wl.N))}")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = workloads.OSCILLATORY
    pool, cores = oracle_pool(wl)
    try:
        for w in range(args.warmup):
            oracle_measure(pool, cores, wl, 1000 + w)
        vals, walls = [], []
        for s in range(args.steps):
            v, wall, _ = oracle_measure(pool, cores, wl, s)
            vals.append(v)
            walls.append(wall)
    finally:
        pool.close()
        pool.join()
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * statistics.mean(walls), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.describe()},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": cpu_sample_text(wl, cores)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
# ------------------------------------------------------------------ precision study
_PS_EMB = {}


def _ps_task(task):
    """Oracle QoIs (outflow, point value, L2 norm) of one sample of the study."""
    import numpy as np
    from oracle import embedding as oem
    from oracle import mlmc as omlmc
    ps = workloads.PRECISION_STUDY
    nu, sample, prec = task
    if nu not in _PS_EMB:
        _PS_EMB[nu] = oem.setup_embedding(0, nu, ps.lam, ps.sigma2, ps.n, ps.pad_mode, J=ps.J)
    e = _PS_EMB[nu]
    full = np.ones(e.Lam.shape, dtype=bool)
    Qf, _ = omlmc.level_qois(e, full, None, ps.seed, 0, [sample], f=ps.f, precision=prec,
                             coarse=False)
    return nu, sample, prec, Qf[0]


def smoothing_study(args):
    """workloads.SMOOTHING_STUDY: per covariance and grid, the level-0 QoI
    with the full and with the smoothed spectrum (same normals), the sup-norm
    of the field difference and the Theorem 1 bound shape
    s^(-1/2) (Lambda^ord_(s-tau+1))^(1/2) tau (p = 1)."""
    import numpy as np
    import torch
    from paper_2306_13493_gb300 import build, sce
    build.build_library()
    sce.load()
    ss = workloads.SMOOTHING_STUDY
    dev = torch.device("cuda", 0)
    out = {"study": "smoothing", "sigma2": ss.sigma2, "qoi": "L2 norm", "f": ss.f, "tau": "sqrt(s)",
           "cases": []}
    for kind, nu, lam in ss.covs:
        pad = sce.CE_PAD_NONE if kind == sce.CE_COV_SEP_EXP else sce.CE_PAD_SMOOTH
        rows = []
        for n, N in zip(ss.ns, ss.samples):
            ep = sce.ce_setup_embedding(kind, nu, lam, ss.sigma2, n, pad_mode=pad,
                                        J=0 if pad == sce.CE_PAD_NONE else -1)
            es = sce.ce_setup_embedding(kind, nu, lam, ss.sigma2, n, pad_mode=pad,
                                        J=0 if pad == sce.CE_PAD_NONE else -1,
                                        keep_fine=sce.CE_KEEP_TAU_SQRT_S,
                                        keep_coarse=sce.CE_KEEP_TAU_SQRT_S)
            P, s_ = ep.P, ep.info.s
            tau = s_ - es.info.keep_eff_fine
            lam_all = torch.empty(s_, dtype=torch.float64)
            sce.ce_get_eigenvalues(ep, lam_all)
            lam_ord = np.sort(lam_all.numpy())[::-1]
            lam_cut = float(lam_ord[s_ - tau]) if tau > 0 else 0.0   # Lambda^ord_(s-tau+1)
            q = {}
            zdiff = []
            for tag, e in (("full", ep), ("smooth", es)):
                qf = torch.empty(N, 3, dtype=torch.float64, device=dev)
                sce.mlmc_level_estimate(e, ss.seed, 0, 0, N, qoi_index=ss.qoi, f=ss.f, rtol=1e-10,
                                        maxit=4000, precision=64, qoi_f=qf,
                                        allow_not_converged=True)
                q[tag] = qf[:, ss.qoi].cpu().numpy()
            # sup-norm of Z - Z~ on the grid (FP64 fields, chunks of 64 samples)
            for c0 in range(0, N, 64):
                c = min(64, N - c0)
                ka = torch.empty(c, n + 1, n + 1, dtype=torch.float64, device=dev)
                kb = torch.empty_like(ka)
                sce.ce_sample_batch(ep, ss.seed, 0, c0, c, 64, k_fine=ka)
                sce.ce_sample_batch(es, ss.seed, 0, c0, c, 64, k_fine=kb)
                zdiff.append((ka.log() - kb.log()).abs().amax(dim=(1, 2)).cpu().numpy())
            zdiff = np.concatenate(zdiff)
            d = q["full"] - q["smooth"]
            bound = s_ ** -0.5 * lam_cut ** 0.5 * tau
            rows.append({"n": n, "P": P, "s": s_, "tau": int(tau), "N": N,
                         "lambda_ord_s_minus_tau_plus_1": lam_cut,
                         "mean_abs_dQ": float(abs(d.mean())), "mean_dQ_std_error":
                             float(d.std(ddof=1) / np.sqrt(N)),
                         "var_dQ": float(d.var(ddof=1)),
                         "E_sup_dZ": float(zdiff.mean()), "thm1_bound_shape": bound,
                         "ratio_E_sup_dZ_to_bound": float(zdiff.mean() / bound) if bound > 0 else None})
            ep.close()
            es.close()
        hs = np.log2([1.0 / r["n"] for r in rows])
        def rate(key):
            y = np.log2(np.maximum([r[key] for r in rows], 1e-300))
            return float(np.polyfit(hs, y, 1)[0])
        out["cases"].append({"kind": "sep_exp" if kind == sce.CE_COV_SEP_EXP else "matern",
                             "nu": nu, "lambda": lam,
                             "padding": "none (P = 2n)" if pad == sce.CE_PAD_NONE else
                             "smooth periodisation",
                             "rate_mean_abs_dQ_in_h": rate("mean_abs_dQ"),
                             "rate_var_dQ_in_h": rate("var_dQ"),
                             "rate_E_sup_dZ_in_h": rate("E_sup_dZ"), "rows": rows})
    print(json.dumps(out), flush=True)
    return 0


def qmc_study(args):
    """workloads.QMC_STUDY: standard error of each level mean with the lattice
    sampler (R shifts x N points; error from the spread of the shift means)
    against Philox Monte Carlo with the same R N samples."""
    import numpy as np
    import torch
    from paper_2306_13493_gb300 import build, sce
    build.build_library()
    sce.load()
    qs = workloads.QMC_STUDY
    dev = torch.device("cuda", 0)
    L = qs.levels - 1
    out = {"study": "qmc", "nu": qs.nu, "lambda": qs.lam, "sigma2": qs.sigma2, "N": qs.N,
           "R": qs.R, "a": qs.a, "qoi": ["outflow", "u(7/15,7/15)", "L2 norm"][qs.qoi],
           "levels": []}
    for l in range(qs.levels):
        n = qs.n0 << l
        e0 = sce.ce_setup_embedding(0, qs.nu, qs.lam, qs.sigma2, n, pad_mode=sce.CE_PAD_SMOOTH)
        kf, kc = workloads.keep_counts(e0.P, l == L, True)
        e0.close()
        emb = sce.ce_setup_embedding(0, qs.nu, qs.lam, qs.sigma2, n, pad_mode=sce.CE_PAD_SMOOTH,
                                     keep_fine=kf, keep_coarse=kc)
        lat = sce.QmcLattice(emb, qs.N, qs.a)
        Y = torch.empty(qs.N * qs.R, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sce.mlmc_level_estimate(emb, qs.seed, l, 0, qs.N * qs.R, qoi_index=qs.qoi, f=qs.f,
                                rtol=1e-10, maxit=2000, precision=32, Y=Y,
                                allow_not_converged=True)
        torch.cuda.synchronize()
        t_mc = time.perf_counter() - t0
        y_mc = Y.cpu().numpy()
        means = []
        t0 = time.perf_counter()
        for r in range(qs.R):
            Yq = torch.empty(qs.N, dtype=torch.float64, device=dev)
            o, _ = sce.mlmc_level_estimate_qmc(lat, qs.seed, l, r, 0, qs.N, qoi_index=qs.qoi,
                                               f=qs.f, rtol=1e-10, maxit=2000, precision=32, Y=Yq,
                                               allow_not_converged=True)
            means.append(o.sumY / o.N)
        torch.cuda.synchronize()
        t_qmc = time.perf_counter() - t0
        means = np.array(means)
        se_mc = float(y_mc.std(ddof=1) / np.sqrt(y_mc.size))
        se_qmc = float(means.std(ddof=1) / np.sqrt(qs.R))
        out["levels"].append({"level": l, "n": n, "P": emb.P,
                              "mean_mc": float(y_mc.mean()), "mean_qmc": float(means.mean()),
                              "std_error_mc": se_mc, "std_error_qmc": se_qmc,
                              "variance_reduction": (se_mc / se_qmc) ** 2 if se_qmc > 0 else None,
                              "seconds_mc": round(t_mc, 4), "seconds_qmc": round(t_qmc, 4)})
        lat.close()
        emb.close()
    print(json.dumps(out), flush=True)
    return 0


# ------------------------------------------------------------------ three dimensions
_ORACLE3 = None


def _oracle3_init(wl):
    global _ORACLE3
    try:
        import math as _m
        from oracle import embedding as oem
        from oracle import field3d as of3
        levels = {}
        for l in range(len(wl.cpu_samples)):
            e = of3.setup_embedding3(0, wl.nu, wl.lam, wl.sigma2, wl.n0 << l, oem.PAD_SMOOTH)
            s = e.Lam.size
            keep = s - _m.isqrt(s)
            mask = oem.smoothing_mask(e.Lam, keep)
            levels[l] = (e, mask)
        _ORACLE3 = (wl, levels)
    except Exception as exc:
        _ORACLE3 = exc


def _oracle3_task(task):
    from oracle import darcy3d as od3
    from oracle import field3d as of3
    if isinstance(_ORACLE3, Exception):
        raise RuntimeError(f"oracle worker set-up failed: {_ORACLE3!r}")
    wl, levels = _ORACLE3
    l, sample = task
    e, mask = levels[l]
    t0 = time.perf_counter()
    kf, kc = of3.sample_k3(e, mask, mask if l > 0 else None, wl.seed, l, sample, 64)
    y = od3.solve_qois3(kf, wl.f)[wl.qoi]
    if l > 0:
        y -= od3.solve_qois3(kc, wl.f)[wl.qoi]
    return l, time.perf_counter() - t0


def _oracle3_ready(_):
    time.sleep(0.2)
    return isinstance(_ORACLE3, Exception)


def three_d_study(args):
    """workloads.THREE_D: one step = one MLMC sweep over the 3D levels through
    mlmc3_estimate_levels (all levels in one call, --concurrency of them in
    flight; fields by the three-pass FFT sampler, Kuhn-P1 solves on the fine
    and coarse grids, level sums).  Prints one JSON line."""
    import numpy as np
    import torch
    from paper_2306_13493_gb300 import build, sce
    build.build_library()
    sce.load()
    wl = workloads.THREE_D
    dev = torch.device("cuda", 0)
    L = len(wl.N) - 1
    t0 = time.perf_counter()
    embs = []
    for (l, n, N) in wl.levels:
        embs.append(sce.ce3_setup_embedding(
            0, wl.nu, wl.lam, wl.sigma2, n, pad_mode=sce.CE_PAD_SMOOTH,
            keep_fine=-1 if l == L else sce.CE_KEEP_TAU_SQRT_S,
            keep_coarse=sce.CE_KEEP_TAU_SQRT_S))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0

    conc = max(1, min(args.concurrency, len(wl.N)))

    def sweep(step, c=None):
        tasks = [{"emb": embs[l], "level": l, "first_sample": step * N, "count": N}
                 for (l, n, N) in wl.levels]
        outs, _, _ = sce.mlmc3_estimate_levels(tasks, wl.seed, qoi_index=wl.qoi, f=wl.f,
                                               rtol=wl.rtol, maxit=2000,
                                               max_concurrency=conc if c is None else c,
                                               allow_not_converged=True)
        return outs

    steps = args.steps if args.steps else 3
    warmup = max(3, args.warmup if args.warmup is not None else 3)
    for w in range(warmup):
        sweep(100000 + w)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    acc = [[0, 0.0, 0.0, 0, 0] for _ in wl.N]     # N, sumY, sumY2, failed, max iters
    ms = []
    clocks = ClockSampler(0)
    clocks.start()
    for k in range(steps):
        flush.fill_(k & 255)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        outs = sweep(k)
        ev1.record()
        torch.cuda.synchronize()
        ms.append(ev0.elapsed_time(ev1))
        for l, o in enumerate(outs):
            a = acc[l]
            a[0] += o.N
            a[1] += o.sumY
            a[2] += o.sumY2
            a[3] += o.n_failed
            a[4] = max(a[4], o.max_iters)
    clk = clocks.stop()
    ms_step = statistics.mean(ms)
    total = sum(wl.N)

    sce.sce_profile_enable(1)
    sweep(900000, c=1)      # levels one after another: each launch's events time it alone
    prof = sce.sce_profile_read()
    sce.sce_profile_enable(0)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    prof = {k: v for k, v in prof.items() if v[2] > 0}
    ptot = sum(v[0] for v in prof.values())
    kernels = {name: {"ms": round(m, 3), "launches": nl, "share": round(m / ptot, 4),
                      "GBps": round(by / (m * 1e6), 1) if m > 0 else None}
               for name, (m, by, nl) in sorted(prof.items(), key=lambda kv: -kv[1][0])}
    roof = None
    hbm_kernels = {k: v for k, v in prof.items() if k not in ("ce3_x", "reduce", "mg_coarsest")}
    if hbm_kernels:
        name, (m, by, nl) = max(hbm_kernels.items(), key=lambda kv: kv[1][0])
        ach = by / (m * 1e6)
        roof = {"bound": "hbm", "kernel": name, "achieved": round(ach, 1), "peak": hbm,
                "unit": "GB/s", "frac": round(ach / hbm, 4), "traffic": None,
                "algorithmic_bytes_per_launch": round(by / nl), "peak_source": peak_src,
                "avg_launch_us": round(1000 * m / nl, 2),
                "timed": "one extra sweep with CUDA events around every launch"}
    x3 = prof.get("ce3_x")
    per_level = []
    for (l, n, N), a in zip(wl.levels, acc):
        mean = a[1] / a[0]
        var = (a[2] - a[0] * mean * mean) / (a[0] - 1)
        per_level.append({"level": l, "n": n, "P": embs[l].P, "N": N, "mean_Y": mean,
                          "var_Y": var, "failed": a[3], "max_iters": a[4]})
    line = {"study": "3d", "metric": "MLMC level-samples/s, all levels of one 3D sweep (each: "
                                     "field + fine and coarse Darcy solves + QoI + Y_l)",
            "value": total / (ms_step / 1000.0), "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "dtype": DTYPE_MIXED, "data": "synthetic",
            "config": {"workload": wl.describe(), "levels_in_flight": conc,
                       "l2": "flushed before every timed step (258 MB write)"},
            "setup_seconds": round(setup_s, 3), "clocks": clk, "per_level": per_level,
            "kernels": kernels, "roofline": roof,
            "field_x_pass": ({"ms": round(x3[0], 3), "launches": x3[2],
                              "bound": "alu (Philox + Box-Muller + FFT)"} if x3 else None)}
    if not args.no_cpu_baseline:
        import multiprocessing as mp
        cores = os.cpu_count() or 1
        os.environ.update({"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1",
                           "MKL_NUM_THREADS": "1"})
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores, initializer=_oracle3_init, initargs=(wl,)) as pool:
            pool.map(_oracle3_ready, range(2 * cores), chunksize=1)
            tasks = [(l, 20_000_000 + i) for l in range(len(wl.cpu_samples))
                     for i in range(wl.cpu_samples[l])]
            tw = time.perf_counter()
            res = pool.map(_oracle3_task, sorted(tasks, key=lambda t: -t[0]), chunksize=1)
            wall = time.perf_counter() - tw
        per = {}
        for l, t in res:
            per.setdefault(l, []).append(t)
        mean = {l: sum(v) / len(v) for l, v in per.items()}
        lv = range(len(wl.cpu_samples))
        sec = sum(wl.N[l] * mean[l] for l in lv) / sum(wl.N[l] for l in lv)
        line["cpu_baseline"] = {
            "value": cores / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"oracle (numpy/scipy FP64, direct sparse solves) on {cores} host cores, "
                       f"{'/'.join(map(str, wl.cpu_samples))} samples on levels "
                       f"0..{len(wl.cpu_samples) - 1} (n = "
                       f"{'/'.join(str(wl.n0 << l) for l in lv)}), per-sample times scaled to "
                       f"their N_l mix; level 3 not sampled (one direct solve on 65^3 takes "
                       f"minutes), so this rate is an upper bound for the full mix"),
            "wall_seconds": round(wall, 2),
            "per_level_seconds": {str(l): round(mean[l], 4) for l in lv}}
    for e in embs:
        e.close()
    print(json.dumps(line), flush=True)
    return 0


def precision_study(args):
    """Config of workloads.PRECISION_STUDY: per nu, the mixed and the all-FP64
    GPU paths on the same samples (per-sample QoIs), the FP64 oracle on the
    first oracle_samples of them (with FP64 normals, and with the FP32 normals
    the mixed path draws), and the bias of the mixed mean against its
    statistical error."""
    import multiprocessing as mp
    import numpy as np
    ps = workloads.PRECISION_STUDY
    K = args.study_oracle if args.study_oracle is not None else ps.oracle_samples
    os.environ.update({"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1"})
    cores = os.cpu_count() or 1
    pool = mp.get_context("spawn").Pool(min(cores, 16)) if K > 0 else None
    oracle_async = None
    if pool:   # the oracle runs on the host while the GPU paths run
        tasks = [(nu, i, prec) for nu in ps.nus for prec in (64, 32) for i in range(K)]
        oracle_async = pool.map_async(_ps_task, tasks, chunksize=1)
    import torch
    from paper_2306_13493_gb300 import build, sce
    build.build_library()
    sce.load()
    dev = torch.device("cuda", 0)
    count = args.study_count or ps.count
    out = {"study": "precision", "n": ps.n, "lambda": ps.lam, "sigma2": ps.sigma2, "f": ps.f,
           "count": count, "oracle_samples": K, "rtol": ps.rtol, "per_nu": []}
    gpu = {}
    for nu in ps.nus:
        emb = sce.ce_setup_embedding(0, nu, ps.lam, ps.sigma2, ps.n, pad_mode=ps.pad_mode, J=ps.J)
        rec = {"nu": nu, "P": emb.P, "lambda_min_over_max": emb.info.lambda_min /
               emb.info.lambda_max}
        for prec in (32, 64):
            q = torch.empty(count, 3, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            o, st = sce.mlmc_level_estimate(emb, ps.seed, 0, 0, count, qoi_index=1, f=ps.f,
                                            rtol=ps.rtol, maxit=4000, precision=prec, qoi_f=q,
                                            allow_not_converged=True)
            torch.cuda.synchronize()
            rec[f"seconds_fp{prec}"] = round(time.perf_counter() - t0, 3)
            rec[f"failed_fp{prec}"] = o.n_failed
            rec[f"max_iters_fp{prec}"] = o.max_iters
            gpu[(nu, prec)] = q.cpu().numpy()
        emb.close()
        qm, qd = gpu[(nu, 32)], gpu[(nu, 64)]
        rel = np.abs(qm - qd) / np.maximum(np.abs(qd), 1e-300)
        se = qd.std(axis=0, ddof=1) / np.sqrt(count)
        rec["mixed_vs_fp64_gpu"] = {
            "max_rel": rel.max(axis=0).tolist(), "median_rel": np.median(rel, axis=0).tolist(),
            "mean_diff": (qm - qd).mean(axis=0).tolist(), "std_error_of_mean": se.tolist(),
            "bias_over_std_error": (np.abs((qm - qd).mean(axis=0)) / se).tolist()}
        out["per_nu"].append(rec)
    if oracle_async is not None:
        res = oracle_async.get()
        pool.close()
        pool.join()
        orc = {(nu, i, prec): q for nu, i, prec, q in res}
        for rec in out["per_nu"]:
            nu = rec["nu"]
            for name, gprec, oprec in (("mixed_vs_oracle_fp64_normals", 32, 64),
                                       ("mixed_vs_oracle_fp32_normals", 32, 32),
                                       ("fp64_gpu_vs_oracle", 64, 64)):
                g = gpu[(nu, gprec)][:K]
                o = np.array([orc[(nu, i, oprec)] for i in range(K)])
                r = np.abs(g - o) / np.maximum(np.abs(o), 1e-300)
                rec[name] = {"max_rel": r.max(axis=0).tolist(),
                             "median_rel": np.median(r, axis=0).tolist()}
    out["qoi_order"] = ["outflow", "u(7/15,7/15)", "L2 norm"]
    print(json.dumps(out), flush=True)
    return 0


# bound of each kernel family that HBM bandwidth does not bound (the V(2,2)
# multigrid tiles: 65 % issue active and 34 % of DRAM bandwidth in their n = 512
# capture, the second sweep having doubled their instructions per byte); the coarse
# multigrid tail reads its levels from L2 (judged against the measured L2 read
# bandwidth); the row pass (Philox, Box-Muller, butterflies), the one-block
# solver (whole solve in shared memory) and the fused n = 64 V-cycle (one
# level in registers, the levels below in shared memory) are bound by
# instruction issue and barriers; the reductions and the level sums (one warp
# per sample over a few partials) and the coarsening of the levels of at most
# 64 cells (one block per sample, a few microseconds) by launch latency.  The
# rest are HBM-bound.
KERNEL_BOUND = {"mg_tail": "l2", "ce_row": "issue", "darcy_small": "issue", "mg_v64": "issue",
                "mg_up": "issue", "mg_down": "issue", "mg_up3": "issue", "mg_down3": "issue",
                "reduce": "latency", "level_sums": "latency", "coarsen_tail": "latency"}

# Warp instructions per algorithmic byte of issue-bound families, from one ncu
# capture of the kernel (smsp__inst_executed.sum / the launch's algorithmic
# bytes), with the file, kernel and sha256 of the captured source text: the
# bench's issue fraction = its algorithmic bytes x this ratio / time / the
# measured FMA issue rate, reported only while the source is the captured one.
INSTR_PER_ALG = {
    # n = 512 x 32 launches with 48-row windows and two sweeps per side; the
    # n = 128 launches of the same capture with three (profiles/mg_up_n512x32.md,
    # profiles/mg_down_n512x32.md)
    "mg_up": (40920192 / 176882432, "paper_2306_13493_gb300/csrc/mg_tiles.cuh", "mg_up_kernel",
              "1e6c3d6b2ae324929df37ce45854077b49df36df7edd57bdbf3e5778ac9dd6b9"),
    "mg_down": (34649984 / 143196800, "paper_2306_13493_gb300/csrc/mg_tiles.cuh",
                "mg_down_kernel", "0ce6fbf16c0c0370eaa26537be930a5a137567ada777dd6f46508928316588f9"),
    "mg_up3": (3979584 / 11191040, "paper_2306_13493_gb300/csrc/mg_tiles.cuh", "mg_up_kernel",
               "1e6c3d6b2ae324929df37ce45854077b49df36df7edd57bdbf3e5778ac9dd6b9"),
    "mg_down3": (3466176 / 9060992, "paper_2306_13493_gb300/csrc/mg_tiles.cuh",
                 "mg_down_kernel", "0ce6fbf16c0c0370eaa26537be930a5a137567ada777dd6f46508928316588f9"),
}


def measure_peaks(sce, stream, reps=10):
    """FP32 FMA issue rate and L2 read bandwidth of this GPU, by the library's
    two peak kernels (sce_peak_fma / sce_peak_l2): best of `reps` CUDA-event
    timings after a warm-up launch."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks, dtype=torch.float32, device="cuda")

    def best(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts)

    iters = 2000
    ms = best(lambda: sce.sce_peak_fma(out, blocks, iters, stream=stream.cuda_stream))
    warp_inst = blocks * 8 * iters * 128
    l2_bytes, l2_reps = 32 << 20, 400
    buf = torch.ones(l2_bytes // 4, dtype=torch.float32, device="cuda")
    ms2 = best(lambda: sce.sce_peak_l2(buf, l2_reps, blocks, out, stream=stream.cuda_stream))
    return {"fma_warp_inst_per_s": warp_inst / (ms / 1000.0),
            "fp32_tflops": warp_inst * 32 * 2 / (ms / 1000.0) / 1e12,
            "l2_read_gbs": l2_bytes * l2_reps / (ms2 / 1000.0) / 1e9,
            "sms": sms,
            "how": "sce_peak_fma: %d blocks x 256 threads x %d x 128 FMAs in 8 independent "
                   "chains; sce_peak_l2: %d MiB buffer read %d times by ld.global.cg, %d blocks; "
                   "best of %d CUDA-event timings" % (blocks, iters, l2_bytes >> 20, l2_reps,
                                                       blocks, reps)}


def run_peaks(args):
    import torch
    from paper_2306_13493_gb300 import build, sce
    build.build_library()
    sce.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    clocks.start()
    pk = measure_peaks(sce, stream, reps=20)
    pk["clocks"] = clocks.stop()
    print(json.dumps(pk), flush=True)
    return 0


def cufft_comparison(sce, stream, flush, sizes=(32, 64, 128, 256, 512)):
    """The library's FP32 field passes against cuFFT (through torch.fft, a
    comparison only: the library never calls cuFFT) on the oscillatory
    covariance at n = 32..512 (P = 4n = 128..2048), the finest-level masks
    (fine field unsmoothed).  Accuracy: max relative error of each FP32 field
    against the FP64 field of the library (which matches the FP64 oracle to
    1e-10), from the same normals.  Time (CUDA events, L2 flushed):
    ce_sample_batch for the whole field (normals, sqrt(Lambda~) scaling,
    pruned row and column FFTs, Hartley, exp), against cuFFT for the
    transform alone (a full P x P complex-to-complex +i transform of the
    pre-computed, pre-scaled spectrum) and for transform + Hartley + exp of
    the kept (n+1)^2 vertices."""
    import torch
    wl = workloads.OSCILLATORY
    rows = []
    for n in sizes:
        emb = sce.ce_setup_embedding(wl.kind, wl.nu, wl.lam, wl.sigma2, n, pad_mode=wl.pad_mode)
        P = emb.P
        count = max(2, min(64, (256 << 20) // (P * P * 8)))
        lam = torch.empty(P * P, dtype=torch.float64, device="cuda")
        sce.ce_get_eigenvalues(emb, lam)
        sq = lam.clamp_min(0).sqrt().view(P, P)
        xi64 = torch.empty(count, P * P, dtype=torch.float64, device="cuda")
        xi32 = torch.empty(count, P * P, dtype=torch.float32, device="cuda")
        sce.ce_normals(wl.seed, 0, 0, count, P * P, 64, xi64)
        sce.ce_normals(wl.seed, 0, 0, count, P * P, 32, xi32)
        k64 = torch.empty(count, n + 1, n + 1, dtype=torch.float64, device="cuda")
        k32 = torch.empty(count, n + 1, n + 1, dtype=torch.float32, device="cuda")
        sce.ce_sample_batch(emb, wl.seed, 0, 0, count, 64, k64)
        sce.ce_sample_batch(emb, wl.seed, 0, 0, count, 32, k32)
        w32 = (xi32.view(count, P, P) * sq.float()).to(torch.complex64)

        def cufft_field(w):
            v = torch.fft.ifft2(w, norm="forward")[:, :n + 1, :n + 1]
            return torch.exp((v.real + v.imag) / P)

        kc = cufft_field(w32)
        # reference: the FP32 normals in FP64 arithmetic (both FP32 fields use them)
        ref = cufft_field((xi32.double().view(count, P, P) * sq).to(torch.complex128))
        rel = lambda a: float(((a.double() - ref).abs().max() / ref.abs().max()).item())

        def t_ms(fn, reps=5):
            fn()
            ts = []
            for _ in range(reps):
                flush.zero_()
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            return statistics.median(ts)

        ours = t_ms(lambda: sce.ce_sample_batch(emb, wl.seed, 0, 0, count, 32, k32,
                                                stream=stream.cuda_stream))
        tr = t_ms(lambda: torch.fft.ifft2(w32, norm="forward"))
        full = t_ms(lambda: cufft_field(w32))
        rows.append({"n": n, "P": P, "count": count,
                     "ours_ms": round(ours, 4), "cufft_transform_ms": round(tr, 4),
                     "cufft_field_ms": round(full, 4),
                     "ours_rel_err_vs_fp64": rel(k32), "cufft_rel_err_vs_fp64": rel(kc),
                     "ours_fp64_vs_ref": float(((k64 - cufft_field(
                         (xi64.view(count, P, P) * sq).to(torch.complex128))).abs().max() /
                         k64.abs().max()).item())})
        emb.close()
        del xi64, xi32, w32, k64, k32, kc, ref
    return {"note": cufft_comparison.__doc__.split("\n\n")[0].replace("\n", " "),
            "rows": rows}


def time_to_rmse_study(sce, stream, prec, eps=1e-3, n_max=2048):
    """Cost to a total root-mean-square error eps of the oscillatory covariance
    (Matern nu = 0.5, lambda = 0.02, sigma^2 = 1, smooth periodisation J = n,
    f = 1) for the QoI ||u||_L2 -- the paper's QoI for its Matern experiments
    (§4.3); for the point value u(7/15, 7/15) the Richardson bias is still
    ~1.5e-3 on the 2048^2 grid, so eps = 1e-3 is out of reach below it.
    Variants: MLMC-CES (tau_l = sqrt(s_l), finest level unsmoothed) from
    h0 = 1/4, 1/8, 1/16, and plain MLMC from its own coarsest mesh,
    Eq. (3.8): the largest h0 = 2^-k <= sqrt(8 nu) lambda = 0.04, i.e. 1/32.
    Each runs mlmc.run_adaptive: levels added (pilot 100 on the first three,
    50 on each added one) until the Richardson bias (alpha fitted on the three
    finest levels, at most 2; the three-level form of the test) is at most
    eps/sqrt(2) -- and at least until the finest mesh is 4 x finer than the
    plain-MLMC mesh of Eq. (3.8), so that the levels of the bias test are all
    in the range where plain MLMC may start (below it E[Y_l] can be small by
    accident and end the loop early) -- up to the 2048^2 grid; there, with
    the bias below eps, the variance target becomes eps^2 - bias^2
    (fill_variance).  Cost = GPU seconds of every level
    estimate (CUDA events), the samples of levels rebuilt when they stopped
    being the finest included; embedding set-up is not counted (reported
    apart as wall time).  cost_vs_eps predicts each variant's cost for other
    eps from its measured level statistics with the finest level each eps
    needs (the same bias test), and plain MC on that level's grid from
    V[Q_L] and its cost per sample."""
    import math as _m
    from paper_2306_13493_gb300 import mlmc as gm
    wl = workloads.OSCILLATORY
    qoi = 2
    seed = wl.seed + 1000
    plain_n0 = gm.coarsest_cells(wl.kind, wl.nu, wl.lam)
    variants = [("mlmc_ces", 4), ("mlmc_ces", 8), ("mlmc_ces", 16), ("mlmc_plain", plain_n0)]
    out = {"eps": eps, "qoi": "||u||_L2", "f": wl.f,
           "note": " ".join(time_to_rmse_study.__doc__.split())}
    eps_list = [1e-2, 5e-3, 2e-3, 1e-3, 5e-4]
    for name, n0 in variants:
        smooth = name == "mlmc_ces"
        L_max = int(round(_m.log2(n_max // n0)))
        created = []

        def make_runner(l, finest, n0=n0, smooth=smooth, created=created):
            n = n0 << l
            e0 = sce.ce_setup_embedding(wl.kind, wl.nu, wl.lam, wl.sigma2, n,
                                        pad_mode=wl.pad_mode)
            kf, kc = workloads.keep_counts(e0.P, finest, smooth)
            e0.close()
            e = sce.ce_setup_embedding(wl.kind, wl.nu, wl.lam, wl.sigma2, n,
                                       pad_mode=wl.pad_mode, keep_fine=kf, keep_coarse=kc)
            created.append(e)
            return gm.LevelRunner(e, l, seed, qoi=qoi, f=wl.f, rtol=wl.rtol, precision=prec,
                                  stream=stream)

        t0 = time.perf_counter()
        # the three finest levels of the bias test at or below the plain-MLMC mesh
        L_min = min(L_max, max(0, int(round(_m.log2(4 * plain_n0 / n0)))))
        res = gm.run_adaptive(make_runner, eps, L0=min(2, L_max), L_max=L_max, pilot=100,
                              pilot_new=50, alpha_levels=3, alpha_max=2.0, bias_levels=3,
                              fill_variance=True, restart_previous_finest=smooth, L_min=L_min)
        wall = time.perf_counter() - t0
        for e in created:
            e.close()
        key = "%s_h0_1/%d" % (name, n0)
        out[key] = {
            "h0": 1.0 / n0, "levels_n": [x.n for x in res.levels], "L_min": L_min,
            "gpu_seconds": round(res.seconds, 4), "wall_seconds": round(wall, 2),
            "estimate": res.estimate, "stat_error": res.stat_error, "bias_est": res.bias,
            "rmse_est": res.rmse, "rmse_met": bool(res.rmse <= eps),
            "var_share": round(res.var_share, 4), "alpha_finest3": res.alpha,
            "N": [x.N for x in res.levels], "mean_Y": [x.mean for x in res.levels],
            "var_Y": [x.var for x in res.levels],
            "cost_per_sample_s": [x.cost for x in res.levels],
            "cost_vs_eps": [{"eps": c["eps"], "finest_n": res.levels[c["L"]].n,
                             "mlmc_s": round(c["mlmc_seconds"], 5),
                             "mc_s": round(c["mc_seconds"], 5)}
                            for c in gm.cost_versus_eps(res.levels, eps_list, choose_levels=True,
                                                        alpha_levels=3, alpha_max=2.0,
                                                        bias_levels=3, L_min=L_min)]}
    ces = [v["gpu_seconds"] for k, v in out.items() if k.startswith("mlmc_ces")]
    pl = out["mlmc_plain_h0_1/%d" % plain_n0]["gpu_seconds"]
    out["cost_ratio_plain_over_best_ces"] = round(pl / min(ces), 3) if ces else None
    return out


def plain_small_bench(sce, stream, flush):
    """The plain small workload (workloads.PLAIN_SMALL: 33 x 33 vertices,
    doubled embedding, no smoothing, f = 0, outflow): its 256 samples in one
    level call, FP64 (as quoted) and on the mixed path; CUDA events, L2 flushed."""
    import torch
    wl = workloads.PLAIN_SMALL
    n, N = wl.n0, wl.N[0]
    emb = sce.ce_setup_embedding(wl.kind, wl.nu, wl.lam, wl.sigma2, n, pad_mode=wl.pad_mode)
    Y = torch.empty(N, dtype=torch.float64, device="cuda")
    out = {"workload": wl.describe(), "P": emb.P}
    for prec in (64, 32):
        ms = []
        for r in range(6):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sce.mlmc_level_estimate(emb, wl.seed, 0, r * N, N, qoi_index=wl.qoi, f=wl.f,
                                    rtol=wl.rtol, maxit=2000, precision=prec, Y=Y,
                                    stream=stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if r >= 2:
                ms.append(e0.elapsed_time(e1))
        m = statistics.mean(ms)
        out["f64" if prec == 64 else "mixed"] = {"ms": round(m, 3),
                                                  "samples_per_s": round(N / (m / 1000.0), 1)}
    emb.close()
    return out


def mixed_launch_bench(args, sce, stream):
    """workloads.MIXED_LAUNCH: the level-pair buckets of several grid sizes
    in one mlmc_estimate_levels call (all buckets in flight at once), timed
    with CUDA events on the caller's stream after warm-up, L2 flushed."""
    import torch
    mw = workloads.MIXED_LAUNCH
    embs, tasks = [], []
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    for l, (n, c) in enumerate(mw.buckets):
        e = sce.ce_setup_embedding(0, mw.nu, mw.lam, mw.sigma2, n, pad_mode=mw.pad_mode)
        embs.append(e)
        tasks.append({"emb": e, "level": 2 + l, "count": c,
                      "Y": torch.empty(c, dtype=torch.float64, device=dev)})

    persistent_ok = args.precision == 32

    def launch(i, persistent=False):
        for t in tasks:
            t["first_sample"] = i * t["count"]
        outs, _, st = sce.mlmc_estimate_levels(tasks, mw.seed, qoi_index=mw.qoi, f=mw.f,
                                               rtol=mw.rtol, maxit=2000, precision=args.precision,
                                               max_concurrency=args.concurrency,
                                               stream=stream.cuda_stream, allow_not_converged=True,
                                               persistent=persistent)
        return outs

    def timed(fn, reps=3):
        fn(1000)
        fn(1001)
        tot, last = 0.0, None
        for i in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            last = fn(i)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / reps, last

    ms, outs = timed(launch)
    iters = [o.total_iters / (2 * o.N) for o in outs]
    nsamp = sum(c for _, c in mw.buckets)
    out = {"workload": mw.describe(), "P": [2 * n for n, _ in mw.buckets],
           "samples_per_launch": nsamp, "ms_per_launch": round(ms, 2),
           "samples_per_s": round(nsamp / (ms / 1e3), 1),
           "mean_iters_per_solve": [round(x, 2) for x in iters],
           "levels_in_flight": args.concurrency,
           "tile_heights": "as tuned before the timed steps"}
    if persistent_ok:
        pms, _ = timed(lambda i: launch(i, persistent=True))
        # the fields alone: one persistent launch for every bucket against one
        # ce_sample_batch call per bucket on the same stream
        ks = [(torch.empty(c, n + 1, n + 1, dtype=torch.float32, device=dev),
               torch.empty(c, n // 2 + 1, n // 2 + 1, dtype=torch.float32, device=dev))
              for n, c in mw.buckets]
        ftasks = [{"emb": t["emb"], "level": t["level"], "first_sample": 0, "count": t["count"],
                   "k_fine": kf, "k_coarse": kc} for t, (kf, kc) in zip(tasks, ks)]

        def fields_one(i):
            sce.ce_sample_levels(ftasks, mw.seed, stream=stream.cuda_stream)

        def fields_each(i):
            for ft in ftasks:
                sce.ce_sample_batch(ft["emb"], mw.seed, ft["level"], 0, ft["count"], 32,
                                    ft["k_fine"], ft["k_coarse"], stream=stream.cuda_stream)

        f1, _ = timed(fields_one)
        fe, _ = timed(fields_each)
        # the persistent field launch together with cached solver graphs
        os.environ["SCE_GRAPHS"] = "1"
        try:
            gms, _ = timed(lambda i: launch(i, persistent=True))
        finally:
            os.environ.pop("SCE_GRAPHS", None)
            sce.darcy_solver_cache_clear(stream=stream.cuda_stream)
        out["persistent"] = {
            "ms_per_launch": round(pms, 2), "samples_per_s": round(nsamp / (pms / 1e3), 1),
            "note": "every bucket's fields in one persistent launch (ce_sample_levels: device "
                    "work queue over all row and column blocks, bounded per-sample waits), "
                    "then the solves as in the streams path; bit-identical results",
            "fields_one_launch_ms": round(f1, 3), "fields_per_bucket_calls_ms": round(fe, 3),
            "with_cached_graphs": {"ms_per_launch": round(gms, 2),
                                   "samples_per_s": round(nsamp / (gms / 1e3), 1),
                                   "note": "the persistent path with SCE_GRAPHS=1: every "
                                           "solve shape keeps its buffers and a captured "
                                           "graph of four CG iterations, replayed"}}
        del ks
    for e in embs:
        e.close()
    return out


def serving_bench(args, sce):
    """The served loop (workloads.SERVED): a request server with `slots`
    concurrent requests, HBM-footprint admission and a resident embedding
    cache; Poisson arrivals at load x the measured service capacity, while an
    adaptive MLMC client (Eq. (3.6) loop to RMSE mlmc_eps on the oscillatory
    covariance, levels 0..4) drives its own level requests through the same
    server.  Latency = completion - submission of each background request."""
    import numpy as np
    from paper_2306_13493_gb300 import mlmc as gm
    sw = workloads.SERVED
    tenants = sw.draw_tenants()
    rng = np.random.default_rng(sw.arrival_seed + 1)
    next_first = {}

    def place(req):
        key = (req["tenant"], req["level"])
        req["first_sample"] = next_first.get(key, 0)
        next_first[key] = req["first_sample"] + req["count"]
        return req

    out = {"workload": "levels 0-%d (n=%d..%d), counts log-uniform %d-%d, %d tenants (nu in %s, "
                       "lambda log-uniform %s, sigma2 uniform %s), smoothing tau=sqrt(s)" % (
                           sw.levels - 1, sw.n0, sw.n0 << (sw.levels - 1), *sw.count_range,
                           sw.tenants, list(sw.nu_choices), list(sw.lam_range),
                           list(sw.sigma2_range)),
           "slots": args.serve_slots}
    with sce.Server(slots=args.serve_slots, max_embeddings=256, precision=args.precision,
                    slice_vertices=args.serve_slice_vertices,
                    rtol=1e-10, maxit=2000) as srv:
        # 1. every (tenant, level) embedding becomes resident
        t0 = time.perf_counter()
        tk = [srv.submit(place({**tenants[t], "tenant": t, "level": l, "n": sw.n0 << l,
                                "count": 1}))
              for t in range(len(tenants)) for l in range(sw.levels)]
        for t in tk:
            srv.wait(t)
        out["cache_warmup_s"] = round(time.perf_counter() - t0, 2)
        # 2. service capacity: a closed batch of requests of the mix
        batch = [place(sw.draw_request(rng, tenants)) for _ in range(48)]
        t0 = time.perf_counter()
        tk = [srv.submit(r) for r in batch]
        for t in tk:
            srv.wait(t)
        cap = len(batch) / (time.perf_counter() - t0)
        rate = sw.load * cap
        out["capacity_req_per_s"] = round(cap, 3)
        out["arrival_rate_per_s"] = round(rate, 3)
        # 3. open loop: Poisson arrivals for serve_seconds, the MLMC client alongside
        n_req = max(8, int(rate * args.serve_seconds))
        gaps = rng.exponential(1.0 / rate, n_req)
        reqs = [place(sw.draw_request(rng, tenants)) for _ in range(n_req)]
        tickets = [None] * n_req
        submitted = threading.Event()

        def submitter():
            t_start = time.perf_counter()
            at = 0.0
            for i, (g, r) in enumerate(zip(gaps, reqs)):
                at += g
                d = t_start + at - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets[i] = srv.submit(r)
            submitted.set()

        osc = workloads.OSCILLATORY
        client = {"nu": osc.nu, "lam": osc.lam, "sigma2": osc.sigma2}
        mres = {}

        def mlmc_client():
            runners = [gm.ServedLevelRunner(srv, client, l, osc.n0 << l,
                                            l == sw.mlmc_levels - 1, sw.mlmc_seed, qoi=osc.qoi,
                                            f=osc.f) for l in range(sw.mlmc_levels)]
            t0 = time.perf_counter()
            res = gm.run_to_rmse(runners, sw.mlmc_eps, pilot=[400, 200, 100, 50, 20])
            mres.update({"eps": sw.mlmc_eps, "wall_s": round(time.perf_counter() - t0, 3),
                         "estimate": res.estimate, "stat_error": res.stat_error,
                         "bias_est": res.bias, "N": [s.N for s in res.levels]})

        st0 = srv.stats()
        th = [threading.Thread(target=submitter), threading.Thread(target=mlmc_client)]
        for t in th:
            t.start()
        submitted.wait()
        res = [srv.wait(t) for t in tickets]
        for t in th:
            t.join()
        st1 = srv.stats()
    lat = np.array([r.t_done - r.t_submit for r in res]) * 1e3
    span = max(r.t_done for r in res) - min(r.t_submit for r in res)
    samples = sum(r.sums.N for r in res)
    # latency per size class: work = count x (n+1)^2 fine vertices
    work = np.array([q["count"] * (q["n"] + 1) ** 2 for q in reqs], dtype=np.float64)
    classes = {}
    for name, lo, hi in (("small", 0, 2 ** 20), ("medium", 2 ** 20, 2 ** 26),
                         ("large", 2 ** 26, np.inf)):
        sel = (work >= lo) & (work < hi)
        if sel.any():
            cl = lat[sel]
            classes[name] = {"work_vertices": [lo, hi if np.isfinite(hi) else None],
                             "requests": int(sel.sum()),
                             "p50_ms": round(float(np.percentile(cl, 50)), 2),
                             "p99_ms": round(float(np.percentile(cl, 99)), 2),
                             "max_ms": round(float(cl.max()), 2)}
    out.update({
        "requests": n_req, "p50_ms": round(float(np.percentile(lat, 50)), 2),
        "p99_ms": round(float(np.percentile(lat, 99)), 2),
        "mean_ms": round(float(lat.mean()), 2), "max_ms": round(float(lat.max()), 2),
        "samples_per_s": round(samples / span, 1),
        "failed": int(sum(r.status not in (0, -5) for r in res)),
        "cache_hits": st1["cache_hits"] - st0["cache_hits"],
        "cache_misses": st1["cache_misses"] - st0["cache_misses"],
        "peak_in_flight": st1["peak_in_flight"],
        "peak_reserved_gb": round(st1["peak_reserved"] / 2 ** 30, 2),
        "budget_gb": round(st1["budget"] / 2 ** 30, 2),
        "mlmc_client": mres,
        "by_size": classes,
        "slice_vertices": args.serve_slice_vertices or 2 ** 24,
    })
    return out


def sharded_step_sums(run_levels, levels, step, rank, world, device=None):
    """One step of the multi-GPU path: this rank runs its contiguous block of
    every level's samples (workloads.shard_first_sample: the blocks of all
    (step, rank) pairs tile the sample indices, so any partition draws the
    samples of a single-rank run) and the per-level sums (N, sum Y, sum Y^2,
    sum Q_f, sum Q_f^2) are all-reduced -- the estimator's one exchange.

    run_levels(tasks) takes [(level, first_sample, count)] and returns one
    5-tuple of sums per task.  device: where the all-reduce runs (the GPU
    under NCCL, None = CPU under gloo).  Returns a (levels, 5) float64 tensor
    on the CPU."""
    import torch
    tasks = [(l, workloads.shard_first_sample(step, rank, world, N), N) for (l, n, N) in levels]
    sums = torch.tensor([list(r) for r in run_levels(tasks)], dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist
        t = sums.to(device) if device is not None else sums
        dist.all_reduce(t)
        sums = t.cpu()
    return sums


def max_over_ranks(value, world, device=None):
    """The largest of every rank's `value` (all ranks must call it)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu_pool = None
    wl = workloads.OSCILLATORY
    if args.scale != 1.0:
        wl = workloads.MLMCWorkload(**{**wl.__dict__, "N": [max(1, int(N * args.scale)) for N in wl.N]})
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    if want_cpu:   # spawn the oracle pool before the first GPU call
        cpu_pool, cpu_cores = oracle_pool(wl)

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2306_13493_gb300 import build, sce
    build.build_library()
    sce.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    prec = args.precision
    L = len(wl.N) - 1

    embs = []
    for (l, n, N) in wl.levels:
        P = 4 * n if wl.pad_mode == 2 else None
        e0 = sce.ce_setup_embedding(wl.kind, wl.nu, wl.lam, wl.sigma2, n, pad_mode=wl.pad_mode)
        kf, kc = workloads.keep_counts(e0.P, l == L, wl.smoothing)
        e0.close()
        embs.append(sce.ce_setup_embedding(wl.kind, wl.nu, wl.lam, wl.sigma2, n,
                                           pad_mode=wl.pad_mode, keep_fine=kf, keep_coarse=kc))
    # FFT launch shapes per embedding size, tuned before anything is timed
    autotune = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        shapes = {}
        for (l, n, N) in wl.levels:
            shapes[str(embs[l].P)] = sce.ce_autotune_fft(embs[l], prec, count=min(N, 64), reps=3)
        # multigrid window heights of the tiled levels (n <= 64 runs fused), smallest
        # first; 1024 is a level of the mixed-level launch
        tiles = {}
        for nn in (128, 256, 512, 1024):
            cnt = max(4, min(256, (1 << 24) // ((nn + 1) * (nn + 1))))
            tiles[str(nn)] = sce.darcy_autotune_tiles(nn, prec, count=cnt, reps=2,
                                                      stream=stream.cuda_stream)
        autotune = {"fft_shapes_by_P": {P: {"row_tpf_F": v["row"], "col_tpf_F": v["col"]}
                                        for P, v in shapes.items()},
                    "tile_height_by_n": tiles,
                    "seconds": round(time.perf_counter() - t0, 2)}
    Ybuf = [torch.empty(N, dtype=torch.float64, device=dev) for (_, _, N) in wl.levels]
    Yhost = [torch.empty(N, dtype=torch.float64, pin_memory=True) for (_, _, N) in wl.levels]
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    sums_acc = np.zeros((len(wl.N), 5))
    iters_max = [0] * len(wl.N)
    iters_tot = [0] * len(wl.N)
    solves = [0] * len(wl.N)

    def step(i, copy_y=False, record=True, conc=None, precision=None):
        def run_levels(tl):
            tasks = [{"emb": embs[l], "level": l, "count": N, "Y": Ybuf[l],
                      "first_sample": first} for (l, first, N) in tl]
            outs, _, _ = sce.mlmc_estimate_levels(
                tasks, wl.seed, qoi_index=wl.qoi, f=wl.f, rtol=wl.rtol, maxit=2000,
                precision=prec if precision is None else precision,
                max_concurrency=args.concurrency if conc is None else conc,
                stream=stream.cuda_stream, allow_not_converged=True)
            for (l, n, N), out in zip(wl.levels, outs):
                iters_max[l] = max(iters_max[l], out.max_iters)
                if record:
                    iters_tot[l] += out.total_iters
                    solves[l] += N * (2 if l > 0 else 1)
                if copy_y:
                    Yhost[l].copy_(Ybuf[l], non_blocking=True)
            return [(o.N, o.sumY, o.sumY2, o.sumQf, o.sumQf2) for o in outs]

        sums = sharded_step_sums(run_levels, wl.levels, i, rank, world, dev)
        if copy_y:
            stream.synchronize()
        if record:
            sums_acc[:] += sums.numpy()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    for w in range(args.warmup):
        step(10_000 + w, record=False)

    # device-timed steps (inputs resident; L2 flushed before each step)
    clocks = ClockSampler(local if "CUDA_VISIBLE_DEVICES" not in os.environ
                          else os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local])
    clocks.start()
    total_ms = 0.0
    for i in range(args.steps):
        flush.zero_()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(i)
        e1.record(stream)
        barrier()
        total_ms += e0.elapsed_time(e1)
    clk = clocks.stop()
    total_ms = max_over_ranks(total_ms, world, dev)
    ms_per_step = total_ms / args.steps
    Ntot = sum(wl.N)
    value = world * Ntot / (ms_per_step / 1000.0)

    # end to end: public API from the host, per-sample Y read back to pinned host memory
    e2e_steps = max(1, args.steps // 2)
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        step(100 + i, copy_y=True, record=False)
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, dev)
    e2e = {"value": world * Ntot / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 8 * Ntot + 56 * len(wl.N),
           "note": "inputs are the scalar sample ranges (normals are drawn on the device); "
                   "per-sample Y and the level sums are read back every step"}

    # roofline: one extra step with the launch profiler on, levels one after
    # another so that every launch's event pair times that launch alone
    barrier()
    sce.sce_profile_enable(1)
    step(200, record=False, conc=1)
    barrier()
    prof = sce.sce_profile_read()
    sce.sce_profile_enable(0)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    # the roofline of the HBM-bound family with the largest share of device time
    # (families bound by issue, barriers or launch latency have no HBM fraction)
    hbm_fams = [kv for kv in prof.items()
                if KERNEL_BOUND.get(kv[0], "hbm") == "hbm" and kv[1][2] > 0]
    top = max(hbm_fams, key=lambda kv: kv[1][0]) if hbm_fams else None
    top_all = max(prof.items(), key=lambda kv: kv[1][0])[0] if prof else None
    roof = None
    kernels = {}
    prof_total = sum(v[0] for v in prof.values()) if prof else 0.0
    mpk = measure_peaks(sce, stream)
    for name, (ms, by, nl) in sorted(prof.items(), key=lambda kv: -kv[1][0]):
        gbs = by / (ms * 1e6) if ms > 0 else None
        bound = KERNEL_BOUND.get(name, "hbm")
        frac = None
        if gbs is not None and bound == "hbm":
            frac = round(gbs / hbm, 4)
        elif gbs is not None and bound == "l2":
            frac = round(gbs / mpk["l2_read_gbs"], 4)
        elif gbs is not None and bound == "issue" and name in INSTR_PER_ALG:
            ipb, src, kname, digest = INSTR_PER_ALG[name]
            if kernel_source_digest(src, kname) == digest:
                frac = round(by * ipb / (ms * 1e-3) / mpk["fma_warp_inst_per_s"], 4)
        kernels[name] = {"ms": round(ms, 3), "launches": nl, "share": round(ms / prof_total, 4),
                         "GBps": round(gbs, 1) if gbs is not None else None, "bound": bound,
                         "frac": frac}
    if top:
        name, (ms, by, nl) = top
        ach = by / (ms * 1e6)
        traffic = None
        if name in TRAFFIC_PER_ALG:
            ratio, src, kname, digest = TRAFFIC_PER_ALG[name]
            if kernel_source_digest(src, kname) == digest:
                traffic = round(ratio * by / nl)   # bytes per launch
        roof = {"bound": "hbm", "kernel": name, "achieved": round(ach, 1), "peak": hbm,
                "unit": "GB/s", "frac": round(ach / hbm, 4), "traffic": traffic,
                "algorithmic_bytes_per_launch": round(by / nl),
                "peak_source": peak_src, "avg_launch_us": round(1000 * ms / nl, 2),
                "dominant_family_overall": top_all,
                "timed": "one extra step after the timed ones, levels one after another, "
                         "CUDA events around every launch on its stream"}

    # each level alone (one mlmc_level_estimate call of its N_l samples, CUDA
    # events, L2 flushed): its samples/s when it has the GPU to itself
    alone = []
    for (l, n, N) in wl.levels:
        ms = []
        for r in range(3):
            flush.zero_()
            barrier()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            sce.mlmc_level_estimate(embs[l], wl.seed, l, 70_000_000 + r * N, N, qoi_index=wl.qoi,
                                    f=wl.f, rtol=wl.rtol, maxit=2000, precision=prec,
                                    Y=Ybuf[l], stream=stream.cuda_stream,
                                    allow_not_converged=True)
            a1.record(stream)
            barrier()
            if r:
                ms.append(a0.elapsed_time(a1))
        alone.append(statistics.mean(ms))

    # the same sweep on the all-FP64 batched path (FP64 field, FP64 multigrid-CG)
    fp64_batched = None
    if not args.no_fp64_path and prec == 32:
        step(300, record=False, precision=64)
        ms = []
        for i in range(2):
            flush.zero_()
            barrier()
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            step(310 + i, record=False, precision=64)
            b1.record(stream)
            barrier()
            ms.append(b0.elapsed_time(b1))
        fms = statistics.mean(ms)
        fp64_batched = {"value": world * Ntot / (fms / 1000.0), "unit": UNIT,
                        "ms_per_step": round(fms, 3),
                        "fine_level_samples_per_s": round(world * wl.N[-1] / (fms / 1000.0), 1),
                        "dtype": "f64", "steps": 2,
                        "note": "the same sweep, all levels in flight, FP64 field and FP64 "
                                "multigrid-preconditioned CG; CUDA events, L2 flushed"}

    # level statistics of the timed steps
    per_level = []
    for (l, n, N) in wl.levels:
        Nn, s1, s2, q1, q2 = sums_acc[l]
        mean = s1 / Nn
        var = (s2 - Nn * mean * mean) / (Nn - 1)
        qm = q1 / Nn
        qv = (q2 - Nn * qm * qm) / (Nn - 1)
        per_level.append({"level": l, "n": n, "N": N, "mean_Y": mean, "var_Y": var,
                          "var_Qf": qv, "max_iters": iters_max[l],
                          "mean_iters": round(iters_tot[l] / max(1, solves[l]), 2),
                          "samples_per_s_in_sweep": round(world * N / (ms_per_step / 1000.0), 1),
                          "ms_alone": round(alone[l], 3),
                          "samples_per_s_alone": round(N / (alone[l] / 1000.0), 1)})

    # plain FP64 per-sample path (batch 1, FP64 field and solver), bounded sample
    fp64 = None
    if not args.no_fp64_path:
        per, ks = [], []
        for (l, n, N) in wl.levels:
            # at least 20 samples, or at least 2 s, per level
            barrier()
            t0 = time.perf_counter()
            k = 0
            while k < 20 and time.perf_counter() - t0 < 2.0:
                sce.mlmc_level_estimate(embs[l], wl.seed, l, 50_000_000 + k, 1, qoi_index=wl.qoi,
                                        f=wl.f, rtol=wl.rtol, maxit=2000, precision=64,
                                        stream=stream.cuda_stream, allow_not_converged=True)
                k += 1
            barrier()
            per.append((time.perf_counter() - t0) / k)
            ks.append(k)
        sec = sum(N * per[l] for (l, _, N) in wl.levels) / Ntot
        fp64 = {"value": 1.0 / sec, "unit": UNIT, "speedup": value / world * sec,
                "per_level_ms": [round(1000 * x, 3) for x in per],
                "sample": "batch-1 FP64 calls (host wall clock), " + "/".join(map(str, ks)) +
                " samples on levels 0..5 (20 per level, or as many as 2 s allow), "
                "scaled to the N_l mix"}

    # MLMC to a total RMSE of 1e-3 (§4.2-4.3): MLMC-CES from coarse meshes and plain
    # MLMC from its own coarsest mesh (Eq. (3.8)), levels added adaptively
    ttr = None
    if rank == 0 and world == 1 and not args.no_fp64_path:
        ttr = time_to_rmse_study(sce, stream, prec)

    plain_small = None
    cufft = None
    if rank == 0 and world == 1 and not args.no_mixed:
        plain_small = plain_small_bench(sce, stream, flush)
        cufft = cufft_comparison(sce, stream, flush)

    mixed = None
    if rank == 0 and world == 1 and not args.no_mixed:
        mixed = mixed_launch_bench(args, sce, stream)

    serving = None
    if rank == 0 and world == 1 and args.serve_seconds > 0:
        serving = serving_bench(args, sce)

    cpu = None
    if want_cpu:
        try:
            v, wall, mean = oracle_measure(cpu_pool, cpu_cores, wl, 0)
            cpu = {"value": v, "unit": UNIT, "cores": cpu_cores, "kind": "oracle",
                   "sample": cpu_sample_text(wl, cpu_cores), "wall_s": round(wall, 2)}
        finally:
            cpu_pool.close()
            cpu_pool.join()

    for e in embs:
        e.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE_MIXED if prec == 32 else "f64", "data": "synthetic",
            "config": {"workload": wl.describe(), "precision": prec,
                       "levels_in_flight": args.concurrency,
                       "l2": "flushed before every timed step (256 MB write)",
                       "parallelism": f"dp{world} (samples sharded, level sums all-reduced)"},
            "clocks": clk, "e2e": e2e,
            "gpu_launches": int(sum(v[2] for v in prof.values())) * args.steps,
            "gpu_launches_per_step": int(sum(v[2] for v in prof.values())),
            "sweeps_per_s": round(1000.0 / ms_per_step, 3),
            "fine_level": {"value": round(world * wl.N[-1] / (ms_per_step / 1000.0), 1),
                           "unit": "finest-level samples/s",
                           "n": wl.levels[-1][1],
                           "note": "the finest level's N_L samples (n = %d fine, %d coarse) per "
                                   "second of the full sweep; alone on the GPU: %.1f samples/s"
                                   % (wl.levels[-1][1], wl.levels[-1][1] // 2,
                                      per_level[-1]["samples_per_s_alone"])},
            "fp64_batched": fp64_batched,
            "roofline": roof, "kernels": kernels, "per_level": per_level,
            "measured_peaks": {k: (round(v, 4) if isinstance(v, float) else v)
                               for k, v in mpk.items()},
            "autotune": autotune,
            "fp64_per_sample_path": fp64, "time_to_rmse": ttr, "mixed_launch": mixed,
            "plain_small": plain_small, "cufft_comparison": cufft,
            "serving": serving,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.case:
        return run_case(args)
    if args.peaks:
        return run_peaks(args)
    if args.study == "precision":
        return precision_study(args)
    if args.study == "smoothing":
        return smoothing_study(args)
    if args.study == "qmc":
        return qmc_study(args)
    if args.study == "3d":
        return three_d_study(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
