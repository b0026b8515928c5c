"""Benchmark: Nystrom-PCG time-to-relres on kernel-ridge-regression workloads.

One step = the whole hot path on one batch of resident synthetic inputs:
kop_create (centre + BF16 split), nys_build (sketch K Omega on the fused
operator, r x r FP64 core, U), pcg_solve until the float64 relative residual
is certified <= 1e-6 (the solver's checks are corrected by an exact FP64
residual of sampled rows).  The hyper-parameter workload adds the validation
loss and its gradient (pcg_adjoint_val) to the step.

Workloads (--workload; default krr_laplace_mix):
  krr_laplace_mix   n = 200000, d = 64, 20-cluster Gaussian mixture, Laplace
                    sigma = 8, lam = 1e-6 n, rank 500, one right-hand side
  krr_rbf_small     n = 4096, d = 16, RBF sigma = 4, lam = 1e-4 n, rank 100
  krr_matern_large  n = 1e6, d = 32, z-scored uniform, Matern-5/2 l = 1
                    (--lengthscale for the sqrt(d) variant), lam = 1e-7 n,
                    rank 1000, refinement every 20 iterations
  krr_rbf_hyper     train n = 1e5, val n = 2e4, d = 32, RBF sigma = sqrt(d),
                    lam = 1e-4 n, rank 500: solve + validation-loss gradient

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on a bounded sample of the same workload instead.
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
sys.path.insert(0, ROOT)

METRIC = "PCG time-to-relres 1e-6 & fused kernel-matvec TFLOP/s vs plain FP32 path"
TOL = 1e-6
# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of the FAST
# single-vector product, keyed by (kernel, n, d); mean of two launches at
# full size, taken on the kernel as it stands
TRAFFIC_BYTES = {(1, 200_000, 64): 94.67e6 + 570.85e6}

# name: (generator kwargs, description, refine_every, maxit)
WORKLOADS = {
    "krr_laplace_mix": ("krr_laplace_mix n=200000 d=64 laplace sigma=8 lam=0.2 r=500 rhs=1", 30, 500),
    "krr_rbf_small": ("krr_rbf_small n=4096 d=16 rbf sigma=4 lam=0.4096 r=100 rhs=1", 30, 500),
    "krr_matern_large": ("krr_matern_large n=1000000 d=32 matern52 l={l} lam=0.1 r=1000 rhs=1", 20, 500),
    "krr_rbf_hyper": ("krr_rbf_hyper n=100000 nval=20000 d=32 rbf sigma=sqrt(32) lam=10 r=500: solve + "
                      "validation-loss gradient", 30, 500),
}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--workload", default="krr_laplace_mix", choices=sorted(WORKLOADS))
    p.add_argument("--lengthscale", type=float, default=1.0, help="krr_matern_large: Matern lengthscale")
    p.add_argument("--n", type=int, default=None, help="override the workload's n (parity / probing only)")
    p.add_argument("--rank", type=int, default=None)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--plain", action="store_true", help="time the plain FP32 path on workloads other than the default")
    p.add_argument("--no-fp64-check", action="store_true")
    p.add_argument("--no-check-cache", action="store_true",
                   help="recompute the checks' kernel matrix instead of keeping it in HBM (n^2 * 4 bytes)")
    return p.parse_args()


def _workload(a, seed):
    from paper_2609_08136_b300 import workloads as W
    kw = {}
    if a.n is not None:
        kw["n"] = a.n
    if a.rank is not None:
        kw["rank"] = a.rank
    if a.workload == "krr_laplace_mix":
        return W.krr_laplace_mix(seed=seed, **kw)
    if a.workload == "krr_rbf_small":
        wl = W.krr_rbf_small(seed=seed, **{k: v for k, v in kw.items() if k == "n"})
        if a.rank is not None:
            wl.rank = a.rank
        return wl
    if a.workload == "krr_matern_large":
        return W.krr_matern_large(seed=seed, lengthscale=a.lengthscale, **kw)
    return W.krr_rbf_hyper(seed=seed, **kw)


def _describe(a):
    d = WORKLOADS[a.workload][0].format(l=a.lengthscale)
    if a.n is not None or a.rank is not None:
        d += f" (override n={a.n} rank={a.rank})"
    return d


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_seed(seed: int, rank: int, instance: int = 0, n_instances: int = 1) -> int:
    """Each rank solves its own independent problems (weak scaling replicas):
    rank r's instance j has seed seed + j + n_instances * r."""
    return seed + instance + n_instances * rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The job's step time is the slowest rank's (no data-path collective:
    this reduction of one scalar is the only communication)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _cpu_oracle_rate(wl, iters, rank_r, budget_s=15.0, extra_matvecs=0.0):
    """FP64 oracle (host C, all cores): matvec and sketch times extrapolated
    from a bounded sample of rows.  Returns (solve_seconds, sample text, cores)."""
    import numpy as np
    from oracle import cmatvec
    X = wl.X
    n = wl.n
    cores = cmatvec.max_threads()
    v = np.random.default_rng(1).standard_normal(n)
    rows = min(n, 64)
    t0 = time.perf_counter()
    cmatvec.kernel_matvec(wl.kernel, X, v, wl.bandwidth, Z=X[:rows])
    t_rows = time.perf_counter() - t0
    # scale the row sample to the time budget
    rows2 = int(max(rows, min(n, rows * (budget_s * 0.5) / max(t_rows, 1e-3))))
    t0 = time.perf_counter()
    cmatvec.kernel_matvec(wl.kernel, X, v, wl.bandwidth, Z=X[:rows2])
    t_mv = (time.perf_counter() - t0) * n / rows2
    om = np.random.default_rng(2).standard_normal((n, rank_r)) / np.sqrt(n)
    rows3 = max(8, rows2 // 16)
    t0 = time.perf_counter()
    cmatvec.kernel_matvec(wl.kernel, X, om, wl.bandwidth, Z=X[:rows3])
    t_sk = (time.perf_counter() - t0) * n / rows3
    total = t_sk + (iters + extra_matvecs) * t_mv
    extra = f" + {extra_matvecs:.1f} matvec-equivalents of validation products" if extra_matvecs else ""
    sample = (f"FP64 oracle K(X[:{rows2}],X)v and K(X[:{rows3}],X)Omega (r={rank_r}) on {cores} threads, "
              f"extrapolated to full n: sketch {t_sk:.1f}s + {iters} matvecs x {t_mv:.1f}s{extra}")
    return total, sample, cores


# iterations of the native solve on each workload (seed 0; the native arm
# reports its own), used to extrapolate the oracle arm
NATIVE_ITERS = {"krr_laplace_mix": 60, "krr_rbf_small": 45, "krr_matern_large": 3, "krr_rbf_hyper": 80}


def _extra_matvecs(wl):
    # the validation loss gradient: K(Xv, X) x, K(X, Xv) e, dK(Xv, X)/dbw x and
    # the train derivative product, in units of one n x n product
    if wl.Xval is None:
        return 0.0
    return 3.0 * wl.Xval.shape[0] / wl.n + 1.0


def run_reference(a):
    world, rank, _ = _dist()
    if rank != 0:
        return
    wl = _workload(a, a.seed)
    iters = NATIVE_ITERS[a.workload] * (2 if wl.Xval is not None else 1)
    times = []
    sample = ""
    cores = 0
    for s in range(a.warmup + a.steps):
        t, sample, cores = _cpu_oracle_rate(wl, iters, wl.rank, budget_s=8.0, extra_matvecs=_extra_matvecs(wl))
        if s >= a.warmup:
            times.append(t)
    t = statistics.mean(times)
    out = {"metric": METRIC, "value": 1.0 / t, "unit": "solves/s", "impl": "reference", "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": _describe(a), "n": wl.n, "d": wl.d, "rank": wl.rank, "extrapolated_iters": iters},
           "cpu_baseline": {"value": 1.0 / t, "unit": "solves/s", "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": 1.0 / t, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def _fp64_relres(wl, x, full_limit=200_000, rows=4096):
    """The oracle's FP64 relative residual of x (host cores): every row when
    n <= full_limit, else a random sample of rows scaled to n."""
    import numpy as np
    from oracle import cmatvec
    b = wl.B[:, 0].astype(np.float64)
    lam = float(wl.lambdas[0])
    if wl.n <= full_limit:
        kx = cmatvec.kernel_matvec(wl.kernel, wl.X, x, wl.bandwidth)
        return float(np.linalg.norm(b - kx - lam * x) / np.linalg.norm(b)), "all rows"
    idx = np.sort(np.random.default_rng(7).choice(wl.n, size=rows, replace=False))
    kx = cmatvec.kernel_matvec(wl.kernel, wl.X, x, wl.bandwidth, Z=wl.X[idx])
    r = b[idx] - kx - lam * x[idx]
    return float(np.sqrt(wl.n / rows) * np.linalg.norm(r) / np.linalg.norm(b)), f"{rows} random rows"


def run_native(a):
    import numpy as np
    import torch
    from paper_2609_08136_b300 import _ffi
    from paper_2609_08136_b300 import ops
    from paper_2609_08136_b300 import workloads as W

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    desc, refine_every, maxit = _describe(a), WORKLOADS[a.workload][1], WORKLOADS[a.workload][2]
    hyper = a.workload == "krr_rbf_hyper"
    # each rank solves its own independent problems (weak scaling, no data-path
    # collective); timed step j solves the instance of seed a.seed + (j mod 3)
    n_inst = 3
    insts = []
    for j in range(n_inst):
        seed = replica_seed(a.seed, rank, j, n_inst)
        wl_j = _workload(a, seed)
        host = {"X": torch.from_numpy(wl_j.X).pin_memory(), "B": torch.from_numpy(wl_j.B).pin_memory(),
                "Om": torch.from_numpy(W.gaussian_sketch(wl_j.n, wl_j.rank, seed=seed)).pin_memory()}
        if hyper:
            host["Xv"] = torch.from_numpy(wl_j.Xval).pin_memory()
            host["yv"] = torch.from_numpy(wl_j.yval).pin_memory()
        insts.append({"seed": seed, "wl": wl_j, "host": host, "dev": {k: v.to(dev) for k, v in host.items()}})
    wl = insts[0]["wl"]
    n, d, r_rank = wl.n, wl.d, wl.rank
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()
    # device memory for the kernel matrix of the checks (n^2 * 4 bytes), held
    # across steps like any workspace; each solve recomputes its contents
    kbuf = None
    if not a.no_check_cache:
        need = n * ((n + 127) // 128 * 128)
        if 4 * need + (16 << 30) <= torch.cuda.mem_get_info(dev)[0]:
            kbuf = torch.empty(need, dtype=torch.float32, device=dev)

    # refinement and acceptance with the direct-difference operator (the
    # tensor-core accurate operator's own residual floor on clustered data is
    # as large as the residuals it would replace); stops certified in FP64
    def step(tensors, w, inner=ops.FAST, refine=ops.PLAIN, check=ops.PLAIN, build=ops.FAST, cache=True):
        op = ops.KernelOperator(tensors["X"], w.kernel, w.bandwidth)
        if cache and kbuf is not None:
            op.set_check_cache(True, kbuf)
        ny = ops.Nystrom(op, tensors["Om"], mode=build)
        kw = dict(tol=TOL, maxit=maxit, refine_every=refine_every, inner_mode=inner, refine_mode=refine,
                  check_mode=check)
        res = ops.pcg_solve(op, tensors["B"], [float(w.lambdas[0])], nys=ny, **kw)
        if hyper:
            h = ops.pcg_adjoint_val(op, res.x, tensors["Xv"], tensors["yv"], float(w.lambdas[0]), nys=ny, **kw)
            return op, ny, res, h[:3]
        return op, ny, res, None

    for _ in range(a.warmup):
        op, ny, res, _h = step(insts[0]["dev"], insts[0]["wl"])
        del ny, op
    # SFU rates for the roofline, measured before and after the timed region
    # (the larger of the two counts)
    rates0 = ops.sfu_rates()
    times, iters_seen, launches, by_seed, certified = [], [], [], {}, []
    clk = ClockSampler(local)
    clk.start()
    for j in range(a.steps):
        ins = insts[j % n_inst]
        flush.fill_(1.0)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        l0 = _ffi.lib().kop_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        op, ny, res, hres = step(ins["dev"], ins["wl"])
        e1.record(stream)
        torch.cuda.synchronize()
        launches.append(_ffi.lib().kop_launch_count() - l0)
        times.append(e0.elapsed_time(e1) / 1e3)
        iters_seen.append(res.iters[0])
        certified.append(res.true_relres[0])
        by_seed.setdefault(ins["seed"], []).append(times[-1])
        last = (op, ny, res, hres, ins["wl"])
        del ny, op
    clocks = clk.stop()
    t_step = max_over_ranks(statistics.mean(times), dist, dev)
    op, ny, res, hres, wl_last = last
    value = world / t_step
    seed_t = [statistics.mean(v) for v in by_seed.values()]
    # the same PCG on the plain FP32 CUDA-core path: direct-difference kernel
    # values and FP32 FMAs for every product (sketch, iterations, refinement)
    plain_path = None
    if (a.workload == "krr_laplace_mix" and not a.no_plain) or a.plain:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        opp, nyp, resp, _h = step(insts[0]["dev"], insts[0]["wl"], inner=ops.PLAIN, refine=ops.PLAIN,
                                  check=ops.PLAIN, build=ops.PLAIN, cache=False)
        e1.record(stream)
        torch.cuda.synchronize()
        tp = e0.elapsed_time(e1) / 1e3
        plain_path = {"time_to_relres_s": tp, "pcg_iters": resp.iters[0], "converged": bool(resp.converged),
                      "fused_speedup": tp / statistics.mean(by_seed[insts[0]["seed"]])
                      if insts[0]["seed"] in by_seed else None}
        del nyp, opp

    # fused operator products alone, timed on the launching stream: the PCG
    # product (m = 1), the block product with m = r columns in the form the
    # solver's block products take (accumulator restarted every 4 tiles,
    # 128-column chunks), and the whole Nystrom build (whose sketch uses
    # 256-column chunks)
    V = torch.randn(n, 1, device=dev)
    O = torch.empty_like(V)
    Om0 = insts[0]["dev"]["Om"]
    Osk = torch.empty_like(Om0)

    def time_mv(mode, reps, Vin=V, Oout=O):
        op.matvec(Vin, mode=mode, out=Oout)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            op.matvec(Vin, mode=mode, out=Oout)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    t_fast = time_mv(ops.FAST, 5)
    t_plain = None if plain_path is None else time_mv(ops.PLAIN, 1)
    t_sketch = time_mv(ops.FAST, 2, Om0, Osk)
    del Osk
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t_build = []
    for _ in range(2):
        torch.cuda.synchronize()
        e0.record(stream)
        nyb = ops.Nystrom(op, Om0, mode=ops.FAST, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t_build.append(e0.elapsed_time(e1) / 1e3)
        del nyb
    flops = 2.0 * n * n * (d + 1)  # distance GEMM + contraction per K v
    flops_sketch = 2.0 * n * n * (d + r_rank)
    peaks, peak_src = _peaks()
    # SFU roofline of the m = 1 product, with the SFU rates measured live on
    # this GPU by the library's probe (MEASURED_PEAKS.json has no SFU figure):
    # an RBF entry needs one ex2; Laplace and Matern one sqrt and one ex2
    rates1 = ops.sfu_rates()
    rates = {k: max(rates0[k], rates1[k]) for k in rates0}
    if wl.kernel == W.RBF:
        peak_entries, per_entry = rates["ex2"], "1 ex2"
    else:
        peak_entries, per_entry = 1.0 / (1.0 / rates["ex2"] + 1.0 / rates["rsqrt"]), "1 rsqrt + 1 ex2"
    # the single-vector product evaluates each pair of 128-point blocks once:
    # nb (nb + 1) / 2 tiles of 128 x 128 entries (nb = ceil(n / 128)), and
    # represents all n^2 entries of K
    nb = (n + 127) // 128
    evaluated = (nb // 2 + 1) * nb * 128 * 128 if nb % 2 else (nb * nb // 2 + nb // 2) * 128 * 128
    achieved_entries = evaluated / t_fast
    # DRAM bytes per launch of that kernel, from one ncu capture of this
    # workload (the ncu summary of this kernel); algorithmic bytes: X as two
    # BF16 splits, scaled norms, v and the output, each once
    traffic = TRAFFIC_BYTES.get((wl.kernel, n, d))
    dp = 16 if d <= 16 else (32 if d <= 32 else (64 if d <= 64 else 128))
    # X as two BF16 splits, scaled norms, v, the output, and the column parts
    # written once (nb x floor(nb / 2) x 128 FP32)
    alg_bytes = n * dp * 2 * 2 + 3 * n * 4 + nb * (nb // 2) * 128 * 4
    knames = {W.RBF: "RBF", W.LAPLACE: "LAPLACE", W.MATERN52: "MATERN"}
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x2-split/f32/f64", "data": "synthetic",
        "config": {"workload": desc, "n": n, "d": d, "rank": r_rank, "tol": TOL,
                   "acceptance": "float64 relative residual, certified by the solver (FP64 residual of sampled "
                                 "rows corrects its FP32 check)",
                   "l2": "flushed (256 MB write) before each step", "parallelism": f"replicas x{world}",
                   "check_matrix": ("stored in HBM, recomputed by every solve" if kbuf is not None
                                    else "recomputed in every check product")},
        "time_to_relres_s": t_step,
        "time_to_relres_by_seed_s": {"seeds": sorted(by_seed), "median": statistics.median(seed_t),
                                     "min": min(seed_t), "max": max(seed_t)},
        "plain_path": plain_path,
        "pcg_iters": iters_seen,
        "certified_fp64_relres": certified,
        "matvec_ms": {"fused_fast_m1": t_fast * 1e3, "plain_fp32_m1": None if t_plain is None else t_plain * 1e3,
                      "block_fast_m%d" % r_rank: t_sketch * 1e3},
        "nys_build_ms": min(t_build) * 1e3,
        "matvec_tflops": {"fused_fast_m1": flops / t_fast / 1e12,
                          "plain_fp32_m1": None if t_plain is None else flops / t_plain / 1e12,
                          "block_fast_m%d" % r_rank: flops_sketch / t_sketch / 1e12,
                          "block_frac_of_bf16_burst": flops_sketch / t_sketch / 1e12 / peaks["bf16_tflops"]},
        "kernel_evals_per_s": achieved_entries,
        "kernel_entries_represented_per_s": n * n / t_fast,
        "roofline": {"bound": "alu", "achieved": achieved_entries / 1e12, "peak": peak_entries / 1e12,
                     "unit": "Tentries/s", "frac": achieved_entries / peak_entries, "traffic": traffic,
                     "traffic_unit": "bytes per launch (DRAM read + write, ncu)", "algorithmic_bytes": alg_bytes,
                     "kernel": "k1_sym_kernel<%s> (K v, m = 1, each block pair once)" % knames[wl.kernel],
                     "entries": "evaluated (%d of the n^2 = %d represented)" % (evaluated, n * n),
                     "peak_source": ("SFU rates measured live by the library's own probe kop_sfu_rates (ex2 %.2f, "
                                     "rsqrt %.2f Tops/s); one entry = %s" % (rates["ex2"] / 1e12,
                                                                            rates["rsqrt"] / 1e12, per_entry))},
        "clocks": clocks,
        "gpu_launches": int(statistics.mean(launches)),
        "peaks_source": peak_src,
    }
    if hres is not None:
        out["hypergradient"] = {"loss": hres[0], "dL_dsigma": hres[1], "dL_dlam": hres[2]}
    if not a.no_e2e:
        # end to end through the public API with host buffers: H2D of the inputs
        # from pinned memory, the solve, D2H of x (and of the gradient scalars),
        # inside the timed region; one run per seed, averaged like `value`
        ets, hb = [], 0
        for ins in insts:
            w = ins["wl"]
            xh = torch.empty(n, dtype=torch.float64).pin_memory()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tens = {k: v.to(dev, non_blocking=True) for k, v in ins["host"].items()}
            op2, ny2, r2, _h = step(tens, w)
            xh.copy_(r2.x.reshape(-1), non_blocking=True)
            torch.cuda.synchronize()
            ets.append(time.perf_counter() - t0)
            hb = sum(v.numel() * v.element_size() for v in ins["host"].values())
            del ny2, op2, tens
        te = statistics.mean(ets)
        out["e2e"] = {"value": world / te, "unit": "solves/s", "h2d_bytes_per_step": hb, "d2h_bytes_per_step": n * 8,
                      "estimator": "mean over seeds 0-2, one run each"}
    if not a.no_fp64_check:
        # the oracle's FP64 residual of the last timed solve (host cores,
        # outside the timed region)
        try:
            t0 = time.perf_counter()
            rr, how = _fp64_relres(wl_last, res.x.reshape(-1).cpu().numpy())
            out["fp64_relres_oracle"] = {"value": rr, "rows": how, "certified_by_solver": res.true_relres[0],
                                         "seconds": time.perf_counter() - t0}
        except Exception as e:  # the check is informational
            out["fp64_relres_oracle"] = f"unavailable: {e}"
    if rank == 0 and not a.no_cpu_baseline:
        it_cpu = int(statistics.mean(iters_seen)) * (2 if hyper else 1)
        total, sample, cores = _cpu_oracle_rate(wl, it_cpu, r_rank, extra_matvecs=_extra_matvecs(wl))
        out["cpu_baseline"] = {"value": 1.0 / total, "unit": "solves/s", "cores": cores, "kind": "oracle",
                               "sample": sample}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)
