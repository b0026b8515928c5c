"""Benchmark: Nystrom-PCG time-to-relres on the Laplace-mixture KRR workload.

One step = the whole hot path on one batch of resident synthetic inputs:
kop_create (centre + BF16 split), nys_build (sketch K Omega on the fused
operator, r x r FP64 core, U), pcg_solve to relative residual <= 5e-7 with
true-residual replacement (so that the FP64 relative residual is <= 1e-6).
Workload: n = 200000, d = 64, 20-cluster Gaussian mixture, Laplace kernel
sigma = 8, lam = 1e-6 n, Nystrom rank 500, one right-hand side.

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
# single-column product, keyed by (n, d); mean of two launches at full size
TRAFFIC_BYTES = {(200_000, 64): 74.46e6}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--n", type=int, default=200_000)
    p.add_argument("--rank", type=int, default=500)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--check-cache", action="store_true",
                   help="keep the kernel matrix of the checks in HBM (n^2 * 4 bytes); each solve recomputes it")
    return p.parse_args()


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


def _cpu_oracle_rate(wl, iters, rank_r, budget_s=15.0):
    """FP64 oracle (host C, all cores): matvec and sketch times extrapolated
    from a bounded sample of rows.  Returns (solve_seconds, sample text, cores)."""
    import numpy as np
    from oracle import cmatvec
    X = wl.X
    n = wl.n
    cores = cmatvec.max_threads()
    v = np.random.default_rng(1).standard_normal(n)
    rows = 64
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
    total = t_sk + iters * t_mv
    sample = (f"FP64 oracle K(X[:{rows2}],X)v and K(X[:{rows3}],X)Omega (r={rank_r}) on {cores} threads, "
              f"extrapolated to full n: sketch {t_sk:.1f}s + {iters} matvecs x {t_mv:.1f}s")
    return total, sample, cores


def run_reference(a):
    world, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2609_08136_b300 import workloads as W
    wl = W.krr_laplace_mix(seed=a.seed, n=a.n, rank=a.rank)
    iters = 62  # the native solve's iteration count on this workload (it reports its own)
    times = []
    sample = ""
    cores = 0
    for s in range(a.warmup + a.steps):
        t, sample, cores = _cpu_oracle_rate(wl, iters, a.rank, budget_s=8.0)
        if s >= a.warmup:
            times.append(t)
    t = statistics.mean(times)
    out = {"metric": METRIC, "value": 1.0 / t, "unit": "solves/s", "impl": "reference", "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "krr_laplace_mix n=200000 d=64 laplace sigma=8 lam=0.2 r=500 rhs=1",
                      "n": wl.n, "d": wl.d, "rank": a.rank, "extrapolated_iters": iters},
           "cpu_baseline": {"value": 1.0 / t, "unit": "solves/s", "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": 1.0 / t, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


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
    # each rank solves its own independent problems (weak scaling, no data-path
    # collective); timed step j solves the instance of seed a.seed + (j mod 3)
    n_inst = 3
    insts = []
    for j in range(n_inst):
        seed = replica_seed(a.seed, rank, j, n_inst)
        wl_j = W.krr_laplace_mix(seed=seed, n=a.n, rank=a.rank)
        Omh_j = torch.from_numpy(W.gaussian_sketch(wl_j.n, a.rank, seed=seed)).pin_memory()
        Xh_j = torch.from_numpy(wl_j.X).pin_memory()
        Bh_j = torch.from_numpy(wl_j.B).pin_memory()
        insts.append({"seed": seed, "wl": wl_j, "Xh": Xh_j, "Bh": Bh_j, "Omh": Omh_j, "X": Xh_j.to(dev),
                      "B": Bh_j.to(dev), "Om": Omh_j.to(dev)})
    wl, Xh, Bh, Omh = insts[0]["wl"], insts[0]["Xh"], insts[0]["Bh"], insts[0]["Omh"]
    lam = float(wl.lambdas[0])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()
    # device memory for the kernel matrix of the checks (n^2 * 4 bytes), held
    # across steps like any workspace; each solve recomputes its contents
    kbuf = None
    if a.check_cache:
        need = a.n * ((a.n + 127) // 128 * 128)
        if 4 * need + (8 << 30) <= torch.cuda.mem_get_info(dev)[0]:
            kbuf = torch.empty(need, dtype=torch.float32, device=dev)

    # refinement and acceptance both with the direct-difference operator: the
    # tensor-core accurate operator's own residual floor on this data (~1.2e-6)
    # is as large as the residuals it would replace
    def step(j, inner=ops.FAST, refine=ops.PLAIN, check=ops.PLAIN, build=ops.FAST, cache=True):
        ins = insts[j % n_inst]
        w = ins["wl"]
        op = ops.KernelOperator(ins["X"], w.kernel, w.bandwidth)
        if cache and kbuf is not None:
            op.set_check_cache(True, kbuf)
        ny = ops.Nystrom(op, ins["Om"], mode=build)
        res = ops.pcg_solve(op, ins["B"], [float(w.lambdas[0])], nys=ny, tol=TOL, maxit=500, refine_every=30,
                            inner_mode=inner, refine_mode=refine, check_mode=check)
        return op, ny, res

    for _ in range(a.warmup):
        op, ny, res = step(0)
        del ny, op
    times, iters_seen, launches, by_seed = [], [], [], {}
    clk = ClockSampler(local)
    clk.start()
    for j in range(a.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        l0 = _ffi.lib().kop_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        op, ny, res = step(j)
        e1.record(stream)
        torch.cuda.synchronize()
        launches.append(_ffi.lib().kop_launch_count() - l0)
        times.append(e0.elapsed_time(e1) / 1e3)
        iters_seen.append(res.iters[0])
        by_seed.setdefault(insts[j % n_inst]["seed"], []).append(times[-1])
        last = (op, ny, res, insts[j % n_inst]["wl"])
        del ny, op
    clocks = clk.stop()
    t_step = max_over_ranks(statistics.mean(times), dist, dev)
    op, ny, res, wl_last = last
    value = world / t_step
    seed_t = [statistics.mean(v) for v in by_seed.values()]
    # the same PCG on the plain FP32 CUDA-core path: direct-difference kernel
    # values and FP32 FMAs for every product (sketch, iterations, refinement)
    plain_path = None
    if not a.no_plain:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        opp, nyp, resp = step(0, inner=ops.PLAIN, refine=ops.PLAIN, check=ops.PLAIN, build=ops.PLAIN, cache=False)
        e1.record(stream)
        torch.cuda.synchronize()
        tp = e0.elapsed_time(e1) / 1e3
        plain_path = {"time_to_relres_s": tp, "pcg_iters": resp.iters[0], "converged": bool(resp.converged),
                      "fused_speedup": tp / statistics.mean(by_seed[insts[0]["seed"]])
                      if insts[0]["seed"] in by_seed else None}
        del nyp, opp

    # fused operator product alone (m = 1), timed on the launching stream
    V = torch.randn(wl.n, 1, device=dev)
    O = torch.empty_like(V)

    def time_mv(mode, reps):
        op.matvec(V, mode=mode, out=O)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            op.matvec(V, mode=mode, out=O)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    t_fast = time_mv(ops.FAST, 5)
    t_plain = None if a.no_plain else time_mv(ops.PLAIN, 1)
    n, d = wl.n, wl.d
    flops = 2.0 * n * n * (d + 1)  # distance GEMM + contraction per K v
    peaks, peak_src = _peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
    # SFU roofline of the m = 1 product, with the SFU rates measured live on
    # this GPU: a Laplace entry needs one sqrt and one ex2
    rates = ops.sfu_rates()
    peak_entries = 1.0 / (1.0 / rates["ex2"] + 1.0 / rates["sqrt"])
    achieved_entries = n * n / t_fast
    # DRAM bytes per launch of that kernel, from one ncu capture of this
    # workload (the ncu summary of this kernel); algorithmic bytes: X as
    # two BF16 splits, scaled norms, v and the output, each once
    traffic = TRAFFIC_BYTES.get((n, d))
    alg_bytes = n * d * 2 * 2 + 3 * n * 4
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x2-split/f32/f64", "data": "synthetic",
        "config": {"workload": "krr_laplace_mix n=200000 d=64 laplace sigma=8 lam=0.2 r=500 rhs=1",
                   "n": n, "d": d, "rank": a.rank, "tol": TOL, "l2": "flushed (256 MB write) before each step",
                   "parallelism": f"replicas x{world}",
                   "check_matrix": ("stored in HBM, recomputed by every solve" if kbuf is not None
                                    else "recomputed in every check product")},
        "time_to_relres_s": t_step,
        "time_to_relres_by_seed_s": {"seeds": sorted(by_seed), "median": statistics.median(seed_t),
                                     "min": min(seed_t), "max": max(seed_t)},
        "plain_path": plain_path,
        "pcg_iters": iters_seen,
        "true_relres_accurate_op": res.true_relres[0],
        "matvec_ms": {"fused_fast": t_fast * 1e3, "plain_fp32": None if t_plain is None else t_plain * 1e3},
        "matvec_tflops": {"fused_fast": flops / t_fast / 1e12,
                          "plain_fp32": None if t_plain is None else flops / t_plain / 1e12},
        "kernel_evals_per_s": achieved_entries,
        "roofline": {"bound": "alu", "achieved": achieved_entries / 1e12, "peak": peak_entries / 1e12,
                     "unit": "Tentries/s", "frac": achieved_entries / peak_entries, "traffic": traffic,
                     "traffic_unit": "bytes per launch (DRAM read + write, ncu)", "algorithmic_bytes": alg_bytes,
                     "kernel": "k1_fma_kernel<LAPLACE,2,1,128,4> (K v, m = 1)",
                     "peak_source": ("SFU rates measured live by kop_sfu_rates (ex2 %.2f, sqrt %.2f Tops/s); "
                                     "one Laplace entry = 1 sqrt + 1 ex2" % (rates["ex2"] / 1e12, rates["sqrt"] / 1e12))},
        "clocks": clocks,
        "gpu_launches": int(statistics.mean(launches)),
        "peaks_source": peak_src,
    }
    if not a.no_e2e:
        # end to end through the public API with host buffers: H2D of X, y, Omega
        # from pinned memory, the solve, D2H of x, all inside the timed region
        xh = torch.empty(n, dtype=torch.float64).pin_memory()
        ets = []
        for i in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Xd = Xh.to(dev, non_blocking=True)
            Bd = Bh.to(dev, non_blocking=True)
            Omd = Omh.to(dev, non_blocking=True)
            op2 = ops.KernelOperator(Xd, wl.kernel, wl.bandwidth)
            if kbuf is not None:
                op2.set_check_cache(True, kbuf)
            ny2 = ops.Nystrom(op2, Omd, mode=ops.FAST)
            r2 = ops.pcg_solve(op2, Bd, [lam], nys=ny2, tol=TOL, maxit=500, refine_every=30,
                               refine_mode=ops.PLAIN, check_mode=ops.PLAIN)
            xh.copy_(r2.x.reshape(-1), non_blocking=True)
            torch.cuda.synchronize()
            ets.append(time.perf_counter() - t0)
            del ny2, op2
        te = min(ets)
        hb = Xh.numel() * 4 + Bh.numel() * 4 + Omh.numel() * 4
        out["e2e"] = {"value": world / te, "unit": "solves/s", "h2d_bytes_per_step": hb, "d2h_bytes_per_step": n * 8}
    # FP64 check of the returned x on sampled rows (host oracle, outside the timed region)
    try:
        from oracle import cmatvec
        xs = res.x.reshape(-1).cpu().numpy()
        wv = wl_last
        rows = np.random.default_rng(7).choice(wv.n, size=min(256, wv.n), replace=False)
        kx = cmatvec.kernel_matvec(wv.kernel, wv.X, xs, wv.bandwidth, Z=wv.X[rows])
        bvec = wv.B[:, 0].astype(np.float64)
        r_s = bvec[rows] - kx - float(wv.lambdas[0]) * xs[rows]
        out["fp64_relres_sampled"] = float(np.sqrt(wv.n / len(rows)) * np.linalg.norm(r_s) / np.linalg.norm(bvec))
    except Exception as e:  # the check is informational
        out["fp64_relres_sampled"] = f"unavailable: {e}"
    if rank == 0 and not a.no_cpu_baseline:
        total, sample, cores = _cpu_oracle_rate(wl, int(statistics.mean(iters_seen)), a.rank)
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
