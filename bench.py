"""Benchmark: approximate Gaussian samples per second on GB300.

One step = one pass of the sampling hot path over the configured workload:
2^28 Philox4x32-10 uniforms turned into piecewise-linear approximate Gaussian
variates (15 dyadic intervals + the zero row, FP32 output, 1 GiB written --
larger than the 129 MB L2, so no flush is needed between steps).

Printed (one JSON line on rank 0): the headline Gsamples/s, the roofline of
the sampler kernel against the measured HBM bandwidth, the same metric end to
end through the host-delivery ABI call, the exact-Phi^{-1} and other variants
on the same GPU, SM clocks sampled during the timed region, and the CPU
oracle timed on the host as a reported baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SAMPLES = 1 << 28
METRIC = "approx Gaussian Gsamples/s (piecewise linear, Philox uniforms, FP32 out)"
UNIT = "Gsamples/s"
WORKLOAD = {"workload": "piecewise-linear Phi^-1, 16-entry dyadic table, 2^28 Philox4x32-10 "
                        "uniforms -> FP32 (1 GiB out)",
            "n_samples": N_SAMPLES, "table": "K=15 dyadic intervals + zero row",
            "uniforms": "Philox4x32-10 seed 0, in registers", "l2": "output 1 GiB > L2 (129 MB): no flush"}
KERNEL_SOURCES = ["paper_2012_09715_gb300/csrc/sample.cu", "paper_2012_09715_gb300/csrc/device_common.cuh",
                  "paper_2012_09715_gb300/csrc/phiinv_coefs.h"]
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "ncu_sample_pwl_f32_2p28.md")


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def _kernel_sha() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    m_sha = re.search(r"source_sha:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_tr or m_sha.group(1) != _kernel_sha():
        return None
    return float(m_tr.group(1))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        if not getattr(self, "lines", None):
            return {"error": "nvidia-smi unavailable"}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"error": "no samples"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _time_device(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(steps):
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    return t0.elapsed_time(t1), per


def cpu_baseline(budget_s: float = 12.0, chunk: int = 1 << 20):
    """The oracle (plain C, single thread) on a bounded sample of the workload:
    Philox uniforms for consecutive sample indices + the piecewise-linear map."""
    import numpy as np
    import oracle
    a, b = oracle.pwl_table(15, 0.5)
    a32, b32 = a.astype(np.float32), b.astype(np.float32)
    done, t = 0, 0.0
    while t < budget_s and done < N_SAMPLES:
        t0 = time.perf_counter()
        u = oracle.uniforms(0, done, chunk)
        oracle.sample_pwl(a32, b32, u)
        t += time.perf_counter() - t0
        done += chunk
    return {"value": done / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {done} of the 2^28 samples (Philox + piecewise-linear map, FP64 "
                      f"arithmetic), single thread, {t:.1f} s"}


def mlmc_time_to_rmse(P, tl, dev, eps: float = 1e-4):
    """GBM European call (S0 = K = 1, r = 0.05, sigma = 0.2, T = 1), Euler-Maruyama:
    wall time to RMSE eps of nested MLMC (PWL + exact correction), regular MLMC
    (exact variates) and plain Monte Carlo with exact variates at the finest
    level the nested run chose -- all on this GPU, through aicdf_mlmc_run."""
    import torch
    ws = torch.empty(P.mlmc_run_workspace_bytes(), dtype=torch.uint8, device=dev)
    prm = P.sde_params()
    P.mlmc_run(prm, tl, 1e-3, ws, estimator=P.EST_NESTED, seed=99)   # warm-up
    res = {}
    nested = P.mlmc_run(prm, tl, eps, ws, estimator=P.EST_NESTED, seed=1)
    regular = P.mlmc_run(prm, tl, eps, ws, estimator=P.EST_REGULAR, seed=2)
    L = nested.L
    plain = P.mlmc_run(prm, tl, eps, ws, estimator=P.EST_PLAIN, fixed_L=L, seed=3)
    for name, r in (("nested", nested), ("regular", regular), ("plain_exact", plain)):
        res[name] = {"estimate": r.estimate, "rmse_est": (r.variance + r.bias ** 2) ** 0.5,
                     "L": r.L, "wall_ms": r.wall_ms, "gpu_ms": r.gpu_ms, "launches": r.launches,
                     "converged": bool(r.converged)}
    res["eps"] = eps
    res["speedup_vs_plain_exact_wall"] = plain.wall_ms / nested.wall_ms
    res["speedup_vs_regular_mlmc_wall"] = regular.wall_ms / nested.wall_ms
    res["speedup_vs_plain_exact_gpu"] = plain.gpu_ms / nested.gpu_ms
    res["speedup_vs_regular_mlmc_gpu"] = regular.gpu_ms / nested.gpu_ms
    return res


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    import numpy as np
    a, b = oracle.pwl_table(15, 0.5)
    a32, b32 = a.astype(np.float32), b.astype(np.float32)
    chunk = 1 << 20   # bounded sample per step

    def step(i):
        u = oracle.uniforms(0, i * chunk, chunk)
        oracle.sample_pwl(a32, b32, u)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    dt = time.perf_counter() - t0
    val = args.steps * chunk / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, reference_sample_per_step=chunk),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{chunk} samples per step (of the 2^28 workload), single thread"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--n-log2", type=int, default=28, help="workload size (profiling runs only)")
    args = ap.parse_args()
    global N_SAMPLES
    N_SAMPLES = 1 << args.n_log2
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    rank, world, local = _env_rank()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2012_09715_gb300 as P
    from paper_2012_09715_gb300 import build as B
    B.build()
    P.lib()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    tl = P.table_build(P.PWL, 15)
    out = torch.empty(N_SAMPLES, dtype=torch.float32, device=dev)
    seed = rank  # replicas draw disjoint streams

    def step():
        P.sample(tl, P.PWL, out, seed=seed, stream=stream)

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        total_ms, per = _time_device(step, args.steps, args.warmup, stream)
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms = total_ms / args.steps
    value = world * N_SAMPLES * args.steps / (total_ms / 1e3) / 1e9
    kernel_ms = statistics.mean(per)
    bytes_per_launch = 4.0 * N_SAMPLES
    peak, peak_kind = _peaks()
    achieved = bytes_per_launch / (kernel_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": _profile_traffic(), "peak_source": peak_kind,
            "kernel": "k_sample_vec<PWL,F32,PHILOX>", "algorithmic_bytes_per_launch": bytes_per_launch}

    extras = {}
    e2e = None
    if not args.no_extras:
        # same metric end to end: the ABI call that delivers samples to pinned host memory
        host = torch.empty(N_SAMPLES, dtype=torch.float32).pin_memory()
        staging = torch.empty(64 << 20, dtype=torch.uint8, device=dev)
        for _ in range(2):
            P.sample_to_host(tl, P.PWL, host, staging, seed=seed)
        t0 = time.perf_counter()
        e2e_steps = max(2, min(args.steps, 5))
        for _ in range(e2e_steps):
            P.sample_to_host(tl, P.PWL, host, staging, seed=seed)
        dt = time.perf_counter() - t0
        e2e = {"value": world * N_SAMPLES * e2e_steps / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": 4 * N_SAMPLES, "steps": e2e_steps,
               "call": "aicdf_sample_to_host (pinned host buffer, 64 MiB device staging)"}
        del host, staging
        # other methods / dtypes on the same GPU, same workload size
        out16 = torch.empty(N_SAMPLES, dtype=torch.float16, device=dev)
        tc = P.table_build(P.PWC, 1024)
        variants = {
            "pwl_f16": lambda: P.sample(tl, P.PWL, out16, seed=seed, stream=stream),
            "pwc_f32": lambda: P.sample(tc, P.PWC, out, seed=seed, stream=stream),
            "exact_f32": lambda: P.sample(None, P.EXACT, out, seed=seed, stream=stream),
            "exact_lib_f32": lambda: P.sample(None, P.EXACT_LIB, out, seed=seed, stream=stream),
        }
        for name, fn in variants.items():
            tot, _ = _time_device(fn, max(5, args.steps // 2), 3, stream)
            extras[name + "_gsamples_per_s"] = N_SAMPLES * max(5, args.steps // 2) / (tot / 1e3) / 1e9
        extras["pwl_over_exact"] = value / world / extras["exact_f32_gsamples_per_s"]
        extras["pwl_over_exact_lib"] = value / world / extras["exact_lib_f32_gsamples_per_s"]
        # the small piecewise-constant configuration: 2^20 samples (launch-latency bound)
        small = torch.empty(1 << 20, dtype=torch.float32, device=dev)
        tot, _ = _time_device(lambda: P.sample(tc, P.PWC, small, seed=seed, stream=stream), 50, 5, stream)
        extras["pwc_2p20_gsamples_per_s"] = (1 << 20) * 50 / (tot / 1e3) / 1e9
        del out16, small
        extras["mlmc"] = mlmc_time_to_rmse(P, tl, dev)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(WORKLOAD, parallelism="replicas" if world > 1 else "single GPU"),
            "roofline": roof, "clocks": clk.summary(), "gpu_launches": args.steps,
            "e2e": e2e, "variants": extras}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
