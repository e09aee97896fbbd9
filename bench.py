#!/usr/bin/env python
"""Benchmark of the spheroidal Laplace BIO apply (S and D at every node).

Workload (default): 200 polydisperse prolate/oblate spheroids, aspect ratio
U[1.2, 5], major semi-axis U[0.5, 1.5], 20 % volume fraction, gap >= 0.05,
p = 16 (17 x 34 nodes, N = 115,600 targets), coefficients N(0,1)/(n+1)^2,
mixed precision (FP32 compensated far field, FP64 near field and self term).

One step = one BIO apply (S[sigma] and D[mu] at all N nodes) with the
geometry resident.  `value` is whole-job applies/s from CUDA events around
each apply on the launch stream (L2 flushed by a 256 MiB write before every
timed step, outside the events); `e2e` is the same metric through the
host-memory entry point (pinned coefficients in, results out, copies inside
the timed region).  Multi-GPU runs are independent replicas (weak scaling).

`--impl reference` times the CPU oracle (plain FP64 restatement of the
method) on a bounded sample of targets of the same workload.
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

FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12     # SMs x FP32 lanes x FMA x max SM clock
FP64_PEAK_TFLOPS = 1.25                               # nominal GB300 FP64 rate
FAR_FLOP_PER_PAIR = {"SD": 19, "S": 10, "D": 14}
METRIC = "BIO applies/s (Laplace S+D, all surface nodes)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-context", action="store_true")
    ap.add_argument("--oracle-sample", type=int, default=48, help="targets in the oracle's timed sample")
    return ap.parse_args()


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    lrank = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=ws)
    return ws, rank, lrank


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def allmax(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample_time(npz_path, n_sample, p_threads=1):
    """Time the oracle's O-method apply on a bounded sample of targets in a
    fresh single-threaded process; returns (seconds, targets, N)."""
    code = f"""
import os, sys, time, json
import numpy as np
sys.path.insert(0, {ROOT!r})
from paper_2506_20809_gb300 import inputs as I
from oracle import geometry as OG, laplace as OL
d = np.load({npz_path!r})
s = I.Suspension(d['kind'], d['A'], d['C'], d['center'], d['quat'], int(d['p']))
og = OG.SuspensionGeom.from_suspension(s)
O = OL.LaplaceOracle(og)
tg = np.sort(np.random.default_rng(1).choice(og.N, {n_sample}, replace=False))
near = og.near_matrix(tg)
og.near_matrix = lambda targets=None: near
t0 = time.perf_counter()
O.apply(d['sig'], d['mu'], 'method', targets=tg)
t1 = time.perf_counter()
print(json.dumps({{"seconds": t1 - t0, "targets": len(tg), "N": og.N}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS=str(p_threads), OPENBLAS_NUM_THREADS=str(p_threads),
               MKL_NUM_THREADS=str(p_threads), CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return out["seconds"], out["targets"], out["N"]


def make_workload():
    import numpy as np

    from paper_2506_20809_gb300 import inputs as I

    # the draw is deterministic; reuse it across runs on the same machine
    cache = os.path.join(tempfile.gettempdir(), "sbio_poly200_seed0_v1.npz")
    if os.path.exists(cache):
        d = np.load(cache)
        susp = I.Suspension(d["kind"], d["A"], d["C"], d["center"], d["quat"], int(d["p"]), "poly200")
    else:
        susp = I.config_suspension(2, seed=0)
        np.savez(cache + ".tmp.npz", kind=susp.kind, A=susp.A, C=susp.C, center=susp.center, quat=susp.quat,
                 p=susp.p)
        os.replace(cache + ".tmp.npz", cache)
    coef = I.config_coefficients(susp, 0)
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    np.savez(path, kind=susp.kind, A=susp.A, C=susp.C, center=susp.center, quat=susp.quat, p=susp.p,
             sig=coef[0], mu=coef[1])
    return susp, coef, path


def config_dict(susp, n_near, n_far, N):
    return {"workload": "poly200_p16_laplace_SD", "M": susp.M, "p": susp.p, "nodes": f"{susp.p + 1}x{2 * (susp.p + 1)}",
            "targets": N, "near_pairs": n_near, "far_pairs_per_apply": n_far, "operators": "S+D",
            "geometry": "AR U[1.2,5], major U[0.5,1.5], phi=20%, gap>=0.05, RSA seed 0",
            "l2": "flushed by a 256 MiB write before every timed step (outside the events)"}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    susp, coef, path = make_workload()
    times = []
    for k in range(args.warmup + args.steps):
        sec, nt, N = oracle_sample_time(path, args.oracle_sample)
        if k >= args.warmup:
            times.append(sec * N / nt)       # seconds per full apply
    os.unlink(path)
    per_apply = statistics.mean(times)
    val = 1.0 / per_apply
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "applies/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_apply * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "poly200_p16_laplace_SD", "M": susp.M, "p": susp.p,
                       "sample": f"{args.oracle_sample} random targets per step, scaled to all {N}"},
            "cpu_baseline": {"value": val, "unit": "applies/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.oracle_sample} of {N} targets per step, single thread"},
            "e2e": {"value": val, "unit": "applies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, ws, rank, lrank):
    import numpy as np
    import torch

    import __graft_entry__ as GE

    GE.build()
    from paper_2506_20809_gb300 import sbio as S

    torch.cuda.set_device(lrank)
    dev = torch.device("cuda", lrank)
    susp, coef, path = make_workload()
    ctx = S.sbio_ctx_create(lrank, 0)
    prec = S.SBIO_MIXED if args.precision == "mixed" else S.SBIO_FP64
    geom = S.Geometry(ctx, susp, precision=prec)
    tune = S.sbio_geom_autotune(geom.h)
    S.sbio_geom_enable_timing(geom.h, True)
    N = geom.N
    sig = torch.from_numpy(coef[0]).to(dev)
    mu = torch.from_numpy(coef[1]).to(dev)
    So = torch.empty(N, dtype=torch.float64, device=dev)
    Do = torch.empty(N, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        S.sbio_apply_laplace(geom.h, sig, mu, So, Do)
    torch.cuda.synchronize()

    clocks = ClockSampler(lrank)
    clocks.start()
    time.sleep(0.3)
    step_ms, far_ms, near_ms, synth_ms = [], [], [], []
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    l0 = S.sbio_launch_count()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        S.sbio_apply_laplace(geom.h, sig, mu, So, Do)
        evs[k][1].record(stream)
        a, b, c = S.sbio_geom_phase_times(geom.h)    # synchronises on this step's events
        synth_ms.append(a)
        near_ms.append(b)
        far_ms.append(c)
    torch.cuda.synchronize()
    launches = S.sbio_launch_count() - l0
    barrier(ws)
    clk = clocks.stop()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_s = allmax(ws, sum(step_ms) / 1e3)
    value = args.steps * ws / total_s

    # end to end through the host-memory entry point (pinned buffers)
    hs = torch.from_numpy(coef[0]).pin_memory().numpy()
    hm = torch.from_numpy(coef[1]).pin_memory().numpy()
    hS = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
    hD = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
    S.sbio_apply_laplace_host(geom.h, hs, hm, hS, hD)
    e2e_s = []
    barrier(ws)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        S.sbio_apply_laplace_host(geom.h, hs, hm, hS, hD)
        e2e_s.append(time.perf_counter() - t0)
    e2e_total = allmax(ws, sum(e2e_s))
    e2e_val = args.steps * ws / e2e_total

    # accuracy of this precision against the FP64 GPU path, and FP64 context
    extra = {}
    if not args.no_fp64_context:
        S64 = torch.empty_like(So)
        D64 = torch.empty_like(Do)
        S.sbio_geom_set_precision(geom.h, S.SBIO_FP64)
        S.sbio_apply_laplace(geom.h, sig, mu, S64, D64)
        torch.cuda.synchronize()
        t64 = []
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            S.sbio_apply_laplace(geom.h, sig, mu, S64, D64)
            e1.record(stream)
            torch.cuda.synchronize()
            t64.append(e0.elapsed_time(e1))
        f64_phase = S.sbio_geom_phase_times(geom.h)
        S.sbio_geom_set_precision(geom.h, prec)
        S.sbio_apply_laplace(geom.h, sig, mu, So, Do)
        torch.cuda.synchronize()
        relS = float((So - S64).abs().max() / S64.abs().max())
        relD = float((Do - D64).abs().max() / D64.abs().max())
        extra = {"fp64_gpu_applies_per_s": 1e3 / statistics.mean(t64), "fp64_gpu_far_ms": f64_phase[2],
                 "rel_err_vs_fp64_gpu": {"S": relS, "D": relD}}

    far_mean = statistics.mean(far_ms)
    far_flop = FAR_FLOP_PER_PAIR["SD"] * geom.n_far
    achieved = far_flop / (far_mean * 1e-3) / 1e12
    lat = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": "applies/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if prec == S.SBIO_MIXED else "f64",
        "data": "synthetic", "config": dict(config_dict(susp, geom.n_near, geom.n_far, N),
                                            far_launch={"targets_per_thread": tune[0], "source_splits": tune[1],
                                                        "autotuned_far_ms": tune[2]}),
        "gpairs_per_s": geom.n_far / (statistics.mean(step_ms) * 1e-3) / 1e9,
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "phase_ms": {"synth": statistics.mean(synth_ms), "near": statistics.mean(near_ms), "far": far_mean},
        "roofline": {"kernel": "far_mixed_kernel" if prec == S.SBIO_MIXED else "far_fp64_kernel",
                     "bound": "alu", "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS if prec == S.SBIO_MIXED else FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / (FP32_PEAK_TFLOPS if prec == S.SBIO_MIXED else FP64_PEAK_TFLOPS),
                     "traffic": None,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz" if prec == S.SBIO_MIXED
                     else "nominal FP64 1.25 TFLOP/s"},
        "e2e": {"value": e2e_val, "unit": "applies/s", "h2d_bytes_per_step": int(hs.nbytes + hm.nbytes),
                "d2h_bytes_per_step": int(hS.nbytes + hD.nbytes)},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    line.update(extra)
    geom.close()
    S.sbio_ctx_destroy(ctx)
    if rank == 0 and not args.no_cpu_baseline:
        sec, nt, NN = oracle_sample_time(path, args.oracle_sample)
        per_apply = sec * NN / nt
        line["cpu_baseline"] = {"value": 1.0 / per_apply, "unit": "applies/s", "cores": 1, "kind": "oracle",
                                "sample": f"{nt} random targets of {NN} ({sec:.1f} s), scaled to a full apply"}
    os.unlink(path)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, lrank = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, lrank)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
