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
# MUFU rsqrt rate of the XU pipe: one warp instruction per 4 cycles per SM
# sub-partition (ncu's XU peak), i.e. 32 per clock per SM
SFU_PEAK_PER_S = 152 * 32 * 2.070e9
FAR_FLOP_PER_PAIR = {"SD": 19, "S": 10, "D": 14}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the mixed S+D far kernel on the 200-spheroid p = 16 suspension, from one ncu
# capture per launch shape (targets per thread, source splits) of the current
# kernel code; other shapes report null
FAR_DRAM_BYTES_POLY200 = {(-8, 44): 11.57e6}
# the same for the mixed S' + D' far kernel (packed, expanded distance)
DERIV_FAR_DRAM_BYTES_POLY200 = {(-8, 44): 14.35e6}


def near_flop_per_pair(p: int) -> int:
    """Algorithmic FP64 flops of one near (target, source) pair for S and D:
    the two contractions (FMA over (p+1)^2 coefficients each), the radial x
    angular product per (n, |m|), the order recurrence of Q (3 flops) and the
    Ferrers recurrence (4 flops) per (n, |m|), and about 12 flops of angle
    recurrence and cos/sin combination per order m.  The data-dependent Miller
    start of Q_n^0, Q_n^1 is not counted."""
    nm = (p + 1) * (p + 2) // 2
    return 4 * (p + 1) ** 2 + nm * (1 + 3 + 4) + 12 * (p + 1)
METRIC = "BIO applies/s (Laplace S+D, all surface nodes)"
# far pair of S' + D': 3 sub, 5 (r^2), 2 (r^-2, r^-3), 5 (r.nu_x), 3 (S' product
# and FMA), 5 (d.r), 5 (d.nu_x), 2 (products), 2 + 2 (the two FMAs) = 34
DERIV_FAR_FLOP_PER_PAIR = 34
# far pair of the Stokeslet: 3 sub, 5 (r^2), 5 (f.r), 3 (r^-1 r^-2 products),
# 12 (three component FMA pairs) = 28; with the pressure (f.r) r^-3 of the same
# pair one more FMA = 30.  Stresslet: 3 sub, 5 (r^2), 5 (q.r), 5 (nu.r), 4
# (products with r^-5), 6 (three FMAs) = 28.
STOKES_FAR_FLOP_PER_PAIR = 28
STOKES_P_FAR_FLOP_PER_PAIR = 30
STRESSLET_FAR_FLOP_PER_PAIR = 28


def sdl_near_flop_per_pair(p: int) -> int:
    """Algorithmic FP64 flops of one Stokes double-layer near pair, as the
    one-pass term evaluation does them, expansions of order P1 = p + 1.  Per
    (n, m >= 1) term (cos and sin parts together): 20 for the recurrences and
    the radial-angular factors, 21 for the local Cartesian gradient basis, 60
    for the contraction with the thirteen expansions (30 FMA); per m = 0 term
    47; per pair about 120 for coordinates, frame constants and the output.
    The data-dependent Miller start of Q_n^0, Q_n^1 is not counted."""
    p1 = p + 1
    return (p1 * (p1 + 1) // 2) * (20 + 21 + 60) + (p1 + 1) * 47 + 120


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-context", action="store_true")
    ap.add_argument("--no-all-cores", action="store_true", help="skip the all-cores oracle timing")
    ap.add_argument("--oracle-sample", type=int, default=48, help="targets in the oracle's timed sample")
    ap.add_argument("--far-shape", default="", help="TT,SPLITS: fixed far-field launch shape (skips the autotuner)")
    ap.add_argument("--workload", default="poly200",
                    choices=["poly200", "stokes100", "batch64", "serve", "deriv200", "targets200", "derivpoints200",
                             "dirichlet200", "stokespoints100", "stokesdl100", "stokesdlpoints100"])
    ap.add_argument("--rates", default="50,100,200,500,1000,2000", help="serve: arrival rates (req/s)")
    ap.add_argument("--requests", type=int, default=48, help="serve: requests per rate")
    ap.add_argument("--slots", type=int, default=4, help="serve: concurrent request slots")
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


def oracle_sample_time(npz_path, n_sample, p_threads=1, seed=1, start_at=None):
    """Time the oracle's O-method apply on a bounded sample of targets in a
    fresh single-threaded process; returns (seconds, targets, N).  With
    start_at (a time.time() value) the process waits until then before the
    timed part, so that several processes run it together."""
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
tg = np.sort(np.random.default_rng({seed}).choice(og.N, {n_sample}, replace=False))
near = og.near_matrix(tg)
og.near_matrix = lambda targets=None: near
start_at = {start_at!r}
if start_at is not None:
    time.sleep(max(0.0, start_at - time.time()))
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


def oracle_all_cores(npz_path, n_sample, cores):
    """The same oracle sample on `cores` concurrent single-threaded processes
    (disjoint random target samples), started together; returns
    (targets per second over all processes, wall seconds, processes)."""
    import concurrent.futures as cf

    start_at = time.time() + 20.0       # after every process has loaded numpy and the geometry
    with cf.ThreadPoolExecutor(cores) as ex:
        res = list(ex.map(lambda k: oracle_sample_time(npz_path, n_sample, 1, seed=100 + k, start_at=start_at),
                          range(cores)))
    wall = max(r[0] for r in res)
    return sum(r[1] for r in res) / wall, wall, cores


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
    if args.far_shape:
        tt, sp = (int(x) for x in args.far_shape.split(","))
        S.sbio_geom_set_launch_shape(geom.h, tt, sp)
        tune = (tt, sp, None)
    else:
        tune = S.sbio_geom_autotune(geom.h)
    tuning = S.sbio_geom_get_tuning(geom.h)
    setup_ms = S.sbio_geom_setup_times(geom.h)
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
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    l0 = S.sbio_launch_count()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        S.sbio_apply_laplace(geom.h, sig, mu, So, Do)    # near (FP64) overlaps far (FP32)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    launches = S.sbio_launch_count() - l0
    barrier(ws)
    clk = clocks.stop()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_s = allmax(ws, sum(step_ms) / 1e3)
    value = args.steps * ws / total_s

    # per-kernel durations: a phase-timed pass (phases in order, events on the launch stream)
    S.sbio_geom_enable_timing(geom.h, True)
    far_ms, near_ms, synth_ms, inorder_ms = [], [], [], []
    for _ in range(min(args.steps, 10)):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        S.sbio_apply_laplace(geom.h, sig, mu, So, Do)
        e1.record(stream)
        a, b, c = S.sbio_geom_phase_times(geom.h)
        synth_ms.append(a)
        near_ms.append(b)
        far_ms.append(c)
        torch.cuda.synchronize()
        inorder_ms.append(e0.elapsed_time(e1))
    S.sbio_geom_enable_timing(geom.h, False)

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
        S.sbio_geom_enable_timing(geom.h, True)
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
        S.sbio_geom_enable_timing(geom.h, False)
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
                                                        "autotuned_far_ms": tune[2],
                                                        "near_ctas_per_sm_overlapped": tuning["near_ctas_per_sm"]}),
        "gpairs_per_s": geom.n_far / (statistics.mean(step_ms) * 1e-3) / 1e9,
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "phase_ms": {"synth": statistics.mean(synth_ms), "near": statistics.mean(near_ms), "far": far_mean,
                     "in_order_apply": statistics.mean(inorder_ms)},
        "roofline": {"kernel": "far_mixed_kernel" if prec == S.SBIO_MIXED else "far_fp64_kernel",
                     "bound": "alu", "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS if prec == S.SBIO_MIXED else FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / (FP32_PEAK_TFLOPS if prec == S.SBIO_MIXED else FP64_PEAK_TFLOPS),
                     "traffic": (FAR_DRAM_BYTES_POLY200.get((tune[0], tune[1]))
                                 if prec == S.SBIO_MIXED and args.workload == "poly200" else None),
                     "traffic_unit": "bytes per launch (ncu dram read + write, one capture at this launch shape)",
                     "algorithmic_bytes": None,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz" if prec == S.SBIO_MIXED
                     else "nominal FP64 1.25 TFLOP/s"},
        "sfu": {"kernel": "far_mixed_kernel" if prec == S.SBIO_MIXED else "far_fp64_kernel",
                "unit": "rsqrt/s", "achieved": geom.n_far / (far_mean * 1e-3), "peak": SFU_PEAK_PER_S,
                "frac": geom.n_far / (far_mean * 1e-3) / SFU_PEAK_PER_S,
                "note": "one rsqrt per far pair; FP32 MUFU in the mixed form"},
        "roofline_near": {"kernel": "near_kernel", "bound": "alu", "unit": "TFLOP/s",
                          "achieved": near_flop_per_pair(susp.p) * geom.n_near / (statistics.mean(near_ms) * 1e-3) / 1e12,
                          "peak": FP64_PEAK_TFLOPS,
                          "frac": near_flop_per_pair(susp.p) * geom.n_near / (statistics.mean(near_ms) * 1e-3) / 1e12
                          / FP64_PEAK_TFLOPS, "flop_per_pair": near_flop_per_pair(susp.p),
                          "peak_source": "nominal GB300 FP64 1.25 TFLOP/s"},
        "e2e": {"value": e2e_val, "unit": "applies/s", "h2d_bytes_per_step": int(hs.nbytes + hm.nbytes),
                "d2h_bytes_per_step": int(hS.nbytes + hD.nbytes)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "geometry_setup_ms": {"host_nodes": setup_ms[0], "host_near_sets": setup_ms[1],
                              "device_tables_upload": setup_ms[2]},
    }
    line.update(extra)
    geom.close()
    S.sbio_ctx_destroy(ctx)
    if rank == 0 and not args.no_cpu_baseline:
        sec, nt, NN = oracle_sample_time(path, args.oracle_sample)
        per_apply = sec * NN / nt
        line["cpu_baseline"] = {"value": 1.0 / per_apply, "unit": "applies/s", "cores": 1, "kind": "oracle",
                                "sample": f"{nt} random targets of {NN} ({sec:.1f} s), scaled to a full apply"}
        cores = max(1, min(os.cpu_count() or 1, 16))
        if cores > 1 and not args.no_all_cores:
            tps, wall, nproc = oracle_all_cores(path, args.oracle_sample, cores)
            line["cpu_baseline_all_cores"] = {
                "value": tps / NN, "unit": "applies/s", "cores": nproc, "kind": "oracle",
                "sample": f"{nproc} concurrent single-threaded processes, {args.oracle_sample} targets each "
                          f"({wall:.1f} s wall), scaled to a full apply"}
    os.unlink(path)
    if rank == 0:
        print(json.dumps(line), flush=True)


def _event_time(stream, fn):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_stokes100(args, ws, rank, lrank):
    import torch

    import __graft_entry__ as GE

    GE.build()
    from paper_2506_20809_gb300 import inputs as I
    from paper_2506_20809_gb300 import sbio as S

    torch.cuda.set_device(lrank)
    susp = I.config_suspension(3)
    f = I.config_coefficients(susp, 0, ndens=3).transpose(1, 0, 2).copy()
    ctx = S.sbio_ctx_create(lrank, 0)
    g = S.Geometry(ctx, susp, precision=S.SBIO_MIXED)
    tune = S.sbio_geom_autotune_stokes(g.h)
    near_cap = S.sbio_geom_get_stokes_tuning(g.h)["near_ctas_per_sm"]
    fd = torch.from_numpy(f).cuda()
    u = torch.empty((g.N, 3), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        S.sbio_apply_stokes_sl(g.h, fd, u)
    clocks = ClockSampler(lrank)
    clocks.start()
    ms = []
    l0 = S.sbio_launch_count()
    for _ in range(args.steps):                 # near (FP64) overlaps the Stokeslet far field (FP32)
        flush.zero_()
        ms.append(_event_time(st, lambda: S.sbio_apply_stokes_sl(g.h, fd, u)))
    launches = S.sbio_launch_count() - l0
    clk = clocks.stop()
    # end to end through the host entry point: pinned host forces in, velocities out
    fh = torch.from_numpy(f).pin_memory()
    uh = torch.empty((g.N, 3), dtype=torch.float64).pin_memory()
    fh_np, uh_np = fh.numpy(), uh.numpy()
    for _ in range(2):
        S.sbio_apply_stokes_sl_host(g.h, fh_np, uh_np)
    e2e = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.sbio_apply_stokes_sl_host(g.h, fh_np, uh_np)
        e2e.append((time.perf_counter() - t0) * 1e3)
    S.sbio_geom_enable_timing(g.h, True)        # phase-timed pass, phases in order
    ph = []
    for _ in range(min(args.steps, 10)):
        flush.zero_()
        S.sbio_apply_stokes_sl(g.h, fd, u)
        ph.append(S.sbio_geom_phase_times(g.h))
    S.sbio_geom_enable_timing(g.h, False)
    um = u.clone()
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    S.sbio_apply_stokes_sl(g.h, fd, u)
    t64 = _event_time(st, lambda: S.sbio_apply_stokes_sl(g.h, fd, u))
    err = float((um - u).abs().max() / u.abs().max())
    far_ms = statistics.mean(x[2] for x in ph)
    ach = STOKES_FAR_FLOP_PER_PAIR * g.n_far / (far_ms * 1e-3) / 1e12
    line = {"metric": "Stokes single-layer applies/s (all surface nodes)", "value": 1e3 / statistics.mean(ms),
            "unit": "applies/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(ms), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "stokes100_p12", "M": susp.M, "p": susp.p, "targets": g.N,
                       "near_pairs": g.n_near, "far_pairs_per_apply": g.n_far,
                       "far_launch": {"targets_per_thread": tune[0], "source_splits": tune[1]},
                       "near_ctas_per_sm_overlapped": near_cap, "l2": "flushed (256 MiB write) before each step"},
            "e2e": {"value": 1e3 / statistics.mean(e2e), "unit": "applies/s", "h2d_bytes_per_step": int(fh.nbytes),
                    "d2h_bytes_per_step": int(uh.nbytes)},
            "phase_ms": {"prep_and_self": statistics.mean(x[0] for x in ph), "near": statistics.mean(x[1] for x in ph),
                         "far": far_ms},
            "roofline": {"kernel": "stokes_far_mixed_kernel", "bound": "alu", "achieved": ach,
                         "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS,
                         "flop_per_pair": STOKES_FAR_FLOP_PER_PAIR, "traffic": None},
            "fp64_gpu_applies_per_s": 1e3 / t64, "rel_err_vs_fp64_gpu": err, "gpu_launches": int(launches),
            "clocks": clk}
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_batch64(args, ws, rank, lrank):
    import numpy as np
    import torch

    from paper_2506_20809_gb300 import inputs as I

    all_susps = I.batch_suspensions(64, workers=min(16, os.cpu_count() or 1))   # before CUDA starts
    from paper_2506_20809_gb300 import replicas as RP

    # several GPUs: each rank owns whole suspensions (no exchange between them)
    cost = [float((s.M * (s.p + 1) * 2 * (s.p + 1)) ** 2) for s in all_susps]
    susps = [all_susps[k] for k in RP.shard(len(all_susps), rank, ws, cost)]
    import __graft_entry__ as GE

    GE.build()
    from paper_2506_20809_gb300 import sbio as S

    torch.cuda.set_device(lrank)
    ctx = S.sbio_ctx_create(lrank, 0)
    geoms = [S.Geometry(ctx, s, precision=S.SBIO_MIXED) for s in susps]
    coefs = [I.config_coefficients(s, 1) for s in susps]
    sig = [torch.from_numpy(c[0]).cuda() for c in coefs]
    mu = [torch.from_numpy(c[1]).cuda() for c in coefs]
    So = [torch.empty(g.N, dtype=torch.float64, device="cuda") for g in geoms]
    Do = [torch.empty_like(o) for o in So]
    st = torch.cuda.current_stream()
    b = S.sbio_batch_create(ctx, geoms)
    best = None
    for tt in (1, 2, 4, 8, -2, -4, -8):                # autotune the persistent far kernel
        S.sbio_batch_set_far_tt(b, tt)
        S.sbio_batch_apply(b, sig, mu, So, Do)
        t = min(_event_time(st, lambda: S.sbio_batch_apply(b, sig, mu, So, Do)) for _ in range(2))
        if best is None or t < best[1]:
            best = (tt, t)
    S.sbio_batch_set_far_tt(b, best[0])
    for _ in range(args.warmup):
        S.sbio_batch_apply(b, sig, mu, So, Do)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    clocks = ClockSampler(lrank)
    clocks.start()
    ms = []
    l0 = S.sbio_launch_count()
    for _ in range(args.steps):
        flush.zero_()
        ms.append(_event_time(st, lambda: S.sbio_batch_apply(b, sig, mu, So, Do)))
    launches = S.sbio_launch_count() - l0
    clk = clocks.stop()
    info = S.sbio_batch_info(b)
    # the same work as one apply per suspension, one after another (mixed)
    seq = _event_time(st, lambda: [S.sbio_apply_laplace(g.h, sig[k], mu[k], So[k], Do[k]) for k, g in enumerate(geoms)])
    # plain FP64 form, one apply per suspension
    for g in geoms:
        S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    f64 = _event_time(st, lambda: [S.sbio_apply_laplace(g.h, sig[k], mu[k], So[k], Do[k]) for k, g in enumerate(geoms)])
    mean = RP.max_over_ranks(statistics.mean(ms), ws)
    line = {"metric": "BIO applies/s (batched Laplace S+D, 64 suspensions per step)",
            "value": 64 * 1e3 / mean, "unit": "applies/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "batch64", "suspensions": 64, "suspensions_on_rank0": len(susps),
                       "M": [s.M for s in susps], "p": [s.p for s in susps],
                       "far_pairs_per_step": info["far_pairs"], "work_items": info["n_items"],
                       "persistent_grid": info["grid"], "far_targets_per_thread": best[0],
                       "l2": "flushed by a 256 MiB write before every timed step"},
            "gpairs_per_s": info["far_pairs"] / (mean * 1e-3) / 1e9,
            "roofline": {"kernel": "whole step (far_persistent_kernel dominant)", "bound": "alu",
                         "achieved": FAR_FLOP_PER_PAIR["SD"] * info["far_pairs"] / (mean * 1e-3) / 1e12,
                         "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": FAR_FLOP_PER_PAIR["SD"] * info["far_pairs"] / (mean * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                         "flop_per_pair": FAR_FLOP_PER_PAIR["SD"], "traffic": None},
            "sequential_mixed_ms": seq, "fp64_plain_ms": f64,
            "speedup_vs_fp64_plain": f64 / mean, "speedup_vs_sequential_mixed": seq / mean,
            "gpu_launches": int(launches), "clocks": clk}
    S.sbio_batch_destroy(b)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serve(args, ws, rank, lrank):
    import math
    import numpy as np
    import torch

    from paper_2506_20809_gb300 import inputs as I

    # a pool of request geometries (drawn before CUDA starts), sampled by the stream
    rng = np.random.default_rng(2024)
    specs = []
    for k in range(16):
        M = int(round(math.exp(rng.uniform(math.log(20), math.log(500)))))
        specs.append((M, int(rng.choice([8, 12, 16]))))
    import concurrent.futures as cf
    import multiprocessing as mp

    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        pool = list(ex.map(I.rsa_suspension, [m for m, _ in specs], [0.20] * 16, range(1000, 1016),
                           [p for _, p in specs]))
    import __graft_entry__ as GE

    GE.build()
    from paper_2506_20809_gb300 import sbio as S

    torch.cuda.set_device(lrank)
    ctx = S.sbio_ctx_create(lrank, 0)
    free, total = torch.cuda.mem_get_info()
    budget = int(0.5 * free)

    def stream_of(rate, seed, precision, n_req):
        reqs = I.poisson_requests(rate, 1e9, seed=seed, M_range=(20, 500), max_requests=n_req)
        prepared = []
        for k, r in enumerate(reqs):
            s = pool[r["seed"] % len(pool)]
            op = S.SBIO_OP_LAPLACE if r["op"] == "laplace" else S.SBIO_OP_STOKES
            N = s.M * (s.p + 1) * 2 * (s.p + 1)
            nc = (s.p + 1) ** 2
            crng = np.random.default_rng([seed, k])
            if op == S.SBIO_OP_LAPLACE:
                coef = np.ascontiguousarray(np.stack([I.coefficients(crng, s.M, s.p, 2).transpose(1, 0, 2)
                                                      for _ in range(10)]))
                out = np.zeros((10, 2 * N))
            else:
                coef = np.ascontiguousarray(np.stack([I.coefficients(crng, s.M, s.p, 3) for _ in range(10)]))
                out = np.zeros((10, N, 3))
            sph = S.make_spheroids(s.kind, s.A, s.C, s.center, s.quat)
            prepared.append((r["t"], op, sph, s.p, coef, out))
        srv = S.sbio_server_create(ctx, args.slots, budget)
        t0 = time.perf_counter()
        tickets = []
        for (ta, op, sph, p, coef, out) in prepared:
            delay = t0 + ta - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(S.sbio_server_submit(srv, op, sph, p, coef, out, 10, precision=precision))
        lat = []
        for t in tickets:
            stt, l, svc = S.sbio_server_wait(srv, t, 3600.0)
            assert stt == 0
            lat.append(l)
        makespan = time.perf_counter() - t0
        S.sbio_server_destroy(srv)
        lat.sort()
        return {"rate": rate, "requests": len(lat), "applies_per_s": 10 * len(lat) / makespan,
                "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                "makespan_s": makespan}

    # where a request's time goes: geometry set-up (host phases) against its
    # ten applies (Laplace S + D, mixed, one at a time)
    prof = []
    st = torch.cuda.current_stream()
    for s in pool:
        t0 = time.perf_counter()
        g = S.Geometry(ctx, s, precision=S.SBIO_MIXED)
        torch.cuda.synchronize()
        create_ms = (time.perf_counter() - t0) * 1e3
        host, near, dev = S.sbio_geom_setup_times(g.h)
        c = I.config_coefficients(s, 0)
        sg, mg = torch.from_numpy(c[0]).cuda(), torch.from_numpy(c[1]).cuda()
        So = torch.empty(g.N, dtype=torch.float64, device="cuda")
        Do = torch.empty_like(So)
        S.sbio_apply_laplace(g.h, sg, mg, So, Do)
        ap = _event_time(st, lambda: [S.sbio_apply_laplace(g.h, sg, mg, So, Do) for _ in range(10)])
        prof.append({"M": s.M, "p": s.p, "create_ms": create_ms, "host_nodes_ms": host, "near_sets_ms": near,
                     "device_tables_ms": dev, "ten_applies_ms": ap})
        g.close()
    profile = {"geometries": prof, "total_create_ms": sum(x["create_ms"] for x in prof),
               "total_ten_applies_ms": sum(x["ten_applies_ms"] for x in prof)}

    rates = [float(x) for x in args.rates.split(",")]
    rows = [stream_of(r, 7, S.SBIO_MIXED, args.requests) for r in rates]
    ref = stream_of(rates[-1], 7, S.SBIO_FP64, min(12, args.requests))
    mixed_same = stream_of(rates[-1], 7, S.SBIO_MIXED, min(12, args.requests))
    best = max(rows, key=lambda r: r["applies_per_s"])
    line = {"metric": "served BIO applies/s (Poisson stream, 10 applies per request) and p50/p99 latency",
            "value": best["applies_per_s"], "unit": "applies/s", "n_gpus": ws, "steps": len(rates),
            "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "serve", "slots": args.slots, "requests_per_rate": args.requests,
                       "pool": [{"M": m, "p": p} for m, p in specs], "mem_budget_bytes": budget,
                       "ops": "Laplace S+D or Stokes single layer, probability 1/2"},
            "sweep": rows, "pool_profile": profile, "fp64_plain_at_max_rate": ref,
            "mixed_same_requests_as_fp64": mixed_same,
            "speedup_vs_fp64_plain": mixed_same["applies_per_s"] / ref["applies_per_s"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_deriv200(args, ws, rank, lrank):
    """S' + D' (normal derivatives) at all nodes of the 200-spheroid, p = 16
    suspension, mixed precision, L2 flushed before every step."""
    import torch

    import __graft_entry__ as GE

    GE.build()
    from paper_2506_20809_gb300 import inputs as I
    from paper_2506_20809_gb300 import sbio as S

    torch.cuda.set_device(lrank)
    susp = I.config_suspension(2)
    c = I.config_coefficients(susp, 0)
    ctx = S.sbio_ctx_create(lrank, 0)
    g = S.Geometry(ctx, susp, precision=S.SBIO_MIXED)
    dtune = S.sbio_geom_autotune(g.h)           # far shape and near CTA cap for the overlapped near field
    sg, mg = torch.from_numpy(c[0]).cuda(), torch.from_numpy(c[1]).cuda()
    Sp = torch.empty(g.N, dtype=torch.float64, device="cuda")
    Dp = torch.empty_like(Sp)
    st = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        S.sbio_apply_laplace_deriv(g.h, sg, mg, Sp, Dp)
    clocks = ClockSampler(lrank)
    clocks.start()
    ms = []
    l0 = S.sbio_launch_count()
    for _ in range(args.steps):
        flush.zero_()
        ms.append(_event_time(st, lambda: S.sbio_apply_laplace_deriv(g.h, sg, mg, Sp, Dp)))
    launches = S.sbio_launch_count() - l0
    clk = clocks.stop()
    S.sbio_geom_enable_timing(g.h, True)
    ph = []
    for _ in range(min(args.steps, 10)):
        flush.zero_()
        S.sbio_apply_laplace_deriv(g.h, sg, mg, Sp, Dp)
        ph.append(S.sbio_geom_phase_times(g.h))
    S.sbio_geom_enable_timing(g.h, False)
    spm, dpm = Sp.clone(), Dp.clone()
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    S.sbio_apply_laplace_deriv(g.h, sg, mg, Sp, Dp)
    t64 = _event_time(st, lambda: S.sbio_apply_laplace_deriv(g.h, sg, mg, Sp, Dp))
    err = {"Sp": float((spm - Sp).abs().max() / Sp.abs().max()), "Dp": float((dpm - Dp).abs().max() / Dp.abs().max())}
    far_ms = statistics.mean(x[2] for x in ph)
    ach = DERIV_FAR_FLOP_PER_PAIR * g.n_far / (far_ms * 1e-3) / 1e12
    line = {"metric": "BIO applies/s (Laplace S'+D', all surface nodes)", "value": 1e3 / statistics.mean(ms),
            "unit": "applies/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(ms), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "poly200_p16_laplace_SpDp", "M": susp.M, "p": susp.p, "targets": g.N,
                       "near_pairs": g.n_near, "far_pairs_per_apply": g.n_far,
                       "l2": "flushed (256 MiB write) before each step"},
            "phase_ms": {"self": statistics.mean(x[0] for x in ph), "near": statistics.mean(x[1] for x in ph),
                         "far": far_ms},
            "roofline": {"kernel": "far_deriv_mixed_kernel", "bound": "alu", "achieved": ach,
                         "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS,
                         "flop_per_pair": DERIV_FAR_FLOP_PER_PAIR,
                         "traffic": DERIV_FAR_DRAM_BYTES_POLY200.get((dtune[0], dtune[1])),
                         "traffic_unit": "bytes per launch (ncu dram read + write, one capture at this launch shape)"},
            "fp64_gpu_applies_per_s": 1e3 / t64, "rel_err_vs_fp64_gpu": err, "gpu_launches": int(launches),
            "clocks": clk}
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_targets200(args, ws, rank, lrank, deriv=False):
    """S + D of the 200-spheroid, p = 16 suspension at about 124,000 points:
    shells at distances 1e-1 .. 1e-6 from every surface (20 points per
    spheroid and distance) plus 100,000 points spread through the box;
    mixed precision, L2 flushed before every step.  With deriv: the
    directional derivatives of S and D at the same points along seeded random
    unit directions."""
    import torch

    import __graft_entry__ as GE

    GE.build()
    from paper_2506_20809_gb300 import inputs as I
    from paper_2506_20809_gb300 import sbio as S

    torch.cuda.set_device(lrank)
    susp = I.config_suspension(2)
    c = I.config_coefficients(susp, 0)
    X = I.shell_points(susp, per_particle=20, seed=0, far_points=100000)
    ctx = S.sbio_ctx_create(lrank, 0)
    g = S.Geometry(ctx, susp, precision=S.SBIO_MIXED)
    tune = S.sbio_geom_autotune(g.h)
    t0 = time.perf_counter()
    ts = S.TargetSet(g, X)
    setup_ms = (time.perf_counter() - t0) * 1e3
    sg, mg = torch.from_numpy(c[0]).cuda(), torch.from_numpy(c[1]).cuda()
    So = torch.empty(ts.T, dtype=torch.float64, device="cuda")
    Do = torch.empty_like(So)
    if deriv:
        import numpy as np

        E = np.random.default_rng(1).standard_normal((ts.T, 3))
        E /= np.linalg.norm(E, axis=1, keepdims=True)
        Ed = torch.from_numpy(E).cuda()

        def step():
            S.sbio_eval_targets_deriv(ts.h, Ed, sg, mg, So, Do)
    else:
        def step():
            S.sbio_eval_targets(ts.h, sg, mg, So, Do)
    st = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(lrank)
    clocks.start()
    ms = []
    l0 = S.sbio_launch_count()
    for _ in range(args.steps):
        flush.zero_()
        ms.append(_event_time(st, step))
    launches = S.sbio_launch_count() - l0
    clk = clocks.stop()
    som, dom = So.clone(), Do.clone()
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    step()
    t64 = _event_time(st, step)
    err = {"S": float((som - So).abs().max() / So.abs().max()), "D": float((dom - Do).abs().max() / Do.abs().max())}
    mean = statistics.mean(ms)
    ach = (DERIV_FAR_FLOP_PER_PAIR if deriv else 19) * ts.n_far / (mean * 1e-3) / 1e12
    metric = ("point evaluations/s (Laplace grad S . e + grad D . e at arbitrary points)" if deriv else
              "point evaluations/s (Laplace S+D at arbitrary points)")
    line = {"metric": metric, "value": ts.T * 1e3 / mean,
            "unit": "points/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": "derivpoints200_p16" if deriv else "targets200_p16", "M": susp.M, "p": susp.p,
                       "points": ts.T,
                       "near_pairs": ts.n_near, "far_pairs": ts.n_far,
                       "points_recipe": "shells at 1e-1..1e-6 (20 per spheroid and distance) + 100,000 in the box",
                       "far_launch": {"targets_per_thread": tune[0], "source_splits": tune[1]},
                       "l2": "flushed (256 MiB write) before each step"},
            "evaluations_per_s": 1e3 / mean, "target_set_setup_ms": setup_ms,
            "roofline": {"kernel": "whole evaluation (%s dominant)" % ("far_deriv_mixed_kernel" if deriv else
                                                                         "far_mixed_kernel"), "bound": "alu",
                         "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS,
                         "traffic": None},
            "fp64_gpu_points_per_s": ts.T * 1e3 / t64, "rel_err_vs_fp64_gpu": err, "gpu_launches": int(launches),
            "clocks": clk}
    ts.close()
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def _charges_potential(xs, qs, X, chunk=4096):
    import numpy as np

    out = np.zeros(len(X))
    for c0 in range(0, len(X), chunk):
        r = np.linalg.norm(X[c0:c0 + chunk, None, :] - xs[None], axis=-1)
        out[c0:c0 + chunk] = (qs / (4 * np.pi * r)).sum(1)
    return out


def run_dirichlet200(args, ws, rank, lrank):
    """The paper's exterior Dirichlet test at full size: two point charges
    near the centre of each of the 200 spheroids (p = 16), boundary data their
    potential, completed double layer with the eta S completion, GMRES(50)
    to 1e-6 in mixed precision; then u at the targets200 shell points
    against the charges' potential."""
    import numpy as np
    import torch

    import __graft_entry__ as GE

    GE.build()
    from paper_2506_20809_gb300 import inputs as I
    from paper_2506_20809_gb300 import sbio as S

    torch.cuda.set_device(lrank)
    susp = I.config_suspension(2)
    xs, qs = I.interior_charges(susp, 2, seed=0)
    ctx = S.sbio_ctx_create(lrank, 0)
    g = S.Geometry(ctx, susp, precision=S.SBIO_MIXED)
    S.sbio_geom_autotune(g.h)
    xyz, nrm, _ = S.sbio_geom_nodes(g.h)
    f = torch.from_numpy(_charges_potential(xs, qs, xyz)).cuda()
    nc = (susp.p + 1) ** 2
    mu = torch.empty((susp.M, nc), dtype=torch.float64, device="cuda")
    st = torch.empty_like(mu)
    q = torch.empty(susp.M, dtype=torch.float64, device="cuda")
    kw = dict(completion=S.SBIO_COMPLETION_ETA_S, tol=1e-6, max_iter=400, restart=50, sigma_tilde_out=st,
              charges_out=q)
    for _ in range(max(1, min(args.warmup, 2))):
        S.sbio_solve_dirichlet(g.h, f, mu, **kw)
    clocks = ClockSampler(lrank)
    clocks.start()
    infos = []
    l0 = S.sbio_launch_count()
    steps = max(1, min(args.steps, 5))
    for _ in range(steps):
        infos.append(S.sbio_solve_dirichlet(g.h, f, mu, **kw))
    launches = S.sbio_launch_count() - l0
    clk = clocks.stop()
    # one plain apply for the per-iteration comparison
    stream = torch.cuda.current_stream()
    So = torch.empty(g.N, dtype=torch.float64, device="cuda")
    Do = torch.empty_like(So)
    S.sbio_apply_laplace(g.h, st, mu, So, Do)
    apply_ms = statistics.median(_event_time(stream, lambda: S.sbio_apply_laplace(g.h, st, mu, So, Do))
                                 for _ in range(5))
    X = I.shell_points(susp, per_particle=20, seed=0, far_points=20000)
    ts = S.TargetSet(g, X)
    Su = torch.empty(ts.T, dtype=torch.float64, device="cuda")
    Du = torch.empty_like(Su)
    S.sbio_eval_targets(ts.h, st, mu, Su, Du)
    torch.cuda.synchronize()
    ref = _charges_potential(xs, qs, X)
    err = float(np.max(np.abs((Su + Du).cpu().numpy() - ref)) / np.max(np.abs(ref)))
    ms = statistics.mean(i["ms"] for i in infos)
    its = statistics.mean(i["iterations"] for i in infos)
    line = {"metric": "BIE solves/s (exterior Dirichlet, completed double layer)", "value": 1e3 / ms,
            "unit": "solves/s", "n_gpus": ws, "steps": steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": "dirichlet200_p16_etaS", "M": susp.M, "p": susp.p, "unknowns": susp.M * nc,
                       "charges": int(len(xs)), "tol": 1e-6, "restart": 50,
                       "check_points": ts.T},
            "gmres_iterations": its, "converged": all(i["converged"] for i in infos),
            "rel_residual": max(i["rel_residual"] for i in infos),
            "ms_per_iteration": ms / its if its else None, "apply_ms": apply_ms,
            "iteration_over_apply": (ms / its) / apply_ms if its else None,
            "max_rel_err_at_shell_points": err,
            "roofline": {"kernel": "whole solve (far_mixed_kernel dominant; Arnoldi applies only)", "bound": "alu",
                         "achieved": FAR_FLOP_PER_PAIR["SD"] * g.n_far * its / (ms * 1e-3) / 1e12,
                         "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": FAR_FLOP_PER_PAIR["SD"] * g.n_far * its / (ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                         "flop_per_pair": FAR_FLOP_PER_PAIR["SD"], "traffic": None},
            "gpu_launches": int(launches), "clocks": clk}
    ts.close()
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_stokespoints100(args, ws, rank, lrank, dl=False):
    """Stokes velocity and pressure of the 100-spheroid, p = 12 suspension at
    shell points (1e-1 .. 1e-6, 10 per spheroid and distance) plus 30,000
    points in the box; mixed precision, L2 flushed before every step.  With
    dl: the Stokes double layer of three densities at the same points."""
    import torch

    import __graft_entry__ as GE

    GE.build()
    from paper_2506_20809_gb300 import inputs as I
    from paper_2506_20809_gb300 import sbio as S

    torch.cuda.set_device(lrank)
    susp = I.config_suspension(3)
    f = I.config_coefficients(susp, 0, ndens=3).transpose(1, 0, 2).copy()
    X = I.shell_points(susp, per_particle=10, seed=0, far_points=30000)
    ctx = S.sbio_ctx_create(lrank, 0)
    g = S.Geometry(ctx, susp, precision=S.SBIO_MIXED)
    stune = S.sbio_geom_autotune_stokes(g.h)
    scap = S.sbio_geom_get_stokes_tuning(g.h)["near_ctas_per_sm"]
    ts = S.TargetSet(g, X)
    fd = torch.from_numpy(f).cuda()
    u = torch.empty((ts.T, 3), dtype=torch.float64, device="cuda")
    pr = torch.empty(ts.T, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    if dl:
        def step():
            S.sbio_eval_targets_stokes_dl(ts.h, fd, u)
    else:
        def step():
            S.sbio_eval_targets_stokes(ts.h, fd, u, pr)
    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(lrank)
    clocks.start()
    ms = []
    l0 = S.sbio_launch_count()
    for _ in range(args.steps):
        flush.zero_()
        ms.append(_event_time(st, step))
    launches = S.sbio_launch_count() - l0
    clk = clocks.stop()
    um, pm = u.clone(), pr.clone()
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    step()
    t64 = _event_time(st, step)
    err = {"u": float((um - u).abs().max() / u.abs().max())}
    if not dl:
        err["p"] = float((pm - pr).abs().max() / pr.abs().max())
    mean = statistics.mean(ms)
    far_flop = STRESSLET_FAR_FLOP_PER_PAIR if dl else STOKES_P_FAR_FLOP_PER_PAIR
    line = {"metric": ("point evaluations/s (Stokes double layer at arbitrary points)" if dl else
                       "point evaluations/s (Stokes velocity + pressure at arbitrary points)"),
            "value": ts.T * 1e3 / mean, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "stokesdlpoints100_p12" if dl else "stokespoints100_p12", "M": susp.M, "p": susp.p, "points": ts.T,
                       "near_pairs": ts.n_near, "far_pairs": ts.n_far,
                       "far_launch": {"targets_per_thread": stune[0], "source_splits": stune[1]},
                       "near_ctas_per_sm_overlapped": scap,
                       "points_recipe": "shells at 1e-1..1e-6 (10 per spheroid and distance) + 30,000 in the box",
                       "l2": "flushed (256 MiB write) before each step"},
            "evaluations_per_s": 1e3 / mean, "fp64_gpu_points_per_s": ts.T * 1e3 / t64,
            "roofline": {"kernel": ("whole evaluation (stresslet_far_mixed_kernel dominant)" if dl else
                                    "whole evaluation (stokes_far_mixed_kernel with pressure dominant)"),
                         "bound": "alu",
                         "achieved": far_flop * ts.n_far / (mean * 1e-3) / 1e12,
                         "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": far_flop * ts.n_far / (mean * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                         "flop_per_pair": far_flop, "traffic": None},
            "rel_err_vs_fp64_gpu": err, "gpu_launches": int(launches), "clocks": clk}
    ts.close()
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_stokesdl100(args, ws, rank, lrank):
    """Stokes double layer (principal value) at all nodes of the 100-spheroid,
    p = 12 suspension; mixed precision, L2 flushed before every step."""
    import torch

    import __graft_entry__ as GE

    GE.build()
    from paper_2506_20809_gb300 import inputs as I
    from paper_2506_20809_gb300 import sbio as S

    torch.cuda.set_device(lrank)
    susp = I.config_suspension(3)
    q = I.config_coefficients(susp, 1, ndens=3).transpose(1, 0, 2).copy()
    ctx = S.sbio_ctx_create(lrank, 0)
    g = S.Geometry(ctx, susp, precision=S.SBIO_MIXED)
    stune = S.sbio_geom_autotune_stokes(g.h)
    scap = S.sbio_geom_get_stokes_tuning(g.h)["near_ctas_per_sm"]
    qd = torch.from_numpy(q).cuda()
    u = torch.empty((g.N, 3), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        S.sbio_apply_stokes_dl(g.h, qd, u)
    clocks = ClockSampler(lrank)
    clocks.start()
    ms = []
    l0 = S.sbio_launch_count()
    for _ in range(args.steps):
        flush.zero_()
        ms.append(_event_time(st, lambda: S.sbio_apply_stokes_dl(g.h, qd, u)))
    launches = S.sbio_launch_count() - l0
    clk = clocks.stop()
    S.sbio_geom_enable_timing(g.h, True)        # phase-timed pass, phases in order
    ph = []
    for _ in range(min(args.steps, 10)):
        flush.zero_()
        S.sbio_apply_stokes_dl(g.h, qd, u)
        ph.append(S.sbio_geom_phase_times(g.h))
    S.sbio_geom_enable_timing(g.h, False)
    um = u.clone()
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    S.sbio_apply_stokes_dl(g.h, qd, u)
    t64 = _event_time(st, lambda: S.sbio_apply_stokes_dl(g.h, qd, u))
    err = float((um - u).abs().max() / u.abs().max())
    mean = statistics.mean(ms)
    near_ms = statistics.mean(x[1] for x in ph)
    far_ms = statistics.mean(x[2] for x in ph)
    near_flop = sdl_near_flop_per_pair(susp.p)
    near_ach = near_flop * g.n_near / (near_ms * 1e-3) / 1e12
    far_ach = STRESSLET_FAR_FLOP_PER_PAIR * g.n_far / (far_ms * 1e-3) / 1e12
    line = {"metric": "Stokes double-layer applies/s (all surface nodes)", "value": 1e3 / mean, "unit": "applies/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": "stokesdl100_p12", "M": susp.M, "p": susp.p, "targets": g.N,
                       "near_pairs": g.n_near, "far_pairs_per_apply": g.n_far,
                       "far_launch": {"targets_per_thread": stune[0], "source_splits": stune[1]},
                       "near_ctas_per_sm_overlapped": scap,
                       "l2": "flushed (256 MiB write) before each step"},
            "phase_ms": {"prep_and_self": statistics.mean(x[0] for x in ph), "near": near_ms, "far": far_ms},
            "roofline": {"kernel": "stokes_dl_near_kernel (FP64 pipe)", "bound": "alu", "achieved": near_ach,
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": near_ach / FP64_PEAK_TFLOPS,
                         "flop_per_pair": near_flop, "traffic": None,
                         "peak_source": "nominal GB300 FP64 1.25 TFLOP/s"},
            "roofline_far": {"kernel": "stresslet_far_mixed_kernel", "bound": "alu", "achieved": far_ach,
                             "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": far_ach / FP32_PEAK_TFLOPS,
                             "flop_per_pair": STRESSLET_FAR_FLOP_PER_PAIR, "traffic": None},
            "fp64_gpu_applies_per_s": 1e3 / t64, "rel_err_vs_fp64_gpu": err, "gpu_launches": int(launches),
            "clocks": clk}
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, lrank = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "stokes100":
        run_stokes100(args, ws, rank, lrank)
    elif args.workload == "batch64":
        run_batch64(args, ws, rank, lrank)
    elif args.workload == "serve":
        run_serve(args, ws, rank, lrank)
    elif args.workload == "deriv200":
        run_deriv200(args, ws, rank, lrank)
    elif args.workload == "targets200":
        run_targets200(args, ws, rank, lrank)
    elif args.workload == "derivpoints200":
        run_targets200(args, ws, rank, lrank, deriv=True)
    elif args.workload == "dirichlet200":
        run_dirichlet200(args, ws, rank, lrank)
    elif args.workload == "stokespoints100":
        run_stokespoints100(args, ws, rank, lrank)
    elif args.workload == "stokesdlpoints100":
        run_stokespoints100(args, ws, rank, lrank, dl=True)
    elif args.workload == "stokesdl100":
        run_stokesdl100(args, ws, rank, lrank)
    else:
        run_ours(args, ws, rank, lrank)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
