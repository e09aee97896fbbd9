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

# Roofline basis: the device's multiprocessor count and the median SM clock
# sampled during the timed region (set by set_peak_basis; the defaults are
# GB300's 152 SMs at the 2070 MHz maximum until a run has measured them).
_PEAK_BASIS = {"sms": 152, "mhz": 2070.0, "source": "default: 152 SMs at 2070 MHz (not yet measured)"}
FP64_NOMINAL_TFLOPS = 1.25                            # GB300 FP64 rate (datasheet), context only


def set_peak_basis(device, clk):
    """SM count from the device properties, clock from the sampled median
    (nvidia-smi during the timed region), else the device's maximum."""
    import torch

    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz = clk["sm_mhz"] if clk and clk.get("sm_mhz") else 2070.0
    _PEAK_BASIS.update(sms=sms, mhz=mhz,
                       source=f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz (median sampled SM clock)"
                       if clk and clk.get("sm_mhz") else f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x 2070 MHz")


def fp32_peak():
    """FP32 FMA peak in TFLOP/s: SMs x 128 lanes x 2 flop x clock."""
    return _PEAK_BASIS["sms"] * 128 * 2 * _PEAK_BASIS["mhz"] * 1e6 / 1e12


def sfu_peak():
    """MUFU rsqrt peak per second: 16 per clock per SM, the rate the rsqrt
    chains of sbio_measure_peaks reach on GB300 (4.99e12 /s on 152 SMs at
    2.06 GHz; ncu's XU percentage is relative to twice that)."""
    return _PEAK_BASIS["sms"] * 16 * _PEAK_BASIS["mhz"] * 1e6


_MEASURED = {}


def measure_device_peaks(S, device):
    """Pipe rates of this GPU from the library's microbenchmarks (measured
    once per process, outside every timed region)."""
    if not _MEASURED:
        _MEASURED.update(S.sbio_measure_peaks(device))
    return dict(_MEASURED)


def fp64_peak():
    """FP64 FMA peak in TFLOP/s: the measured DFMA rate when this process has
    measured it, else the nominal 1.25 TFLOP/s."""
    return _MEASURED.get("fp64_dfma_tflops") or FP64_NOMINAL_TFLOPS


def fp64_peak_source():
    return ("measured: FP64 FMA chains at full occupancy (sbio_measure_peaks)" if _MEASURED.get("fp64_dfma_tflops")
            else "nominal GB300 FP64 1.25 TFLOP/s")


FAR_FLOP_PER_PAIR = {"SD": 19, "S": 10, "D": 14}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the mixed S+D far kernel on the 200-spheroid p = 16 suspension, from one ncu
# capture per launch shape (targets per thread, source splits) of the current
# kernel code, with the profile summary it comes from; other shapes report null
FAR_DRAM_BYTES_POLY200 = {(-8, 44): (11.57e6, "profiles/far_mixed_packed_expanded_poly200.md")}
# the same for the mixed S' + D' far kernel (packed, expanded distance)
DERIV_FAR_DRAM_BYTES_POLY200 = {(-8, 44): (14.35e6, "profiles/far_deriv_packed_poly200.md")}


def near_flop_per_pair(p: int) -> int:
    """Algorithmic FP64 flops of one near (target, source) pair for S and D
    without its data-dependent Miller start: the two contractions (FMA over
    (p+1)^2 coefficients each), the radial x angular product per (n, |m|),
    the order recurrence of Q (3 flops) and the Ferrers recurrence (4 flops)
    per (n, |m|), about 12 flops of angle recurrence and cos/sin combination
    per order m, about 40 for the local and spheroidal coordinates, and the
    unrolled part of the two Miller sweeps (p + 2 steps of two three-term
    recurrences, 6 flops each, and the normalisation of 2 (p + 2) values)."""
    nm = (p + 1) * (p + 2) // 2
    return 4 * (p + 1) ** 2 + nm * (1 + 3 + 4) + 12 * (p + 1) + 40 + 12 * (p + 2) + 2 * (p + 2)


# one rolled Miller step (m = 0 and m = 1 together): 5 + 4 flops for the two
# recurrences (FMA = 2) and 2 for the running index and (2n + 1) u
MILLER_FLOP_PER_STEP = 11
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
    ap.add_argument("--oracle-sample", type=int, default=96, help="targets in the oracle's timed sample")
    ap.add_argument("--far-shape", default="", help="TT,SPLITS: fixed far-field launch shape (skips the autotuner)")
    ap.add_argument("--workload", default="poly200",
                    choices=["poly200", "stokes100", "batch64", "serve", "deriv200", "targets200", "derivpoints200",
                             "dirichlet200", "stokespoints100", "stokesdl100", "stokesdlpoints100",
                             "lattice8", "far_sweep"])
    ap.add_argument("--rates", default="5,10,20,30,50,200", help="serve: arrival rates (req/s)")
    ap.add_argument("--requests", type=int, default=2000, help="serve: at most this many requests per rate")
    ap.add_argument("--slots", type=int, default=4, help="serve: concurrent request slots")
    ap.add_argument("--serve-seconds", type=float, default=30.0, help="serve: arrival window per rate (s)")
    ap.add_argument("--serve-pool", type=int, default=32, help="serve: distinct suspensions drawn for the stream")
    ap.add_argument("--serve-direct", action="store_true", help="serve: direct far field for Laplace requests")
    ap.add_argument("--headline-only", action="store_true",
                    help="poly200: skip the batched, served and Stokes sub-objects")
    ap.add_argument("--sweep-M", default="200,500,1000,2000", help="far_sweep: particle counts")
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


def stratified_targets(near_count, n, offset=0.5, seed=0):
    """n targets spread evenly over the targets ordered by their number of
    near particles (ties in a seeded random order), so near-heavy and
    far-only targets enter the sample in proportion; `offset` in (0, 1)
    shifts the picks, giving disjoint samples for different offsets."""
    import numpy as np

    N = len(near_count)
    perm = np.random.default_rng(seed).permutation(N)
    order = perm[np.argsort(near_count[perm], kind="stable")]
    pick = np.minimum(((np.arange(n) + offset) * N / n).astype(np.int64), N - 1)
    return np.sort(order[pick])


def oracle_sample_time(npz_path, targets, start_at=None):
    """Time the oracle's O-method apply on the given targets in a fresh
    single-threaded process (the near sets of the sample are computed before
    the timed part); returns (seconds, targets, N).  With start_at (a
    time.time() value) the process waits until then before the timed part,
    so that several processes run it together."""
    import numpy as np

    fd, tpath = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    np.save(tpath, np.asarray(targets, dtype=np.int64))
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
tg = np.load({tpath!r})
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
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    finally:
        os.unlink(tpath)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return out["seconds"], out["targets"], out["N"]


def oracle_all_cores(npz_path, near_count, n_sample, cores):
    """The oracle on `cores` concurrent single-threaded processes, each on
    its own stratified sample of n_sample targets (disjoint picks), started
    together; returns (targets per second over all processes, wall seconds,
    processes)."""
    import concurrent.futures as cf

    start_at = time.time() + 30.0       # after every process has loaded numpy and the geometry
    samples = [stratified_targets(near_count, n_sample, offset=(k + 0.5) / cores, seed=1) for k in range(cores)]
    with cf.ThreadPoolExecutor(cores) as ex:
        res = list(ex.map(lambda k: oracle_sample_time(npz_path, samples[k], start_at=start_at), range(cores)))
    wall = max(r[0] for r in res)
    return sum(r[1] for r in res) / wall, wall, cores


def cpu_model():
    """CPU model name from lscpu (or /proc/cpuinfo), for the CPU baseline."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


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
    import numpy as np

    from oracle import geometry as OG

    susp, coef, path = make_workload()
    near_count = OG.SuspensionGeom.from_suspension(susp).near_matrix().sum(axis=1)
    times = []
    for k in range(args.warmup + args.steps):
        tg = stratified_targets(near_count, args.oracle_sample, offset=(k + 0.5) / (args.warmup + args.steps))
        sec, nt, N = oracle_sample_time(path, tg)
        if k >= args.warmup:
            times.append(sec * N / nt)       # seconds per full apply
    os.unlink(path)
    per_apply = statistics.mean(times)
    val = 1.0 / per_apply
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "applies/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_apply * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "poly200_p16_laplace_SD", "M": susp.M, "p": susp.p,
                       "sample": f"{args.oracle_sample} stratified targets per step (by near-particle count), "
                                 f"scaled to all {N}"},
            "cpu_baseline": {"value": val, "unit": "applies/s", "cores": 1, "kind": "oracle", "cpu": cpu_model(),
                             "sample": f"{args.oracle_sample} of {N} targets per step, stratified by near-particle "
                                       f"count, single thread"},
            "e2e": {"value": val, "unit": "applies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, ws, rank, lrank):
    """The headline line: poly200 S + D applies/s (device-timed, L2 flushed),
    end to end through the host-memory entry point, the far and near
    rooflines against derived and measured peaks, the FP64 GPU form and the
    oracle's CPU time.  Returns the line (printed by the caller)."""
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
    peaks = measure_device_peaks(S, lrank)
    if args.far_shape:
        tt, sp = (int(x) for x in args.far_shape.split(","))
        S.sbio_geom_set_launch_shape(geom.h, tt, sp)
        tune = (tt, sp, None)
    else:
        tune = S.sbio_geom_autotune(geom.h)
    tuning = S.sbio_geom_get_tuning(geom.h)
    setup_ms = S.sbio_geom_setup_times(geom.h)
    n_pairs, miller_steps = S.sbio_geom_near_work(geom.h)
    near_t, _ = S.sbio_geom_near_pairs(geom.h)
    N = geom.N
    near_count = np.bincount(near_t, minlength=N)
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
    set_peak_basis(lrank, clk)
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
                 "fp64_gpu_near_ms": f64_phase[1],
                 "rel_err_vs_fp64_gpu": {"S": relS, "D": relD}}
        if prec == S.SBIO_MIXED:
            # the same apply with the treecode far field (order 16, theta 0.5)
            S.sbio_geom_set_far_method(geom.h, S.SBIO_FAR_TREE, 0.5, 16)
            info = S.sbio_geom_tree_info(geom.h)
            for _ in range(3):
                S.sbio_apply_laplace(geom.h, sig, mu, So, Do)
            tms = []
            for _ in range(args.steps):
                flush.zero_()
                tms.append(_event_time(stream, lambda: S.sbio_apply_laplace(geom.h, sig, mu, So, Do)))
            S.sbio_geom_enable_timing(geom.h, True)
            S.sbio_apply_laplace(geom.h, sig, mu, So, Do)
            tph = S.sbio_geom_tree_phase_times(geom.h)
            tfar = S.sbio_geom_phase_times(geom.h)[2]
            S.sbio_geom_enable_timing(geom.h, False)
            S.sbio_apply_laplace(geom.h, sig, mu, So, Do)
            torch.cuda.synchronize()
            extra["tree"] = {
                "far_method": "particle treecode, solid-harmonic multipoles order 16, theta 0.5",
                "applies_per_s": 1e3 / statistics.mean(tms), "ms_per_step": statistics.mean(tms),
                "far_ms": tfar, "phase_ms": dict(zip(("leaf_multipoles", "translations", "direct", "evaluations"), tph)),
                "rel_err_vs_fp64_gpu": {"S": float((So - S64).abs().max() / S64.abs().max()),
                                        "D": float((Do - D64).abs().max() / D64.abs().max())},
                "m2p_evaluations": info["m2p_pairs"], "direct_pairs": info["direct_pairs"],
                "m2p_evaluations_by_order": S.sbio_geom_tree_order_counts(geom.h, S.SBIO_OP_LAPLACE),
                "near_ctas_per_sm_beside_tree": S.sbio_geom_get_tree_near_cap(geom.h),
                "note": "same apply with the far field by the treecode instead of the direct sum; the headline "
                        "value above is the direct tiled sum"}
            S.sbio_geom_set_far_method(geom.h, S.SBIO_FAR_DIRECT)

    far_mean = statistics.mean(far_ms)
    far_flop = FAR_FLOP_PER_PAIR["SD"] * geom.n_far
    achieved = far_flop / (far_mean * 1e-3) / 1e12
    pk32 = fp32_peak() if prec == S.SBIO_MIXED else fp64_peak()
    traffic = FAR_DRAM_BYTES_POLY200.get((tune[0], tune[1])) if prec == S.SBIO_MIXED else None
    near_mean = statistics.mean(near_ms)
    near_fixed = near_flop_per_pair(susp.p)
    near_flop = near_fixed * n_pairs + MILLER_FLOP_PER_STEP * miller_steps
    # the FP64 near kernel's roofline: its time from the plain FP64 apply
    # (phases in order); a mixed geometry runs the FP32-contraction form,
    # reported beside it
    near64_ms = extra.get("fp64_gpu_near_ms") if prec == S.SBIO_MIXED else near_mean
    near_ach = near_flop / (near64_ms * 1e-3) / 1e12 if near64_ms else None
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
        "phase_ms": {"synth": statistics.mean(synth_ms), "near": near_mean, "far": far_mean,
                     "in_order_apply": statistics.mean(inorder_ms)},
        "roofline": {"kernel": "far_mixed_kernel" if prec == S.SBIO_MIXED else "far_fp64_kernel",
                     "bound": "alu", "achieved": achieved, "peak": pk32, "unit": "TFLOP/s",
                     "frac": achieved / pk32,
                     "traffic": traffic[0] if traffic else None,
                     "traffic_source": (f"{traffic[1]} (ncu dram read + write, one capture at this launch shape)"
                                        if traffic else None),
                     "algorithmic_bytes": None,
                     "flop_per_pair": FAR_FLOP_PER_PAIR["SD"], "pairs_per_launch": geom.n_far,
                     "peak_source": _PEAK_BASIS["source"] if prec == S.SBIO_MIXED else fp64_peak_source(),
                     "measured_peaks": {
                         "ffma2_tflops": peaks["fp32_ffma2_tflops"],
                         "frac_of_measured_ffma2": achieved / peaks["fp32_ffma2_tflops"],
                         "pairmix_pairs_per_s": peaks["pairmix_pairs_per_s"],
                         "frac_of_pairmix": geom.n_far / (far_mean * 1e-3) / peaks["pairmix_pairs_per_s"],
                         "pairsmem_pairs_per_s": peaks["pairsmem_pairs_per_s"],
                         "frac_of_pairsmem": geom.n_far / (far_mean * 1e-3) / peaks["pairsmem_pairs_per_s"],
                         "note": "measured by sbio_measure_peaks on this GPU: f32x2 FMA chains; the packed far "
                                 "pair's register arithmetic (11 f32x2 + 2 MUFU per 2 pairs) with no memory "
                                 "traffic (pairmix); the same fed from shared memory as the kernel does, without "
                                 "tiles or barriers (pairsmem)"} if prec == S.SBIO_MIXED else None},
        "sfu": {"kernel": "far_mixed_kernel" if prec == S.SBIO_MIXED else "far_fp64_kernel",
                "unit": "rsqrt/s", "achieved": geom.n_far / (far_mean * 1e-3), "peak": sfu_peak(),
                "frac": geom.n_far / (far_mean * 1e-3) / sfu_peak(),
                "measured_peak": peaks["rsqrt_per_s"],
                "frac_of_measured": geom.n_far / (far_mean * 1e-3) / peaks["rsqrt_per_s"],
                "note": "one rsqrt per far pair; FP32 MUFU in the mixed form"},
        "roofline_near": {"kernel": "near_kernel (FP64 form)", "bound": "alu", "unit": "TFLOP/s",
                          "achieved": near_ach, "ms": near64_ms,
                          "peak": fp64_peak(), "frac": near_ach / fp64_peak() if near_ach else None,
                          "frac_of_nominal": near_ach / FP64_NOMINAL_TFLOPS if near_ach else None,
                          "flop_per_pair": near_flop / max(1, n_pairs),
                          "flop_count": f"{near_fixed} per pair without the Miller start + {MILLER_FLOP_PER_STEP} per "
                                        f"rolled Miller step ({miller_steps} steps over {n_pairs} pairs, counted "
                                        f"by sbio_geom_near_work)",
                          "peak_source": fp64_peak_source(),
                          "timed_in": "the plain FP64 apply, phases in order" if prec == S.SBIO_MIXED else
                                      "this apply, phases in order"},
        "near_mixed": {"kernel": "near_kernel_mixed", "ms": near_mean,
                       "pairs_per_s": n_pairs / (near_mean * 1e-3),
                       "speedup_vs_fp64_near": (near64_ms / near_mean) if near64_ms else None,
                       "note": "coordinates, Miller sweep, Q order recurrence and angle recurrence in FP64; "
                               "rho = extS q rounded to FP32, normalised Ferrers recurrence and TwoSum-compensated "
                               "n and m sums in FP32"}
        if prec == S.SBIO_MIXED else None,
        "measured_peaks": peaks,
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
        tg = stratified_targets(near_count, args.oracle_sample)
        sec, nt, NN = oracle_sample_time(path, tg)
        per_apply = sec * NN / nt
        line["cpu_baseline"] = {"value": 1.0 / per_apply, "unit": "applies/s", "cores": 1, "kind": "oracle",
                                "cpu": cpu_model(),
                                "sample": f"{nt} of {NN} targets stratified by near-particle count ({sec:.1f} s), "
                                          f"scaled to a full apply"}
        cores = os.cpu_count() or 1
        if cores > 1 and not args.no_all_cores:
            tps, wall, nproc = oracle_all_cores(path, near_count, args.oracle_sample, cores)
            line["cpu_baseline_all_cores"] = {
                "value": tps / NN, "unit": "applies/s", "cores": nproc, "kind": "oracle", "cpu": cpu_model(),
                "sample": f"{nproc} concurrent single-threaded processes (os.cpu_count()), {args.oracle_sample} "
                          f"stratified targets each, disjoint ({wall:.1f} s wall), scaled to a full apply"}
    os.unlink(path)
    return line


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
    set_peak_basis(lrank, clk)
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
    # the same apply with the treecode far field (order 16, theta 0.5)
    S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, 0.5, 16)
    for _ in range(3):
        S.sbio_apply_stokes_sl(g.h, fd, u)
    tms = []
    for _ in range(args.steps):
        flush.zero_()
        tms.append(_event_time(st, lambda: S.sbio_apply_stokes_sl(g.h, fd, u)))
    ut = u.clone()
    S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_DIRECT)
    S.sbio_geom_set_precision(g.h, S.SBIO_FP64)
    S.sbio_apply_stokes_sl(g.h, fd, u)
    t64 = _event_time(st, lambda: S.sbio_apply_stokes_sl(g.h, fd, u))
    err = float((um - u).abs().max() / u.abs().max())
    tree_line = {"applies_per_s": 1e3 / statistics.mean(tms), "ms_per_step": statistics.mean(tms),
                 "rel_err_vs_fp64_gpu": float((ut - u).abs().max() / u.abs().max()),
                 "far_method": "particle treecode, 4 charge + 4 dipole channels, order 16, theta 0.5"}
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
                         "peak": fp32_peak(), "unit": "TFLOP/s", "frac": ach / fp32_peak(),
                         "flop_per_pair": STOKES_FAR_FLOP_PER_PAIR, "traffic": None},
            "fp64_gpu_applies_per_s": 1e3 / t64, "rel_err_vs_fp64_gpu": err, "tree": tree_line,
            "gpu_launches": int(launches), "clocks": clk}
    g.close()
    return line


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
    # the library's batch autotuner: far targets per thread, near CTA size, persistent grid
    t0 = time.perf_counter()
    best = S.sbio_batch_autotune(b, sig, mu, So, Do)
    tune_s = time.perf_counter() - t0
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
    set_peak_basis(lrank, clk)
    info = S.sbio_batch_info(b)
    # the same work as one apply per suspension, one after another (mixed)
    seq = _event_time(st, lambda: [S.sbio_apply_laplace(g.h, sig[k], mu[k], So[k], Do[k]) for k, g in enumerate(geoms)])
    Sd = [o.clone() for o in So]
    Dd = [o.clone() for o in Do]
    # the same batch with the treecode far field on every suspension
    for g in geoms:
        S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, 0.5, 16)
    bt = S.sbio_batch_create(ctx, geoms)
    for _ in range(3):
        S.sbio_batch_apply(bt, sig, mu, So, Do)
    tms = []
    for _ in range(args.steps):
        flush.zero_()
        tms.append(_event_time(st, lambda: S.sbio_batch_apply(bt, sig, mu, So, Do)))
    torch.cuda.synchronize()
    terr = {"S": max(float((a - b_).abs().max() / b_.abs().max()) for a, b_ in zip(So, Sd)),
            "D": max(float((a - b_).abs().max() / b_.abs().max()) for a, b_ in zip(Do, Dd))}
    tree_line = {"applies_per_s": len(geoms) * 1e3 / statistics.mean(tms), "ms_per_step": statistics.mean(tms),
                 "rel_err_vs_direct_mixed": terr,
                 "far_method": "particle treecode per suspension (order 16, theta 0.5), on the graph's branches"}
    S.sbio_batch_destroy(bt)
    for g in geoms:
        S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_DIRECT)
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
                       "persistent_grid": info["grid"],
                       "autotuned": {"far_targets_per_thread": best[0], "near_threads_per_cta": best[1],
                                     "far_ctas_per_sm": best[2], "step_ms": best[3], "tuner_s": tune_s},
                       "l2": "flushed by a 256 MiB write before every timed step"},
            "gpairs_per_s": info["far_pairs"] / (mean * 1e-3) / 1e9,
            "roofline": {"kernel": "whole step (far_persistent_kernel dominant)", "bound": "alu",
                         "achieved": FAR_FLOP_PER_PAIR["SD"] * info["far_pairs"] / (mean * 1e-3) / 1e12,
                         "peak": fp32_peak(), "unit": "TFLOP/s",
                         "frac": FAR_FLOP_PER_PAIR["SD"] * info["far_pairs"] / (mean * 1e-3) / 1e12 / fp32_peak(),
                         "flop_per_pair": FAR_FLOP_PER_PAIR["SD"], "traffic": None},
            "sequential_mixed_ms": seq, "fp64_plain_ms": f64, "fp64_plain_applies_per_s": len(geoms) * 1e3 / f64,
            "speedup_vs_fp64_plain": f64 / mean, "speedup_vs_sequential_mixed": seq / mean,
            "tree": tree_line,
            "gpu_launches": int(launches), "clocks": clk}
    S.sbio_batch_destroy(b)
    return line


def run_serve(args, ws, rank, lrank):
    """Served form: a Poisson stream of BIO-apply requests (Laplace S + D or
    Stokes single layer with probability 1/2, 10 applies each with fresh
    coefficients) into the library's continuous-batching server.  Every
    request brings its own geometry: a suspension of the pool (M log-uniform
    in [20, 500], p from {8, 12, 16}) moved by a seeded random rigid motion,
    so the server builds a new geometry for every request, inside the
    request's latency.  Rates span below and above the saturation knee; per
    rate the stream runs `--serve-seconds` of arrivals (at most `--requests`
    requests).  The plain FP64 server and the mixed server run the same
    eight requests submitted together (throughput at saturation)."""
    import queue
    import threading

    import numpy as np
    import torch

    from paper_2506_20809_gb300 import inputs as I

    pool = I.serve_pool(args.serve_pool, seed=0, workers=min(32, os.cpu_count() or 1))   # before CUDA starts
    import __graft_entry__ as GE

    GE.build()
    from paper_2506_20809_gb300 import sbio as S

    torch.cuda.set_device(lrank)
    ctx = S.sbio_ctx_create(lrank, 0)
    free, total = torch.cuda.mem_get_info()
    budget = int(0.5 * free)
    # ten coefficient sets per pool member, per operator (read-only, shared by its requests)
    crng = np.random.default_rng([rank, 4242])
    coefs = []
    for s in pool:
        lap = np.ascontiguousarray(np.stack([I.coefficients(crng, s.M, s.p, 2).transpose(1, 0, 2)
                                             for _ in range(10)]))
        sto = np.ascontiguousarray(np.stack([I.coefficients(crng, s.M, s.p, 3) for _ in range(10)]))
        coefs.append((lap, sto))

    def request(k, op_is_laplace):
        s = I.rigid_motion(pool[k % len(pool)], seed=k)
        sph = S.make_spheroids(s.kind, s.A, s.C, s.center, s.quat)
        N = s.M * (s.p + 1) * 2 * (s.p + 1)
        lap, sto = coefs[k % len(pool)]
        if op_is_laplace:
            return S.SBIO_OP_LAPLACE, sph, s.p, lap, (10, 2 * N)
        return S.SBIO_OP_STOKES, sph, s.p, sto, (10, N, 3)

    tree_flag = 0 if args.serve_direct else S.SBIO_REQ_TREE

    def run_stream(arrivals, precision, flags=None):
        """arrivals: list of (t, k, op_is_laplace).  Returns latencies (ms)
        and the makespan (s) from the first arrival to the last result."""
        srv = S.sbio_server_create(ctx, args.slots, budget)
        done = queue.Queue()
        lat = []

        def waiter():
            while True:
                item = done.get()
                if item is None:
                    return
                t, keep = item
                st, l, _ = S.sbio_server_wait(srv, t, 3600.0)
                assert st == 0, st
                lat.append(l)
                del keep                      # the request's host buffers can go now

        th = threading.Thread(target=waiter)
        th.start()
        prepared = [(ta,) + request(k, lapl) for ta, k, lapl in arrivals]
        t0 = time.perf_counter()
        for ta, op, sph, p, coef, oshape in prepared:
            delay = t0 + ta - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            out = np.empty(oshape)
            fl = (tree_flag if flags is None else flags) if precision == S.SBIO_MIXED else 0
            t = S.sbio_server_submit(srv, op, sph, p, coef, out, 10, precision=precision, flags=fl)
            done.put((t, (out, sph)))
        done.put(None)
        th.join()
        makespan = time.perf_counter() - t0
        S.sbio_server_destroy(srv)
        return sorted(lat), makespan

    rates = [float(x) for x in args.rates.split(",")]
    rows = []
    for rate in rates:
        reqs = I.poisson_requests(rate, args.serve_seconds, seed=7, max_requests=args.requests)
        arrivals = [(r["t"], r["seed"], r["op"] == "laplace") for r in reqs]
        lat, makespan = run_stream(arrivals, S.SBIO_MIXED)
        rows.append({"rate": rate, "requests": len(lat), "window_s": args.serve_seconds,
                     "applies_per_s": 10 * len(lat) / makespan,
                     "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                     "makespan_s": makespan})
    # the knee: the highest rate whose median latency stays within 1.5x of the lowest rate's
    base = rows[0]["p50_ms"]
    flat = [r["rate"] for r in rows if r["p50_ms"] <= 1.5 * base]
    sat = max(rows, key=lambda r: r["applies_per_s"])
    eight = [(0.0, 900 + k, k % 2 == 0) for k in range(8)]
    lat64, mk64 = run_stream(eight, S.SBIO_FP64)
    latm, mkm = run_stream(eight, S.SBIO_MIXED)
    latd, mkd = run_stream(eight, S.SBIO_MIXED, flags=0)
    line = {"metric": "served BIO applies/s (Poisson stream, 10 applies per request) and p50/p99 latency",
            "value": sat["applies_per_s"], "unit": "applies/s", "n_gpus": ws, "steps": len(rates),
            "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "serve", "slots": args.slots, "window_s_per_rate": args.serve_seconds,
                       "max_requests_per_rate": args.requests, "pool": [{"M": s.M, "p": s.p} for s in pool],
                       "request_geometry": "pool suspension moved by a seeded random rigid motion (new geometry "
                                           "built by the server inside every request's latency)",
                       "mem_budget_bytes": budget, "ops": "Laplace S+D or Stokes single layer, probability 1/2",
                       "laplace_far_field": "direct sum" if args.serve_direct else
                       "treecode (order 16, theta 0.5; SBIO_REQ_TREE), built inside each request"},
            "sweep": rows,
            "knee": {"flat_up_to_rate": max(flat), "p50_ms_at_lowest_rate": base,
                     "saturation_applies_per_s": sat["applies_per_s"]},
            "fp64_plain": {"requests": 8, "applies_per_s": 80 / mk64, "p50_ms": lat64[4]},
            "mixed_same_requests": {"requests": 8, "applies_per_s": 80 / mkm, "p50_ms": latm[4]},
            "mixed_direct_far_same_requests": {"requests": 8, "applies_per_s": 80 / mkd, "p50_ms": latd[4]},
            "speedup_vs_fp64_plain": mk64 / mkm}
    S.sbio_ctx_destroy(ctx)
    return line


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
    set_peak_basis(lrank, clk)
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
                         "peak": fp32_peak(), "unit": "TFLOP/s", "frac": ach / fp32_peak(),
                         "flop_per_pair": DERIV_FAR_FLOP_PER_PAIR,
                         "traffic": DERIV_FAR_DRAM_BYTES_POLY200.get((dtune[0], dtune[1])),
                         "traffic_unit": "bytes per launch (ncu dram read + write, one capture at this launch shape)"},
            "fp64_gpu_applies_per_s": 1e3 / t64, "rel_err_vs_fp64_gpu": err, "gpu_launches": int(launches),
            "clocks": clk}
    g.close()
    return line


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
    set_peak_basis(lrank, clk)
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
                         "achieved": ach, "peak": fp32_peak(), "unit": "TFLOP/s", "frac": ach / fp32_peak(),
                         "traffic": None},
            "fp64_gpu_points_per_s": ts.T * 1e3 / t64, "rel_err_vs_fp64_gpu": err, "gpu_launches": int(launches),
            "clocks": clk}
    ts.close()
    g.close()
    return line


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
    set_peak_basis(lrank, clk)
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
                         "peak": fp32_peak(), "unit": "TFLOP/s",
                         "frac": FAR_FLOP_PER_PAIR["SD"] * g.n_far * its / (ms * 1e-3) / 1e12 / fp32_peak(),
                         "flop_per_pair": FAR_FLOP_PER_PAIR["SD"], "traffic": None},
            "gpu_launches": int(launches), "clocks": clk}
    ts.close()
    g.close()
    return line


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
    set_peak_basis(lrank, clk)
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
                       # the double layer's near pairs run at the tuned cap but at least 4 CTAs per SM
                       "near_ctas_per_sm_overlapped": max(4, scap) if (dl and scap > 0) else scap,
                       "points_recipe": "shells at 1e-1..1e-6 (10 per spheroid and distance) + 30,000 in the box",
                       "l2": "flushed (256 MiB write) before each step"},
            "evaluations_per_s": 1e3 / mean, "fp64_gpu_points_per_s": ts.T * 1e3 / t64,
            "roofline": {"kernel": ("whole evaluation (stresslet_far_mixed_kernel dominant)" if dl else
                                    "whole evaluation (stokes_far_mixed_kernel with pressure dominant)"),
                         "bound": "alu",
                         "achieved": far_flop * ts.n_far / (mean * 1e-3) / 1e12,
                         "peak": fp32_peak(), "unit": "TFLOP/s",
                         "frac": far_flop * ts.n_far / (mean * 1e-3) / 1e12 / fp32_peak(),
                         "flop_per_pair": far_flop, "traffic": None},
            "rel_err_vs_fp64_gpu": err, "gpu_launches": int(launches), "clocks": clk}
    ts.close()
    g.close()
    return line


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
    set_peak_basis(lrank, clk)
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
                       "near_ctas_per_sm_overlapped": max(4, scap) if scap > 0 else scap,
                       "l2": "flushed (256 MiB write) before each step"},
            "phase_ms": {"prep_and_self": statistics.mean(x[0] for x in ph), "near": near_ms, "far": far_ms},
            "roofline": {"kernel": "stokes_dl_near_kernel (FP64 pipe)", "bound": "alu", "achieved": near_ach,
                         "peak": fp64_peak(), "unit": "TFLOP/s", "frac": near_ach / fp64_peak(),
                         "flop_per_pair": near_flop, "traffic": None,
                         "peak_source": "nominal GB300 FP64 1.25 TFLOP/s"},
            "roofline_far": {"kernel": "stresslet_far_mixed_kernel", "bound": "alu", "achieved": far_ach,
                             "peak": fp32_peak(), "unit": "TFLOP/s", "frac": far_ach / fp32_peak(),
                             "flop_per_pair": STRESSLET_FAR_FLOP_PER_PAIR, "traffic": None},
            "fp64_gpu_applies_per_s": 1e3 / t64, "rel_err_vs_fp64_gpu": err, "gpu_launches": int(launches),
            "clocks": clk}
    g.close()
    return line


def run_lattice8(args, ws, rank, lrank):
    """The 8-spheroid lattice at p = 8 (1296 targets) in plain FP64: a
    latency-bound apply; per-apply CUDA-event times give p50 / p99."""
    import torch

    from paper_2506_20809_gb300 import inputs as I

    import __graft_entry__ as GE

    GE.build()
    from paper_2506_20809_gb300 import sbio as S

    torch.cuda.set_device(lrank)
    susp = I.config_suspension(1)
    coef = I.config_coefficients(susp, 0)
    ctx = S.sbio_ctx_create(lrank, 0)
    g = S.Geometry(ctx, susp, precision=S.SBIO_FP64)
    sig, mu = torch.from_numpy(coef[0]).cuda(), torch.from_numpy(coef[1]).cuda()
    So = torch.empty(g.N, dtype=torch.float64, device="cuda")
    Do = torch.empty_like(So)
    st = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(3, args.warmup)):
        S.sbio_apply_laplace(g.h, sig, mu, So, Do)
    clocks = ClockSampler(lrank)
    clocks.start()
    steps = max(args.steps, 200)
    ms = []
    l0 = S.sbio_launch_count()
    for _ in range(steps):
        flush.zero_()
        ms.append(_event_time(st, lambda: S.sbio_apply_laplace(g.h, sig, mu, So, Do)))
    launches = S.sbio_launch_count() - l0
    clk = clocks.stop()
    set_peak_basis(lrank, clk)
    hs = torch.from_numpy(coef[0]).pin_memory().numpy()
    hm = torch.from_numpy(coef[1]).pin_memory().numpy()
    hS = torch.empty(g.N, dtype=torch.float64).pin_memory().numpy()
    hD = torch.empty(g.N, dtype=torch.float64).pin_memory().numpy()
    S.sbio_apply_laplace_host(g.h, hs, hm, hS, hD)
    e2e = []
    for _ in range(steps):
        t0 = time.perf_counter()
        S.sbio_apply_laplace_host(g.h, hs, hm, hS, hD)
        e2e.append((time.perf_counter() - t0) * 1e3)
    S.sbio_geom_set_precision(g.h, S.SBIO_MIXED)
    mixed = [_event_time(st, lambda: S.sbio_apply_laplace(g.h, sig, mu, So, Do)) for _ in range(50)]
    lat = sorted(ms)
    el = sorted(e2e)
    line = {"metric": "BIO applies/s (Laplace S+D, all surface nodes, plain FP64) and p50/p99 latency",
            "value": 1e3 / statistics.mean(ms), "unit": "applies/s", "n_gpus": ws, "steps": steps,
            "warmup": max(3, args.warmup), "ms_per_step": statistics.mean(ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "lattice8_p8_laplace_SD_fp64", "M": susp.M, "p": susp.p, "targets": g.N,
                       "near_pairs": g.n_near, "far_pairs_per_apply": g.n_far,
                       "l2": "flushed (256 MiB write) before each step"},
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
            "e2e": {"value": 1e3 / statistics.mean(e2e), "unit": "applies/s",
                    "h2d_bytes_per_step": int(hs.nbytes + hm.nbytes), "d2h_bytes_per_step": int(hS.nbytes + hD.nbytes),
                    "p50_ms": el[len(el) // 2], "p99_ms": el[min(len(el) - 1, int(0.99 * len(el)))]},
            "mixed_applies_per_s": 1e3 / statistics.mean(mixed),
            "gpu_launches": int(launches), "clocks": clk}
    g.close()
    S.sbio_ctx_destroy(ctx)
    return line


def _sweep_member(args):
    M, seed = args
    from paper_2506_20809_gb300 import inputs as I

    return I.rsa_suspension(M, 0.20, seed, 16, ar_range=(1.2, 5.0), name=f"poly{M}")


def run_far_sweep(args, ws, rank, lrank):
    """The poly200 recipe (AR U[1.2, 5], major U[0.5, 1.5], 20 %, gap 0.05,
    p = 16) at growing particle counts: the direct far field's time and pair
    rate per apply, and the whole mixed apply, to show where the O(N^2) sum
    stops being the kernel of choice."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import torch

    Ms = [int(x) for x in args.sweep_M.split(",")]
    with cf.ProcessPoolExecutor(max_workers=len(Ms), mp_context=mp.get_context("spawn")) as ex:
        susps = list(ex.map(_sweep_member, [(M, 0) for M in Ms]))   # before CUDA starts
    from paper_2506_20809_gb300 import inputs as I

    import __graft_entry__ as GE

    GE.build()
    from paper_2506_20809_gb300 import sbio as S

    torch.cuda.set_device(lrank)
    ctx = S.sbio_ctx_create(lrank, 0)
    st = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    rows = []
    clocks = ClockSampler(lrank)
    clocks.start()
    for susp in susps:
        coef = I.config_coefficients(susp, 0)
        g = S.Geometry(ctx, susp, precision=S.SBIO_MIXED)
        tune = S.sbio_geom_autotune(g.h)
        sig, mu = torch.from_numpy(coef[0]).cuda(), torch.from_numpy(coef[1]).cuda()
        So = torch.empty(g.N, dtype=torch.float64, device="cuda")
        Do = torch.empty_like(So)
        for _ in range(2):
            S.sbio_apply_laplace(g.h, sig, mu, So, Do)
        reps = 5 if g.n_far < 1e11 else 3
        whole = []
        for _ in range(reps):
            flush.zero_()
            whole.append(_event_time(st, lambda: S.sbio_apply_laplace(g.h, sig, mu, So, Do)))
        S.sbio_geom_enable_timing(g.h, True)
        far = []
        for _ in range(reps):
            flush.zero_()
            S.sbio_apply_laplace(g.h, sig, mu, So, Do)
            far.append(S.sbio_geom_phase_times(g.h)[2])
        S.sbio_geom_enable_timing(g.h, False)
        far_ms = statistics.median(far)
        Sd, Dd = So.clone(), Do.clone()
        row = {"M": susp.M, "targets": g.N, "near_pairs": g.n_near, "far_pairs": g.n_far,
               "far_launch": {"targets_per_thread": tune[0], "source_splits": tune[1]},
               "direct_far_ms": far_ms, "direct_gpairs_per_s": g.n_far / (far_ms * 1e-3) / 1e9,
               "apply_ms": statistics.median(whole),
               "far_frac_of_fp32_peak": FAR_FLOP_PER_PAIR["SD"] * g.n_far / (far_ms * 1e-3) / 1e12 / fp32_peak()}
        # the same applies with the treecode far field (order 16, theta 0.5)
        t0 = time.perf_counter()
        S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, 0.5, 16)
        build_ms = (time.perf_counter() - t0) * 1e3
        info = S.sbio_geom_tree_info(g.h)
        for _ in range(2):
            S.sbio_apply_laplace(g.h, sig, mu, So, Do)
        twhole = []
        for _ in range(reps):
            flush.zero_()
            twhole.append(_event_time(st, lambda: S.sbio_apply_laplace(g.h, sig, mu, So, Do)))
        S.sbio_geom_enable_timing(g.h, True)
        tfar, tph = [], []
        for _ in range(reps):
            flush.zero_()
            S.sbio_apply_laplace(g.h, sig, mu, So, Do)
            tfar.append(S.sbio_geom_phase_times(g.h)[2])
            tph.append(S.sbio_geom_tree_phase_times(g.h))
        S.sbio_geom_enable_timing(g.h, False)
        S.sbio_apply_laplace(g.h, sig, mu, So, Do)
        torch.cuda.synchronize()
        row["tree"] = {"order": 16, "theta": 0.5, "far_ms": statistics.median(tfar),
                       "apply_ms": statistics.median(twhole), "setup_ms": build_ms,
                       "speedup_far_vs_direct": far_ms / statistics.median(tfar),
                       "rel_err_vs_direct_mixed": {"S": float((So - Sd).abs().max() / Sd.abs().max()),
                                                   "D": float((Do - Dd).abs().max() / Dd.abs().max())},
                       "m2p_evaluations": info["m2p_pairs"], "direct_pairs": info["direct_pairs"],
                       "m2p_evaluations_by_order": S.sbio_geom_tree_order_counts(g.h, S.SBIO_OP_LAPLACE),
                       "near_ctas_per_sm_beside_tree": S.sbio_geom_get_tree_near_cap(g.h),
                       "direct_pair_fraction": info["direct_pairs"] / g.n_far, "tree_nodes": info["nodes"],
                       "phase_ms": dict(zip(("leaf_multipoles", "translations", "direct", "evaluations"),
                                            [statistics.median(x[k] for x in tph) for k in range(4)]))}
        # the Stokes single layer on the same suspension, direct and treecode
        S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_DIRECT)
        f = I.config_coefficients(susp, 1, ndens=3).transpose(1, 0, 2).copy()
        fd = torch.from_numpy(f).cuda()
        u = torch.empty((g.N, 3), dtype=torch.float64, device="cuda")
        S.sbio_apply_stokes_sl(g.h, fd, u)
        sd = []
        for _ in range(reps):
            flush.zero_()
            sd.append(_event_time(st, lambda: S.sbio_apply_stokes_sl(g.h, fd, u)))
        ud = u.clone()
        S.sbio_geom_set_far_method(g.h, S.SBIO_FAR_TREE, 0.5, 16)
        S.sbio_apply_stokes_sl(g.h, fd, u)
        stt = []
        for _ in range(reps):
            flush.zero_()
            stt.append(_event_time(st, lambda: S.sbio_apply_stokes_sl(g.h, fd, u)))
        torch.cuda.synchronize()
        row["stokes"] = {"direct_apply_ms": statistics.median(sd), "tree_apply_ms": statistics.median(stt),
                         "rel_err_tree_vs_direct_mixed": float((u - ud).abs().max() / ud.abs().max())}
        rows.append(row)
        g.close()
    clk = clocks.stop()
    set_peak_basis(lrank, clk)
    for r in rows:
        r["far_frac_of_fp32_peak"] = FAR_FLOP_PER_PAIR["SD"] * r["far_pairs"] / (r["direct_far_ms"] * 1e-3) / 1e12 / fp32_peak()
    big = rows[-1]
    line = {"metric": "Laplace S+D apply time vs suspension size (direct tiled far field and treecode, mixed)",
            "value": 1e3 / big["tree"]["apply_ms"], "unit": "applies/s", "n_gpus": ws, "steps": len(rows), "warmup": 2,
            "ms_per_step": big["tree"]["apply_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "far_sweep_p16", "M": Ms, "p": 16,
                       "geometry": "AR U[1.2,5], major U[0.5,1.5], phi=20%, gap>=0.05, RSA seed 0",
                       "l2": "flushed (256 MiB write) before each step"},
            "sweep": rows, "clocks": clk}
    S.sbio_ctx_destroy(ctx)
    return line


def _sub(fn, keys, *a, **k):
    """Run a secondary workload for the headline line and keep the keys a
    reader needs; a failure is recorded instead of losing the line."""
    try:
        line = fn(*a, **k)
    except Exception as e:   # noqa: BLE001
        return {"error": f"{type(e).__name__}: {e}"[:500]}
    return {key: line[key] for key in keys if key in line}


def main():
    args = parse()
    ws, rank, lrank = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        line = None
    elif args.workload == "stokes100":
        line = run_stokes100(args, ws, rank, lrank)
    elif args.workload == "batch64":
        line = run_batch64(args, ws, rank, lrank)
    elif args.workload == "serve":
        line = run_serve(args, ws, rank, lrank)
    elif args.workload == "deriv200":
        line = run_deriv200(args, ws, rank, lrank)
    elif args.workload == "targets200":
        line = run_targets200(args, ws, rank, lrank)
    elif args.workload == "derivpoints200":
        line = run_targets200(args, ws, rank, lrank, deriv=True)
    elif args.workload == "dirichlet200":
        line = run_dirichlet200(args, ws, rank, lrank)
    elif args.workload == "stokespoints100":
        line = run_stokespoints100(args, ws, rank, lrank)
    elif args.workload == "stokesdlpoints100":
        line = run_stokespoints100(args, ws, rank, lrank, dl=True)
    elif args.workload == "stokesdl100":
        line = run_stokesdl100(args, ws, rank, lrank)
    elif args.workload == "lattice8":
        line = run_lattice8(args, ws, rank, lrank)
    elif args.workload == "far_sweep":
        line = run_far_sweep(args, ws, rank, lrank)
    else:
        line = run_ours(args, ws, rank, lrank)
        if not args.headline_only:
            # the batched (64 suspensions per step), served (Poisson stream)
            # and Stokes single-layer forms, each beside its plain FP64 form
            line["batched"] = _sub(run_batch64, ["metric", "value", "unit", "ms_per_step", "gpairs_per_s",
                                                 "roofline", "fp64_plain_ms", "fp64_plain_applies_per_s",
                                                 "speedup_vs_fp64_plain", "speedup_vs_sequential_mixed",
                                                 "tree", "config"], args, ws, rank, lrank)
            line["served"] = _sub(run_serve, ["metric", "value", "unit", "sweep", "knee", "fp64_plain",
                                              "mixed_same_requests", "mixed_direct_far_same_requests",
                                              "speedup_vs_fp64_plain", "config"],
                                  args, ws, rank, lrank)
            line["stokes100"] = _sub(run_stokes100, ["metric", "value", "unit", "ms_per_step", "e2e", "roofline",
                                                     "fp64_gpu_applies_per_s", "rel_err_vs_fp64_gpu", "tree",
                                                     "config"],
                                     args, ws, rank, lrank)
            line["lattice8"] = _sub(run_lattice8, ["metric", "value", "unit", "ms_per_step", "latency_ms", "e2e",
                                                   "mixed_applies_per_s", "config"], args, ws, rank, lrank)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
