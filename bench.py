#!/usr/bin/env python3
"""Benchmark of the L-QSW time-series path on GB300.

One step = one pass of the whole path over one synthetic walk: build the
superoperator from the host graph (normalisation, CSR assembly, 1-norm series),
run the Al-Mohy--Higham series on the device (parameter choice, Taylor blocks,
populations).  Default workload: Erdos-Renyi digraph N = 1000, p = 0.01,
weights U(0.5, 1.5), omega = 0.3, uniform-superposition rho0, complex128,
50 steps of dt = 0.1 (superoperator 10^6 rows, ~4.07e7 nnz).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Metric: walk time-steps/s (output times of the series per second, whole job).
Walks are independent, so N > 1 runs one walk per rank (weak scaling, no
collective on the data path).  `--impl reference` times the FP64 CPU oracle on
a bounded sample of the same workload.
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

PROCESS_T0 = time.time()
ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "walk time-steps/s (L-QSW expmv series, whole path incl. superoperator build)"
UNIT = "time-steps/s"
WORKLOAD = "er1000"
SAMPLE_STEPS = 2   # output times of the oracle sample


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--warmup-seconds", type=float, default=0.0,
                    help="default line: keep warming up until this many seconds after process "
                         "start (in addition to --warmup steps)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--operator", default="matfree", choices=["matfree", "csr"],
                    help="how the series applies the superoperator")
    ap.add_argument("--no-csr-line", action="store_true",
                    help="skip the extra CSR-operator series measurement")
    ap.add_argument("--requests", type=int, default=2000, help="serve2000: number of requests")
    ap.add_argument("--walks", type=int, default=256, help="batch256: number of walks")
    ap.add_argument("--est-networks", type=int, default=4, help="est: dipole networks")
    ap.add_argument("--est-omegas", type=int, default=64, help="est: omega values per network")
    ap.add_argument("--est-precision", default="c128", choices=["c128", "c64"], help="est: precision")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "batch256", "serve2000", "grid45", "est", "gqsw", "nmgqsw"],
                    help="er1000: one walk per step (default); batch256: 256 random 4-regular "
                         "walks with 4 pure states each, complex64, one batched launch per step")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--grid-oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--batch-oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--serve-oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--record-traffic", metavar="NCU_CSV",
                    help="write profiles/series_kernel_er1000_traffic.json from an ncu --csv log")
    ap.add_argument("--record-command", default="", help="the ncu command the CSV came from")
    ap.add_argument("--profile-workload", default="er1000", choices=["er1000", "grid45"],
                    help="--profile-steps case: the ER-1000 walk or the 45x45 lattice")
    ap.add_argument("--profile-c128", action="store_true", help="grid45 profile case in complex128")
    ap.add_argument("--profile-fixed", action="store_true",
                    help="profile case without schedule tuning (QSW_BUILD_FIXED_SCHEDULE)")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="run one build + one series of this many output times and exit "
                         "(small case for ncu captures)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(x: float, device="cpu") -> float:
    """Max of a per-rank float over the process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps_per_walk: int, ms_per_step: float) -> float:
    """Whole-job time-steps/s: every rank runs its own walk (weak scaling), the
    job's step time is the slowest rank's."""
    return world * steps_per_walk * 1000.0 / ms_per_step


# ------------------------------------------------------------------ oracle --

def oracle_sample() -> dict:
    """Oracle as it stands on the ER-1000 workload: Kronecker assembly plus
    Algorithm 5.2 over the first SAMPLE_STEPS output times."""
    from oracle import expmv, graph, superop
    from paper_2003_02450_gb300 import workloads as W
    cfg = W.er1000()
    t = time.perf_counter()
    walk = graph.lqsw_walk(graph.adjacency(cfg.graph))
    L = superop.superoperator(walk, cfg.omega)
    X = expmv.expmv_series(L, W.vec(cfg.rho0), cfg.t0, cfg.dt, SAMPLE_STEPS)
    superop.populations(X, walk.n_tilde)
    sec = time.perf_counter() - t
    return {"seconds": sec, "steps": SAMPLE_STEPS}


def run_oracle_subprocess(flag: str = "--oracle-sample") -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    res = subprocess.run([sys.executable, os.path.abspath(__file__), flag],
                         capture_output=True, text=True, env=env, cwd=ROOT)
    if res.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + res.stderr[-2000:])
    return json.loads(res.stdout.strip().splitlines()[-1])


def oracle_all_cores(flag: str = "--oracle-sample", per_proc_gb: float = 4.0) -> dict:
    """The oracle sample run as one single-threaded process per host core, all
    at once (independent walks): aggregate throughput = processes x outputs /
    wall time.  The process count is bounded by the host's available memory
    (per_proc_gb each)."""
    cores = os.cpu_count() or 1
    try:
        with open("/proc/meminfo") as fh:
            avail_kb = next(int(l.split()[1]) for l in fh if l.startswith("MemAvailable"))
        cores = max(1, min(cores, int(avail_kb / 1e6 / per_proc_gb)))
    except (OSError, StopIteration, ValueError):
        pass
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    t = time.perf_counter()
    procs = [subprocess.Popen([sys.executable, os.path.abspath(__file__), flag],
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                              env=env, cwd=ROOT) for _ in range(cores)]
    outs = [pr.communicate() for pr in procs]
    wall = time.perf_counter() - t
    if any(pr.returncode for pr in procs):
        raise RuntimeError("oracle sample failed:\n" + outs[0][1][-1000:])
    samples = [json.loads(o[0].strip().splitlines()[-1]) for o in outs]
    return {"processes": cores, "wall_s": wall, "steps_each": samples[0]["steps"],
            "mean_process_s": statistics.mean(x["seconds"] for x in samples)}


def cpu_baseline_block(sample: dict) -> dict:
    return {"value": sample["steps"] / sample["seconds"], "unit": UNIT, "cores": 1,
            "kind": "oracle",
            "sample": (f"FP64 numpy/scipy oracle, single thread: Kronecker-product superoperator "
                       f"of the ER-1000 walk + Algorithm 5.2 over its first {sample['steps']} "
                       f"output times (dt=0.1), {sample['seconds']:.1f} s")}


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms.

    start() launches the sampler and waits until its first sample has arrived,
    so that nvidia-smi's own start-up (driver queries that can hold up the
    CUDA calls of the process being measured) is over before the caller's
    work; mark() records the start of the timed region, and stop() keeps only
    the samples taken after it."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None
        self.t_mark = None

    def start(self, settle_s: float = 5.0):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        t_end = time.time() + settle_s
        while time.time() < t_end and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)

    def mark(self):
        self.t_mark = time.time()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        import datetime
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            if self.t_mark is not None:
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    if ts < self.t_mark - 0.2:
                        continue
                except ValueError:
                    pass
            try:
                sm.append(float(parts[2]))
                smax.append(float(parts[3]))
            except ValueError:
                continue
            for name, v in zip(names, parts[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# -------------------------------------------------------------------- ours --

def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# FP64 FMA issue rate of GB300: 304 thread-FMAs per cycle for the whole GPU
# (2 per SM per clock; ncu sm__sass_thread_inst_executed_op_dfma_pred_on
# .sum.peak_sustained), 2 flops each, at the maximum SM clock.
DFMA_PER_CYCLE = 304


KERNEL_SOURCES = ["paper_2003_02450_gb300/csrc/series.cu", "paper_2003_02450_gb300/csrc/matfree.cuh",
                  "paper_2003_02450_gb300/csrc/params.cuh", "paper_2003_02450_gb300/csrc/gqsw.cuh"]


TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "series_kernel_er1000_traffic.json")


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def series_traffic():
    """DRAM bytes (read + write) of one full-size series launch, from the record
    written by `bench.py --record-traffic` out of an ncu capture, or None when
    the kernel sources changed since that capture."""
    try:
        with open(TRAFFIC_RECORD) as fh:
            rec = json.load(fh)
        if rec["kernel_sources_sha256"] != kernel_sources_sha256():
            return None
        return int(rec["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def record_traffic(csv_path: str, command: str) -> None:
    """Write TRAFFIC_RECORD from an ncu --csv log of the full-size bench command
    with the metrics dram__bytes_read.sum, dram__bytes_write.sum and
    gpu__time_duration.sum captured on the series kernel (-k regex:series_kernel)."""
    import csv
    rows = []
    with open(csv_path, newline="") as fh:
        lines = [ln for ln in fh if ln.startswith('"')]
    for r in csv.DictReader(lines):
        if "series_kernel" in r.get("Kernel Name", ""):
            rows.append(r)
    launches = {}
    for r in rows:
        v = float(r["Metric Value"].replace(",", ""))
        unit = r.get("Metric Unit", "")
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "B": 1, "KB": 1e3,
                 "MB": 1e6, "GB": 1e9, "ns": 1e-9, "us": 1e-6, "ms": 1e-3, "s": 1.0,
                 "nsecond": 1e-9, "usecond": 1e-6, "msecond": 1e-3, "second": 1.0}.get(unit, 1.0)
        launches.setdefault(r["ID"], {})[r["Metric Name"]] = v * scale
    if not launches:
        raise SystemExit(f"no series_kernel launch in {csv_path}")
    first = launches[sorted(launches, key=int)[0]]
    rec = {"kernel": "series_kernel (er1000 bench launch: 50 outputs, complex128, matrix-free)",
           "kernel_sources_sha256": kernel_sources_sha256(),
           "dram_bytes_read": int(first["dram__bytes_read.sum"]),
           "dram_bytes_write": int(first["dram__bytes_write.sum"]),
           "dram_bytes_per_launch": int(first["dram__bytes_read.sum"] + first["dram__bytes_write.sum"]),
           "gpu_time_duration_ms": first["gpu__time_duration.sum"] * 1e3,
           "command": command}
    with open(TRAFFIC_RECORD, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps(rec))


def csr_equivalent(nnz: int, n: int, peak_gbs: float, kernel_ms: float, matvecs: int) -> dict:
    """Time a CSR SpMV of the same superoperator would need at 100 % of the
    measured HBM bandwidth (complex128 values, int32 indices, one term read and
    one written, one output read and written), against the measured time per
    application of L~ in the series kernel."""
    b = nnz * (16 + 4) + (n + 1) * 4 + 2 * n * 16 + 2 * n * 16
    roof_ms = b / (peak_gbs * 1e9) * 1e3
    per_app = kernel_ms / max(1, matvecs)
    return {"csr_bytes_per_application": b, "csr_at_hbm_peak_ms": roof_ms,
            "ms_per_application": per_app, "ratio": roof_ms / per_app}


def fp64_peak_tflops():
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mhz = float(json.load(fh).get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    return DFMA_PER_CYCLE * 2 * mhz * 1e6 / 1e12


def run_ours(args):
    import numpy as np
    import torch
    from paper_2003_02450_gb300 import qsw as C
    from paper_2003_02450_gb300 import workloads as W

    rank, world, local_rank = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    cfg = W.er1000()
    N, n, q = cfg.graph.n, cfg.graph.n ** 2, cfg.steps
    stream = torch.cuda.current_stream(dev)
    ctx = C.qsw_create(local_rank, stream.cuda_stream)
    rho0 = torch.from_numpy(W.vec(cfg.rho0)).to(dev)
    out = torch.empty((q + 1, n), dtype=torch.complex128, device=dev)
    pops = torch.empty((q + 1, N), dtype=torch.float64, device=dev)

    def one_step():
        op = C.qsw_build_superoperator(ctx, cfg.graph, None, cfg.omega, precision="c128",
                                       operator=args.operator)
        st = C.qsw_expmv_series(ctx, op, rho0, cfg.t0, cfg.dt, q, out, pops)
        info = C.qsw_op_info(ctx, op)
        C.qsw_op_destroy(op)
        st["nnz"] = info["nnz"]
        return st

    # the clock sampler starts before the warm-up: its start-up is over before
    # the timed region, whose samples alone are kept
    sampler = ClockSampler(local_rank)
    sampler.start()
    warm = 0
    while warm < args.warmup or time.time() - PROCESS_T0 < args.warmup_seconds:
        one_step()
        warm += 1
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    sampler.mark()
    l0 = C.qsw_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    # L2 (129 MB) is flushed between timed steps by a 256 MB device-to-device
    # copy (the copy engine, cudaMemcpyAsync): a fill kernel of the framework
    # measured ~28 ms per call in the first process on a fresh box
    flush_src = torch.zeros(256 << 20, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    flush.copy_(flush_src)
    ev0.record(stream)
    stats = []
    for k in range(args.steps):
        if k:
            flush.copy_(flush_src)
        stats.append(one_step())
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    launches = (C.qsw_kernel_launches() - l0) / args.steps
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dev)
    value = job_value(world, q, ms)

    kern_ms = statistics.mean(s["kernel_ms"] for s in stats)
    alg_bytes = statistics.mean(s["algorithmic_bytes"] for s in stats)
    alg_flops = statistics.mean(s["algorithmic_flops"] for s in stats)
    peak, peak_kind = measured_peak_gbs()
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    fp64_peak = fp64_peak_tflops()
    achieved_tf = alg_flops / (kern_ms * 1e-3) / 1e12
    s0 = stats[0]

    # ---- the CSR-operator series on the same walk (secondary line)
    csr_line = None
    if not args.no_csr_line:
        op = C.qsw_build_superoperator(ctx, cfg.graph, None, cfg.omega, precision="c128",
                                       operator="csr")
        C.qsw_expmv_series(ctx, op, rho0, cfg.t0, cfg.dt, q, out, pops)
        cs = C.qsw_expmv_series(ctx, op, rho0, cfg.t0, cfg.dt, q, out, pops)
        C.qsw_op_destroy(op)
        csr_line = {"kernel_ms": cs["kernel_ms"], "matvecs": cs["matvecs"],
                    "bytes_per_matvec": cs["bytes_per_matvec"],
                    "achieved_gbs": cs["algorithmic_bytes"] / (cs["kernel_ms"] * 1e-3) / 1e9,
                    "achieved_tflops_fp64": cs["algorithmic_flops"] / (cs["kernel_ms"] * 1e-3) / 1e12,
                    "series_time_steps_per_s": q * 1000.0 / cs["kernel_ms"]}

    # ---- end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        h_rho0 = torch.from_numpy(W.vec(cfg.rho0)).pin_memory()
        h_out = torch.empty((q + 1, n), dtype=torch.complex128).pin_memory()
        h_pops = torch.empty((q + 1, N), dtype=torch.float64).pin_memory()

        def e2e_step():
            op = C.qsw_build_superoperator(ctx, cfg.graph, None, cfg.omega, precision="c128",
                                           operator=args.operator)
            C.qsw_expmv_series_host(ctx, op, h_rho0, cfg.t0, cfg.dt, q, h_out, h_pops)
            C.qsw_op_destroy(op)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        barrier()
        t0 = time.perf_counter()
        marks = []
        for _ in range(args.steps):
            e2e_step()   # returns with the step's results on the host
            marks.append(time.perf_counter())
        torch.cuda.synchronize(dev)
        e_ms = max_over_ranks((time.perf_counter() - t0) * 1000.0 / args.steps, dev)
        step_ms = [(y - x) * 1000.0 for x, y in zip([t0] + marks[:-1], marks)]
        g = cfg.graph
        h2d = g.rowptr.nbytes + g.col.nbytes + g.w.nbytes + h_rho0.numel() * 16
        d2h = h_out.numel() * 16 + h_pops.numel() * 8
        e2e = {"value": job_value(world, q, e_ms), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e_ms,
               "step_ms": [round(v, 2) for v in step_ms],
               "api": "qsw_build_superoperator + qsw_expmv_series_host (host buffers)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            single = cpu_baseline_block(run_oracle_subprocess())
            allc = oracle_all_cores()
            cpu = {"value": allc["processes"] * allc["steps_each"] / allc["wall_s"], "unit": UNIT,
                   "cores": allc["processes"], "kind": "oracle",
                   "sample": (f"FP64 numpy/scipy oracle, one single-threaded process per host core "
                              f"({allc['processes']} processes at once, independent walks): each "
                              f"the Kronecker superoperator of the ER-1000 walk + Algorithm 5.2 over "
                              f"its first {allc['steps_each']} output times; wall "
                              f"{allc['wall_s']:.1f} s, {allc['mean_process_s']:.1f} s per process"),
                   "single_core": single}
        except Exception as exc:   # reported, not fatal
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": str(exc)[:300]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128 (complex128 / FP64)",
            "data": "synthetic (seeded Erdos-Renyi digraph; the paper's graph sets are not available)",
            "config": {"workload": WORKLOAD, "graph": "Erdos-Renyi digraph N=1000 p=0.01 w~U(0.5,1.5)",
                       "omega": cfg.omega, "rho0": "uniform superposition (dense)",
                       "t0": cfg.t0, "dt": cfg.dt, "series_steps": q, "rows": n, "nnz": s0["nnz"],
                       "parallelism": f"replicas x{world} (one walk per GPU)",
                       "l2": "flushed between timed steps (256 MB device-to-device copy); each step also writes its 51 output states (816 MB)",
                       "warmup_steps_run": warm, "warmup_until_s_after_start": args.warmup_seconds},
            "roofline": {"bound": "alu", "pipe": "fp64",
                         "kernel": f"series_kernel ({args.operator} operator, fused Taylor update)",
                         "achieved": achieved_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": achieved_tf / fp64_peak,
                         "peak_source": "304 DFMA/cycle x 2 flop x max SM clock (ncu peak_sustained)",
                         "traffic": series_traffic() if args.operator == "matfree" else None, "traffic_unit": "bytes per launch (ncu dram read + write)", "algorithmic_flops_per_launch": alg_flops,
                         "kernel_ms": kern_ms,
                         "hbm_view": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                                      "frac": achieved / peak, "peak_source": peak_kind,
                                      "algorithmic_bytes_per_launch": alg_bytes},
                         # the CSR formulation's bytes per application (matrix +
                         # row pointers + term read/write + output update) at the
                         # measured HBM peak, against this kernel's time per application
                         "csr_equivalent": csr_equivalent(s0["nnz"], n, peak, kern_ms,
                                                          s0["matvecs"])},
            "csr_operator_series": csr_line,
            "series": {"m_star": s0["m_star"], "s": s0["s"], "outputs_per_block": s0["outputs_per_block"],
                       "matvecs": s0["matvecs"], "bytes_per_matvec": s0["bytes_per_matvec"],
                       "series_time_steps_per_s": q * 1000.0 / kern_ms,
                       "build_and_other_ms": ms - kern_ms},
            "gpu_launches": launches,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    C.qsw_destroy(ctx)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# --------------------------------------------------------------- reference --

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(min(args.warmup, 1)):   # one untimed sample: page in numpy/scipy
        run_oracle_subprocess()
    samples = [run_oracle_subprocess() for _ in range(args.steps)]
    sec = sum(s["seconds"] for s in samples)
    steps = sum(s["steps"] for s in samples)
    value = steps / sec
    cpu = cpu_baseline_block({"seconds": sec / len(samples), "steps": SAMPLE_STEPS})
    cpu["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sec / len(samples),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128 (complex128 / FP64)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_output_times": SAMPLE_STEPS},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_gqsw_workload(args):
    """G-QSW (Section 2.5.2: one global Lindblad operator L = G) on a directed
    Erdos-Renyi digraph, N = 400, p = 0.025, w ~ U(0.5, 1.5), omega = 0.3,
    uniform superposition, 50 steps of dt = 0.1, complex128.  One step = build
    (Q = -i(1-omega)H - omega/2 G^T G on the host, norms on the device) + the
    series with populations."""
    import numpy as np
    import torch
    from paper_2003_02450_gb300 import qsw as C
    from paper_2003_02450_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = C.qsw_create(0, stream.cuda_stream)
    g = W.erdos_renyi_digraph(400, 0.025, W.SEED_ER1000 + 1)
    omega, steps, dt = 0.3, 50, 0.1
    rho0 = torch.from_numpy(W.vec(W.uniform_superposition(400))).to(dev)
    pops = torch.empty((steps + 1, 400), dtype=torch.float64, device=dev)

    def step():
        op = C.qsw_build_gqsw(ctx, g, None, omega)
        st = C.qsw_expmv_series(ctx, op, rho0, 0.0, dt, steps, None, pops)
        C.qsw_op_destroy(op)
        return st

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(0)
    sampler.start()
    sampler.mark()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = C.qsw_kernel_launches()
    e0.record(stream)
    stats = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    launches = (C.qsw_kernel_launches() - l0) / args.steps
    C.qsw_destroy(ctx)
    s0 = stats[-1]
    peak = fp64_peak_tflops()
    achieved = s0["algorithmic_flops"] / (s0["kernel_ms"] * 1e-3) / 1e12
    cpu = None
    if not args.no_cpu_baseline:
        import time
        from oracle import expmv, gqsw
        t = time.perf_counter()
        walk = gqsw.global_walk(g.dense())
        L = gqsw.superoperator(walk, omega)
        expmv.expmv_series(L, W.vec(W.uniform_superposition(400)), 0.0, dt, 2)
        sec = time.perf_counter() - t
        cpu = {"value": 2.0 / sec, "unit": "time-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"Kronecker G-QSW superoperator + Algorithm 5.2 over the first 2 output "
                         f"times, {sec:.1f} s"}
    line = {"metric": "G-QSW walk time-steps/s (global Lindblad operator, whole path)",
            "value": steps * 1000.0 / ms, "unit": "time-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic (seeded Erdos-Renyi digraph)",
            "config": {"workload": "gqsw", "graph": "Erdos-Renyi digraph N=400 p=0.025",
                       "omega": omega, "series_steps": steps, "dt": dt},
            "roofline": {"bound": "alu", "pipe": "fp64", "kernel": "series_kernel (global walk)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak},
            "series": {"kernel_ms": s0["kernel_ms"], "matvecs": s0["matvecs"],
                       "m_star": s0["m_star"], "s": s0["s"]},
            "gpu_launches": launches, "clocks": clocks, "cpu_baseline": cpu}
    print(json.dumps(line))


def run_nm_workload(args):
    """NM-G-QSW (Section 2.5.2, Eq. nm_gqsw) of a directed Erdos-Renyi digraph,
    N = 60, p = 0.06, w ~ U(0.5, 1.5), demoralised to N^D = sum_v deg_{G^u}(v)
    copies; omega = 0.3, uniform vertex populations, 20 steps of dt = 0.1,
    complex128.  One step = demoralise + build + series + population map."""
    import numpy as np
    import torch
    from paper_2003_02450_gb300 import qsw as C
    from paper_2003_02450_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = C.qsw_create(0, stream.cuda_stream)
    g = W.erdos_renyi_digraph(60, 0.06, W.SEED_ER1000 + 2)
    omega, steps, dt = 0.3, 20, 0.1
    probe = C.qsw_build_nm_gqsw(ctx, g, omega)
    nd = C.qsw_op_info(ctx, probe)["n_tilde"]
    C.qsw_op_destroy(probe)
    state = torch.empty(nd * nd, dtype=torch.complex128, device=dev)
    pe = torch.empty((steps + 1, nd), dtype=torch.float64, device=dev)
    p = torch.empty((steps + 1, 60), dtype=torch.float64, device=dev)
    pops0 = np.full(60, 1.0 / 60)

    def step():
        op = C.qsw_build_nm_gqsw(ctx, g, omega)
        C.qsw_nm_initial_state(ctx, op, pops0, state)
        st = C.qsw_expmv_series(ctx, op, state, 0.0, dt, steps, None, pe)
        C.qsw_nm_populations(ctx, op, pe, steps + 1, p)
        C.qsw_op_destroy(op)
        return st

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(0)
    sampler.start()
    sampler.mark()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = C.qsw_kernel_launches()
    e0.record(stream)
    stats = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    launches = (C.qsw_kernel_launches() - l0) / args.steps
    C.qsw_destroy(ctx)
    s0 = stats[-1]
    peak = fp64_peak_tflops()
    achieved = s0["algorithmic_flops"] / (s0["kernel_ms"] * 1e-3) / 1e12
    cpu = None
    if not args.no_cpu_baseline:
        import time
        from oracle import expmv, gqsw, nm
        t = time.perf_counter()
        walk, vs = nm.nm_walk(g.dense())
        L = gqsw.superoperator(walk, omega)
        expmv.expmv_series(L, W.vec(nm.initial_state(pops0, vs)), 0.0, dt, 1)
        sec = time.perf_counter() - t
        cpu = {"value": 1.0 / sec, "unit": "time-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"demoralisation + Kronecker superoperator + Algorithm 5.2 over the first "
                         f"output time, {sec:.1f} s"}
    line = {"metric": "NM-G-QSW walk time-steps/s (demoralised digraph, whole path)",
            "value": steps * 1000.0 / ms, "unit": "time-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic (seeded Erdos-Renyi digraph)",
            "config": {"workload": "nmgqsw", "graph": "Erdos-Renyi digraph N=60 p=0.06",
                       "expanded_vertices": nd, "omega": omega, "series_steps": steps, "dt": dt},
            "roofline": {"bound": "alu", "pipe": "fp64", "kernel": "series_kernel (global walk)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak},
            "series": {"kernel_ms": s0["kernel_ms"], "matvecs": s0["matvecs"],
                       "m_star": s0["m_star"], "s": s0["s"]},
            "gpu_launches": launches, "clocks": clocks, "cpu_baseline": cpu}
    print(json.dumps(line))


def run_est_workload(args):
    """Expected-survival-time sweep (Section 4.1.4): `--est-networks` dipole
    networks of 10 points uniform in the unit ball (V = -d^-3, source and sink of
    rate 0.5), omega = k / `--est-omegas`, k = 1..; eta by Simpson over 600
    intervals of [0, 300] (1 - p_sink(300) < 1e-6).  One step = build every
    operator + one qsw_batch_survival_time launch (complex128).  The oracle times
    one walk of the sweep as the CPU baseline."""
    import numpy as np
    import torch
    from paper_2003_02450_gb300 import qsw as C
    from paper_2003_02450_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = C.qsw_create(0, stream.cuda_stream)
    walks = W.est_dipole(count=args.est_networks, omegas=args.est_omegas, t_end=300.0, q=600)
    rhos = [torch.from_numpy(W.vec(w["rho0"])).to(dev) for w in walks]

    def step():
        ops = [C.qsw_build_superoperator(ctx, w["graph"], w["H"], w["omega"], w["sources"],
                                         w["sinks"], precision=args.est_precision, defer_norms=True)
               for w in walks]
        etas, st = C.qsw_batch_survival_time(ctx, ops, rhos, [w["t_end"] for w in walks],
                                             [w["q"] for w in walks], [w["sink"] for w in walks])
        for o in ops:
            C.qsw_op_destroy(o)
        return etas, st

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(0)
    sampler.start()
    sampler.mark()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = C.qsw_kernel_launches()
    ev0.record(stream)
    res = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = (C.qsw_kernel_launches() - l0) / args.steps
    etas, s0 = res[-1]
    C.qsw_destroy(ctx)
    cpu = None
    if not args.no_cpu_baseline:
        cpu = est_cpu_baseline(walks, args.est_omegas)
    line = {"metric": "expected survival times/s (dipole networks, omega sweep, batched)",
            "value": len(walks) * 1000.0 / ms, "unit": "EST evaluations/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.est_precision, "data": "synthetic (seeded dipole networks in the unit ball)",
            "config": {"workload": "est", "networks": args.est_networks, "points": 10,
                       "omegas": args.est_omegas, "t_end": 300.0, "q": 600},
            "batch": {"norms_ms": s0["norms_ms"], "series_ms": s0["series_ms"],
                      "matvecs": s0["matvecs"], "clusters": s0["clusters"]},
            "eta": {"min": float(np.min(etas)), "max": float(np.max(etas)),
                    "first_network": [float(e) for e in etas[:args.est_omegas]]},
            "gpu_launches": launches, "clocks": clocks, "cpu_baseline": cpu}
    print(json.dumps(line))


def est_cpu_baseline(walks, omegas):
    """The oracle's survival time for one walk of each network (omega = 0.5),
    single thread; the rate is walks / total time."""
    import time
    from oracle import est, graph, superop
    from paper_2003_02450_gb300 import workloads as W
    sample = [w for k, w in enumerate(walks) if k % omegas == omegas // 2 - 1]
    t = time.perf_counter()
    for w in sample:
        walk = graph.lqsw_walk(graph.adjacency(w["graph"]), H=w["H"], sources=w["sources"],
                               sinks=w["sinks"])
        L = superop.superoperator(walk, w["omega"])
        est.survival_time(L, walk.n_tilde, W.vec(w["rho0"]), w["t_end"], w["q"], w["sink"])
    sec = time.perf_counter() - t
    return {"value": len(sample) / sec, "unit": "EST evaluations/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(sample)} walks (one per network, omega={sample[0]['omega']:.3f}): "
                      f"Kronecker superoperator + Algorithm 5.2 over 600 intervals + Simpson, "
                      f"{sec:.1f} s"}


def batch_oracle_sample(count: int = 6) -> dict:
    """Oracle as it stands on the first `count` walks of the batch256 workload:
    per walk the Kronecker superoperator and Algorithm 5.2 on its n x 4 block of
    initial states over 10 steps of 0.2 (populations of every output)."""
    import numpy as np
    from oracle import expmv, graph, superop
    from paper_2003_02450_gb300 import workloads as W
    walks = W.batch_regular(count=256)[:count]
    t = time.perf_counter()
    for g, omega, states in walks:
        walk = graph.lqsw_walk(graph.adjacency(g))
        L = superop.superoperator(walk, omega)
        B = np.stack([W.vec(x) for x in states], axis=1)
        X = expmv.expmv_series(L, B, 0.0, 0.2, 10, n0=4)
        np.real(X[:, np.arange(g.n) * (g.n + 1), :])
    return {"seconds": time.perf_counter() - t, "walks": count}


def serve_oracle_sample(budget_s: float = 20.0) -> dict:
    """Oracle as it stands replaying the serve2000 request list serially from the
    start (Kronecker superoperator + Algorithm 5.2 per request) until
    `budget_s` seconds have passed."""
    import numpy as np
    from oracle import expmv, graph, superop
    from paper_2003_02450_gb300 import workloads as W
    specs = W.serve_requests(count=2000)
    t = time.perf_counter()
    done = 0
    for sp in specs:
        g = W.erdos_renyi_mean_degree(sp["n"], 8.0, sp["graph_seed"])
        walk = graph.lqsw_walk(graph.adjacency(g))
        L = superop.superoperator(walk, sp["omega"])
        X = expmv.expmv_series(L, W.vec(W.basis_state(sp["n"], 0)), 0.0, sp["dt"], sp["steps"])
        superop.populations(X, walk.n_tilde)
        done += 1
        if time.perf_counter() - t >= budget_s:
            break
    return {"seconds": time.perf_counter() - t, "requests": done}


def run_batch_workload(args):
    """256 random 4-regular walks (N ~ U{16..512}), omega ~ U(0,1), 4 random pure
    states each, 10 steps of dt = 0.2.  One step = build the 256 operators from
    the host graphs + one batched series launch (complex64 bulk) with populations.
    Also times the plain complex128 single-walk form on the same walks (one
    series call per initial state) for the walks/s comparison."""
    import numpy as np
    import torch
    from paper_2003_02450_gb300 import qsw as C
    from paper_2003_02450_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = C.qsw_create(0, stream.cuda_stream)
    walks = W.batch_regular(count=args.walks)
    q, dt, n0 = 10, 0.2, 4
    rhos = [torch.from_numpy(np.concatenate([W.vec(s) for s in st])).to(dev) for _, _, st in walks]
    pops = [torch.empty((q + 1) * n0 * g.n, dtype=torch.float64, device=dev) for g, _, _ in walks]

    def batch_step():
        ops = [C.qsw_build_superoperator(ctx, g, None, om, precision="c64", defer_norms=True)
               for g, om, _ in walks]
        st = C.qsw_batch_series(ctx, ops, rhos, n0, [0.0] * len(walks), [dt] * len(walks),
                                [q] * len(walks), pops)
        for o in ops:
            C.qsw_op_destroy(o)
        return st

    for _ in range(max(1, args.warmup)):
        batch_step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(0)
    sampler.start()
    sampler.mark()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = C.qsw_kernel_launches()
    ev0.record(stream)
    stats = [batch_step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = (C.qsw_kernel_launches() - l0) / args.steps

    # plain complex128 single-walk form: one op per walk, one series per state
    out1 = {g.n: torch.empty((q + 1) * g.n, dtype=torch.float64, device=dev) for g, _, _ in walks}
    def single_step():
        for (g, om, st), rho in zip(walks, rhos):
            op = C.qsw_build_superoperator(ctx, g, None, om, precision="c128")
            n = g.n * g.n
            for c in range(n0):
                C.qsw_expmv_series(ctx, op, rho[c * n:(c + 1) * n], 0.0, dt, q, None, out1[g.n])
            C.qsw_op_destroy(op)
    single_step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    single_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    single_ms = e0.elapsed_time(e1)
    # the same single-walk calls with every operator (and its 1-norm series)
    # built before the timed region: the series alone, no build cost at all
    ops1 = [C.qsw_build_superoperator(ctx, g, None, om, precision="c128") for g, om, _ in walks]

    def single_series():
        for (g, _, _), op, rho in zip(walks, ops1, rhos):
            n = g.n * g.n
            for c in range(n0):
                C.qsw_expmv_series(ctx, op, rho[c * n:(c + 1) * n], 0.0, dt, q, None, out1[g.n])
    single_series()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    single_series()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    series_only_ms = e0.elapsed_time(e1)
    for op in ops1:
        C.qsw_op_destroy(op)
    C.qsw_destroy(ctx)
    cpu = None
    if not args.no_cpu_baseline:
        try:
            smp = run_oracle_subprocess("--batch-oracle-sample")
            cpu = {"value": smp["walks"] / smp["seconds"], "unit": "walks/s", "cores": 1,
                   "kind": "oracle",
                   "sample": f"FP64 numpy/scipy oracle, single thread, on a fixed subset: the first "
                             f"{smp['walks']} of the 256 walks (Kronecker superoperator + "
                             f"Algorithm 5.2 on the n x 4 block, 10 steps), {smp['seconds']:.1f} s; "
                             f"walks/s extrapolated from that subset"}
        except Exception as exc:   # reported, not fatal
            cpu = {"value": None, "unit": "walks/s", "cores": 1, "kind": "oracle",
                   "error": str(exc)[:300]}
    s0 = stats[-1]
    line = {"metric": "walks/s (256 random 4-regular walks x 4 pure states, 10 steps, batched)",
            "value": len(walks) * 1000.0 / ms, "unit": "walks/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 bulk (complex64 terms, FP64 Taylor sums / norms / (m,s))",
            "data": "synthetic (seeded random 4-regular graphs)",
            "config": {"workload": "batch256", "walks": len(walks), "rhs_per_walk": n0,
                       "steps": q, "dt": dt, "clusters": s0["clusters"]},
            "batch": {"norms_ms": s0["norms_ms"], "series_ms": s0["series_ms"],
                      "matvecs": s0["matvecs"], "fupdates": s0["fupdates"],
                      "schedule": {"cluster_size": s0["cluster_size"],
                                   "small_limit_bytes": s0["small_limit"],
                                   "how": "autotuned on the first (warm-up) step: every "
                                          "candidate (clusters of 4/8/16 CTAs x one-CTA "
                                          "limit 0/32/64 KB) timed on this batch"}},
            "roofline": {
                "bound": "latency (FP32 operator products + FP64 output sums, L2-resident terms)",
                "kernel": "batch_series_kernel + batch_small_kernel (series phase)",
                "achieved_tflops": s0["algorithmic_flops"] / (s0["series_ms"] * 1e-3) / 1e12,
                "hbm_view_gbs": s0["algorithmic_bytes"] / (s0["series_ms"] * 1e-3) / 1e9,
                "hbm_peak_gbs": measured_peak_gbs()[0],
                "hbm_frac": s0["algorithmic_bytes"] / (s0["series_ms"] * 1e-3) / 1e9 / measured_peak_gbs()[0],
                "algorithmic_flops_per_step": s0["algorithmic_flops"],
                "algorithmic_bytes_per_step": s0["algorithmic_bytes"]},
            "single_walk_c128": {"ms": single_ms, "walks_per_s": len(walks) * 1000.0 / single_ms,
                                 "what": "per walk: build (incl. its 1-norm series) + one "
                                         "qsw_expmv_series per initial state"},
            "single_walk_c128_series_only": {
                "ms": series_only_ms, "walks_per_s": len(walks) * 1000.0 / series_only_ms,
                "what": "the same series calls with every operator built before the timed "
                        "region (no build or norm cost, unlike the batched step)"},
            "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line))


def run_serve_workload(args):
    """Request stream: ER digraphs with mean out-degree 8, N log-uniform in
    [32, 1024], omega ~ U(0,1), 1..100 output times of dt = 0.1, complex64 /
    complex128 50/50, rho0 = |0><0|.  First the capacity (all requests submitted
    at once), then Poisson arrivals at 0.5x and 0.9x that capacity and at a fixed 60 requests/s; latency =
    submit -> populations on the host."""
    import threading
    import numpy as np
    from paper_2003_02450_gb300 import qsw as C
    from paper_2003_02450_gb300 import workloads as W
    specs = W.serve_requests(count=args.requests)
    graphs = {}

    def make(spec):
        g = graphs.get(spec["graph_seed"])
        if g is None:
            g = W.erdos_renyi_mean_degree(spec["n"], 8.0, spec["graph_seed"])
            graphs[spec["graph_seed"]] = g
        return C.Request(g, spec["omega"], 0.0, spec["dt"], spec["steps"], spec["precision"],
                         populations=np.eye(1, spec["n"])[0])

    def run(rate):
        srv = C.qsw_server_create(0, workers=4, max_batch=64)
        reqs = [make(sp) for sp in specs]
        rng = np.random.default_rng(123)
        gaps = rng.exponential(1.0 / rate, size=len(reqs)) if rate else np.zeros(len(reqs))
        t_start = time.perf_counter()

        def producer():
            t = time.perf_counter()
            for r, gap in zip(reqs, gaps):
                t += gap
                delay = t - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                C.qsw_server_submit(srv, r)
        th = threading.Thread(target=producer)
        th.start()
        th.join()
        lat = [C.qsw_server_wait(srv, r, 3600.0)["latency_ms"] for r in reqs]
        wall = time.perf_counter() - t_start
        st = C.qsw_server_stats(srv)
        C.qsw_server_destroy(srv)
        return {"requests": len(reqs), "wall_s": wall, "throughput_rps": len(reqs) / wall,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "batches": st["batches"]}

    run(None) if args.warmup else None          # warm-up: page in, fill the memory pool
    cap = run(None)
    loads = {}
    for load in (0.5, 0.9):
        loads[str(load)] = run(load * cap["throughput_rps"])
    # one fixed absolute rate, so that runs with different capacities compare
    loads["60rps"] = run(60.0)
    cpu = None
    if not args.no_cpu_baseline:
        try:
            smp = run_oracle_subprocess("--serve-oracle-sample")
            cpu = {"value": smp["requests"] / smp["seconds"], "unit": "requests/s", "cores": 1,
                   "kind": "oracle",
                   "sample": f"FP64 numpy/scipy oracle, single thread, replaying the request list "
                             f"serially from its start: {smp['requests']} requests in "
                             f"{smp['seconds']:.1f} s"}
        except Exception as exc:   # reported, not fatal
            cpu = {"value": None, "unit": "requests/s", "cores": 1, "kind": "oracle",
                   "error": str(exc)[:300]}
    line = {"metric": "served walk requests/s and p50/p99 latency (Poisson arrivals)",
            "value": cap["throughput_rps"], "unit": "requests/s", "n_gpus": 1,
            "steps": 1, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "mixed c64 bulk / c128 (50/50)",
            "data": "synthetic (seeded Erdos-Renyi digraphs, mean out-degree 8)",
            "config": {"workload": "serve2000", "requests": len(specs), "N": "log-uniform [32, 1024]",
                       "steps": "U{1..100}", "dt": 0.1, "workers": 4, "max_batch": 64},
            "capacity": cap, "offered_load": loads, "cpu_baseline": cpu}
    print(json.dumps(line))


def grid_oracle_sample(steps: int) -> dict:
    """Oracle as it stands on the 45 x 45 lattice: Kronecker assembly plus
    Algorithm 5.2 over the first `steps` output times of its grid."""
    from oracle import expmv, graph, superop
    from paper_2003_02450_gb300 import workloads as W
    cfg = W.grid45("c128")
    t = time.perf_counter()
    walk = graph.lqsw_walk(graph.adjacency(cfg.graph))
    L = superop.superoperator(walk, cfg.omega)
    X = expmv.expmv_series(L, W.vec(cfg.rho0), cfg.t0, cfg.dt, steps)
    superop.populations(X, walk.n_tilde)
    return {"seconds": time.perf_counter() - t, "steps": steps}


def run_grid_workload(args):
    """45 x 45 lattice (N = 2025, n = 4.1e6), omega = 0.1, rho0 = |centre><centre|,
    20 steps of dt = 0.5: complex64 bulk (FP64 sums) and complex128, whole path
    per step (build + series + populations).  The complex64 result's population
    error is reported per output time against the FP64 oracle's stored series
    (tests/golden/grid45_series.npz, written by the oracle alone) and against
    the complex128 run."""
    import numpy as np
    import torch
    from paper_2003_02450_gb300 import qsw as C
    from paper_2003_02450_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = C.qsw_create(0, stream.cuda_stream)
    out, final_pops = {}, {}
    fp64_peak = fp64_peak_tflops()
    peak_gbs, peak_kind = measured_peak_gbs()
    sampler = ClockSampler(0)
    sampler.start()
    sampler.mark()
    for prec in ("c64", "c128"):
        cfg = W.grid45(prec)
        rho0 = torch.from_numpy(W.vec(cfg.rho0)).to(dev)
        pops = torch.empty((cfg.steps + 1, 2025), dtype=torch.float64, device=dev)

        def step():
            op = C.qsw_build_superoperator(ctx, cfg.graph, None, cfg.omega, precision=prec,
                                           operator=args.operator)
            st = C.qsw_expmv_series(ctx, op, rho0, cfg.t0, cfg.dt, cfg.steps, None, pops)
            info = C.qsw_op_info(ctx, op)
            st["lanes_per_row"], st["unroll"] = C.qsw_op_schedule(op, with_unroll=True)
            C.qsw_op_destroy(op)
            st["nnz"] = info["nnz"]
            return st
        for _ in range(max(1, args.warmup)):
            step()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = [step() for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / args.steps
        s0 = stats[-1]
        kms = statistics.mean(x["kernel_ms"] for x in stats)
        tf = s0["algorithmic_flops"] / (kms * 1e-3) / 1e12
        out[prec] = {"time_steps_per_s": cfg.steps * 1000.0 / ms, "ms_per_step": ms,
                     "series_kernel_ms": kms, "build_and_other_ms": ms - kms,
                     "matvecs": s0["matvecs"], "m_star": s0["m_star"], "s": s0["s"],
                     "operator": args.operator,
                     "roofline": {"bound": "alu" if args.operator == "matfree" or prec == "c128" else "hbm",
                                  "pipe": "fp64" if prec == "c128" else "fp32 + fp64",
                                  "achieved_tflops": tf, "fp64_peak_tflops": fp64_peak,
                                  "frac_of_fp64_peak": tf / fp64_peak,
                                  "hbm_view_gbs": s0["algorithmic_bytes"] / (kms * 1e-3) / 1e9,
                                  "hbm_frac": s0["algorithmic_bytes"] / (kms * 1e-3) / 1e9 / peak_gbs,
                                  "hbm_peak_gbs": peak_gbs, "hbm_peak_source": peak_kind,
                                  "algorithmic_bytes_per_launch": s0["algorithmic_bytes"],
                                  "bytes_per_term_spmv": s0["bytes_per_matvec"]},
                     "csr_lanes_per_row": s0["lanes_per_row"] or None,
                     "csr_unroll": s0["unroll"] or None,
                     "csr_equivalent": csr_equivalent(s0["nnz"], 2025 ** 2, peak_gbs, kms,
                                                      s0["matvecs"])}
        final_pops[prec] = pops.cpu().numpy()
    clocks = sampler.stop()
    C.qsw_destroy(ctx)
    # accuracy of the complex64 bulk result, per output time
    acc = {}
    try:
        g = np.load(os.path.join(ROOT, "tests", "golden", "grid45_series.npz"))
        e_or = np.max(np.abs(final_pops["c64"] - g["pops"]), axis=1)
        e_c128_or = np.max(np.abs(final_pops["c128"] - g["pops"]), axis=1)
        acc["c64_pop_err_vs_oracle_per_output"] = [float(x) for x in e_or]
        acc["c64_pop_err_vs_oracle_max"] = float(e_or.max())
        acc["c128_pop_err_vs_oracle_max"] = float(e_c128_or.max())
    except OSError:
        acc["oracle_series"] = "tests/golden/grid45_series.npz not found"
    e_c = np.max(np.abs(final_pops["c64"] - final_pops["c128"]), axis=1)
    acc["c64_pop_err_vs_c128_per_output"] = [float(x) for x in e_c]
    acc["bound"] = "c64 populations <= 1e-4; c128 <= 1e-10 (tests/test_gpu_full_series.py)"
    cpu = None
    if not args.no_cpu_baseline:
        try:
            smp = run_oracle_subprocess("--grid-oracle-sample")
            cpu = {"value": smp["steps"] / smp["seconds"], "unit": UNIT, "cores": 1,
                   "kind": "oracle",
                   "sample": f"FP64 numpy/scipy oracle, single thread: Kronecker superoperator of "
                             f"the 45x45 lattice walk + Algorithm 5.2 over its first "
                             f"{smp['steps']} output times (dt=0.5), {smp['seconds']:.1f} s"}
        except Exception as exc:   # reported, not fatal
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": str(exc)[:300]}
    print(json.dumps({"metric": "walk time-steps/s (45x45 lattice, 20 steps of 0.5)",
                      "value": out["c64"]["time_steps_per_s"], "unit": "time-steps/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": out["c64"]["ms_per_step"], "higher_is_better": True,
                      "dtype": "c64 bulk (complex64 terms, FP64 Taylor sums / norms / (m,s)); "
                               "c128 beside it", "data": "synthetic (45x45 lattice)",
                      "config": {"workload": "grid45", "N": 2025, "omega": 0.1, "dt": 0.5,
                                 "series_steps": 20, "operator": args.operator},
                      "c64": out["c64"], "c128": out["c128"], "accuracy": acc,
                      "cpu_baseline": cpu, "clocks": clocks}))


def run_profile_case(args):
    """One series call for profilers: the ER-1000 walk (complex128) or the 45 x 45
    lattice (--profile-workload grid45, complex64 bulk unless --profile-c128),
    over the first --profile-steps output times, with --operator."""
    import torch
    from paper_2003_02450_gb300 import qsw as C
    from paper_2003_02450_gb300 import workloads as W
    q = args.profile_steps
    if args.profile_workload == "grid45":
        prec = "c128" if args.profile_c128 else "c64"
        cfg = W.grid45(prec)
    else:
        prec = "c128"
        cfg = W.er1000()
    dev = torch.device("cuda", 0)
    ctx = C.qsw_create(0, torch.cuda.current_stream(dev).cuda_stream)
    rho0 = torch.from_numpy(W.vec(cfg.rho0)).to(dev)
    out = torch.empty((q + 1, cfg.graph.n ** 2), dtype=torch.complex128, device=dev)
    op = C.qsw_build_superoperator(ctx, cfg.graph, None, cfg.omega, precision=prec,
                                   operator=args.operator, fixed_schedule=args.profile_fixed)
    st = C.qsw_expmv_series(ctx, op, rho0, cfg.t0, cfg.dt, q, out, None)
    lanes, unroll = C.qsw_op_schedule(op, with_unroll=True)
    C.qsw_op_destroy(op)
    C.qsw_destroy(ctx)
    print(json.dumps({"profile_case": cfg.name, "precision": prec, "operator": args.operator,
                      "series_steps": q, "matvecs": st["matvecs"], "kernel_ms": st["kernel_ms"],
                      "algorithmic_bytes": st["algorithmic_bytes"], "csr_lanes_per_row": lanes,
                      "csr_unroll": unroll,
                      "schedule_measurements": C.qsw_tune_measurements()}))


def main():
    args = parse_args()
    if args.profile_steps:
        run_profile_case(args)
        return
    if args.oracle_sample:
        print(json.dumps(oracle_sample()))
        return
    if args.grid_oracle_sample:
        print(json.dumps(grid_oracle_sample(2)))
        return
    if args.batch_oracle_sample:
        print(json.dumps(batch_oracle_sample()))
        return
    if args.serve_oracle_sample:
        print(json.dumps(serve_oracle_sample()))
        return
    if args.record_traffic:
        record_traffic(args.record_traffic, args.record_command)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch256":
        run_batch_workload(args)
        return
    if args.workload == "serve2000":
        run_serve_workload(args)
        return
    if args.workload == "grid45":
        run_grid_workload(args)
        return
    if args.workload == "est":
        run_est_workload(args)
        return
    if args.workload == "gqsw":
        run_gqsw_workload(args)
        return
    if args.workload == "nmgqsw":
        run_nm_workload(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
