#!/usr/bin/env python
"""Benchmark of the coherent F-statistic template loop on one GB300 (or N).

One step = one pass of the whole path over one segment: segment preparation
(time/ephemeris tables, Fourier x2 upsampling, spline) followed by the coarse
search of every template (resample/demodulate per sky, two-pass zero-padded
transform per template, F on every bin up to Nyquist, candidate compaction).
Workload "grid_2d": 2 sidereal days at dt = 2 s (N = 86,164 float32 samples),
Nfft = 2^18, 256 sky positions x 16 spindowns in [-1e-8, 0] Hz/s, F written
for all 2^17 bins (4096 x 512 KiB), candidates above F = 20; seeded white
noise with 4 simulated signals.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1003_0844_gb300 import workloads as W  # noqa: E402

METRIC = "F-stat templates/s (N=86,164, 2^18 FFT) on 1 GB300; % HBM roofline; max rel dF vs FP64"
METRICS = {
    "grid_2d": METRIC,
    "wide_6d": "F-stat templates/s (N=1,033,968, 2^21 FFT) on 1 GB300; max rel dF vs FP64",
    "uneven_64": "F-stat templates/s (64 segments of 1/2/3/6 days, 2^16-2^20 FFT) on 1 GB300",
    "grid_2d_ib": "F-stat templates/s (N=86,164, 2^17 FFT + interbinning) on 1 GB300; max rel dF vs FP64",
    "refine_2d": "fine-search candidates/s (20 Newton steps on the exact F, N=86,164) on 1 GB300",
    "adjoint_2d": ("adjoint fine-search candidates/s (F of the resampled series and dF/d(f0, f1, delta, alpha) "
                   "recomputing the series, 20 quasi-Newton steps, N=86,164) on 1 GB300"),
    "lattice_2d": "F-stat templates/s (N=86,164, 2^18 FFT, constrained A4* lattice of a sky patch) on 1 GB300",
}

# the constrained-lattice workload: the 2-day data of grid_2d and the A4* lattice of a
# sky patch (Sec. IV), built by the library's host functions
LATTICE_BOX = W.LATTICE_BOX
LATTICE_MATCH = W.LATTICE_MATCH


def metric_name(workload: str) -> str:
    """The metric string of a named workload (test-size workloads get a descriptive one)."""
    if workload in METRICS:
        return METRICS[workload]
    if workload in W.BATCHES:
        return "F-stat templates/s (%s batch of segments) on 1 GB300" % workload
    wl = W.WORKLOADS[workload]
    return "F-stat templates/s (N=%d, 2^%d FFT, %s) on 1 GB300" % (wl.n, wl.nfft.bit_length() - 1, workload)


REFINE_FLOP_PER_SAMPLE = 5540.0  # FP32 flops per sample and point of a climb pass: F and gradient
                                 # (1514) and the Hessian's 46 sums computed once (4026), from ncu's
                                 # FADD/FFMA/FMUL counts (profiles/k_points_refine_2d.md); the
                                 # per-signal Hessian kernels' recomputation is not counted
ADJOINT_FLOP_PER_SAMPLE = 424.0  # FP32 flops per output sample and point of the adjoint's backward
                                 # kernel (F and the 26 sums of its gradient), from ncu's FADD/FFMA/FMUL
                                 # counts (profiles/k_resampled_refine_2d.md)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x FMA x max SM clock


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1, help="GPUs (one process each under torchrun)")
    p.add_argument("--steps", type=int, default=100, help="timed steps")
    p.add_argument("--warmup", type=int, default=5, help="untimed warm-up steps (at least 3 for a valid number)")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"],
                   help="ours: the CUDA library; reference: the CPU oracle on the host cores")
    p.add_argument("--workload", default="grid_2d",
                   help="grid_2d (default), grid_2d_ib, wide_6d, lattice_2d, refine_2d, adjoint_2d, a batch (uneven_64, "
                        "uneven_small) or a test-size workload (tiny, small)")
    p.add_argument("--cpu-templates", type=int, default=320,
                   help="oracle sample size: templates of the 2-day size per 20 host cores (~10 s)")
    p.add_argument("--fp64-skies", type=int, default=16,
                   help="skies of the plain FP64 form comparison (the FP32 error is taken over all their templates)")
    p.add_argument("--quick", action="store_true", help="skip the CPU baseline and FP64 comparison")
    p.add_argument("--nsky", type=int, default=None, help="override the sky count (profiling runs, batch sky subset)")
    p.add_argument("--tune", action="store_true", help="run the launch tuner for each transform length first")
    p.add_argument("--n1", type=int, default=0, help="first-pass length N1 of the transform split (0: default)")
    p.add_argument("--cands", type=int, default=1024,
                   help="fine-search and adjoint workloads: candidates refined per step")
    p.add_argument("--stub", action="store_true",
                   help="launcher self-test on the CPU: every rank takes its sky shard and reports it over gloo; "
                        "no GPU work")
    return p.parse_args()


def _free_port() -> int:
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def launch_ranks(args):
    """--gpus N: one process per GPU.  Under torchrun (WORLD_SIZE set) the world size
    must equal N.  Without it and N > 1, this script re-runs itself under
    torch.distributed.run with N ranks on this node (rendezvous on 127.0.0.1) and
    returns their exit status; None means: run here as the only rank or as a rank."""
    ws = os.environ.get("WORLD_SIZE")
    if ws is not None:
        if int(ws) != args.gpus:
            raise SystemExit("bench.py: WORLD_SIZE=%s but --gpus %d" % (ws, args.gpus))
        return None
    if args.gpus <= 1:
        return None
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(args.gpus),
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def run_stub(args):
    """Launcher self-test without a GPU: each rank takes its sky shard of the workload
    exactly as the GPU path does, the shards and a per-rank time go through gloo, and
    rank 0 prints the line the GPU path would print with the shard of every rank."""
    import torch.distributed as dist
    from paper_1003_0844_gb300 import shard
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        dist.init_process_group("gloo")
    wl = W.WORKLOADS[args.workload]
    mine = shard.sky_shard(wl.nsky, rank, world)
    parts = [mine.tolist()]
    if world > 1:
        parts = [None] * world
        dist.all_gather_object(parts, mine.tolist())
    ms = shard.max_over_ranks(1.0 + rank)
    if rank == 0:
        print(json.dumps({"metric": metric_name(args.workload), "value": None, "unit": "templates/s",
                          "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                          "stub": True, "rank_shards": parts,
                          "config": {"workload": wl.name, "nsky": wl.nsky, "nspin": wl.nspin,
                                     "parallelism": "sky shards x%d" % world}}), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _profile_traffic(kernel_profile: str):
    """DRAM bytes per template of the persistent kernel from the committed ncu summary,
    or None when the kernel's sources changed since that capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", kernel_profile)
    if not os.path.exists(path):
        return None, "no profile"
    fields = {}
    for line in open(path):
        if ":" in line and line.split(":")[0] in ("traffic_bytes_per_template", "kernel_sources_sha256",
                                                  "kernel_sources"):
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    try:
        h = hashlib.sha256()
        for f in fields["kernel_sources"].split():
            h.update(open(os.path.join(ROOT, f), "rb").read())
    except (KeyError, OSError):
        return None, "profile incomplete"
    if h.hexdigest() != fields.get("kernel_sources_sha256"):
        return None, "kernel changed since the ncu capture"
    return float(fields["traffic_bytes_per_template"]), "ncu capture, scaled by templates per launch"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(device), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cufft_comparison(nfft, nbins, reps=10):
    """cuFFT (through torch.fft), timed for comparison only, on the transforms a
    template needs: two zero-padded complex series of length nfft per template
    (chirp and padding already applied: not timed), batched C2C FP32 FFT, the same
    followed by F on nbins bins from |X|^2 with PyTorch elementwise kernels, and the
    batched Z2Z FP64 FFT (beside the plain FP64 form).  Each batch is larger than
    L2.  Returns templates/s for each."""
    import torch

    def timed(fn, B):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return {"value": B * reps / (e0.elapsed_time(e1) / 1e3), "unit": "templates/s", "batch_templates": B}

    out = {}
    g = torch.Generator(device="cuda").manual_seed(7)
    for dt, esz in ((torch.complex64, 8), (torch.complex128, 16)):
        B = max(4, (256 << 20) // (2 * nfft * esz))
        x = torch.randn((B, 2, nfft), dtype=dt, device="cuda", generator=g)
        X = torch.empty_like(x)
        if dt == torch.complex64:
            F = torch.empty((B, nbins), dtype=torch.float32, device="cuda")
            w = torch.tensor([0.6, 0.4], dtype=torch.float32, device="cuda").view(1, 2, 1)
            out["fft_only"] = timed(lambda: torch.fft.fft(x, dim=-1, out=X), B)

            def fft_and_F():
                torch.fft.fft(x, dim=-1, out=X)
                torch.sum(torch.view_as_real(X[..., :nbins]).square().sum(-1) * w, dim=1, out=F)

            out["fft_and_F"] = timed(fft_and_F, B)
            del F
        else:
            out["fft_only_fp64"] = timed(lambda: torch.fft.fft(x, dim=-1, out=X), B)
        del x, X
    out["note"] = ("cuFFT via torch.fft, batched C2C FP32 (and Z2Z FP64) of 2 x %d points per template; "
                   "chirp and zero padding not timed (an upper bound on a cuFFT-based search)" % nfft)
    return out


# ------------------------------------------------------------------ the oracle on the host cores
def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_worker_init():
    import oracle.adjoint, oracle.fstat, oracle.refine, oracle.resample  # noqa: F401  (imports before any timed region)


def _oracle_worker_ready(_):
    return os.getpid()


def _oracle_templates(task):
    """One worker's share of a sample, the oracle as it stands: its own preparation
    of the segment, then F of its templates (FFT mode; items are (alpha, delta, f1,
    bin offset or None))."""
    x, wl, det, items = task
    from oracle import fstat as ofs, resample as ors
    seg = ors.Segment(np.asarray(x, dtype=np.float64), wl.dt)
    for a, d, f, off in items:
        if getattr(wl, "interbin", False):
            ofs.fstat_interbinned(seg, a, d, f, wl.fl, det, wl.S0, wl.nfft)
        elif off is None:
            ofs.fstat(seg, a, d, f, wl.fl, det, wl.S0, wl.nfft)
        else:
            ofs.fstat(seg, a, d, f, wl.fl, det, wl.S0, wl.nfft, bin_offset=off)
    return len(items)


def _oracle_points(task):
    """One worker's share of fine-search work: exact-F passes with gradient and
    Hessian at points (kind "pass"), Nelder-Mead climbs from points ("climb"), or the
    resampled F with its gradient at points after the worker's own segment
    preparation ("adjoint")."""
    kind, x, dt, pts, fl, det, S0 = task
    from oracle import adjoint as oad, refine as orf, resample as ors
    seg = ors.Segment(np.asarray(x, dtype=np.float64), dt) if kind == "adjoint" else None
    for p in pts:
        if kind == "pass":
            orf.fstat_point(np.asarray(x), dt, p, fl, det, S0, grad=True, hess=True)
        elif kind == "adjoint":
            oad.resampled_fstat_point(seg, p, fl, det, S0, grad=True)
        else:
            orf.fine_search(np.asarray(x), dt, p, fl, det, S0)
    return len(pts)


class OraclePool:
    """The oracle as it stands on every host core: one worker process per core
    (started with spawn, so no CUDA state is inherited), BLAS/OpenMP threads at one
    per worker.  Work is dealt round-robin; a timed call is one pool.map."""

    def __init__(self, cores: int | None = None):
        import multiprocessing as mp
        self.cores = int(cores or host_cores())
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(k, "1")
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init)
        self.pool.map(_oracle_worker_ready, range(self.cores), chunksize=1)  # every worker up

    def deal(self, items):
        return [items[i::self.cores] for i in range(self.cores) if items[i::self.cores]]

    def templates(self, tasks):
        """tasks: [(x, wl, det, items)], one per worker -> (templates, seconds)."""
        t0 = time.perf_counter()
        n = sum(self.pool.map(_oracle_templates, tasks, chunksize=1))
        return n, time.perf_counter() - t0

    def points(self, tasks):
        t0 = time.perf_counter()
        n = sum(self.pool.map(_oracle_points, tasks, chunksize=1))
        return n, time.perf_counter() - t0

    def record(self, value, unit, sample):
        return {"value": value, "unit": unit, "cores": self.cores, "cpu": host_cpu_model(), "kind": "oracle",
                "sample": sample}

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_grid_baseline(x, wl, det, alpha, delta, f1, ntempl):
    """cpu_baseline of a grid workload: ntempl templates of the grid (sky-major)
    dealt over the host cores, each worker preparing the segment itself."""
    items = [(float(alpha[s]), float(delta[s]), float(f1[m]), None) for s in range(len(alpha))
             for m in range(len(f1))][:ntempl]
    pool = OraclePool()
    try:
        n, secs = pool.templates([(x, wl, det, it) for it in pool.deal(items)])
        return pool.record(n / secs, "templates/s", "%d templates (FFT mode) over %d worker processes, each with its "
                           "own segment preparation, %.1f s" % (n, pool.cores, secs))
    finally:
        pool.close()


def _grid_config(wl, nsky, nspin, world):
    """config of a single-segment workload (both arms)."""
    return {"workload": wl.name, "n": wl.n, "nfft": wl.nfft, "nsky": nsky, "nspin": nspin,
            "templates_per_gpu": nsky * nspin, "nbins": wl.nbins, "F_thr": wl.F_thr, "F_written": True,
            "l2": "flushed between timed steps (256 MiB write)", "parallelism": "sky shards x%d" % world}


def _lattice_config(wl, nsky, nspin, world):
    """config of the constrained-lattice workload (both arms)."""
    return {"workload": "lattice_2d", "n": wl.n, "nfft": wl.nfft, "nsky": nsky, "nspin": nspin,
            "templates_per_gpu": nsky * nspin // world, "nbins": wl.nbins, "F_thr": wl.F_thr, "F_written": True,
            "lattice": "constrained A4*, minimal match %.2f, sky patch n_x in [%.2f, %.2f], n_y in [%.2f, %.2f]"
                       % ((LATTICE_MATCH,) + LATTICE_BOX),
            "l2": "flushed between timed steps (256 MiB write)", "parallelism": "sky rows dealt over %d ranks" % world}


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on every host core (one worker
    process per core), each step a bounded sample of the workload dealt over the
    workers, each worker preparing its segment itself (grid and lattice workloads:
    templates of the grid; batches: one template of each segment kind per worker;
    the fine search: exact-F passes with gradient and Hessian, 1/21 of a
    candidate's climb each)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import earth as oe, response as orsp
    metric, unit = metric_name(args.workload), "templates/s"
    pool = OraclePool()
    C = pool.cores
    if args.workload in W.BATCHES:
        b = W.BATCHES[args.workload]
        det = W.detector_for(b)
        kinds = {}
        for wl, t0 in zip(b.segments(), b.epochs()):
            kinds.setdefault((wl.days, wl.nfft), (wl, float(t0)))
        a_all, d_all = W.sky_grid(b.nsky)
        f1 = W.spin_grid(b.nspin, *b.f1_range)
        tasks = []
        for wl, t0 in kinds.values():
            dk = oe.detector_at_epoch(det, t0)
            x = (W.noise(wl) + orsp.inject(wl.n, wl.dt, W.injections(wl), wl.fl, dk, wl.sigma)).astype(np.float32)
            tasks += [(x, wl, dk, [(float(a_all[i % b.nsky]), float(d_all[i % b.nsky]), float(f1[0]), None)])
                      for i in range(C)]

        def sample():
            return pool.templates(tasks)[0]
        nsub = min(args.nsky or 64, b.nsky)
        config = {"workload": args.workload, "segments": len(b.segments()),
                  "segment_kinds": [list(p) for p in b.parts], "dt": b.dt, "nsky": nsub, "nsky_lattice": b.nsky,
                  "nspin": b.nspin, "templates_per_gpu": len(b.segments()) * nsub * b.nspin, "F_thr": b.F_thr,
                  "F_written": False, "l2": "flushed between timed steps (256 MiB write)",
                  "parallelism": "sky shards x%d" % args.gpus, "graph": "one CUDA graph per batch, two branches"}
        what = "one template of each of the %d segment kinds with its preparation, on each of %d workers" % (
            len(kinds), C)
        per_unit = 1.0
    elif args.workload == "lattice_2d":
        from oracle import grid as og
        wl = W.WORKLOADS["grid_2d"]
        det = W.detector_for(wl)
        x = (W.noise(wl) + orsp.inject(wl.n, wl.dt, W.injections(wl), wl.fl, det, wl.sigma)).astype(np.float32)
        G = og.linear_model_fisher(wl.n, wl.dt, det)
        B, _, _ = og.constrained_lattice(G, LATTICE_MATCH, 2 * math.pi / (wl.nfft * wl.dt))
        T = og.lattice_templates(B, det, wl.fl, wl.nfft, wl.dt, *wl.f1_range, box=LATTICE_BOX)
        tm = [(float(al), float(de), float(fr), float(dr)) for al, de, rows in T for fr, dr, _ in rows]
        per_worker = 16
        tasks = [(x, wl, det, it) for it in pool.deal(tm[:per_worker * C])]

        def sample():
            return pool.templates(tasks)[0]
        config = _lattice_config(wl, len(T), max(len(r) for _, _, r in T), args.gpus)
        what = "%d lattice templates (FFT mode) over %d workers, each with its own segment preparation" % (
            min(len(tm), per_worker * C), C)
        per_unit = 1.0
    elif args.workload == "refine_2d":
        wl = W.WORKLOADS["grid_2d"]
        det = W.detector_for(wl)
        x = (W.noise(wl) + orsp.inject(wl.n, wl.dt, W.injections(wl), wl.fl, det, wl.sigma)).astype(np.float64)
        inj = W.injections(wl)[0]
        th = np.array([inj.f0, inj.f1, inj.alpha, inj.delta])
        tasks = [("pass", x, wl.dt, [th], wl.fl, det, wl.S0) for _ in range(C)]

        def sample():
            return pool.points(tasks)[0]
        metric, unit = METRICS["refine_2d"], "candidates/s"
        config = {"workload": "refine_2d", "n": wl.n, "candidates": args.cands, "newton_steps": 20,
                  "coarse": "grid_2d search (256 sky x 16 spindowns), strongest %d crossings" % args.cands,
                  "l2": "flushed between timed steps (256 MiB write)", "parallelism": "sky shards x%d" % args.gpus}
        what = "one exact-F pass with gradient and Hessian on each of %d workers (a candidate's climb takes 21)" % C
        per_unit = 1.0 / 21.0
    elif args.workload == "adjoint_2d":
        wl = W.WORKLOADS["grid_2d"]
        det = W.detector_for(wl)
        x = (W.noise(wl) + orsp.inject(wl.n, wl.dt, W.injections(wl), wl.fl, det, wl.sigma)).astype(np.float32)
        inj = W.injections(wl)[0]
        th = np.array([inj.f0, inj.f1, inj.alpha, inj.delta])
        tasks = [("adjoint", x, wl.dt, [th, th], wl.fl, det, wl.S0) for _ in range(C)]

        def sample():
            return pool.points(tasks)[0]
        metric, unit = METRICS["adjoint_2d"], "candidates/s"
        config = _adjoint_config(wl, args.cands, args.gpus)
        what = ("two evaluations of the resampled F and its gradient after the segment's preparation on each of "
                "%d workers (a candidate's 20 steps take 21)" % C)
        per_unit = 1.0 / 21.0
    else:
        wl = W.WORKLOADS[args.workload]
        det = W.detector_for(wl)
        x = (W.noise(wl) + orsp.inject(wl.n, wl.dt, W.injections(wl), wl.fl, det, wl.sigma)).astype(np.float32)
        alpha, delta = W.sky_grid(wl.nsky)
        f1 = W.spin_grid(wl.nspin, *wl.f1_range)
        per_worker = max(1, int(16 * 86164 / wl.n))
        items = [(float(alpha[s]), float(delta[s]), float(f1[m]), None) for s in range(len(alpha))
                 for m in range(len(f1))][:per_worker * C]
        tasks = [(x, wl, det, it) for it in pool.deal(items)]

        def sample():
            return pool.templates(tasks)[0]
        config = _grid_config(wl, wl.nsky, wl.nspin, args.gpus)
        what = "%d templates (FFT mode) over %d workers, each with its own segment preparation" % (len(items), C)
        per_unit = 1.0
    try:
        for _ in range(args.warmup):
            sample()
        t0 = time.perf_counter()
        total = 0
        for _ in range(args.steps):
            total += sample()
        wall = time.perf_counter() - t0
    finally:
        pool.close()
    value = total * per_unit / wall
    config["sample_per_step"] = what
    line = {
        "impl": "reference", "metric": metric, "value": value, "unit": unit, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": pool.record(value, unit, "%s per step, %d steps" % (what, args.steps)),
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main_batch(args):
    """One step = reload every segment of the batch (preparation) + the batched search
    of the same sky/spindown grid in all of them (candidates only)."""
    import torch
    import torch.distributed as dist
    from paper_1003_0844_gb300 import build, fstat as fs, shard

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    b = W.BATCHES[args.workload]
    det = W.detector_for(b)
    ctx = fs.Context(det, device=local)
    segs_wl, t0s = b.segments(), b.epochs()
    xs, segs = [], []
    for wl, t0 in zip(segs_wl, t0s):
        x64 = torch.as_tensor(W.noise(wl), device="cuda")
        fs.inject(ctx, x64, wl.dt, wl.fl, wl.sigma, W.injections(wl), t0=float(t0))
        x32 = x64.float().contiguous()
        xs.append(x32)
        segs.append(fs.Segment(ctx, x32, wl.dt, wl.nfft, wl.fl, wl.S0, t0=float(t0)))
    nsky_sub = min(args.nsky or 64, b.nsky)   # sky subset of the batch's lattice (templates/s is per template)
    a_all, d_all = W.sky_grid(b.nsky)
    mine = shard.sky_shard(nsky_sub, rank, world)
    alpha = torch.as_tensor(np.ascontiguousarray(a_all[mine]), device="cuda")
    delta = torch.as_tensor(np.ascontiguousarray(d_all[mine]), device="cuda")
    f1 = torch.as_tensor(W.spin_grid(b.nspin, *b.f1_range), device="cuda")
    nsky, nspin, nseg = alpha.numel(), f1.numel(), len(segs)
    ntempl = nseg * nsky * nspin
    cap = 1 << 20  # candidates per segment (16 MiB each)
    cand = torch.empty((nseg, cap, 4), dtype=torch.int32, device="cuda")
    ncand = torch.zeros(nseg, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    tuning = {}
    if args.tune:
        for s in sorted({wl.nfft for wl in segs_wl}):
            i = [wl.nfft for wl in segs_wl].index(s)
            tuning[str(s)] = ctx.autotune(segs[i], alpha[:min(nsky, 32)].contiguous(),
                                          delta[:min(nsky, 32)].contiguous(), f1)

    def step():
        for sg, x in zip(segs, xs):
            sg.load(x)
        fs.search_batch(ctx, segs, alpha, delta, f1, b.F_thr, cand=cand, n_cand=ncand, cand_cap=cap)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    ctx.check()
    ctx.stats(reset=True)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    stats = ctx.stats(reset=True)
    ctx.check()
    total_ms = shard.max_over_ranks(sum(a.elapsed_time(c) for a, c in ev), device="cuda")
    ms_per_step = total_ms / args.steps
    value = ntempl * world / (ms_per_step / 1e3)
    # whole-step FP32 rate: 2 transforms of 5 Nfft log2 Nfft flops per template
    flops = sum(2 * 5 * wl.nfft * math.log2(wl.nfft) for wl in segs_wl) * nsky * nspin
    achieved = flops / (ms_per_step / 1e3) / 1e12
    hbm_gbs, hbm_kind = _peaks()
    line = {
        "metric": metric_name(args.workload), "value": value, "unit": "templates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64/double-float phases)", "data": "synthetic",
        "config": {"workload": args.workload, "segments": nseg,
                   "segment_kinds": [list(p) for p in b.parts], "dt": b.dt, "nsky": nsky, "nsky_lattice": b.nsky,
                   "nspin": nspin, "templates_per_gpu": ntempl, "F_thr": b.F_thr, "F_written": False,
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": "sky shards x%d" % world,
                   "graph": "one CUDA graph per batch, two branches"},
        "roofline": {"kernel": "whole step (graph of demodulation + persistent transform launches)",
                     "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                     "traffic_note": "not captured for the batch graph",
                     "peak_kind": "FP32 CUDA-core peak from unit counts and max clock (152 SM x 128 x 2 x 2070 MHz)",
                     "flop_convention": "5 Nfft log2 Nfft per complex FFT, 2 FFTs per template"},
        "hbm_peak_gbs": hbm_gbs, "hbm_peak_kind": hbm_kind,
        "gpu_launches": int(stats["launches"]),
        "clocks": ck,
        "n_candidates": int(ncand.sum().item()),
    }
    if tuning:
        line["tuning"] = tuning
    if rank == 0 and not args.quick:
        # the oracle on the host cores: one template of each segment kind per worker, each
        # worker preparing its segment (the kinds are equally frequent in the batch, so the
        # sample follows its mix)
        from oracle import earth as oe
        f1h = W.spin_grid(b.nspin, *b.f1_range)
        kinds_seen, tasks = set(), []
        pool = OraclePool()
        for i, wl in enumerate(segs_wl):
            if (wl.days, wl.nfft) in kinds_seen:
                continue
            kinds_seen.add((wl.days, wl.nfft))
            dk = oe.detector_at_epoch(det, float(t0s[i]))
            xh_k = xs[i].cpu().numpy()
            tasks += [(xh_k, wl, dk, [(float(a_all[mine][0]), float(d_all[mine][0]), float(f1h[c % len(f1h)]), None)])
                      for c in range(pool.cores)]
        try:
            done, secs = pool.templates(tasks)
            line["cpu_baseline"] = pool.record(done / secs, "templates/s",
                                               "one template of each of the %d segment kinds on each of %d workers, "
                                               "preparation included, %.1f s" % (len(kinds_seen), pool.cores, secs))
        finally:
            pool.close()
        # end to end: pinned host data of every segment -> device, load, batch, candidates -> host
        xh = [torch.empty(x.numel(), dtype=torch.float32).pin_memory() for x in xs]
        for h, x in zip(xh, xs):
            h.copy_(x.cpu())
        nc_h = torch.empty(nseg, dtype=torch.int64).pin_memory()
        ke = max(2, args.steps)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        d2h = 0
        for _ in range(ke):
            for h, x, sg in zip(xh, xs, segs):
                x.copy_(h, non_blocking=True)
                sg.load(x)
            fs.search_batch(ctx, segs, alpha, delta, f1, b.F_thr, cand=cand, n_cand=ncand, cand_cap=cap)
            nc_h.copy_(ncand, non_blocking=True)
            torch.cuda.synchronize()
            got = [cand[i, :min(int(nc_h[i]), cap)].cpu() for i in range(nseg)]  # the stored candidates
            d2h = nseg * 8 + sum(g.numel() * 4 for g in got)
        e2e_s = (time.perf_counter() - t1) / ke
        line["e2e"] = {"value": ntempl / e2e_s, "unit": "templates/s",
                       "h2d_bytes_per_step": sum(x.numel() * 4 for x in xs), "d2h_bytes_per_step": d2h}
    else:
        line.setdefault("e2e", None)
        line.setdefault("cpu_baseline", None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    for sg in segs:
        sg.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def main_refine(args):
    """Fine search (config 4): the coarse 2-day search gives candidates (untimed);
    one step = starting points from 1024 candidates + 20 Newton steps of the exact F."""
    import torch
    import torch.distributed as dist
    from paper_1003_0844_gb300 import build, fstat as fs, shard

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    wl = W.WORKLOADS["grid_2d"]
    det = W.detector_for(wl)
    ctx = fs.Context(det, device=local)
    x64 = torch.as_tensor(W.noise(wl), device="cuda")
    fs.inject(ctx, x64, wl.dt, wl.fl, wl.sigma, W.injections(wl))
    x32 = x64.float().contiguous()
    a_all, d_all = W.sky_grid(wl.nsky * world)
    mine = shard.sky_shard(wl.nsky, rank, world)
    alpha = torch.as_tensor(np.ascontiguousarray(a_all[mine]), device="cuda")
    delta = torch.as_tensor(np.ascontiguousarray(d_all[mine]), device="cuda")
    f1 = torch.as_tensor(W.spin_grid(wl.nspin, *wl.f1_range), device="cuda")
    seg = fs.Segment(ctx, x32, wl.dt, wl.nfft, wl.fl, wl.S0)
    res = fs.search(ctx, seg, alpha, delta, f1, wl.F_thr, write_F=False, cand_cap=1 << 20)
    ncand_all = min(int(res.n_cand.item()), res.cand.shape[0])
    # the 1024 strongest crossings
    Fc = res.cand[:ncand_all, 3].view(torch.float32)
    top = torch.argsort(Fc, descending=True)[:args.cands]
    cand = res.cand[top].contiguous()
    npt, nsteps = cand.shape[0], 20

    def step():
        pts = fs.points_from_candidates(ctx, seg, cand, npt, alpha, delta, f1)
        return fs.refine(ctx, seg, pts, nsteps=nsteps)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    ctx.check()
    ctx.stats(reset=True)
    stream = torch.cuda.current_stream()
    steps = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    clocks = Clocks(local)
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        out, Fr = step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    stats = ctx.stats(reset=True)
    ctx.check()
    total_ms = shard.max_over_ranks(sum(a.elapsed_time(c) for a, c in ev), device="cuda")
    ms_per_step = total_ms / steps
    value = npt * world / (ms_per_step / 1e3)
    F0 = fs.fstat_points(ctx, seg, fs.points_from_candidates(ctx, seg, cand, npt, alpha, delta, f1), grad=False)[0]
    gain = (Fr / F0).cpu().numpy()
    flops = REFINE_FLOP_PER_SAMPLE * wl.n * npt * (nsteps + 1)
    achieved = flops / (ms_per_step / 1e3) / 1e12
    line = {
        "metric": METRICS["refine_2d"], "value": value, "unit": "candidates/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 double-float sums, FP64 orbital phase", "data": "synthetic",
        "config": {"workload": "refine_2d", "n": wl.n, "candidates": npt, "newton_steps": nsteps,
                   "coarse": "grid_2d search (256 sky x 16 spindowns), strongest 1024 crossings",
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": "sky shards x%d" % world},
        "roofline": {"kernel": "k_points_h + k_points_fg (double-float sums on the FP32 pipe, 21 passes per step)",
                     "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                     "peak_kind": "FP32 CUDA-core peak from unit counts and max clock (152 SM x 128 x 2 x 2070 MHz)",
                     "flop_convention": "%d FP32 flop per sample and point per pass (ncu opcode counts of the two "
                                        "kernels; the whole step's time)" % REFINE_FLOP_PER_SAMPLE},
        "gpu_launches": int(stats["launches"]),
        "clocks": ck,
        "F_gain": {"median": float(np.median(gain)), "max": float(np.max(gain))},
    }
    # the adjoint: the coarse search's F at the starting points (forward) and gF dF/dtheta
    # (backward, recomputing the resampled series), each timed over the same steps
    pts0 = fs.points_from_candidates(ctx, seg, cand, npt, alpha, delta, f1)
    for _ in range(2):
        fs.fstat_resampled_grad(ctx, seg, pts0)
    evf = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    evb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        evf[k][0].record(stream)
        Fres = fs.fstat_resampled(ctx, seg, pts0)
        evf[k][1].record(stream)
        flush.zero_()
        evb[k][0].record(stream)
        _, gres = fs.fstat_resampled_grad(ctx, seg, pts0)
        evb[k][1].record(stream)
    torch.cuda.synchronize()
    ctx.check()
    fwd_ms = sum(a.elapsed_time(c) for a, c in evf) / steps
    bwd_ms = sum(a.elapsed_time(c) for a, c in evb) / steps
    # 20 steps of gradient ascent of the resampled F from the same points
    fs.refine_resampled(ctx, seg, pts0, nsteps=nsteps)
    eva = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        eva[k][0].record(stream)
        _, Fasc = fs.refine_resampled(ctx, seg, pts0, nsteps=nsteps)
        eva[k][1].record(stream)
    torch.cuda.synchronize()
    ctx.check()
    asc_ms = sum(a.elapsed_time(c) for a, c in eva) / steps
    line["adjoint"] = {"forward": {"value": npt / (fwd_ms / 1e3), "unit": "candidates/s", "ms": fwd_ms},
                       "backward": {"value": npt / (bwd_ms / 1e3), "unit": "candidates/s", "ms": bwd_ms},
                       "what": "F of the resampled series at the %d starting points (fs_fstat_resampled) and "
                               "dF/d(f0, f1, alpha, delta) recomputing the series (fs_fstat_resampled_grad), "
                               "FP32 with double-float phases" % npt,
                       "F_res_over_F_exact_median": float(torch.median(Fres / F0).item()),
                       "gradient_ascent": {"value": npt / (asc_ms / 1e3), "unit": "candidates/s", "ms": asc_ms,
                                           "steps": nsteps,
                                           "F_gain_median": float(torch.median(Fasc / Fres).item()),
                                           "what": "fs_refine_resampled: quasi-Newton ascent (BFGS from 2 F G) "
                                                   "of the resampled F, one adjoint evaluation per step"}}
    if rank == 0 and not args.quick:
        # oracle: Nelder-Mead fine search (Sec. VI.C) from the first starting points, one
        # climb per host core
        pool = OraclePool()
        pts0 = fs.points_from_candidates(ctx, seg, cand, min(npt, pool.cores), alpha, delta, f1).cpu().numpy()
        xh = x32.double().cpu().numpy()
        try:
            done, secs = pool.points([("climb", xh, wl.dt, list(pt), wl.fl, det, wl.S0) for pt in pool.deal(list(pts0))])
            line["cpu_baseline"] = pool.record(done / secs, "candidates/s",
                                               "Nelder-Mead on the exact F from %d candidates over %d workers, %.1f s"
                                               % (done, pool.cores, secs))
        finally:
            pool.close()
        # end to end: candidates from the host, refined points and F back to the host
        ch = cand.cpu().pin_memory()
        ke = max(2, steps)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(ke):
            cd = ch.to("cuda", non_blocking=True)
            pts = fs.points_from_candidates(ctx, seg, cd, npt, alpha, delta, f1)
            out, Fr = fs.refine(ctx, seg, pts, nsteps=nsteps)
            out.cpu(), Fr.cpu()
        e2e_s = (time.perf_counter() - t1) / ke
        line["e2e"] = {"value": npt / e2e_s, "unit": "candidates/s", "h2d_bytes_per_step": npt * 16,
                       "d2h_bytes_per_step": npt * 40}
    else:
        line.setdefault("e2e", None)
        line.setdefault("cpu_baseline", None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    seg.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def _adjoint_config(wl, cands, world):
    return {"workload": "adjoint_2d", "n": wl.n, "candidates": cands, "ascent_steps": 20,
            "coarse": "grid_2d search (256 sky x 16 spindowns), strongest %d crossings" % cands,
            "l2": "flushed between timed steps (256 MiB write)", "parallelism": "sky shards x%d" % world}


def main_adjoint(args):
    """The differentiation workload (config 4 of the headline's configs): the coarse
    2-day search gives candidates (untimed); one step = starting points from 1024
    candidates + the adjoint's gradient ascent (fs_refine_resampled: F and the gradient
    of the resampled series recomputed at every step, 20 quasi-Newton steps)."""
    import torch
    import torch.distributed as dist
    from paper_1003_0844_gb300 import build, fstat as fs, shard

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    wl = W.WORKLOADS["grid_2d"]
    det = W.detector_for(wl)
    ctx = fs.Context(det, device=local)
    x64 = torch.as_tensor(W.noise(wl), device="cuda")
    fs.inject(ctx, x64, wl.dt, wl.fl, wl.sigma, W.injections(wl))
    x32 = x64.float().contiguous()
    a_all, d_all = W.sky_grid(wl.nsky * world)
    mine = shard.sky_shard(wl.nsky, rank, world)
    alpha = torch.as_tensor(np.ascontiguousarray(a_all[mine]), device="cuda")
    delta = torch.as_tensor(np.ascontiguousarray(d_all[mine]), device="cuda")
    f1 = torch.as_tensor(W.spin_grid(wl.nspin, *wl.f1_range), device="cuda")
    seg = fs.Segment(ctx, x32, wl.dt, wl.nfft, wl.fl, wl.S0)
    res = fs.search(ctx, seg, alpha, delta, f1, wl.F_thr, write_F=False, cand_cap=1 << 20)
    ncand_all = min(int(res.n_cand.item()), res.cand.shape[0])
    Fc = res.cand[:ncand_all, 3].view(torch.float32)
    top = torch.argsort(Fc, descending=True)[:args.cands]
    cand = res.cand[top].contiguous()
    npt, nsteps = cand.shape[0], 20

    def step():
        pts = fs.points_from_candidates(ctx, seg, cand, npt, alpha, delta, f1)
        return fs.refine_resampled(ctx, seg, pts, nsteps=nsteps)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    ctx.check()
    ctx.stats(reset=True)
    stream = torch.cuda.current_stream()
    steps = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    clocks = Clocks(local)
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        out, Fa = step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    stats = ctx.stats(reset=True)
    ctx.check()
    total_ms = shard.max_over_ranks(sum(a.elapsed_time(c) for a, c in ev), device="cuda")
    ms_per_step = total_ms / steps
    value = npt * world / (ms_per_step / 1e3)
    # the forward and backward calls alone at the starting points, same flushing
    pts0 = fs.points_from_candidates(ctx, seg, cand, npt, alpha, delta, f1)
    evf = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    evb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        evf[k][0].record(stream)
        F0 = fs.fstat_resampled(ctx, seg, pts0)
        evf[k][1].record(stream)
        flush.zero_()
        evb[k][0].record(stream)
        fs.fstat_resampled_grad(ctx, seg, pts0)
        evb[k][1].record(stream)
    torch.cuda.synchronize()
    ctx.check()
    fwd_ms = sum(a.elapsed_time(c) for a, c in evf) / steps
    bwd_ms = sum(a.elapsed_time(c) for a, c in evb) / steps
    gain = (Fa / F0).cpu().numpy()
    flops = ADJOINT_FLOP_PER_SAMPLE * wl.n * npt * (nsteps + 1)
    achieved = flops / (ms_per_step / 1e3) / 1e12
    line = {
        "metric": METRICS["adjoint_2d"], "value": value, "unit": "candidates/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (double-float phases)", "data": "synthetic",
        "config": _adjoint_config(wl, npt, world),
        "roofline": {"kernel": "k_resampled<true> (F and gradient of the resampled series, 21 calls per step)",
                     "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                     "peak_kind": "FP32 CUDA-core peak from unit counts and max clock (152 SM x 128 x 2 x 2070 MHz)",
                     "flop_convention": "%d FP32 flop per output sample and point per call (ncu opcode counts; the "
                                        "whole step's time, which also holds the starting points' metric pass)"
                                        % ADJOINT_FLOP_PER_SAMPLE},
        "gpu_launches": int(stats["launches"]),
        "clocks": ck,
        "forward": {"value": npt / (fwd_ms / 1e3), "unit": "candidates/s", "ms": fwd_ms},
        "backward": {"value": npt / (bwd_ms / 1e3), "unit": "candidates/s", "ms": bwd_ms},
        "F_gain": {"median": float(np.median(gain)), "max": float(np.max(gain))},
    }
    if rank == 0 and not args.quick:
        # oracle: the resampled F with its gradient (FP64) at starting points, on every host core
        pool = OraclePool()
        ptsh = pts0.cpu().numpy()
        xh = x32.double().cpu().numpy()
        try:
            per = 64  # evaluations per worker: ~7 s on the 16 cores of a Grace host
            pts_s = [list(ptsh[i % npt]) for i in range(per * pool.cores)]
            done, secs = pool.points([("adjoint", xh, wl.dt, pp, wl.fl, det, wl.S0) for pp in pool.deal(pts_s)])
            line["cpu_baseline"] = pool.record(done / 21.0 / secs, "candidates/s",
                                               "%d evaluations of the resampled F and its gradient (with each "
                                               "worker's segment preparation) over %d workers, %.1f s; a "
                                               "candidate's 20 steps take 21" % (done, pool.cores, secs))
        finally:
            pool.close()
        # end to end: candidates from the host, refined points and F back to the host
        ch = cand.cpu().pin_memory()
        ke = max(2, steps)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(ke):
            cd = ch.to("cuda", non_blocking=True)
            pts = fs.points_from_candidates(ctx, seg, cd, npt, alpha, delta, f1)
            o, Fo = fs.refine_resampled(ctx, seg, pts, nsteps=nsteps)
            o.cpu(), Fo.cpu()
        e2e_s = (time.perf_counter() - t1) / ke
        line["e2e"] = {"value": npt / e2e_s, "unit": "candidates/s", "h2d_bytes_per_step": npt * 16,
                       "d2h_bytes_per_step": npt * 40}
    else:
        line.setdefault("e2e", None)
        line.setdefault("cpu_baseline", None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    seg.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def main_lattice(args):
    """The constrained A4* lattice of a sky patch on the 2-day data (Sec. IV): per sky
    node a row of spindown nodes, each line one transform whose bins are shifted by its
    fraction of a bin (fs_search_lattice), F written for every bin.  The templates come
    from the library's host functions (linear-model Fisher matrix, lattice, nodes);
    with several ranks the patch's sky rows are dealt out (strong scaling)."""
    import torch
    import torch.distributed as dist
    from paper_1003_0844_gb300 import build, fstat as fs, shard

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    wl = W.WORKLOADS["grid_2d"]
    det = W.detector_for(wl)
    ctx = fs.Context(det, device=local)
    x64 = torch.as_tensor(W.noise(wl), device="cuda")
    fs.inject(ctx, x64, wl.dt, wl.fl, wl.sigma, W.injections(wl))
    x32 = x64.float().contiguous()
    G = fs.linear_model_fisher(det, wl.n, wl.dt)
    B, _ = fs.lattice(G, LATTICE_MATCH, 2 * math.pi / (wl.nfft * wl.dt))
    a, d, f1, off = fs.lattice_templates(B, det, wl.fl, wl.nfft, wl.dt, wl.f1_range, LATTICE_BOX)
    rows = shard.row_shard(a.size, rank, world)
    if args.nsky:
        rows = rows[:args.nsky]

    def dev(v):
        return torch.as_tensor(np.ascontiguousarray(v), device="cuda")
    alpha, delta, f1d, offd = dev(a[rows]), dev(d[rows]), dev(f1[rows]), dev(off[rows])
    nsky, nspin, nbins = rows.size, f1.shape[1], wl.nbins
    ntempl = nsky * nspin
    seg = fs.Segment(ctx, x32, wl.dt, wl.nfft, wl.fl, wl.S0)
    F_out = torch.empty((ntempl, nbins), dtype=torch.float32, device="cuda")
    cap = 1 << 16
    cand = torch.empty((cap, 4), dtype=torch.int32, device="cuda")
    ncand = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)

    def step():
        seg.load(x32)
        fs.search_lattice(ctx, seg, alpha, delta, f1d, offd, wl.F_thr, F_out=F_out, cand=cand, n_cand=ncand,
                          cand_cap=cap)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    ctx.check()
    ctx.stats(reset=True)
    ctx.set_profiling(True)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()  # L2 flushed between timed steps (outside the events)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    total_ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    stats = ctx.stats(reset=True)
    ctx.set_profiling(False)
    ctx.check()
    total_ms = shard.max_over_ranks(total_ms, device="cuda")
    ms_per_step = total_ms / args.steps
    templates_all = a.size * nspin if not args.nsky else ntempl * world
    value = templates_all / (ms_per_step / 1e3)
    # the transform kernel (one persistent launch per sky group) against the FP32 ALU
    # peak on 5 Nfft log2 Nfft flops per complex transform, two transforms per template
    p = int(round(math.log2(wl.nfft)))
    kinds = {k: (stats["ms"][k], stats["count"][k]) for k in ("prepare", "demodulate", "pass1", "pass2")}
    roof = None
    dom_ms, dom_n = kinds["pass2"]
    if dom_n and kinds["pass1"][1] == 0:
        per_launch_ms = dom_ms / dom_n
        tpl = ntempl * args.steps / dom_n
        achieved = 2 * 5 * wl.nfft * p * tpl / (per_launch_ms / 1e3) / 1e12
        tpt, tnote = _profile_traffic("k_passes_lattice_2d.md")
        roof = {"kernel": "k_passes (lattice items, persistent)", "bound": "alu", "achieved": achieved,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "traffic": (tpt * tpl if tpt is not None else None), "traffic_unit": "bytes per launch",
                "traffic_note": tnote,
                "peak_kind": "FP32 CUDA-core peak from unit counts and max clock (152 SM x 128 x 2 x 2070 MHz)",
                "flop_convention": "5 Nfft log2 Nfft per complex FFT, 2 FFTs per template",
                "per_launch_ms": per_launch_ms, "templates_per_launch": tpl}
    total_k = max(sum(v[0] for v in kinds.values()), 1e-9)
    line = {
        "metric": METRICS["lattice_2d"], "value": value, "unit": "templates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
        "dtype": "f32 (FP64/double-float phases)", "data": "synthetic",
        "config": _lattice_config(wl, nsky * world if args.nsky else a.size, nspin, world),
        "roofline": roof,
        "hbm_alg_gbs": ntempl * nbins * 4 / (ms_per_step / 1e3) / 1e9,
        "kernel_ms_share": {k: round(v[0] / total_k, 4) for k, v in kinds.items() if v[1]},
        "gpu_launches": int(stats["launches"]),
        "clocks": ck,
        "e2e": None, "cpu_baseline": None,
    }
    if rank == 0 and not args.quick:
        # the plain FP64 form of the lattice search on a sample of sky rows, and the FP32 error against it
        nsk = min(args.fp64_skies, nsky)
        seg64 = fs.Segment(ctx, x32, wl.dt, wl.nfft, wl.fl, wl.S0, precision="f64")
        sub = (alpha[:nsk].contiguous(), delta[:nsk].contiguous(), f1d[:nsk].contiguous(), offd[:nsk].contiguous())
        fs.search_lattice(ctx, seg64, *sub, wl.F_thr)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r64 = fs.search_lattice(ctx, seg64, *sub, wl.F_thr)
        e1.record()
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        F32 = F_out[: nsk * nspin].double()
        line["fp64_form"] = {"value": nsk * nspin / t64, "unit": "templates/s", "templates": nsk * nspin,
                             "note": "plain all-FP64 lattice search (own FP64 Stockham FFT), search only"}
        line["max_rel_dF_vs_fp64"] = float(((F32 - r64.F).abs() / torch.clamp(r64.F, min=1.0)).max().item())
        seg64.close()
        xh = x32.cpu().numpy()
        items = [(float(a[rows[s_]]), float(d[rows[s_]]), float(f1[rows[s_], m_]), float(off[rows[s_], m_]))
                 for s_ in range(nsky) for m_ in range(nspin)]
        pool = OraclePool()
        try:
            items = items[:max(pool.cores, min(len(items), pool.cores * args.cpu_templates // 16))]
            done, secs = pool.templates([(xh, wl, det, it) for it in pool.deal(items)])
            line["cpu_baseline"] = pool.record(done / secs, "templates/s",
                                               "%d lattice templates (FFT mode) over %d workers, each with its own "
                                               "segment preparation, %.1f s" % (done, pool.cores, secs))
        finally:
            pool.close()
        # end to end through the public API with host buffers, as for the grid workloads
        xh_pin = torch.empty(wl.n, dtype=torch.float32).pin_memory()
        xh_pin.copy_(x32.cpu())
        cand_h = torch.empty((cap, 4), dtype=torch.int32).pin_memory()
        nc_h = torch.empty(1, dtype=torch.int64).pin_memory()
        xd = torch.empty_like(x32)
        ke = max(5, args.steps // 5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            xd.copy_(xh_pin, non_blocking=True)
            seg.load(xd)
            fs.search_lattice(ctx, seg, alpha, delta, f1d, offd, wl.F_thr, F_out=F_out, cand=cand, n_cand=ncand,
                              cand_cap=cap)
            nc_h.copy_(ncand, non_blocking=True)
            cand_h.copy_(cand, non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / ke
        line["e2e"] = {"value": ntempl * world / e2e_s, "unit": "templates/s", "h2d_bytes_per_step": wl.n * 4,
                       "d2h_bytes_per_step": cap * 16 + 8}
    if rank == 0:
        print(json.dumps(line), flush=True)
    seg.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def grid_e2e(fs, ctx, seg, wl, x32, alpha, delta, f1, F_dev, cand, ncand, cap, steps, chunk_skies=16,
             copy_streams=1):
    """End to end through the public API with host buffers, every step: the data from
    pinned host memory to the device, segment preparation, the search, and its whole
    result back on the host: the F map of every template and bin, the candidates and
    their count.  Two ways of returning F are timed: the transform kernel writing F
    straight into a pinned host buffer (the device writes over the host link, no
    staging), and F written to device memory by sky chunks with each chunk copied to
    the pinned host buffer on a second stream while the next chunk runs.  The faster
    is "e2e"; the other and the candidates-only figure (F left on the device) are
    reported beside it.  The F map outweighs the step's compute on the host link
    (2.15 GB per 2-day step at ~190 GB/s from device to pinned host memory on this
    machine), so the staged way reaches ~90% of the copy's own rate with 16-sky
    chunks; more copy streams or alternating the two ways measured slower.
    Returns the fields for the JSON line."""
    import torch
    ntempl, nbins = F_dev.shape
    nsky, nspin = alpha.numel(), f1.numel()
    xh_pin = torch.empty(wl.n, dtype=torch.float32).pin_memory()
    xh_pin.copy_(x32.cpu())
    cand_h = torch.empty((cap, 4), dtype=torch.int32).pin_memory()
    nc_h = torch.empty(1, dtype=torch.int64).pin_memory()
    F_host = torch.empty((ntempl, nbins), dtype=torch.float32).pin_memory()
    xd = torch.empty_like(x32)
    ke = max(5, steps // 5)
    main_st = torch.cuda.current_stream()
    copy_sts = [torch.cuda.Stream() for _ in range(max(1, copy_streams))]
    chunk = max(1, min(nsky, chunk_skies))  # skies per chunk of the staged variant
    nchunk = (nsky + chunk - 1) // chunk
    cand_c = torch.empty((nchunk, cap, 4), dtype=torch.int32, device="cuda")  # per chunk: its own list
    ncand_c = torch.zeros(nchunk, dtype=torch.int64, device="cuda")
    cand_ch = torch.empty((nchunk, cap, 4), dtype=torch.int32).pin_memory()
    nc_ch = torch.empty(nchunk, dtype=torch.int64).pin_memory()

    def direct():
        fs.search(ctx, seg, alpha, delta, f1, wl.F_thr, F_out=F_host, cand=cand, n_cand=ncand, cand_cap=cap)
        nc_h.copy_(ncand, non_blocking=True)
        cand_h.copy_(cand, non_blocking=True)

    def staged():
        for i, s0 in enumerate(range(0, nsky, chunk)):
            s1 = min(nsky, s0 + chunk)
            rows = slice(s0 * nspin, s1 * nspin)
            # chunks write distinct rows; a step's copies end before the next step (synchronised)
            fs.search(ctx, seg, alpha[s0:s1], delta[s0:s1], f1, wl.F_thr, F_out=F_dev[rows], cand=cand_c[i],
                      n_cand=ncand_c[i:i + 1], cand_cap=cap)
            copy_st = copy_sts[i % len(copy_sts)]
            copy_st.wait_stream(main_st)
            with torch.cuda.stream(copy_st):
                F_host[rows].copy_(F_dev[rows], non_blocking=True)
        for copy_st in copy_sts:
            main_st.wait_stream(copy_st)
        nc_ch.copy_(ncand_c, non_blocking=True)
        cand_ch.copy_(cand_c, non_blocking=True)

    def cands_only():
        fs.search(ctx, seg, alpha, delta, f1, wl.F_thr, F_out=F_dev, cand=cand, n_cand=ncand, cand_cap=cap)
        nc_h.copy_(ncand, non_blocking=True)
        cand_h.copy_(cand, non_blocking=True)

    def timed(search):
        search()  # untimed first call
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            xd.copy_(xh_pin, non_blocking=True)
            seg.load(xd)
            search()
            torch.cuda.synchronize()
        return (time.perf_counter() - t0) / ke

    out = {}
    t_direct = timed(direct)
    # the host map equals the device map of the same search (sampled rows)
    cands_only()
    torch.cuda.synchronize()
    rows = torch.linspace(0, ntempl - 1, 16).long()
    same_direct = bool(torch.equal(F_host[rows], F_dev[rows].cpu()))
    F_host.zero_()
    t_staged = timed(staged)
    same_staged = bool(torch.equal(F_host[rows], F_dev[rows].cpu()))
    t_cands = timed(cands_only)
    f_bytes = ntempl * nbins * 4
    ways = {"direct": (t_direct, "the transform kernel writes F into a pinned host buffer", same_direct,
                       cap * 16 + 8),
            "staged": (t_staged, "F to device memory by chunks of %d skies, each copied to a pinned host buffer "
                                 "on %d copy stream(s) while the next chunk runs" % (chunk, len(copy_sts)), same_staged,
                       nchunk * (cap * 16 + 8))}
    best = min(ways, key=lambda k: ways[k][0])
    for k, (t, how, same, cbytes) in ways.items():
        rec = {"value": ntempl / t, "unit": "templates/s", "h2d_bytes_per_step": wl.n * 4,
               "d2h_bytes_per_step": f_bytes + cbytes, "F_returned": True, "how": how,
               "F_host_equals_device": same}
        out["e2e" if k == best else "e2e_F_" + k] = rec
    out["e2e_candidates_only"] = {"value": ntempl / t_cands, "unit": "templates/s", "h2d_bytes_per_step": wl.n * 4,
                                  "d2h_bytes_per_step": cap * 16 + 8, "F_returned": False}
    return out


def main():
    args = _args()
    rc = launch_ranks(args)
    if rc is not None:
        sys.exit(rc)
    if args.stub:
        return run_stub(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in W.BATCHES:
        return main_batch(args)
    if args.workload == "refine_2d":
        return main_refine(args)
    if args.workload == "adjoint_2d":
        return main_adjoint(args)
    if args.workload == "lattice_2d":
        return main_lattice(args)
    import torch
    import torch.distributed as dist
    from paper_1003_0844_gb300 import build, fstat as fs, shard

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    wl = W.WORKLOADS[args.workload]
    if args.nsky:
        import dataclasses
        wl = dataclasses.replace(wl, nsky=args.nsky)
    det = W.detector_for(wl)
    ctx = fs.Context(det, device=local)
    # inputs: seeded noise plus simulated signals (fs_inject, FP64), stored as float32 data
    x64 = torch.as_tensor(W.noise(wl), device="cuda")
    fs.inject(ctx, x64, wl.dt, wl.fl, wl.sigma, W.injections(wl))
    x32 = x64.float().contiguous()
    # weak scaling: rank r searches its own 256-sky shard of a lattice of 256 x world points
    a_all, d_all = W.sky_grid(wl.nsky * world)
    mine = shard.sky_shard(wl.nsky, rank, world)
    alpha = torch.as_tensor(np.ascontiguousarray(a_all[mine]), device="cuda")
    delta = torch.as_tensor(np.ascontiguousarray(d_all[mine]), device="cuda")
    f1 = torch.as_tensor(W.spin_grid(wl.nspin, *wl.f1_range), device="cuda")
    nsky, nspin, nbins = alpha.numel(), f1.numel(), wl.nbins
    ntempl = nsky * nspin
    seg = fs.Segment(ctx, x32, wl.dt, wl.nfft, wl.fl, wl.S0, interbin=wl.interbin)
    F_out = torch.empty((ntempl, nbins), dtype=torch.float32, device="cuda")
    cap = 1 << 16
    cand = torch.empty((cap, 4), dtype=torch.int32, device="cuda")
    ncand = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)

    def step():
        seg.load(x32)
        fs.search(ctx, seg, alpha, delta, f1, wl.F_thr, F_out=F_out, cand=cand, n_cand=ncand, cand_cap=cap)

    tuning = None
    if args.n1:
        ctx.set_tuning(wl.nfft, n1=args.n1)
        tuning = ctx.get_tuning(wl.nfft)
    if args.tune:
        tuning = ctx.autotune(seg, alpha[:min(nsky, 64)].contiguous(), delta[:min(nsky, 64)].contiguous(), f1)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    ctx.check()
    ctx.stats(reset=True)
    ctx.set_profiling(True)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()  # L2 flushed between timed steps (outside the events)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    stats = ctx.stats(reset=True)
    ctx.set_profiling(False)
    ctx.check()
    total_ms = shard.max_over_ranks(total_ms, device="cuda")
    ms_per_step = total_ms / args.steps
    value = ntempl * world / (ms_per_step / 1e3)

    # dominant kernel and its roofline: FFT flops 5 Nfft log2(Nfft) per complex transform,
    # two transforms (a, b) per template.  In the persistent mode one launch per sky
    # group runs both passes (kind "pass2" then covers the whole transform); in the
    # per-batch mode the flops split between the passes by log2 N1 : log2 N2.
    p = int(round(math.log2(wl.nfft)))
    lg1, lg2 = (p + 1) // 2, p // 2
    kinds = {k: (stats["ms"][k], stats["count"][k]) for k in ("prepare", "demodulate", "pass1", "pass2")}
    fused = kinds["pass1"][1] == 0
    names = {"pass1": "k_pass1", "pass2": "k_passes (both passes, persistent)" if fused else "k_pass2",
             "demodulate": "k_demod32", "prepare": "segment preparation"}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms, dom_n = kinds[dom]
    flops_tmpl = {"pass1": 2 * 5 * wl.nfft * lg1, "pass2": 2 * 5 * wl.nfft * (p if fused else lg2)}
    roof = None
    if dom in flops_tmpl and dom_n:
        per_launch_ms = dom_ms / dom_n
        tpl = ntempl * args.steps / dom_n
        achieved = flops_tmpl[dom] * tpl / (per_launch_ms / 1e3) / 1e12
        tpt, tnote = (_profile_traffic("k_passes_%s.md" % args.workload) if fused else (None, "per-batch mode"))
        roof = {"kernel": names[dom], "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "traffic": (tpt * tpl if tpt is not None else None), "traffic_unit": "bytes per launch",
                "traffic_note": tnote,
                "peak_kind": "FP32 CUDA-core peak from unit counts and max clock (152 SM x 128 x 2 x 2070 MHz)",
                "flop_convention": "5 Nfft log2 Nfft per complex FFT, 2 FFTs per template",
                "per_launch_ms": per_launch_ms, "templates_per_launch": tpl}
    hbm_gbs, hbm_kind = _peaks()
    # whole-path HBM view: algorithmic bytes = F written (4 B per bin) per template
    hbm_alg = ntempl * nbins * 4 / (ms_per_step / 1e3) / 1e9
    dram = bound = None
    if roof is not None and roof.get("traffic"):
        # achieved DRAM rate of the transform kernel (ncu bytes per launch over the event-timed
        # launch), and the model bound that binds: HBM on the design's bytes per template
        # (measured traffic) or the FP32 ALU on the algorithmic flops
        dram_gbs = roof["traffic"] / (roof["per_launch_ms"] / 1e3) / 1e9
        dram = {"kernel": roof["kernel"], "achieved_gbs": dram_gbs, "peak_gbs": hbm_gbs, "frac": dram_gbs / hbm_gbs,
                "peak_kind": hbm_kind, "source": "ncu dram bytes per launch / event-timed launch duration"}
        per_tpl = roof["traffic"] / roof["templates_per_launch"]
        hbm_tps = hbm_gbs * 1e9 / per_tpl
        alu_tps = FP32_PEAK_TFLOPS * 1e12 / flops_tmpl[dom]
        bound = {"hbm_templates_per_s": hbm_tps, "alu_templates_per_s": alu_tps,
                 "binding": "hbm" if hbm_tps < alu_tps else "alu", "frac": value / min(hbm_tps, alu_tps),
                 "note": "HBM bound on the measured bytes per template, ALU bound on 5 Nfft log2 Nfft x 2 flops"}
    shares = {names[k]: round(v[0] / max(sum(x[0] for x in kinds.values()), 1e-9), 4)
              for k, v in kinds.items() if v[1]}

    line = {
        "metric": metric_name(args.workload), "value": value, "unit": "templates/s", "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (FP64/double-float phases)", "data": "synthetic",
        "config": _grid_config(wl, nsky, nspin, world),
        "roofline": roof,
        "hbm_alg_gbs": hbm_alg, "hbm_peak_gbs": hbm_gbs, "hbm_peak_kind": hbm_kind,
        "dram": dram, "model_bound": bound,
        "kernel_ms_share": shares,
        "gpu_launches": int(stats["launches"]),
        "clocks": ck,
    }
    if tuning is not None:
        line["tuning"] = tuning
    if rank == 0 and not args.quick:
        # plain FP64 form on a sample of skies (same GPU), and the FP32 path's error against it
        nsk = min(args.fp64_skies, nsky)
        seg64 = fs.Segment(ctx, x32, wl.dt, wl.nfft, wl.fl, wl.S0, precision="f64", interbin=wl.interbin)
        fs.search(ctx, seg64, alpha[:nsk].contiguous(), delta[:nsk].contiguous(), f1, wl.F_thr)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r64 = fs.search(ctx, seg64, alpha[:nsk].contiguous(), delta[:nsk].contiguous(), f1, wl.F_thr)
        e1.record()
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        F64 = r64.F
        F32 = F_out[: nsk * nspin].double()
        drel = float(((F32 - F64).abs() / torch.clamp(F64, min=1.0)).max().item())
        line["fp64_form"] = {"value": nsk * nspin / t64, "unit": "templates/s", "templates": nsk * nspin,
                             "note": "plain all-FP64 path (own FP64 Stockham FFT, radix 16/4/2), search only"}
        line["max_rel_dF_vs_fp64"] = drel
        seg64.close()
        line["cufft_comparison"] = cufft_comparison(wl.nfft, nbins)
        # the oracle on every host core, bounded sample: about 16 templates of the 2-day
        # size per core (a template costs ~N), each worker preparing the segment itself
        ncores = host_cores()
        ntc = max(ncores, min(nsky * nspin, int(ncores * args.cpu_templates / 20 * 86164 / wl.n)))
        line["cpu_baseline"] = oracle_grid_baseline(x32.cpu().numpy(), wl, det, a_all[mine], d_all[mine],
                                                    W.spin_grid(wl.nspin, *wl.f1_range), ntc)
        line.update(grid_e2e(fs, ctx, seg, wl, x32, alpha, delta, f1, F_out, cand, ncand, cap, args.steps))
    else:
        line.setdefault("e2e", None)
        line.setdefault("cpu_baseline", None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    seg.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
