"""Benchmark of the random-sampling multiscale solver on one GB300 (or N replicas).

A step is one pass of the whole hot path over the 2049^2 log-normal workload
(eps = 2^-7, 32 x 32 patches of 64 cells, 16-cell buffers, 128 Gaussian
samples per patch plus the boundary-delta columns of the patches on the
domain boundary):

  build the medium (face coefficients)              msp_build_medium
  offline local solves, restriction                 msp_sample_patches
  basis extraction, edge operators, preconditioner  msp_extract_basis
  online solve of one batch of Dirichlet data       msp_online_solve

Headline metric: local sample-solves per second of the whole step.  The
online latency (p50/p99 over repeated single-request solves on the prebuilt
basis) is reported beside it.  Inputs are synthetic and seeded; every step
rebuilds everything, and the per-step working set (snapshots, 4.7 GB) is far
larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                  [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own replica (weak scaling); the
timed region is bracketed by a barrier and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "elliptic-2049-lognormal-32x32-b16-S128"
METRIC = "local sample-solves/s"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    @staticmethod
    def smi_id(props, index: int) -> str:
        """nvidia-smi's id of the GPU torch calls `index`: its UUID ("GPU-<uuid>"),
        because nvidia-smi numbers GPUs in PCI order and ignores
        CUDA_VISIBLE_DEVICES; the plain index only when the UUID is unknown."""
        u = getattr(props, "uuid", None)
        if u is None:
            return str(index)
        u = str(u)
        return u if u.startswith("GPU-") else "GPU-" + u

    def start(self):
        try:
            import torch
            gid = self.smi_id(torch.cuda.get_device_properties(self.index), self.index)
        except Exception:
            gid = str(self.index)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gid, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0])); smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- multi-rank host logic

def max_over_ranks(x: float, world: int) -> float:
    """The largest value over all ranks (the slowest replica's time); x at one rank.
    NCCL reduces a device tensor, gloo a host tensor."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, t_max: float) -> float:
    """Whole-job throughput of N independent replicas: all ranks' units over the
    slowest rank's time."""
    return units_per_rank * world / t_max


# ---------------------------------------------------------------- CPU oracle arm

def oracle_sample(budget_s: float = 15.0):
    """Time the CPU oracle (as it stands) on a bounded sample of the workload:
    the local solves of whole patches of the 2049^2 medium, interior and
    boundary ones, until the time budget is used.  Returns solves/s."""
    from oracle import elliptic as E
    w = synth.workload_batched()
    t0 = time.time()
    aE, aN = E.face_coefficients(w["medium"])
    t_med = time.time() - t0
    patches = E.patch_boxes(2048, w["patches"])
    order = [0, 33, 528, 17, 1023, 300, 700, 31, 992, 64]
    solves, t_solve, used = 0, 0.0, []
    for m in order:
        P = patches[m]
        t1 = time.time()
        R = E.snapshots(aE, aN, P, w["seed"], 2048)
        t_solve += time.time() - t1
        solves += R.shape[1]
        used.append(m)
        if t_solve > budget_s:
            break
    # SuperLU factorisation and back-substitution run on one thread
    return {"value": solves / t_solve, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{solves} local solves (patches {used}) of the 2049^2 workload by sparse LU + "
                      f"back-substitution; face coefficients {t_med:.1f} s not counted"}


def cpu_model() -> str:
    """CPU model name of the host (lscpu), for the baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


_ORACLE_STATE = {}


def _oracle_worker_init(barrier=None):
    from oracle import elliptic as E
    w = synth.workload_batched()
    _ORACLE_STATE["E"] = E
    _ORACLE_STATE["w"] = w
    _ORACLE_STATE["faces"] = E.face_coefficients(w["medium"])
    _ORACLE_STATE["patches"] = E.patch_boxes(2048, w["patches"])
    if barrier is not None:
        barrier.wait()          # no worker takes a patch before every worker is ready


def _oracle_patch_solves(m):
    E, w = _ORACLE_STATE["E"], _ORACLE_STATE["w"]
    aE, aN = _ORACLE_STATE["faces"]
    t0 = time.time()
    R = E.snapshots(aE, aN, _ORACLE_STATE["patches"][m], w["seed"], 2048)
    return R.shape[1], t0, time.time()


def oracle_sample_all_cores(budget_s: float = 15.0, cores: int | None = None):
    """The CPU oracle on every host core: one process per core (spawned, so it
    is safe after the CUDA context exists), each solving whole patches of the
    2049^2 workload (sparse LU + back-substitution, as the oracle stands).  The
    face coefficients are evaluated once per process before the clock starts.
    Patches are handed out in a fixed seeded order until the time budget is
    spent; returns solves/s over the wall time."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    order = np.random.default_rng(0).permutation(1024).tolist()
    ctx = mp.get_context("spawn")
    # one thread per process: the processes are the parallelism (the children
    # read these before numpy starts its thread pools)
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        barrier = ctx.Barrier(cores)
        with ctx.Pool(cores, initializer=_oracle_worker_init, initargs=(barrier,)) as pool:
            solves, used, t_first, t_last = 0, 0, None, None
            it = pool.imap_unordered(_oracle_patch_solves, order, chunksize=1)
            for n, a, b in it:
                solves += n
                used += 1
                t_first = a if t_first is None else min(t_first, a)
                t_last = b if t_last is None else max(t_last, b)
                if t_last - t_first > budget_s:
                    break
            dt = t_last - t_first
            pool.terminate()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {"value": solves / dt, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{solves} local solves ({used} whole patches, seeded order) of the 2049^2 workload, "
                      f"one spawned single-threaded process per core, sparse LU + back-substitution per patch; "
                      f"face coefficients evaluated before the clock; wall time from the first patch's start "
                      f"to the last finished patch's end"}


def cpu_baselines(budget_s: float):
    """Oracle baseline on one core and on all cores, with the host's core count
    and CPU model."""
    one = oracle_sample(budget_s=budget_s)
    allc = oracle_sample_all_cores(budget_s=budget_s)
    return {**allc, "one_core": one, "nproc": os.cpu_count(), "cpu_model": cpu_model()}


def run_reference(args, rank, world):
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        oracle_sample(budget_s=3.0)
    for _ in range(args.steps):
        vals.append(oracle_sample(budget_s=8.0))
    v = statistics.median(x["value"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "bounded per step (whole patches)"},
            "cpu_baseline": {**vals[-1], "value": v},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def run_profile_case(args):
    """One offline pass (sample + extract) and one online solve on the 513^2
    log-normal medium (8 x 8 patches of 64 cells, 16-cell buffers, 128 samples):
    the small case for detailed profiler captures of the same kernels."""
    import torch
    import paper_1807_08848_gb300 as msp
    torch.cuda.set_device(0)
    N = 512
    ms = synth.lognormal(N, 2.0 ** -5, 64, 11)
    ps = synth.uniform_patches(N, 8, 8, 16, 128)
    med = msp.Medium(ms, ps)
    if args.precision == "mixed" and args.local_solver == "direct":
        med.set_launch("mixed", "direct")
    st = med.sample(1, args.precision, tol=1e-10, max_iter=20000)
    basis = med.extract(1e-6, args.precision)
    from paper_1807_08848_gb300 import _native
    try:
        u, it = basis.solve(torch.tensor(synth.phi_sin_cos(N), device="cuda"), tol=1e-8, max_iter=args.online_iters)
        oi = int(it[0])
    except _native.MspError as e:
        if e.status != _native.MSP_ERR_NOT_CONVERGED:
            raise
        oi = -1
    torch.cuda.synchronize()
    print(json.dumps({"case": "lognormal-513-8x8", "solves": int(st.n_solves), "cg_iters": int(st.total_iters),
                      "online_iters": oi}))


def serve_poisson(srv, phis, arrivals, which, fetch_idx=()):
    """Submit requests at the given arrival times (seconds from the start) with
    boundary data phis[i][j] for request j on medium i = which[j]; a poller thread
    records each request's latency (submit to result on the device) and fetches
    the results of fetch_idx.  Returns (latencies ms, fetched {j: u}, wall s)."""
    n_req = len(arrivals)
    pending, fetched = {}, {}
    lat = np.full(n_req, np.nan)
    lock = threading.Lock()
    finished = threading.Event()
    fetch_idx = set(fetch_idx)

    def poller():
        while not finished.is_set() or pending:
            with lock:
                items = list(pending.items())
            for rid, j in items:
                d, l = srv.poll(rid)
                if d == 0:
                    continue
                lat[j] = l
                if j in fetch_idx:
                    fetched[j] = srv.fetch(rid, int(which[j]))
                else:
                    srv.release(rid)
                with lock:
                    pending.pop(rid, None)
            time.sleep(0.0002)

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    t_start = time.perf_counter()
    for j in range(n_req):
        dt = arrivals[j] - (time.perf_counter() - t_start)
        if dt > 0:
            time.sleep(dt)
        i = int(which[j])
        rid = srv.submit(i, phis[i][j % len(phis[i])])
        with lock:
            pending[rid] = j
    finished.set()
    th.join(timeout=900)
    return lat, fetched, time.perf_counter() - t_start


def pct(x, q):
    x = np.asarray(x)
    x = x[~np.isnan(x)]
    return float(np.percentile(x, q)) if x.size else None


def online_latency_block(basis, n_req: int, rates, seed: int = 5, workers: int = 4):
    """Online latency of one medium under Poisson load: the plain FP64 path
    (the request loop's FP64 engine: FP64 CGLS, FP64 factor applied in FP64) and
    the mixed path (the request loop's map engine: FP32 map GEMM on the tensor
    cores), each fed the same arrival times and the same 64 boundary data sets.
    Reports p50/p99 of submit-to-result latency, throughput, and the error of
    sampled results against an FP64 online solve to 1e-12."""
    import torch
    n = basis.n_cells
    phis = [synth.phi_fourier(n, 16, 3000 + seed, batch=64)]
    which = np.zeros(n_req, dtype=np.int64)
    check = list(range(0, n_req, max(1, n_req // 8)))[:8]
    basis.set_preconditioner("block_rows_fp64")
    refs = {}
    for j in check:
        r, _ = basis.solve(torch.tensor(phis[0][j % 64], device="cuda"), tol=1e-12, max_iter=5000, want_iters=False)
        refs[j] = r.cpu().numpy()
    basis.set_preconditioner("block_rows")
    out = {"n_nodes": f"{n + 1}^2", "requests": n_req, "workers": workers,
           "data": "64 distinct 16-mode Fourier boundary data sets, seeded", "loads": []}
    for rate in rates:
        arr = synth.poisson_arrivals(rate, n_req, 3)
        rec = {"offered_rate_hz": rate}
        for eng, tol in (("iterative_fp64", 1e-8), ("map", None)):
            srv = msp_server(basis, workers)
            try:
                if eng == "map":
                    srv.set_engine("map")
                else:
                    srv.set_engine("iterative_fp64", tol=tol, max_iter=1000)
                lat, fetched, wall = serve_poisson(srv, phis, arr, which, check)
                st = srv.stats()
            finally:
                srv.close()
            errs = [float(np.linalg.norm(fetched[j] - refs[j]) / np.linalg.norm(refs[j])) for j in fetched]
            rec["fp64_iterative" if eng != "map" else "mixed_map"] = {
                "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "throughput_hz": float(st["completed"] / wall),
                "completed": int(st["completed"]), "failed": int(st["failed"]), "batches": int(st["batches"]),
                "max_batch_seen": int(st["max_batch_seen"]),
                "max_rel_err_vs_fp64_1e-12": max(errs) if errs else None,
                "engine": ("FP64 CGLS to 1e-8, FP64 factor applied in FP64" if eng != "map"
                           else "FP32 map on tensor cores (split TF32, FP32/FP64 accumulation)")}
        out["loads"].append(rec)
    return out


def msp_server(basis, workers):
    import paper_1807_08848_gb300 as msp
    return msp.Server([basis], mem_budget_bytes=16 << 30, max_slots=4096, max_batch=32, n_workers=workers)


def serving_summary(bench_basis, n_req: int, rate: float, workers: int = 4):
    """Short serving run over three media (513^2, 1025^2 of the serving workload
    and the bench's own 2049^2 medium, whose basis and map are already built):
    Poisson arrivals on a uniformly chosen medium, map engine."""
    import paper_1807_08848_gb300 as msp
    wl = synth.workload_serving()
    bases, meds = [], []
    t0 = time.time()
    for md in wl["media"][:2]:
        med = msp.Medium(md["medium"], md["patches"])
        med.sample(1, "mixed", tol=1e-10, max_iter=20000, stats=False)
        b = med.extract(1e-6, "mixed")
        b.build_map(tol=1e-10, max_iter=5000)
        meds.append(med)
        bases.append(b)
    bases.append(bench_basis)
    t_setup = time.time() - t0
    rng = np.random.default_rng(wl["seed"])
    arr = synth.poisson_arrivals(rate, n_req, wl["seed"])
    which = rng.integers(0, 3, n_req)
    phis = [synth.phi_fourier(b.n_cells, 16, 3000 + i, batch=64) for i, b in enumerate(bases)]
    srv = msp.Server(bases, mem_budget_bytes=16 << 30, max_slots=4096, max_batch=32, n_workers=workers)
    try:
        lat, _, wall = serve_poisson(srv, phis, arr, which)
        st = srv.stats()
    finally:
        srv.close()
    return {"media": ["513^2 eps 2^-5 (serving workload)", "1025^2 eps 2^-6 (serving workload)",
                      "2049^2 eps 2^-7 (the bench workload)"], "requests": n_req, "offered_rate_hz": rate,
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "throughput_hz": float(st["completed"] / wall),
            "completed": int(st["completed"]), "failed": int(st["failed"]), "batches": int(st["batches"]),
            "max_batch_seen": int(st["max_batch_seen"]), "setup_s_two_media": t_setup}


def measure_peaks():
    """FP32 (CUDA cores), TF32 (tensor cores) and FP64 dense rates of this GPU at
    its current clocks, from torch.matmul timed with CUDA events (best of 5):
    the roofline denominators for kernels bound by those units."""
    import torch
    out = {}
    stream = torch.cuda.current_stream()
    for name, dt, n, tf32 in (("fp32_tflops", torch.float32, 8192, False), ("tf32_tflops", torch.float32, 8192, True),
                              ("fp64_tflops", torch.float64, 4096, False)):
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = tf32
        try:
            a = torch.randn((n, n), dtype=dt, device="cuda")
            b = torch.randn((n, n), dtype=dt, device="cuda")
            c = a @ b
            best = 1e30
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                torch.matmul(a, b, out=c)
                e1.record(stream)
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            out[name] = 2.0 * n ** 3 / best / 1e12
            del a, b, c
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev
    out["how"] = "torch.matmul n^3 (fp32/tf32 8192, fp64 4096), best of 5, CUDA events"
    return out


def run_serving(args):
    """Serving workload: three prebuilt log-normal media (513^2, 1025^2, 2049^2;
    64-cell patches, 16-cell buffers, 128 samples), bases and boundary-to-
    coefficient maps on the device, Poisson arrivals (mean args.rate req/s, seed
    3) of 16-mode Fourier boundary data on a uniformly chosen medium, served by
    the request loop.  Reports p50/p99 latency (submit to result on the device)
    and the throughput, and checks a seeded 1% sample against the FP64 iterative
    online solve of the same data (relative L2 <= 1e-6)."""
    import torch
    import paper_1807_08848_gb300 as msp
    torch.cuda.set_device(0)
    wl = synth.workload_serving()
    t0 = time.time()
    bases, meds = [], []
    for md in wl["media"]:
        med = msp.Medium(md["medium"], md["patches"])
        med.sample(1, "mixed", tol=1e-10, max_iter=20000, stats=False)
        b = med.extract(1e-6, "mixed")
        meds.append(med)
        bases.append(b)
    t_offline = time.time() - t0
    t0 = time.time()
    for b in bases:
        b.build_map(tol=1e-10, max_iter=5000)
    torch.cuda.synchronize()
    t_map = time.time() - t0
    rng = np.random.default_rng(wl["seed"])
    n_req = args.requests
    gaps = rng.exponential(1.0 / args.rate, n_req)
    arrivals = np.cumsum(gaps)
    which = rng.integers(0, len(bases), n_req)
    pool = [synth.phi_fourier(b.n_cells, 16, 3000 + i, batch=64) for i, b in enumerate(bases)]
    check = set(rng.choice(n_req, max(1, n_req // 100), replace=False).tolist())
    srv = msp.Server(bases, mem_budget_bytes=int(args.serve_mem_gb * (1 << 30)), max_slots=4096,
                     max_batch=32, n_workers=args.serve_workers)
    pending = {}
    lat = np.full(n_req, np.nan)
    fetched = {}
    lock = threading.Lock()
    finished = threading.Event()

    def poller():
        while not finished.is_set() or pending:
            with lock:
                items = list(pending.items())
            for rid, j in items:
                d, l = srv.poll(rid)
                if d == 0:
                    continue
                lat[j] = l
                if j in check:
                    fetched[j] = srv.fetch(rid, int(which[j]))
                else:
                    srv.release(rid)
                with lock:
                    pending.pop(rid, None)
            time.sleep(0.0002)

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    t_start = time.perf_counter()
    for j in range(n_req):
        dt = arrivals[j] - (time.perf_counter() - t_start)
        if dt > 0:
            time.sleep(dt)
        i = int(which[j])
        rid = srv.submit(i, pool[i][j % 64])
        with lock:
            pending[rid] = j
    finished.set()
    th.join(timeout=600)
    t_end = time.perf_counter()
    st = srv.stats()
    srv.close()
    # accuracy of the sampled requests against the FP64 iterative online solve
    worst = 0.0
    for j, u in fetched.items():
        i = int(which[j])
        b = bases[i]
        b.set_preconditioner("block_rows_fp64")
        ref, _ = b.solve(torch.tensor(pool[i][j % 64], device="cuda"), tol=1e-12, max_iter=5000)
        b.set_preconditioner("block_rows")
        worst = max(worst, float(np.linalg.norm(u - ref.cpu().numpy()) / np.linalg.norm(ref.cpu().numpy())))
    # single-request latency per medium: the plain FP64 path (iterative online
    # solve, FP64 factor sweeps) beside the map solve, device-resident data
    single = []
    for i, b in enumerate(bases):
        phi_d = torch.tensor(pool[i][0], device="cuda")
        rec = {}
        for name in ("fp64_iterative", "map"):
            ts = []
            for _ in range(6):
                torch.cuda.synchronize()
                a = time.perf_counter()
                if name == "map":
                    b.solve_map(phi_d)
                else:
                    b.set_preconditioner("block_rows_fp64")
                    b.solve(phi_d, tol=1e-8, max_iter=5000, want_iters=False)
                    b.set_preconditioner("block_rows")
                torch.cuda.synchronize()
                ts.append((time.perf_counter() - a) * 1e3)
            rec[name + "_ms"] = float(np.median(ts[1:]))
        single.append({"n_nodes": b.n_cells + 1, **rec})
    ok = lat[~np.isnan(lat)]
    line = {"metric": "online solve latency p50/p99 ms (serving)", "value": float(np.percentile(ok, 99)),
            "unit": "ms (p99)", "higher_is_better": False, "n_gpus": 1,
            "p50_ms": float(np.percentile(ok, 50)), "p99_ms": float(np.percentile(ok, 99)),
            "requests": int(n_req), "completed": int(st["completed"]), "failed": int(st["failed"]),
            "offered_rate_hz": args.rate, "throughput_hz": float(st["completed"] / (t_end - t_start)),
            "batches": int(st["batches"]), "max_batch_seen": int(st["max_batch_seen"]),
            "mem_peak_bytes": int(st["mem_peak"]), "workers": args.serve_workers,
            "sample_checked": len(fetched), "sample_max_rel_err_vs_fp64": worst,
            "single_request": single,
            "setup_s": {"offline_3_media": t_offline, "maps": t_map},
            "config": {"workload": wl["name"], "media": ["513^2 eps 2^-5", "1025^2 eps 2^-6", "2049^2 eps 2^-7"],
                       "patch_cells": 64, "buffer": 16, "samples": 128,
                       "data": "16-mode Fourier data, 64 distinct sets per medium, seeded"}}
    print(json.dumps(line), flush=True)


def run_mapgemm(args):
    """One serving medium (--medium 513/1025/2049) with its basis and map; two
    batch-32 map solves with each GEMM engine, CUDA-event times: the small case for
    profiler captures of the map GEMMs."""
    import torch
    import paper_1807_08848_gb300 as msp
    torch.cuda.set_device(0)
    md = synth.workload_serving()["media"][{513: 0, 1025: 1, 2049: 2}[args.medium]]
    med = msp.Medium(md["medium"], md["patches"])
    med.sample(1, "mixed", tol=1e-10, max_iter=20000, stats=False)
    b = med.extract(1e-6, "mixed")
    b.build_map(tol=1e-10, max_iter=5000)
    n = b.n_cells
    phi = torch.tensor(synth.phi_fourier(n, 16, 5, batch=32), device="cuda")
    u = torch.empty((32, n + 1, n + 1), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    for eng in ("cuda_cores", "tensor_cores"):
        b.set_map_engine(eng)
        ts = []
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.solve_map(phi, u=u)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        res[eng + "_ms"] = ts[-1]
    print(json.dumps({"case": f"mapgemm-{args.medium}", "n_unknowns": b.n_unknowns, **res}), flush=True)


def run_stencil(args):
    """The streaming operator on every patch x 128 samples of one serving medium
    (--medium), FP32 and FP64, CUDA-event times: the small case for profiler captures."""
    import torch
    import paper_1807_08848_gb300 as msp
    torch.cuda.set_device(0)
    md = synth.workload_serving()["media"][{513: 0, 1025: 1, 2049: 2}[args.medium]]
    med = msp.Medium(md["medium"], md["patches"])
    rows, cols = med.tile_shape()
    pitch = (cols + 3) // 4 * 4
    S = 128
    out = {"case": f"stencil-{args.medium}", "tiles": med.n_patches * S}
    nodes = sum((p.X1 - p.X0 + 1) * (p.Y1 - p.Y0 + 1) for p in (med.patch(m) for m in range(med.n_patches)))
    for prec, dt, es in (("mixed", torch.float32, 4), ("fp64", torch.float64, 8)):
        x = torch.randn((med.n_patches, S, rows, pitch), dtype=dt, device="cuda")
        y = torch.empty_like(x)
        med.apply_operator(x, prec, y=y)
        ms = med.apply_operator(x, prec, y=y, timed=True)[1]
        out[prec] = {"ms": ms, "achieved_gbs": (nodes * S * 2 * es + nodes * 2 * es) / ms / 1e6}
        del x, y
    print(json.dumps(out), flush=True)


def kinetic_direct_rates(msp, torch, kw, stream, g, precision, reps=2):
    """The kinetic slab's local solves by the direct block solver: the first call
    (factorisation + solve) and the steady state (factor reused), CUDA events."""
    km = msp.KineticMedium(kw["n_cells"], kw["eps"], kw["n_v"], kw["n_patches"], kw["buffer"], kw["samples"], g=g)
    km.set_solver("direct")
    out = {"g": g}
    for r in range(1 + reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = km.sample(kw["seed"], tol=1e-13, max_iter=16, precision=precision)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if r == 0:
            out["first_call_ms"] = ms
        else:
            out["ms"] = min(out.get("ms", ms), ms)
        out["passes_max"] = int(st.max_iters)
    out["solves_per_s"] = int(st.n_solves) / (out["ms"] / 1e3)
    out["factor_ms"] = out["first_call_ms"] - out["ms"]
    del km
    return out


def run_kinetic(args):
    """The kinetic slab workload alone (8192 cells, 64 GL velocities, 64 patches x 96
    samples): one sample pass per precision and solver, CUDA-event times, for
    profiler captures; the direct solver also with the Henyey-Greenstein
    collision at g = 1/2."""
    import torch
    import paper_1807_08848_gb300 as msp
    torch.cuda.set_device(0)
    kw = synth.workload_kinetic()
    stream = torch.cuda.current_stream()
    out = {"case": kw["name"]}
    for kp in ("mixed", "fp64"):
        km = msp.KineticMedium(kw["n_cells"], kw["eps"], kw["n_v"], kw["n_patches"], kw["buffer"], kw["samples"])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = km.sample(kw["seed"], tol=1e-13, max_iter=200000, precision=kp)
        e1.record(stream)
        torch.cuda.synchronize()
        out[kp] = {"ms": e0.elapsed_time(e1), "solves": int(st.n_solves),
                   "sweeps_per_solve": st.total_iters / max(1, int(st.n_solves))}
        del km
    for g in (0.0, 0.5):
        for kp in ("mixed", "fp64"):
            out[f"direct_g{g}_{kp}"] = kinetic_direct_rates(msp, torch, kw, stream, g, kp)
    print(json.dumps(out), flush=True)


def run_direct(args):
    """The 2049^2 workload's local solves by the direct solver (block LDL^T over
    the grid rows, FP32 inverse Schur complements, FP64 refinement) beside the CG
    tile kernel, same medium and seed, CUDA events; the factorisation is timed on
    its own (first call) and inside steady-state calls it is reused."""
    import torch
    import paper_1807_08848_gb300 as msp
    torch.cuda.set_device(0)
    w = synth.workload_batched()
    stream = torch.cuda.current_stream()
    out = {"case": "direct-2049"}

    def timed(med, reps=3):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            med.sample(w["seed"], "mixed", tol=1e-10, max_iter=20000, stats=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ts

    cg = msp.Medium(w["medium"], w["patches"])
    st = cg.sample(w["seed"], "mixed", tol=1e-10, max_iter=20000)
    out["cg_ms"] = timed(cg)
    d = msp.Medium(w["medium"], w["patches"])
    d.set_launch("mixed", "direct")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    std = d.sample(w["seed"], "mixed", tol=1e-10, max_iter=20000)
    e1.record(stream)
    torch.cuda.synchronize()
    out["direct_first_call_ms"] = e0.elapsed_time(e1)
    out["direct_ms"] = timed(d)
    out["solves"] = int(std.n_solves)
    out["direct_max_passes"] = int(std.max_iters)
    out["direct_not_converged"] = int(std.n_not_converged)
    out["cg_avg_iters"] = st.total_iters / max(1, int(st.n_solves))
    diffs = []
    for m in (0, 17, 528, 1023):
        a = cg.snapshots(m).cpu().numpy()
        b = d.snapshots(m).cpu().numpy()
        diffs.append(float(np.linalg.norm(a - b) / np.linalg.norm(a)))
    out["rel_diff_direct_vs_cg"] = diffs
    out["direct_solves_per_s"] = out["solves"] / (min(out["direct_ms"]) / 1e3)
    out["cg_solves_per_s"] = out["solves"] / (min(out["cg_ms"]) / 1e3)
    print(json.dumps(out), flush=True)


def run_extract(args):
    """Extraction of the 2049^2 workload's bases (Cholesky-QR3, Jacobi SVD,
    projection, online operators and factor) with the FP64 products on the tensor
    cores and on the CUDA cores, same snapshots, CUDA events; the singular values,
    ranks and an online field of the two are compared."""
    import torch
    import paper_1807_08848_gb300 as msp
    torch.cuda.set_device(0)
    w = synth.workload_batched()
    stream = torch.cuda.current_stream()
    med = msp.Medium(w["medium"], w["patches"])
    med.set_launch("mixed", "direct")
    med.sample(w["seed"], "mixed", tol=1e-10, max_iter=20000)
    out = {"case": "extract-2049"}
    bases = {}
    for eng in ("tensor_cores", "cuda_cores", "tensor_cores"):
        msp.set_gemm_engine(eng)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b = med.extract(w["tau"], "mixed")
        e1.record(stream)
        torch.cuda.synchronize()
        out[eng + "_ms"] = e0.elapsed_time(e1)
        bases[eng] = b
    msp.set_gemm_engine("tensor_cores")
    bt, bc = bases["tensor_cores"], bases["cuda_cores"]
    out["max_sigma_diff_rel_sigma1"] = max(float(np.max(np.abs(bt.sigma(m) - bc.sigma(m))) / bc.sigma(m)[0])
                                           for m in range(0, med.n_patches, 37))
    out["k_equal"] = all(bt.k(m) == bc.k(m) for m in range(med.n_patches))
    phi = torch.tensor(w["phi"], device="cuda")
    ut, _ = bt.solve(phi, tol=1e-10, max_iter=1000)
    uc, _ = bc.solve(phi, tol=1e-10, max_iter=1000)
    out["online_rel_diff"] = float(torch.linalg.norm(ut - uc) / torch.linalg.norm(uc))
    out["stats_tc"] = bt.stats()
    # the Jacobi SVD from the identity in FP64 against the FP32-started one (default),
    # tensor-core products both, with the phase times
    msp.set_extract_timing(True)
    for mode in ("fp32_preconditioned", "qr_preconditioned", "fp64"):
        msp.set_svd_mode(mode)
        b = med.extract(w["tau"], "mixed")
        out["svd_" + mode] = {"phases_ms": b.extract_timing(), "max_jacobi_sweeps": b.stats()["max_jacobi_sweeps"],
                              "mean_jacobi_sweeps": b.stats()["mean_jacobi_sweeps"]}
        bases["svd_" + mode] = b
    msp.set_svd_mode()
    msp.set_extract_timing(False)
    b64 = bases["svd_fp64"]
    for mode in ("fp32_preconditioned", "qr_preconditioned"):
        bx = bases["svd_" + mode]
        # singular values at 0.1 tau sigma_1 and above (the sweeps leave pairs of
        # columns far below the truncation level unrotated)
        d = 0.0
        for m in range(0, med.n_patches, 37):
            s64, sx = b64.sigma(m), bx.sigma(m)
            res = s64 >= 0.1 * w["tau"] * s64[0]
            d = max(d, float(np.max(np.abs(sx - s64)[res]) / s64[0]))
        out["svd_" + mode]["max_sigma_diff_rel_sigma1"] = d
        out["svd_" + mode]["k_equal"] = all(bx.k(m) == b64.k(m) for m in range(med.n_patches))
    print(json.dumps(out), flush=True)


def run_uneven(args):
    """The uneven workload: 1025^2 nodes, eps = 2^-6, channel medium of contrast 1e3,
    patches of 16-96 cells with 4-24-cell buffers and 64-256 samples; local solves per
    second of the split launch, the fused persistent launch, and the autotuned choice
    replayed from a CUDA graph (mixed precision, CUDA events)."""
    import torch
    import paper_1807_08848_gb300 as msp
    torch.cuda.set_device(0)
    w = synth.workload_uneven()
    stream = torch.cuda.current_stream()
    out = {"metric": "local sample-solves/s (uneven batch)", "unit": "local sample-solves/s",
           "higher_is_better": True, "n_gpus": 1, "config": {"workload": w["name"]}}

    def timed(med, reps=3):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            med.sample(w["seed"], "mixed", tol=1e-10, max_iter=40000, stats=False)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return float(np.median(ts))

    forms = {}
    for name in ("split", "fused"):
        med = msp.Medium(w["medium"], w["patches"])
        med.set_launch("mixed", name)
        st = med.sample(w["seed"], "mixed", tol=1e-10, max_iter=40000)
        n = int(st.n_solves)
        forms[name] = {"solves_per_s": n / timed(med), "launches": 1 if name == "fused" else 2}
        del med
    med = msp.Medium(w["medium"], w["patches"])
    t0 = time.time()
    rep = med.autotune(w["seed"], "mixed", tol=1e-10, max_iter=40000, max_probe_items=2048)
    t_tune = time.time() - t0
    med.set_graph(True)
    med.sample(w["seed"], "mixed", tol=1e-10, max_iter=40000, stats=False)   # direct run + capture
    forms["autotuned_graph"] = {"solves_per_s": n / timed(med), "choice": rep["best_mode"], "rows": rep["best_rows"],
                                "tune_s": t_tune, "candidates": rep["candidates"]}
    out["value"] = forms["autotuned_graph"]["solves_per_s"]
    out["local_solves"] = n
    out["forms"] = forms
    print(json.dumps(out), flush=True)


def schwarz_block(msp, native, w, basis, phi_dev, prec, tol, direct, online_tol, reps=20, coarse_modes=(True,)):
    """The overlapping Schwarz variant of the online step on `basis`: the set-up
    samples the full-basis medium (one delta per ring node of every buffered patch,
    with the step's local solver and tolerance) and forms B_m = Q_m^T G~_m and the
    coarse space; then single-request solves (restarted GMRES on the reduced fixed
    point) timed with CUDA events, and the relative difference of its field from
    the least-squares glue's (two readings of the online step, not a parity check)."""
    import torch
    out = {}
    try:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        full = msp.Medium(w["medium"], w["patches"], full_basis=True)
        if direct:
            full.set_launch("mixed", "direct")
        full.sample(w["seed"], prec, tol=tol, max_iter=20000, stats=False)
        ev[1].record()
        torch.cuda.synchronize()
        out["full_medium_solves"] = int(sum(full.patch(m).n_ring for m in range(full.n_patches)))
        out["full_sample_ms"] = ev[0].elapsed_time(ev[1])
        u_ls, _ = basis.solve(phi_dev, tol=1e-12, max_iter=20000)
        for coarse in coarse_modes:
            key = "two_level" if coarse else "one_level"
            r = {}
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            basis.setup_schwarz(full, coarse=coarse)
            b.record()
            torch.cuda.synchronize()
            r["setup_ms"] = a.elapsed_time(b)
            a.record()
            u, it = basis.solve(phi_dev, tol=online_tol, max_iter=5000, schwarz=True)
            b.record()
            torch.cuda.synchronize()
            r["first_call_ms"] = a.elapsed_time(b)
            times = []
            for _ in range(reps):
                a.record()
                u, it = basis.solve(phi_dev, tol=online_tol, max_iter=5000, schwarz=True)
                b.record()
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b))
            r["p50_ms"], r["p99_ms"] = pct(times, 50), pct(times, 99)
            r["requests"] = reps
            r["gmres_iters"] = int(it[0])
            r["rel_diff_vs_least_squares"] = float(torch.linalg.norm(u - u_ls) / torch.linalg.norm(u_ls))
            out[key] = r
        del full
    except native.MspError as e:
        out["error"] = str(e)
    return out


def run_schwarz(args):
    """Only the Schwarz variant of the online step at 2049^2: offline stage as in
    the step (mixed, direct local solver), then one- and two-level solves."""
    import torch
    import paper_1807_08848_gb300 as msp
    from paper_1807_08848_gb300 import _native
    torch.cuda.set_device(0)
    msp.load_library()
    n = args.schwarz_n
    if n == 2048:
        w = synth.workload_batched()
    else:   # the smaller log-normal media of the serving workload (same tiles)
        sv = synth.workload_serving()["media"][{512: 0, 1024: 1}[n]]
        w = dict(medium=sv["medium"], patches=sv["patches"], seed=1, tau=1e-6, online_tol=1e-8,
                 phi=synth.phi_sin_cos(n))
    med = msp.Medium(w["medium"], w["patches"])
    med.set_launch("mixed", "direct")
    med.sample(w["seed"], "mixed", tol=1e-10, max_iter=20000, stats=False)
    basis = med.extract(w["tau"], "mixed")
    phi_dev = torch.tensor(w["phi"], dtype=torch.float64, device="cuda").reshape(1, -1)
    t0 = time.perf_counter()
    u, it = basis.solve(phi_dev, tol=w["online_tol"], max_iter=args.online_iters)
    torch.cuda.synchronize()
    out = {"case": f"schwarz-{n + 1}", "least_squares_first_call_ms": (time.perf_counter() - t0) * 1e3,
           "least_squares_iters": int(it[0])}
    out.update(schwarz_block(msp, _native, w, basis, phi_dev, "mixed", 1e-10, True, w["online_tol"],
                             reps=args.schwarz_reps, coarse_modes=(False, True) if args.schwarz_one_level else (True,)))
    print(json.dumps(out), flush=True)


def run_step_case(args):
    """Only the headline step (new medium, local solves, extraction, one online
    solve) of the 2049^2 workload, --warmup then --steps times, CUDA events per
    step: the command of the step's launch list (nothing else launches)."""
    import torch
    import paper_1807_08848_gb300 as msp
    from paper_1807_08848_gb300 import _native
    torch.cuda.set_device(0)
    w = synth.workload_batched()
    stream = torch.cuda.current_stream()
    phi = torch.tensor(w["phi"], dtype=torch.float64).reshape(1, -1).cuda()
    direct = args.precision == "mixed" and args.local_solver == "direct"

    def step():
        med = msp.Medium(w["medium"], w["patches"])
        if direct:
            med.set_launch("mixed", "direct")
        med.sample(w["seed"], args.precision, tol=1e-10, max_iter=20000, stats=False)
        basis = med.extract(w["tau"], args.precision)
        try:
            basis.solve(phi, tol=w["online_tol"], max_iter=args.online_iters, want_iters=False)
        except _native.MspError as e:
            if e.status != _native.MSP_ERR_NOT_CONVERGED:
                raise

    for _ in range(args.warmup):
        step()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    print(json.dumps({"case": "step-2049", "ms_per_step": ms}), flush=True)


def run_ours(args, rank, world):
    import torch
    import paper_1807_08848_gb300 as msp
    from paper_1807_08848_gb300 import _native

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    lib = msp.load_library()
    stream = torch.cuda.current_stream()
    w = synth.workload_batched()
    prec = args.precision
    tol = 1e-10 if prec == "mixed" else 1e-10
    phi_host = torch.tensor(w["phi"], dtype=torch.float64).reshape(1, -1).pin_memory()
    phi_dev = phi_host.cuda()
    n = 2049

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    state = {}
    direct = prec == "mixed" and args.local_solver == "direct"

    def new_medium():
        med = msp.Medium(w["medium"], w["patches"])
        if direct:
            med.set_launch("mixed", "direct")
        return med

    def step(host_io: bool):
        med = new_medium()
        st = med.sample(w["seed"], prec, tol=tol, max_iter=20000, stats=False)
        basis = med.extract(w["tau"], prec)
        if host_io:
            ph = phi_host.cuda(non_blocking=True)
        else:
            ph = phi_dev
        try:
            u, it = basis.solve(ph, tol=w["online_tol"], max_iter=args.online_iters, want_iters=False)
        except _native.MspError as e:
            if e.status != _native.MSP_ERR_NOT_CONVERGED:
                raise
            u = None
        if host_io and u is not None:
            state["u_host"] = u.to("cpu", non_blocking=False)
        state["med"], state["basis"] = med, basis
        return med

    # warm-up
    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    # solve statistics of one step (outside the timed region)
    med = new_medium()
    stats = med.sample(w["seed"], prec, tol=tol, max_iter=20000)
    n_solves = int(stats.n_solves)
    n_gauss = int(np.sum(w["patches"].samples))
    infos = [med.patch(m) for m in range(med.n_patches)]
    # local-solve stage timing with events on the launching stream; the direct
    # solver also times each of its phases with events around its launches
    if direct:
        med.set_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    med.sample(w["seed"], prec, tol=tol, max_iter=20000, stats=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_kernel = ev0.elapsed_time(ev1) / 1e3
    phases = med.direct_timing() if direct else None
    del med
    # the CG tile kernel on the same medium (the mixed path without the direct solver)
    cg = None
    if prec == "mixed" and direct and args.compare_fp64:
        cmed = msp.Medium(w["medium"], w["patches"])
        cst = cmed.sample(w["seed"], "mixed", tol=tol, max_iter=20000)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        cmed.sample(w["seed"], "mixed", tol=tol, max_iter=20000, stats=False)
        c1.record(stream)
        torch.cuda.synchronize()
        tc_ = c0.elapsed_time(c1) / 1e3
        cg = {"kernel": "local_solve_tile<float, 12>", "seconds": tc_, "solves_per_s": n_solves / tc_,
              "avg_cg_iters": cst.total_iters / max(1, n_solves),
              "achieved_tflops": 19.0 * float(cst.unknown_iters) / tc_ / 1e12}
        del cmed

    # ---- timed region (device-resident inputs)
    clocks = ClockSampler(dev)
    barrier(); torch.cuda.synchronize()
    clocks.start()
    launches0 = lib.msp_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(False)
    e1.record(stream)
    torch.cuda.synchronize(); barrier()
    clk = clocks.stop()
    launches = (lib.msp_kernel_launches() - launches0) / args.steps
    t = max_over_ranks(e0.elapsed_time(e1) / 1e3 / args.steps, world)

    # ---- end to end through host buffers (medium description and phi from the
    # host, the reconstructed field back to the host), wall clock with syncs
    barrier(); torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps // 2)):
        step(True)
    torch.cuda.synchronize(); barrier()
    t_e2e = max_over_ranks((time.perf_counter() - t0) / max(1, args.steps // 2), world)
    h2d = int(w["medium"].modes.nbytes + 4 * 4 * (33 + 33 + 1024 + 1024) + phi_host.numel() * 8)
    d2h = int(n * n * 8)

    # ---- online latency on the prebuilt basis: the plain FP64 path and the mixed
    # (map) path under the same Poisson load and data, then a short three-media
    # serving run
    basis = state["basis"]
    online = None
    serving = None
    if args.online_reqs > 0:
        t0 = time.time()
        basis.build_map(tol=1e-10, max_iter=5000)
        torch.cuda.synchronize()
        t_map = time.time() - t0
        online = online_latency_block(basis, args.online_reqs, rates=args.online_rates)
        online["map_build_s"] = t_map
        if args.serve_summary_reqs > 0:
            serving = serving_summary(basis, args.serve_summary_reqs, args.rate)

    # ---- per-stage device times of one step (outside the timed region)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    evs[0].record(stream)
    smed = new_medium()
    evs[1].record(stream)
    smed.sample(w["seed"], prec, tol=tol, max_iter=20000, stats=False)
    evs[2].record(stream)
    msp.set_extract_timing(True)
    sbasis = smed.extract(w["tau"], prec)
    msp.set_extract_timing(False)
    evs[3].record(stream)
    try:
        sbasis.solve(phi_dev, tol=w["online_tol"], max_iter=args.online_iters, want_iters=False)
    except _native.MspError:
        pass
    evs[4].record(stream)
    torch.cuda.synchronize()
    stages = {nm: evs[i].elapsed_time(evs[i + 1]) for i, nm in
              enumerate(("build_medium_ms", "sample_patches_ms", "extract_basis_ms", "online_solve_ms"))}
    stages["basis_stats"] = sbasis.stats()
    ext_phases = sbasis.extract_timing()
    stages["extract_phases_ms"] = {k: v for k, v in ext_phases.items() if k != "jacobi_flop"}
    # the constrained least-squares variant of the online step on the same basis:
    # the first call builds its derived basis (null spaces, online operators and
    # factor), later calls only solve
    cons = {}
    try:
        for key in ("first_call_ms", "solve_ms"):
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            sbasis.solve(phi_dev, tol=w["online_tol"], max_iter=args.online_iters, want_iters=False, constrained=True)
            c1.record(stream)
            torch.cuda.synchronize()
            cons[key] = c0.elapsed_time(c1)
    except _native.MspError as e:
        cons["error"] = str(e)
    stages["online_constrained"] = cons
    # the overlapping Schwarz variant of the online step on the same basis
    stages["online_schwarz"] = schwarz_block(msp, _native, w, sbasis, phi_dev, prec, tol, direct,
                                             online_tol=w["online_tol"])
    del smed, sbasis

    # ---- the streaming matrix-free operator on the same tiles (every patch x every
    # Gaussian sample, FP32): HBM-bound, reported against the measured copy bandwidth
    stencil = None
    if args.stencil:
        omed = msp.Medium(w["medium"], w["patches"])
        rows, cols = omed.tile_shape()
        pitch = (cols + 3) // 4 * 4
        S = int(w["patches"].samples[0])
        xs = torch.randn((omed.n_patches, S, rows, pitch), dtype=torch.float32, device="cuda")
        ys = torch.empty_like(xs)
        for _ in range(3):
            omed.apply_operator(xs, "mixed", y=ys)
        times = [omed.apply_operator(xs, "mixed", y=ys, timed=True)[1] for _ in range(5)]
        t_st = float(np.median(times)) / 1e3
        nodes = sum((p.X1 - p.X0 + 1) * (p.Y1 - p.Y0 + 1) for p in (omed.patch(m) for m in range(omed.n_patches)))
        alg = nodes * S * 8.0 + nodes * 8.0          # x read + y written per sample; faces once per patch
        hbm = peaks().get("hbm_gbs", 6800.0)
        stencil = {"kernel": "stencil_apply_kernel<float>", "tiles": omed.n_patches * S,
                   "tile": f"{rows}x{pitch} (pitch)", "ms": t_st * 1e3, "algorithmic_bytes": alg,
                   "achieved_gbs": alg / t_st / 1e9, "peak_gbs": hbm, "frac": alg / t_st / 1e9 / hbm,
                   "l2": "inputs 5 GB > L2"}
        del xs, ys, omed

    # ---- the kinetic slab workload (8192 cells, 64 GL velocities, 64 patches x 96
    # samples): local solves per second, mixed (FP32 corrections) and plain FP64
    kinetic = None
    if args.kinetic:
        kw = synth.workload_kinetic()
        kinetic = {"workload": kw["name"]}
        for kp in ("mixed", "fp64"):
            km = msp.KineticMedium(kw["n_cells"], kw["eps"], kw["n_v"], kw["n_patches"], kw["buffer"], kw["samples"])
            km.sample(kw["seed"], tol=1e-13, max_iter=200000, precision=kp, stats=False)
            k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k0.record(stream)
            kst = km.sample(kw["seed"], tol=1e-13, max_iter=200000, precision=kp)
            k1.record(stream)
            torch.cuda.synchronize()
            kt = k0.elapsed_time(k1) / 1e3
            kinetic[kp] = {"solves_per_s": int(kst.n_solves) / kt, "ms": kt * 1e3,
                           "sweeps_per_solve": kst.total_iters / max(1, int(kst.n_solves))}
            del km
        # the direct block solver (isotropic, and the Henyey-Greenstein collision at g = 1/2)
        for g in (0.0, 0.5):
            for kp in ("mixed", "fp64"):
                kinetic[f"direct_g{g}_{kp}"] = kinetic_direct_rates(msp, torch, kw, stream, g, kp, reps=1)

    # ---- the plain FP64 path's local solves on the same medium, for comparison
    fp64_rate = None
    if args.compare_fp64 and prec == "mixed":
        med64 = msp.Medium(w["medium"], w["patches"])
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        st64 = med64.sample(w["seed"], "fp64", tol=tol, max_iter=20000)
        f1.record(stream)
        torch.cuda.synchronize()
        fp64_rate = {"solves_per_s": int(st64.n_solves) / (f0.elapsed_time(f1) / 1e3),
                     "avg_cg_iters": st64.total_iters / max(1, int(st64.n_solves))}
        del med64

    # ---- measured FP32 / TF32 / FP64 rates (roofline denominators)
    mpk = measure_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count

    # ---- roofline of the dominant kernel: the CG arithmetic of the tile-resident
    # local solves.  Algorithmic flops per CG iteration and unknown of the
    # symmetrically scaled operator (unit diagonal): 9 for the 5-point apply
    # (4 products, 4 adds, 1 subtract), 2 for p.Ap, 2 + 2 for the x and r
    # updates, 2 for r.r, 2 for the p update: 19.
    pk = peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0)
    fp32_derived = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    peak = mpk["fp32_tflops"] if prec == "mixed" else mpk["fp64_tflops"]
    if direct:
        # the direct solver's sweeps: per column and refinement pass, the forward
        # and the backward sweep each multiply every interior row block by W_j
        # (nx x nx): 4 nx^2 ny flop; passes per column from the statistics
        # (their mean, the columns of one patch share their tiles)
        passes = stats.total_iters / max(1, n_solves)
        flops = passes * sum(4.0 * (p.X1 - p.X0 - 1) ** 2 * (p.Y1 - p.Y0 - 1) * p.cols for p in infos)
        t_roof = phases["solve"]["ms"] / 1e3
        kernel_name = "direct_solve_kernel<3>"
        roof_launches = phases["solve"]["launches"]
        traffic = None
        traffic_source = "not captured for this kernel build"
    else:
        # the CG arithmetic of the tile-resident local solves: per CG iteration and
        # unknown of the symmetrically scaled operator (unit diagonal), 9 flop for the
        # 5-point apply, 2 for p.Ap, 2 + 2 for the x and r updates, 2 for r.r, 2 for p
        flops = 19.0 * float(stats.unknown_iters)
        t_roof = t_kernel
        kernel_name = "local_solve_tile<float, 12>" if prec == "mixed" else "local_solve_tile<double, 12>"
        roof_launches = 1
        # DRAM bytes per local solve of local_solve_tile<float, 12>, from one ncu
        # capture (dram__bytes_read.sum + dram__bytes_write.sum) of the 513^2 case,
        # whose buffered tiles have the same sizes: 1012.35 MB / 11164 solves.
        traffic = (22942720 + 989403648) / 11164.0 * n_solves if prec == "mixed" else None
        traffic_source = "ncu capture of the 513^2 case scaled by solves" if prec == "mixed" else None
    achieved = flops / t_roof / 1e12
    local_roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                  "traffic": traffic, "traffic_source": traffic_source, "kernel": kernel_name,
                  "launches": roof_launches, "seconds": t_roof, "algorithmic_flop": flops}
    # the FP64 one-sided Jacobi SVD of the extraction, timed with events around its
    # launch (22 c flop per column pair and sweep, summed over the patches)
    t_jac = ext_phases["jacobi"] / 1e3
    jac_roof = None
    if t_jac > 0:
        ja = ext_phases["jacobi_flop"] / t_jac / 1e12
        jac_roof = {"bound": "alu", "achieved": ja, "peak": mpk["fp64_tflops"], "unit": "TFLOP/s",
                    "frac": ja / mpk["fp64_tflops"], "traffic": None,
                    "traffic_source": "not captured for this kernel build", "kernel": "jacobi_svd_kernel",
                    "launches": 1, "seconds": t_jac, "algorithmic_flop": ext_phases["jacobi_flop"],
                    "peak_source": "measured: cuBLAS DGEMM (torch.matmul fp64) in this run"}
    value = aggregate_rate(n_solves, world, t)
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_nodes": "2049x2049", "patches": "32x32", "buffer": 16,
                   "gaussian_samples_per_patch": 128, "gaussian_solves": n_gauss, "local_solves": n_solves,
                   "precision": prec, "local_tol": tol, "tau": w["tau"], "online_tol": w["online_tol"],
                   "l2": "working set > L2 (4.7 GB snapshots rebuilt every step)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": aggregate_rate(n_solves, world, t_e2e), "unit": METRIC, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(round(launches)),
        "gaussian_only": {"value": aggregate_rate(n_gauss, world, t), "unit": "Gaussian sample-solves/s",
                          "note": "the same step counted by its Gaussian columns only (the boundary-delta columns "
                                  "of the patches on the domain boundary excluded)"},
        "online": online,
        "serving": serving,
        "measured_peaks": {**mpk, "n_sm": n_sm, "fp32_derived_tflops": fp32_derived},
        "local_solve": {"solver": "direct (block LDL^T, FP32 inverse Schur complements, FP64 refinement)"
                                  if direct else "CG tile kernel",
                        "seconds": t_kernel, "solves_per_s": n_solves / t_kernel,
                        "avg_iters": stats.total_iters / max(1, n_solves),
                        "iters_unit": "refinement passes" if direct else "CG iterations",
                        "max_refinements": stats.max_refinements, "not_converged": stats.n_not_converged,
                        "phases": phases},
        "local_solve_cg_mixed": cg,
        "fp64_path_local_solve": fp64_rate,
        "stencil_apply": stencil,
        "kinetic_local_solve": kinetic,
        "stages": stages,
        "roofline_secondary": None,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_source,
                     "kernel": kernel_name, "launches": roof_launches, "seconds": t_roof,
                     "algorithmic_flop": flops,
                     "peak_source": ("measured: cuBLAS SGEMM (torch.matmul fp32, TF32 off) in this run" if prec == "mixed"
                                     else "measured: cuBLAS DGEMM (torch.matmul fp64) in this run")
                                    + f"; derived FP32 unit peak {fp32_derived:.1f} TFLOP/s "
                                      f"({n_sm} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz)"},
        "clocks": clk,
    }
    # the roofline line is the step's dominant kernel: the local-solve sweeps or the
    # Jacobi SVD, whichever takes longer; the other is reported beside it
    local_roof["peak_source"] = line["roofline"]["peak_source"]
    if jac_roof is not None and jac_roof["seconds"] > local_roof["seconds"]:
        line["roofline"], line["roofline_secondary"] = jac_roof, local_roof
    else:
        line["roofline_secondary"] = jac_roof
    if rank == 0:
        if args.cpu_baseline and world >= 1:
            line["cpu_baseline"] = cpu_baselines(budget_s=args.cpu_budget)
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--local-solver", default="direct", choices=["direct", "cg"],
                    help="local solver of the mixed path: the direct solver (block LDL^T with FP32 inverse Schur "
                         "complements inside FP64 refinement) or the CG tile kernel")
    ap.add_argument("--online-iters", type=int, default=1000)
    ap.add_argument("--online-reqs", type=int, default=200,
                    help="requests per load and engine of the online latency block (0: skip it)")
    ap.add_argument("--online-rates", type=float, nargs="+", default=[2000.0, 50.0],
                    help="Poisson rates (req/s) of the online latency block")
    ap.add_argument("--serve-summary-reqs", type=int, default=2000,
                    help="requests of the three-media serving summary (0: skip it)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-kinetic", dest="kinetic", action="store_false",
                    help="skip timing the kinetic slab local solves")
    ap.add_argument("--no-stencil", dest="stencil", action="store_false",
                    help="skip timing the streaming operator")
    ap.add_argument("--no-fp64-compare", dest="compare_fp64", action="store_false",
                    help="skip timing the plain FP64 local solves beside the mixed ones")
    ap.add_argument("--schwarz-n", type=int, default=2048, choices=[512, 1024, 2048],
                    help="cells per side of the schwarz case (2048: the batched workload; 512/1024: serving media)")
    ap.add_argument("--schwarz-reps", type=int, default=20, help="timed single-request solves of the schwarz case")
    ap.add_argument("--schwarz-one-level", type=int, default=1, help="schwarz case: also time the one-level form")
    ap.add_argument("--case", default="full", choices=["full", "step", "profile513", "serving", "uneven", "mapgemm", "stencil", "kinetic", "schwarz",
                                                      "direct", "extract"],
                    help="profile513: one pass of the small 513^2 case for profiler captures; "
                         "serving: the request loop over three prebuilt media")
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--medium", type=int, default=1025, choices=[513, 1025, 2049],
                    help="serving medium of --case mapgemm / --case stencil")
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-mem-gb", type=float, default=16.0)
    args = ap.parse_args()
    if args.case == "step":
        run_step_case(args)
        return
    if args.case == "profile513":
        run_profile_case(args)
        return
    if args.case == "serving":
        run_serving(args)
        return
    if args.case == "uneven":
        run_uneven(args)
        return
    if args.case == "mapgemm":
        run_mapgemm(args)
        return
    if args.case == "stencil":
        run_stencil(args)
        return
    if args.case == "kinetic":
        run_kinetic(args)
        return
    if args.case == "direct":
        run_direct(args)
        return
    if args.case == "schwarz":
        return run_schwarz(args)
    if args.case == "extract":
        run_extract(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    run_ours(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
