#!/usr/bin/env python3
"""Benchmark of the arrow-decomposition SpMM on GB300 (prints ONE JSON line on rank 0).

Default workload (one step = one arrow_spmm call = the whole hot path once):
  3D 400x400x400 grid, 7-point stencil (n = 64,000,000, nnz = 447,040,000), values
  U(0.5,1.5) row-normalised f32, arrow width b = 4096, X n x 16 f32 N(0,1),
  20 iterations of X <- A X with the FP64 per-column norm rescale.
Inputs (X 4.1 GB, A 3.6 GB) are larger than the 129 MB L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload grid3d|grid2d|rmat|batch|serve|predicates] [--size S] [--iters T] [--k K]
                  [--dtype f32|bf16] [--count M] [--tuning R,E,C,P] [--no-e2e] [--no-cpu] [--no-cusparse]

The line carries the device-timed value, the rows kernel's roofline, per-step min/mean/max,
the clocks seen during the timed region, an end-to-end figure through the public call with
pinned host buffers (copies inside the timed region; two steps in flight on two streams,
and the one-stream form beside it), cuSPARSE on the undecomposed matrix and the CPU oracle.
The rows kernel is autotuned before timing unless --tuning fixes its launch configuration.
--impl reference times the CPU oracle (the FP64 product of the oracle package, as it
stands) on a bounded sample of the same workload on the host cores.
Under torchrun each rank runs its own replica of the workload (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "arrow-SpMM iters/s & HBM GB/s (% of peak) vs plain FP32/cuSPARSE; serve p50/p99"
# the sources the single-matrix kernels are compiled from (the traffic record is tied to them)
KERNEL_SRCS = [os.path.join(ROOT, "paper_2402_19364_gb300", "csrc", f) for f in ("arrow_spmm.cu", "device_common.cuh")]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="grid3d", choices=["grid3d", "grid2d", "rmat", "batch", "serve", "predicates"])
    p.add_argument("--count", type=int, default=0, help="matrices of the batch workload (0 = 512)")
    p.add_argument("--size", type=int, default=0, help="grid side / R-MAT scale (0 = workload default)")
    p.add_argument("--iters", type=int, default=0)
    p.add_argument("--k", type=int, default=0)
    p.add_argument("--dtype", default="", choices=["", "f32", "bf16"])
    p.add_argument("--no-cusparse", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-fp32", action="store_true", help="skip the FP32 arm of a 16-bit workload")
    p.add_argument("--no-device-decompose", action="store_true",
                   help="skip timing the decomposition with its steps on the GPU")
    p.add_argument("--no-sub", action="store_true", help="default workload only: skip the other configurations' records")
    p.add_argument("--sub", default="grid2d,rmat,batch,serve,predicates", help="which other configurations to attach")
    p.add_argument("--tuning", default="", help="tile_rows,tile_nnz,ctas_per_sm,carveout[,fold_permute_in[,fused_small]]: fixed tuning "
                   "instead of autotuning (keeps a profiler's launch list short)")
    return p.parse_args()


def fixed_tuning(a):
    """The --tuning value as a 4-tuple, or None (autotune)."""
    if not a.tuning:
        return None
    t = tuple(int(v) for v in a.tuning.split(","))
    if len(t) not in (4, 5, 6):
        raise SystemExit("--tuning wants tile_rows,tile_nnz,ctas_per_sm,carveout[,fold_permute_in[,fused_small]]")
    return t


def workload_spec(a):
    if a.workload == "grid3d":
        N = a.size or 400
        return dict(name="grid3d", N=N, b=4096, k=a.k or 16, iters=a.iters or 20, rescale=True,
                    dtype=a.dtype or "f32", seed_a=3, seed_x=4,
                    desc=f"3D {N}^3 grid 7-point stencil, U(0.5,1.5) row-normalised, b=4096")
    if a.workload == "grid2d":
        N = a.size or 64
        return dict(name="grid2d", N=N, b=64, k=a.k or 16, iters=a.iters or 10, rescale=False,
                    dtype=a.dtype or "f32", seed_a=1, seed_x=2,
                    desc=f"2D {N}x{N} grid 5-point stencil, U(0.5,1.5) row-normalised, b=64")
    s = a.size or 23
    return dict(name="rmat", N=s, b=8192, k=a.k or 128, iters=a.iters or 8, rescale=False,
                dtype=a.dtype or "bf16", seed_a=5, seed_x=6,
                desc=f"R-MAT scale {s} ef16 (0.57,0.19,0.19,0.05) symmetrised + self-loops, GCN-normalised, b=8192")


def make_matrix(spec):
    import workloads as w
    if spec["name"] == "grid3d":
        return w.grid3d(spec["N"], seed=spec["seed_a"])
    if spec["name"] == "grid2d":
        return w.grid_stencil((spec["N"], spec["N"]), seed=spec["seed_a"])
    return w.rmat_gcn(spec["N"], 16, seed=spec["seed_a"])


def make_sample(spec, rows_target):
    """A smaller matrix of the same family and structure, for the CPU oracle timing."""
    import workloads as w
    if spec["name"] == "grid3d":
        N = spec["N"]
        layers = max(1, min(N, rows_target // (N * N)))
        return w.grid_stencil((layers, N, N), seed=spec["seed_a"]), f"{layers}x{N}x{N} slab of the same grid"
    if spec["name"] == "grid2d":
        return make_matrix(spec), "the whole matrix"
    sc = max(10, min(spec["N"], int(math.log2(max(2, rows_target)))))
    return w.rmat_gcn(sc, 16, seed=spec["seed_a"]), f"R-MAT scale {sc} of the same family"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload_key(spec) -> str:
    """Short name of a single-matrix workload, as the traffic file records it."""
    return f"{spec['name']} N={spec['N']} k={spec['k']} {spec['dtype']} rescale={int(spec['rescale'])}"


def kernel_source_digest() -> str:
    """First 16 hex digits of the SHA-256 of the kernel sources, concatenated in order."""
    h = hashlib.sha256()
    for path in KERNEL_SRCS:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def kernel_traffic(workload: str):
    """DRAM bytes per iteration of the rows (+ split-row) kernels from the committed ncu summary
    (profiles/arrow_rows_traffic.txt: one block per workload, each starting with its
    'workload:' line), if the block for this workload was taken on the current kernel sources;
    else None."""
    path = os.path.join(ROOT, "profiles", "arrow_rows_traffic.txt")
    try:
        digest = kernel_source_digest()
        blocks, kv = [], None
        with open(path) as f:
            for line in f:
                if ":" not in line or line.startswith("#"):
                    continue
                k, v = line.split(":", 1)
                k, v = k.strip(), v.strip()
                if k == "workload":
                    kv = {}
                    blocks.append(kv)
                if kv is not None:
                    kv[k] = v
        for kv in blocks:
            if kv.get("workload") == workload and kv.get("kernel_source_sha256_16") == digest:
                return kv
        return None
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x, device="cuda"):
    """Largest value of x over the ranks (the whole-job time is the slowest rank's)."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms_max):
    """Whole-job throughput: every rank's units over the slowest rank's time (weak scaling)."""
    return world * units_per_rank / (ms_max / 1e3)


def cpu_oracle():
    """(iterate function, host threads it uses, description) of the CPU oracle: the C form of
    the FP64 product over all host cores, or the scipy form on one core if it cannot be built."""
    try:
        import __graft_entry__
        __graft_entry__._build_oracle_c()             # compiled by the build step; no-op when current
        from oracle import cspmm as C
        return C.iterate, C.threads(), "C FP64 CSR product (oracle/c), rows over the host cores"
    except Exception:
        from oracle import spmm as S
        return S.iterate, 1, "scipy FP64 CSR product, one core"


def cpu_oracle_time(spec, rows_target, reps):
    """Seconds per iteration of the FP64 oracle on a bounded sample; (s, rows, desc, cores, kind)."""
    import workloads as w
    it, cores, what = cpu_oracle()
    A, desc = make_sample(spec, rows_target)
    X = w.features(A.n, spec["k"], seed=spec["seed_x"]).astype(np.float64)
    try:
        it(A, X, 1, rescale=spec["rescale"])          # warm the caches once
    except Exception:                                  # the C form failed here: time the scipy form
        from oracle import spmm as S
        it, cores, what = S.iterate, 1, "scipy FP64 CSR product, one core"
        it(A, X, 1, rescale=spec["rescale"])
    t0 = time.perf_counter()
    it(A, X, reps, rescale=spec["rescale"])
    dt = time.perf_counter() - t0
    return dt / reps, A.n, desc, cores, what


def run_reference(a, spec):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import workloads as w
    it, cores, what = cpu_oracle()
    n_full = {"grid3d": spec["N"] ** 3, "grid2d": spec["N"] ** 2, "rmat": 1 << spec["N"]}[spec["name"]]
    A, desc = make_sample(spec, 8_000_000 if cores > 1 else 4_000_000)
    X = w.features(A.n, spec["k"], seed=spec["seed_x"]).astype(np.float64)
    try:
        it(A, X, 1, rescale=spec["rescale"])
    except Exception:                                  # the C form failed here: time the scipy form
        from oracle import spmm as S
        it, cores, what = S.iterate, 1, "scipy FP64 CSR product, one core"
    for _ in range(a.warmup):
        it(A, X, 1, rescale=spec["rescale"])
    t0 = time.perf_counter()
    for _ in range(a.steps):
        it(A, X, 1, rescale=spec["rescale"])
    dt = (time.perf_counter() - t0) / a.steps
    value = (A.n / n_full) / dt                         # full-matrix iterations per second
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": spec["desc"], "k": spec["k"], "iters": spec["iters"]},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
                             "sample": f"one FP64 iteration per step ({what}) on {desc} "
                                       f"({A.n:,} of {n_full:,} rows), scaled by rows"},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _batch_worker(task):
    """Spawned worker: generate one random-geometric matrix, decompose it on the host, save it."""
    i, n, seed, path, vdt = task
    import workloads as w
    import paper_2402_19364_gb300 as arrow
    A = w.rgg(int(n), seed=seed)
    b = int(math.ceil(math.sqrt(A.n)))
    M = arrow.ArrowMatrix(A, b, host_only=True, nthreads=1, value_dtype=vdt)
    M.save(path)
    return i, A.n, A.nnz, b


def run_batch(a):
    """Batched workload: `count` random-geometric graphs (n log-uniform in [1e3, 2e6], b = ceil(sqrt n),
    k in {8,16,32,64}, FP16 values and features, 10 iterations each) advanced by arrow_batch_spmm as one
    CUDA graph, against the FP32 form with one arrow_spmm call (one rows launch per iteration) per matrix."""
    import multiprocessing as mp
    import tempfile
    import torch
    import workloads as w
    from paper_2402_19364_gb300 import build as _build
    _build.build()
    import paper_2402_19364_gb300 as arrow
    count = a.count or 512
    iters = a.iters or 10
    sizes = w.log_uniform_sizes(count, 1e3, 2e6, 7)
    ks = [int(x) for x in np.random.default_rng(8).choice([8, 16, 32, 64], count)]
    tmp = tempfile.mkdtemp(prefix="arrow_batch_", dir="/dev/shm" if os.path.isdir("/dev/shm") else None)
    tasks = sorted([(i, int(sizes[i]), 7000 + i, os.path.join(tmp, f"m{i}.arw"), "f16") for i in range(count)],
                   key=lambda t: -t[1])
    t0 = time.perf_counter()
    info = {}
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        for i, n, nnz, b in pool.imap_unordered(_batch_worker, tasks):
            info[i] = (n, nnz, b)
    t_prep = time.perf_counter() - t0
    torch.cuda.set_device(0)
    mats16, mats32 = [], []
    for i in range(count):
        path = os.path.join(tmp, f"m{i}.arw")
        m16 = arrow.ArrowMatrix.load(path)
        mats16.append(m16)
        mats32.append(m16.copy("f32"))
        os.remove(path)
    os.rmdir(tmp)
    gen = torch.Generator(device="cuda").manual_seed(9)
    X16 = [torch.randn(m.n, k, device="cuda", generator=gen).half() for m, k in zip(mats16, ks)]
    Y16 = [torch.empty_like(x) for x in X16]
    X32 = [x.float() for x in X16]
    Y32 = [torch.empty_like(x) for x in X32]
    if fixed_tuning(a):
        for m in mats16:
            m.set_tuning(*fixed_tuning(a))
    B = arrow.ArrowBatch(mats16)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    if fixed_tuning(a):
        tuned = mats16[0].tuning
    else:
        tuned, tuned_ms = B.autotune(X16, iters, outs=Y16)
    t_tune = time.perf_counter() - t0
    for _ in range(max(3, a.warmup)):
        B.spmm(X16, iters, outs=Y16, graph=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(a.steps):
        B.spmm(X16, iters, outs=Y16, graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) / a.steps
    assert B.status() == 0
    for m, x, y in zip(mats32, X32, Y32):
        m.spmm(x, iters, out=y)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(a.steps):
        for m, x, y in zip(mats32, X32, Y32):
            m.spmm(x, iters, out=y)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_f = e0.elapsed_time(e1) / a.steps
    err = 0.0
    for y16, y32 in zip(Y16, Y32):
        err = max(err, float((torch.linalg.vector_norm(y16.float() - y32, dim=0) /
                              torch.linalg.vector_norm(y32, dim=0)).max()))
    bytes16 = sum(m.algorithmic_bytes_per_iter(k, "f16")["total"] for m, k in zip(mats16, ks)) * iters
    bytes32 = sum(m.algorithmic_bytes_per_iter(k, "f32")["total"] for m, k in zip(mats32, ks)) * iters
    rows = sum(m.n for m in mats16)
    nnz = sum(m.nnz for m in mats16)
    peak, peak_kind = load_peaks()
    out = {"metric": "arrow-SpMM batched matrix-iterations/s (512 random-geometric graphs, one CUDA graph)",
           "value": count * iters / (ms_b / 1e3), "unit": "matrix-iters/s", "n_gpus": 1, "steps": a.steps,
           "warmup": max(3, a.warmup), "ms_per_step": ms_b, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f16", "data": "synthetic",
           "config": {"workload": f"{count} 2D random-geometric graphs, n log-uniform [1e3, 2e6], mean degree 8, "
                                  f"b = ceil(sqrt n), k in {{8,16,32,64}}, {iters} iterations, FP16 values and X",
                      "rows": rows, "nnz": nnz, "sum_k_rows": sum(m.n * k for m, k in zip(mats16, ks)),
                      "launches_per_step": 2 + iters, "prep_s": t_prep, "autotuned": tuned,
                      "autotune_s": t_tune},
           "aggregate_GBps": bytes16 / (ms_b / 1e3) / 1e9, "frac_of_measured_hbm": bytes16 / (ms_b / 1e3) / 1e9 / peak,
           "fp32_one_launch_per_iteration": {"ms_per_step": ms_f, "matrix_iters_per_s": count * iters / (ms_f / 1e3),
                                            "aggregate_GBps": bytes32 / (ms_f / 1e3) / 1e9,
                                            "launches_per_step": count * (2 + iters)},
           "speedup_vs_fp32": ms_f / ms_b, "max_normwise_err_f16_vs_f32": err, "peak_kind": peak_kind}
    print(json.dumps(out), flush=True)


def _pool_worker(task):
    """Spawned worker: generate one matrix of the serving pool, decompose it, save it."""
    i, fam, n, seed, path = task
    import workloads as w
    import paper_2402_19364_gb300 as arrow
    if fam == "grid":
        N = max(8, int(round(n ** (1 / 3))))
        A = w.grid_stencil((N, N, N), seed=seed)
    elif fam == "rgg":
        A = w.rgg(int(n), seed=seed, round_to=None)
    else:
        A = w.rmat_gcn(max(10, int(round(math.log2(n)))), 16, seed=seed)
    b = int(math.ceil(math.sqrt(A.n)))
    M = arrow.ArrowMatrix(A, b, host_only=True, nthreads=4, value_dtype="bf16")
    M.save(path)
    return i, fam, A.n, A.nnz


def run_serve(a):
    """Serving workload: Poisson arrivals of requests on a pool of pre-decomposed matrices
    (grid / random-geometric / R-MAT, n log-uniform in [1e4, 8e6]), k in {16,32,64,128} BF16,
    iterations uniform in [5, 50]; continuous batching with admission by HBM footprint.
    Reports closed-loop capacity, then p50/p99 latency and throughput at 0.5, 0.8, 0.95 of it."""
    import multiprocessing as mp
    import tempfile
    import torch
    import workloads as w
    from paper_2402_19364_gb300 import build as _build
    _build.build()
    import paper_2402_19364_gb300 as arrow
    per_family = 6
    fams = ["grid", "rgg", "rmat"]
    sizes = w.log_uniform_sizes(per_family * 3, 1e4, 8e6, 11)
    tmp = tempfile.mkdtemp(prefix="arrow_pool_", dir="/dev/shm" if os.path.isdir("/dev/shm") else None)
    tasks = [(i, fams[i % 3], int(sizes[i]), 100 + i, os.path.join(tmp, f"p{i}.arw")) for i in range(per_family * 3)]
    t0 = time.perf_counter()
    info = {}
    with mp.get_context("spawn").Pool(4) as pool:
        for i, fam, n, nnz in pool.imap_unordered(_pool_worker, sorted(tasks, key=lambda t: -t[2])):
            info[i] = (fam, n, nnz)
    t_prep = time.perf_counter() - t0
    torch.cuda.set_device(0)
    mats = []
    for i in range(len(tasks)):
        mats.append(arrow.ArrowMatrix.load(os.path.join(tmp, f"p{i}.arw")))
        os.remove(os.path.join(tmp, f"p{i}.arw"))
    os.rmdir(tmp)
    gen = torch.Generator(device="cuda").manual_seed(12)
    xin = [torch.randn(m.n * 128, device="cuda", generator=gen).bfloat16() for m in mats]
    yout = [torch.empty(m.n * 128, device="cuda", dtype=torch.bfloat16) for m in mats]
    rng = np.random.default_rng(13)
    count = a.count or 5000

    def make_requests(cnt):
        return [(int(rng.integers(0, len(mats))), int(rng.choice([16, 32, 64, 128])), int(rng.integers(5, 51)))
                for _ in range(cnt)]

    budget = 64 << 30

    def run(reqs, arrivals):
        srv = arrow.ArrowServer(hbm_budget=budget, max_active=64, x_dtype="bf16", max_inflight=2)
        lat, delay, done_at = {}, {}, {}
        t_start = time.perf_counter()
        i = 0
        n = len(reqs)
        while len(lat) < n:
            now = time.perf_counter() - t_start
            while i < n and arrivals[i] <= now:
                m, k, it = reqs[i]
                X = xin[m][: mats[m].n * k].view(mats[m].n, k)
                Y = yout[m][: mats[m].n * k].view(mats[m].n, k)
                rid = srv.submit(mats[m], X, Y, it)
                delay[rid] = (time.perf_counter() - t_start) - arrivals[i]
                i += 1
            active = srv.step()
            for rid, l in srv.poll():
                lat[rid] = l + delay[rid]
                done_at[rid] = time.perf_counter() - t_start
            if active == 0 and i < n and not srv.stats()["inflight_steps"]:
                time.sleep(max(0.0, min(0.001, arrivals[i] - (time.perf_counter() - t_start))))
        st = srv.stats()
        srv.close()
        span = max(done_at.values()) - min(arrivals)
        v = np.array(list(lat.values()))
        return {"requests": n, "throughput_rps": n / span, "p50_ms": float(np.percentile(v, 50) * 1e3),
                "p99_ms": float(np.percentile(v, 99) * 1e3), "mean_ms": float(v.mean() * 1e3),
                "steps": st["steps"], "peak_state_bytes": st["peak_bytes"],
                "host_s_in_step": st["host_seconds"], "wait_s_for_gpu": st["wait_seconds"],
                "gpu_busy_s": st["gpu_seconds"], "gpu_busy_frac": st["gpu_seconds"] / span, "span_s": span}

    warm = make_requests(64)
    run(warm, np.zeros(len(warm)))
    closed = make_requests(min(count, 1000))
    cap = run(closed, np.zeros(len(closed)))
    C = cap["throughput_rps"]
    results = []
    stream_08 = None
    for frac in (0.5, 0.8, 0.95):
        reqs = make_requests(count if frac == 0.8 else min(count, 1000))
        arrivals = np.cumsum(rng.exponential(1.0 / (frac * C), count))
        arrivals -= arrivals[0]
        r = run(reqs, arrivals)
        r["rate_rps"] = frac * C
        r["load"] = frac
        results.append(r)
        if frac == 0.8:
            stream_08 = (reqs, arrivals)
    main = results[1]

    # The plain FP32 form on the same requests: one arrow_spmm call per request (FP32 values
    # and X, one rows launch per iteration), served one at a time in arrival order.  Each
    # request's device time is measured with CUDA events; the latencies follow from the
    # arrival times of the 0.8 C stream by FIFO order: finish_i = max(arrival_i,
    # finish_{i-1}) + service_i.
    fp32 = None
    if not a.no_fp32:
        n32 = min(len(stream_08[0]), 1000)
        mats32 = [m.copy("f32") for m in mats]
        x32 = [xin[i].float() for i in range(len(mats))]
        y32 = [torch.empty(m.n * 128, device="cuda", dtype=torch.float32) for m in mats]
        stream = torch.cuda.current_stream()
        for m, k, it in stream_08[0][:8]:                  # warm-up
            mats32[m].spmm(x32[m][: mats[m].n * k].view(mats[m].n, k), it, out=y32[m][: mats[m].n * k].view(mats[m].n, k))
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n32)]
        for (m, k, it), (s0, s1) in zip(stream_08[0][:n32], evs):
            s0.record(stream)
            mats32[m].spmm(x32[m][: mats[m].n * k].view(mats[m].n, k), it, out=y32[m][: mats[m].n * k].view(mats[m].n, k))
            s1.record(stream)
        torch.cuda.synchronize()
        service = np.array([s0.elapsed_time(s1) / 1e3 for s0, s1 in evs])
        arr = stream_08[1][:n32]
        finish = np.empty(n32)
        t = 0.0
        for i in range(n32):
            t = max(arr[i], t) + service[i]
            finish[i] = t
        lat = finish - arr
        fp32 = {"requests": n32, "capacity_rps": n32 / service.sum(), "mean_service_ms": float(service.mean() * 1e3),
                "at_0.8C": {"rate_rps": 0.8 * C, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                            "p99_ms": float(np.percentile(lat, 99) * 1e3),
                            "throughput_rps": n32 / (finish[-1] - arr[0])},
                "what": "FP32 values and X, one arrow_spmm call per request, one request at a time (FIFO) on the "
                        "first requests of the 0.8 C stream; latencies from the measured device times"}
        for m in mats32:
            m.close()
        del x32, y32
    out = {"metric": "arrow-SpMM serving p50/p99 latency and throughput (continuous batching)",
           "value": main["throughput_rps"], "unit": "requests/s", "p50_ms": main["p50_ms"], "p99_ms": main["p99_ms"],
           "n_gpus": 1, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
           "config": {"workload": f"{count} requests at 0.8 of capacity (1000 at 0.5 and 0.95), Poisson arrivals, pool of {len(mats)} pre-decomposed "
                                  "matrices (grid / random-geometric / R-MAT, n log-uniform [1e4, 8e6], b = ceil(sqrt n)), "
                                  "k in {16,32,64,128} BF16, iterations U{5..50}, 64 slots, 64 GiB state budget",
                      "pool": [{"family": info[i][0], "n": info[i][1], "nnz": info[i][2]} for i in range(len(mats))],
                      "prep_s": t_prep},
           "closed_loop": cap, "by_rate": results, "fp32_per_request": fp32}
    print(json.dumps(out), flush=True)


def time_calls(arrow, M, Xd, Yd, iters, rescale, steps, warmup, pg, stream, flush=None, sigma=None):
    """Warm-up calls, then `steps` timed arrow_spmm calls with CUDA events on the launching
    stream (barrier + synchronize on both sides, max over ranks).  With `flush` (a buffer
    larger than L2) the buffer is written between calls and each call is timed on its own.
    Per-kernel device times come from the library's own events (ARROW_PROFILE)."""
    import torch
    sigma = sigma or {}
    for _ in range(warmup):
        M.spmm(Xd, iters, rescale=rescale, out=Yd, **sigma)
    torch.cuda.synchronize()
    for kind in (arrow.ARROW_K_ROWS, arrow.ARROW_K_SEGMENTS, arrow.ARROW_K_NORM, arrow.ARROW_K_PERMUTE,
                 arrow.ARROW_K_FUSED):
        M.profile_get(kind)
    barrier(pg)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e0.record(stream)
    for i in range(steps):
        if flush is not None:
            flush.fill_(i & 0xff)
        starts[i].record(stream)
        M.spmm(Xd, iters, rescale=rescale, out=Yd, profile=True, **sigma)
        marks[i].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    step_ms = [starts[i].elapsed_time(marks[i]) for i in range(steps)]
    ms_total = sum(step_ms) if flush is not None else e0.elapsed_time(e1)
    ms_total = max_over_ranks(pg, ms_total)
    km, launches = {}, 0
    for name, kind in (("rows", arrow.ARROW_K_ROWS), ("segments", arrow.ARROW_K_SEGMENTS),
                       ("norm", arrow.ARROW_K_NORM), ("permute", arrow.ARROW_K_PERMUTE),
                       ("fused", arrow.ARROW_K_FUSED)):
        ms, cnt = M.profile_get(kind)
        km[name] = ms
        km[name + "_launches"] = cnt
        launches += cnt
    return {"ms_total": ms_total, "launches": launches,
            "kernel_ms": {c: km[c] for c in ("rows", "segments", "norm", "permute", "fused")},
            "rows_launches": km["rows_launches"], "segments_launches": km["segments_launches"],
            "fused_launches": km["fused_launches"], "iters_per_call": iters,
            "step_ms": {"mean": sum(step_ms) / len(step_ms), "min": min(step_ms), "max": max(step_ms)}}


def roofline_record(M, k, dt_name, tm, spec, peak, peak_kind):
    """roofline of one iteration's rows + split-row kernels: algorithmic bytes (A's values and
    indices, row pointers, every level's active X rows once, Y once) over their device time
    per iteration, against the measured HBM copy bandwidth.  traffic: DRAM bytes of one
    iteration from the committed ncu summary, when it was taken on this kernel source and
    this workload (spec None: not looked up)."""
    ab = M.algorithmic_bytes_per_iter(k, dt_name)
    if tm["fused_launches"]:
        # the one-launch path: the whole call in one kernel; per iteration = its time / iterations
        per_launch_s = tm["kernel_ms"]["fused"] / (tm["fused_launches"] * tm["iters_per_call"]) / 1e3
        kernel = "arrow_fused_small_kernel (whole call, per iteration)"
    else:
        per_launch_s = (tm["kernel_ms"]["rows"] + tm["kernel_ms"]["segments"]) / max(1, tm["rows_launches"]) / 1e3
        kernel = "arrow_rows_kernel" + (" + arrow_segments_kernel + arrow_combine_kernel"
                                        if tm["segments_launches"] else "")
    achieved = ab["total"] / per_launch_s / 1e9
    traffic = None
    tr = kernel_traffic(workload_key(spec)) if spec is not None else None
    if tr is not None:
        try:
            traffic = float(tr["dram_bytes_per_launch_full_size"])
        except (KeyError, ValueError):
            traffic = None
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": peak_kind, "kernel": kernel,
            "algorithmic_bytes_per_launch": ab["total"], "launch_ms": per_launch_s * 1e3,
            "frac_of_nominal_8000": achieved / 8000.0}


def cusparse_record(A, M, Xd, spec, dt_name, stream, reps=5):
    """cusparseSpMM (the bench-only comparator library, baseline/cusparse_spmm.cu) on the
    undecomposed matrix: every algorithm (default, CSR_ALG1..3) with row-major and
    column-major X, in natural vertex order and in the decomposition's first order pi_0, in
    FP32 and (16-bit workloads) in the workload's type; the best of each type is the
    comparator.  With the rescale, the column normalisation is timed as one HBM-speed pass
    (sum of squares, then scale) and added."""
    import ctypes
    import torch
    import __graft_entry__
    lib = ctypes.CDLL(__graft_entry__._build_cusparse_cmp())
    lib.cmp_cusparse_spmm.restype = ctypes.c_int
    lib.cmp_cusparse_spmm.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_float)]
    lib.cmp_column_normalise.restype = ctypes.c_int
    lib.cmp_column_normalise.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    dev = Xd.device
    n, k = A.n, Xd.shape[1]
    sp = ctypes.c_void_p(stream.cuda_stream)
    rowptr = torch.from_numpy(A.rowptr).to(dev)
    col = torch.from_numpy(A.colidx).to(dev).long()
    val = torch.from_numpy(A.values).to(dev, torch.float32)
    # pi_0 order: row p = vertex pi_0^{-1}(p), columns renamed by pi_0 and sorted in each row
    perm = torch.from_numpy(M.level_perm(0)).to(dev).long() if M.num_levels else torch.arange(n, device=dev)
    row = torch.repeat_interleave(torch.arange(n, device=dev), rowptr[1:] - rowptr[:-1])
    key = perm[row] * n + perm[col]
    del row
    key, order = torch.sort(key)
    rp_pi = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    rp_pi[1:] = torch.cumsum(torch.bincount(key // n, minlength=n), 0)
    forms = {"natural": (rowptr.int(), col.int(), val),
             "pi0": (rp_pi.int(), (key % n).int(), val[order])}
    del key, order, rp_pi, col
    types = [("f32", torch.float32, 0)] + ([(dt_name, torch.bfloat16, 1)] if dt_name == "bf16" else [])
    runs = []
    best = {}
    for tname, tdt, tcode in types:
        Xr = Xd.to(tdt).contiguous()
        Xc = Xr.t().contiguous()                      # column-major storage of the same n x k matrix
        Yr = torch.empty_like(Xr)
        for form, (rp, ci, va) in forms.items():
            vt = va.to(tdt)
            for layout, Xb in (("row", Xr), ("col", Xc)):
                for alg, aname in enumerate(("default", "csr_alg1", "csr_alg2", "csr_alg3")):
                    ms = ctypes.c_float(0.0)
                    Yb = Yr if layout == "row" else torch.empty_like(Xc)
                    rc = lib.cmp_cusparse_spmm(n, A.nnz, rp.data_ptr(), ci.data_ptr(), vt.data_ptr(), tcode,
                                               Xb.data_ptr(), Yb.data_ptr(), k, tcode, alg, int(layout == "col"), reps,
                                               sp, ctypes.byref(ms))
                    r = {"dtype": tname, "order": form, "layout": layout, "alg": aname}
                    if rc == 0:
                        r["ms"] = float(ms.value)
                        if tname not in best or r["ms"] < best[tname]["ms"]:
                            best[tname] = dict(r)
                    else:
                        r["error"] = rc
                    runs.append(r)
                    del Yb
            del vt
        del Xr, Xc, Yr
        torch.cuda.synchronize()
    rec = {"what": "cusparseSpMM (CSR, compute FP32) on the undecomposed matrix; best of algorithm x X layout x "
                   "vertex order", "best": best, "runs": runs}
    if "f32" in best:
        ms_it = best["f32"]["ms"]
        if spec["rescale"]:
            # one HBM-speed normalisation pass over the FP32 product (row-major)
            Y = torch.randn(n, k, device=dev)
            Z = torch.empty_like(Y)
            grid = 152 * 8
            part = torch.empty(grid * k, dtype=torch.float64, device=dev)
            inv = torch.empty(k, dtype=torch.float32, device=dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for i in range(reps + 2):
                if i == 2:
                    e0.record(stream)
                rc = lib.cmp_column_normalise(Y.data_ptr(), Z.data_ptr(), n, k, part.data_ptr(), grid, inv.data_ptr(), sp)
                if rc:
                    raise RuntimeError(f"cmp_column_normalise: {rc}")
            e1.record(stream)
            torch.cuda.synchronize()
            ms_norm = e0.elapsed_time(e1) / reps
            rec["ms_column_norm"] = ms_norm
            rec["column_norm_GBps"] = 3 * n * k * 4 / (ms_norm / 1e3) / 1e9
            ms_it += ms_norm
            del Y, Z, part, inv
        rec["ms_per_iter"] = ms_it
        rec["iters_per_s"] = 1e3 / ms_it
    return rec


# Configurations measured beside the headline in the default run (each in its own process,
# after the headline's device memory is released): (key, bench arguments).
SUBRECORDS = [
    ("grid2d", ["--workload", "grid2d", "--steps", "50", "--warmup", "5"]),
    ("rmat", ["--workload", "rmat", "--steps", "5", "--warmup", "3"]),
    ("batch", ["--workload", "batch", "--steps", "5", "--warmup", "3"]),
    ("serve", ["--workload", "serve"]),
    ("predicates", ["--workload", "predicates", "--steps", "3"]),
]


def run_subrecords(keys, timeout_s=1800):
    """Run the other configurations as child processes; their JSON lines, keyed."""
    recs = {}
    for key, args in SUBRECORDS:
        if key not in keys:
            continue
        t0 = time.perf_counter()
        try:
            r = subprocess.run([sys.executable, os.path.abspath(__file__), *args], cwd=ROOT, capture_output=True,
                               text=True, timeout=timeout_s)
            lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
            if r.returncode != 0 or not lines:
                recs[key] = {"error": f"rc={r.returncode}: " + (r.stderr.strip().splitlines() or [""])[-1][:300]}
            else:
                recs[key] = json.loads(lines[-1])
        except Exception as ex:
            recs[key] = {"error": str(ex)[:300]}
        recs[key]["wall_s"] = time.perf_counter() - t0
    return recs


def run_predicates(a):
    """The two arrow shapes on the GPU (Section 1's band |p - q| <= b against the block-diagonal
    tiles of Section 3.1): levels, non-zero b x b tiles, algorithmic bytes per iteration and the
    measured time of the same product on a 3D 200^3 grid (k = 16 FP32, 20 iterations with the
    rescale) and an R-MAT scale 21 graph (k = 128 BF16, 8 iterations); plus the block form's time
    with the fused sigma epilogues (ReLU and row normalisation) on."""
    import torch
    import workloads as w
    from paper_2402_19364_gb300 import build as _build
    _build.build()
    import paper_2402_19364_gb300 as arrow
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    cases = [("3D 200^3 grid, b = 4096, k = 16 FP32, 20 iterations with the rescale", w.grid3d(200, seed=3), 4096, 16,
              "f32", 20, True),
             ("R-MAT scale 21 GCN, b = 8192, k = 128 BF16, 8 iterations", w.rmat_gcn(21, 16, seed=5), 8192, 128, "bf16",
              8, False)]
    out = {"metric": "arrow-SpMM band vs block predicate (levels, tiles, bytes, time)", "data": "synthetic",
           "n_gpus": 1, "cases": []}
    for desc, A, b, k, dt, iters, rs in cases:
        X = torch.from_numpy(w.features(A.n, k, seed=4)).cuda().to({"f32": torch.float32, "bf16": torch.bfloat16}[dt])
        rec = {"workload": desc, "n": A.n, "nnz": A.nnz}
        ref = None
        for pred in ("block", "band"):
            M = arrow.ArrowMatrix(A, b, value_dtype=dt, predicate=pred)
            M.autotune(X, iters, rescale=rs)
            Y = torch.empty_like(X)
            tm = time_calls(arrow, M, X, Y, iters, rs, max(3, a.steps), 3, None, stream)
            rep = M.structure_report()
            ab = M.algorithmic_bytes_per_iter(k, dt)
            rec[pred] = {"levels": M.num_levels, "tiles": rep["tiles"], "level0_nnz_share": rep["levels"][0]["nnz_share"],
                         "algorithmic_bytes_per_iter": ab["total"],
                         "ms_per_iter": tm["ms_total"] / max(3, a.steps) / iters,
                         "rows_segments_ms_per_iter": (tm["kernel_ms"]["rows"] + tm["kernel_ms"]["segments"])
                         / max(1, tm["rows_launches"])}
            if pred == "block":
                # the same product with sigma = rownorm(relu(.)) fused into the row stores
                ts = time_calls(arrow, M, X, torch.empty_like(X), iters, rs, max(3, a.steps), 3, None, stream,
                                sigma={"relu": True, "rownorm": True})
                rec["block_relu_rownorm_ms_per_iter"] = ts["ms_total"] / max(3, a.steps) / iters
            Yf = Y.float()
            if ref is None:
                ref = Yf
            else:
                rec["max_normwise_diff_band_vs_block"] = float(
                    (torch.linalg.vector_norm(Yf - ref, dim=0) / torch.linalg.vector_norm(ref, dim=0)).max())
            M.close()
        out["cases"].append(rec)
        del X, ref
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def main():
    a = parse()
    if a.workload == "predicates":
        run_predicates(a)
        return
    if a.workload == "batch":
        run_batch(a)
        return
    if a.workload == "serve":
        run_serve(a)
        return
    spec = workload_spec(a)
    if a.impl == "reference":
        run_reference(a, spec)
        return
    import torch
    rank, world, local, pg = dist_init()
    torch.cuda.set_device(local)
    from paper_2402_19364_gb300 import build as _build
    _build.build()
    import paper_2402_19364_gb300 as arrow

    t0 = time.perf_counter()
    A = make_matrix(spec)
    t_gen = time.perf_counter() - t0
    k, iters, dt_name = spec["k"], spec["iters"], spec["dtype"]
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[dt_name]
    t0 = time.perf_counter()
    M = arrow.ArrowMatrix(A, spec["b"], value_dtype=dt_name, device=local)
    t_dec = time.perf_counter() - t0
    st = M.stats()
    # the same decomposition with its data-parallel steps on the GPU (ARROW_DEVICE_DECOMPOSE):
    # timed, and checked equal to the host one (first and last level permutations)
    dev_dec = None
    if not a.no_device_decompose:
        t0 = time.perf_counter()
        Md = arrow.ArrowMatrix(A, spec["b"], value_dtype=dt_name, device=local, host_only=False,
                               device_decompose=True)
        t_dd = time.perf_counter() - t0
        same = Md.num_levels == M.num_levels and all(
            np.array_equal(Md.level_perm(i), M.level_perm(i)) for i in {0, M.num_levels - 1} if M.num_levels)
        dev_dec = {"decompose_and_upload": t_dd, "decompose": Md.stats()["decompose_seconds"],
                   "same_permutations_as_host": bool(same)}
        Md.close()
    levels = [M.level_info(i) for i in range(M.num_levels)]
    import workloads as w
    Xh = torch.from_numpy(w.features(A.n, k, seed=spec["seed_x"] + 1000 * rank)).to(tdt)
    Xd = Xh.cuda()
    Yd = torch.empty_like(Xd)
    stream = torch.cuda.current_stream()
    # inputs smaller than L2 (the 2D 64x64 latency case) get an L2 flush between timed steps
    flush = None
    if Xd.numel() * Xd.element_size() * 2 + A.nnz * 8 < 512 << 20:
        flush = torch.empty(512 << 20, dtype=torch.uint8, device=Xd.device)

    t0 = time.perf_counter()
    if fixed_tuning(a):
        M.set_tuning(*fixed_tuning(a))
        tuned = M.tuning
    else:
        tuned, _ = M.autotune(Xd, iters, rescale=spec["rescale"], out=Yd)   # arrow_autotune keeps the fastest
    t_tune = time.perf_counter() - t0

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    tm = time_calls(arrow, M, Xd, Yd, iters, spec["rescale"], a.steps, max(3, a.warmup), pg, stream, flush)
    clk = clocks.stop()
    ms_total = tm["ms_total"]
    ms_step = ms_total / a.steps
    value = job_value(a.steps * iters, world, ms_total)
    peak, peak_kind = load_peaks()
    roofline = roofline_record(M, k, dt_name, tm, spec, peak, peak_kind)

    out = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": a.steps,
           "warmup": max(3, a.warmup), "ms_per_step": ms_step, "step_ms": tm["step_ms"],
           "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": dt_name, "data": "synthetic",
           "config": {"workload": spec["desc"], "n": A.n, "nnz": A.nnz, "b": spec["b"], "k": k, "iters": iters,
                      "rescale_fp64": spec["rescale"], "levels": [list(x) for x in levels],
                      "long_rows": st["long_rows"], "segments": st["segments"], "autotuned": tuned,
                      "l2": ("inputs larger than L2 (no flush)" if flush is None else
                             "inputs smaller than L2: a 512 MiB buffer is written between timed steps, "
                             "which are timed one by one"),
                      "parallelism": f"replicas x{world}"},
           "roofline": roofline, "gpu_launches": tm["launches"], "clocks": clk,
           "kernel_ms": {c: v / a.steps for c, v in tm["kernel_ms"].items()},
           "prep_s": {"generate": t_gen, "decompose_and_upload": t_dec, "decompose_host": st["decompose_seconds"],
                      "autotune": t_tune, "device_decompose": dev_dec}}
    if spec["name"] == "grid2d":
        out["us_per_iter"] = ms_step / iters * 1e3

    # ---- the same workload through the FP32 path (values and X in FP32), beside the 16-bit one ----
    if dt_name != "f32" and not a.no_fp32:
        M32 = M.copy("f32")
        X32 = Xd.float()
        Y32 = torch.empty_like(X32)
        if fixed_tuning(a):
            M32.set_tuning(*fixed_tuning(a))
            tuned32 = M32.tuning
        else:
            tuned32, _ = M32.autotune(X32, iters, rescale=spec["rescale"], out=Y32)
        t32 = time_calls(arrow, M32, X32, Y32, iters, spec["rescale"], a.steps, max(3, a.warmup), pg, stream, flush)
        M.spmm(Xd, iters, rescale=spec["rescale"], out=Yd)
        torch.cuda.synchronize()
        rel = (torch.linalg.vector_norm(Yd.float() - Y32, dim=0) / torch.linalg.vector_norm(Y32, dim=0)).max()
        out["fp32_arm"] = {"value": job_value(a.steps * iters, world, t32["ms_total"]), "unit": "iters/s",
                           "ms_per_step": t32["ms_total"] / a.steps, "autotuned": tuned32,
                           "roofline": roofline_record(M32, k, "f32", t32, None, peak, peak_kind),
                           "kernel_ms": {c: v / a.steps for c, v in t32["kernel_ms"].items()},
                           "max_normwise_diff_vs_16bit": float(rel),
                           "what": "the same decomposition with FP32 values and FP32 X (arrow_handle_copy)"}
        M32.close()
        del X32, Y32
        torch.cuda.empty_cache()

    # ---- end to end through the public call, host buffers, copies inside the timed region ----
    # Every step copies its inputs from pinned host memory, runs arrow_spmm_ws and reads its
    # result back.  Two steps are in flight on two streams (each with its own device buffers
    # and workspace), so one step's copies overlap the other's kernels; the one-stream form
    # (copy, compute, copy, nothing overlapped) is reported beside it.
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if not a.no_e2e:
        Xp = Xh.pin_memory()
        Yps = [torch.empty_like(Xp).pin_memory() for _ in range(2)]
        Xds = [Xd, torch.empty_like(Xd)]
        Yds = [Yd, torch.empty_like(Yd)]
        wss = [torch.empty(M.workspace_size(k, dt_name, spec["rescale"]), dtype=torch.uint8, device=Xd.device)
               for _ in range(2)]
        side = [torch.cuda.Stream(device=Xd.device) for _ in range(2)]

        # the compute of a step waits for the previous step's compute (an event), so the two
        # streams' kernels do not run side by side and split the SMs and L2 between two working
        # sets, while each step's copies still overlap the other step's kernels
        last = [None]

        def e2e_step(i, s):
            with torch.cuda.stream(s):
                Xds[i % 2].copy_(Xp, non_blocking=True)
                if last[0] is not None:
                    s.wait_event(last[0])
                M.spmm_ws(Xds[i % 2], iters, wss[i % 2], rescale=spec["rescale"], out=Yds[i % 2], stream=s)
                ev = torch.cuda.Event()
                ev.record(s)
                last[0] = ev
                Yps[i % 2].copy_(Yds[i % 2], non_blocking=True)

        def e2e_run(steps, streams):
            last[0] = None
            e0.record(stream)
            for s in streams:
                s.wait_stream(stream)
            for i in range(steps):
                e2e_step(i, streams[i % len(streams)])
            for s in streams:
                stream.wait_stream(s)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        e2e_run(2, side)                                  # warm-up
        barrier(pg)
        ms_serial = max_over_ranks(pg, e2e_run(a.steps, side[:1]))
        barrier(pg)
        ms_e2e = max_over_ranks(pg, e2e_run(a.steps, side))
        nb = Xp.numel() * Xp.element_size()
        out["e2e"] = {"value": world * a.steps * iters / (ms_e2e / 1e3), "unit": "iters/s",
                      "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb, "ms_per_step": ms_e2e / a.steps,
                      "steps_in_flight": 2, "compute_serialised_across_streams": True,
                      "one_stream": {"value": world * a.steps * iters / (ms_serial / 1e3),
                                     "ms_per_step": ms_serial / a.steps}}
        del Xp, Yps, Xds, Yds, wss

    # ---- cuSPARSE SpMM on the undecomposed matrix (measured comparison) ----------------------
    if not a.no_cusparse and rank == 0:
        try:
            out["cusparse"] = cusparse_record(A, M, Xd, spec, dt_name, stream)
        except Exception as ex:  # comparator only: report, do not fail the bench
            out["cusparse"] = {"error": str(ex)[:300]}
        torch.cuda.empty_cache()

    # ---- CPU oracle on the host cores (bounded sample) ----------------------------------------
    if not a.no_cpu and rank == 0:
        s_per_iter, rows, desc, cores, what = cpu_oracle_time(spec, 12_000_000, 2)
        v = (rows / A.n) / s_per_iter
        out["cpu_baseline"] = {"value": v, "unit": "iters/s", "cores": cores, "kind": "oracle",
                               "sample": f"2 FP64 iterations ({what}) on {desc} "
                                         f"({rows:,} of {A.n:,} rows), scaled by rows"}
    M.close()
    if (spec["name"] == "grid3d" and not a.no_sub and world == 1 and not a.size and not a.k and not a.iters
            and not a.dtype and not a.tuning):
        del Xd, Yd, Xh
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        out["configs"] = run_subrecords([x for x in a.sub.split(",") if x])
    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
