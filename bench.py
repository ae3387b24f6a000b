#!/usr/bin/env python
"""Benchmark of the generalized H^2-LDL^T inertia path on GB300.

Workload (the n = 1024 configuration): n = 1024 points uniform in the unit
square (SplitMix64 seed 1), A_ij = 1/(|x_i - x_j| + 1e-3) (A_ii = 1e3), leaf
64, rank 16, eta = 1 (box admissibility), FP64.  A step is one batch of 256
shifted matrices A~ - sigma I factorized together (all levels: leaf blocks,
fill-in recompression, Bunch-Kaufman LDL^T, Schur updates, merges, negative
pivot count); the shifts of step i are 64 points spread over the Gershgorin
interval (seeded jitter), resident in HBM before the timed region.

value : LDL-inertia shifts/sec, device-resident shifts (h2_inertia_device).
e2e   : the same metric through h2_inertia with host (pinned) buffers: the H2D
        copy of the 256 shifts and the D2H read of the 256 counts in every step.
Extra keys: k-th eigenvalue solves (k = n/2, tol 1e-8) -- eigs/sec, p50/p99
latency, rounds, shifts per solve, on a 64-lane handle.

Multi-GPU (torchrun): every rank holds its own replica and factorizes its own
batches (independent shifts, no data-path collective); value = all ranks'
shifts / max-over-ranks time ("scaling": "weak").

--impl reference times the CPU oracle (the plain FP64 generalized H^2-LDL) on
the host cores on the same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

WORKLOADS = {
    # the default bench workload: n = 1024 uniform in the unit square, 1/(r+1e-3)
    "laplace2d_n1024": dict(name="laplace2d_n1024", n=1024, d=2, seed=1, kernel=W.LAPLACE_EPS,
                            kparams=(1e-3, 0.0, 0.0, 0.0), leaf=64, rank=16, eta=1.0, k=512, tol=1e-8),
    # the precision configuration: cylindrical lattice (radius 5, spacing 0.14,
    # jitter 0.01), exp(-r^2/2) + 1e-2/(r + 0.1), leaf 256, rank 48
    "cylinder_n262144": dict(name="cylinder_n262144", n=262144, d=3, seed=4, kernel=W.GAUSS_PLUS_INV,
                             kparams=(1e-2, 0.1, 0.0, 0.0), leaf=256, rank=48, eta=1.0, k=131072, tol=1e-8),
    # the 3D Yukawa configuration: n = 65536 uniform in the unit cube
    "yukawa3d_n65536": dict(name="yukawa3d_n65536", n=65536, d=3, seed=2, kernel=W.YUKAWA_EPS,
                            kparams=(1e-3, 0.0, 0.0, 0.0), leaf=256, rank=32, eta=1.0, k=32768, tol=1e-8),
}
WORKLOAD = WORKLOADS["laplace2d_n1024"]


def _points(wl):
    if wl["name"].startswith("cylinder"):
        return W.cylinder_lattice(wl["n"], wl["seed"])
    return W.uniform_cube(wl["n"], wl["d"], wl["seed"])
METRIC = "LDL-inertia shifts/sec (FP64); k-th eigs/sec at tol 1e-8 with p50/p99"
FP64_PEAK_GFLOPS = 1250.0   # nominal GB300 FP64 rate (the measured-peaks file has no FP64 entry)
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per k_schur launch,
# the mean over the 31 launches of one batch, from the committed ncu summary of
# k_schur at this workload under profiles/; valid for that workload and lane
# count while the kernel's source is unchanged (sha256 prefix of its text)
NCU_TRAFFIC = {"kernel": "k_schur", "workload": "laplace2d_n1024", "lanes": 256,
               "bytes_per_launch": 323.52e6, "source_sha": "7ddfe31f5f9903ac"}
KERNEL_REGIONS = {"k_schur": ("h2_factor.cu", "// S_ab[i0:i0+32, j0:j0+32] -= W_a Y_b^T (Eq. blr2-diag-schur).",
                               "// FP64-accurate Schur products on the tensor cores")}


def _fp64_peak_gflops(dev):
    """FP64 peak measured in this run: cuBLAS DGEMM (torch.matmul on float64),
    8192^3, best of 3 after a warm-up, timed with CUDA events."""
    import torch
    n = 8192
    a = torch.randn((n, n), dtype=torch.float64, device=dev)
    b = torch.randn((n, n), dtype=torch.float64, device=dev)
    c = a @ b
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        c = a @ b
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b, c
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / (best * 1e-3) / 1e9


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def _kernel_sha(kernel):
    """sha256 prefix of a kernel's source text (None if it cannot be located)."""
    if kernel not in KERNEL_REGIONS:
        return None
    f, start, end = KERNEL_REGIONS[kernel]
    with open(os.path.join(ROOT, "paper_2311_08618_gb300", "csrc", f)) as fh:
        src = fh.read()
    a = src.find(start)
    b = src.find(end, a + 1)
    if a < 0 or b < 0:
        return None
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:16]


def _shift_batches(lo, hi, lanes, count, seed=7):
    """count batches of lanes shifts spread over [lo, hi] with seeded jitter."""
    u = W.uniform(seed, count * lanes).reshape(count, lanes)
    base = (np.arange(lanes)[None, :] + u) / lanes
    return lo + (hi - lo) * base


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
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
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    import torch
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, local, dist


def _max_over_ranks(x, dist, device):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(dist):
    if dist is not None:
        dist.barrier()


# ------------------------------------------------------------- CPU oracle --
def _oracle_worker(args):
    """Spawned worker: builds the oracle H^2 matrix, waits, times its shifts."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    wl, warm, shifts, barrier = args
    sys.path.insert(0, ROOT)
    import workloads as Wk
    from oracle import h2 as oh2
    X = Wk.uniform_cube(wl["n"], wl["d"], wl["seed"])
    h = oh2.construct(X, wl["kernel"], wl["kparams"], wl["leaf"], wl["rank"], wl["eta"])
    for s in warm:
        oh2.h2_inertia(h, s)
    barrier.wait()
    t0 = time.time()
    counts = [oh2.h2_inertia(h, s)[0] for s in shifts]
    return t0, time.time(), counts


def oracle_throughput(shifts, cores, warm=()):
    """Shifts/sec of the oracle over `shifts`, one process per core (spawn);
    each worker first evaluates its share of `warm` untimed."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    env_before = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_before:
        os.environ[k] = "1"
    try:
        mgr = ctx.Manager()
        bar = mgr.Barrier(cores)
        parts = [list(shifts[i::cores]) for i in range(cores)]
        wparts = [list(warm[i::cores]) for i in range(cores)]
        with ctx.Pool(cores) as pool:
            res = pool.map(_oracle_worker, [(WORKLOAD, w, p, bar) for w, p in zip(wparts, parts)])
    finally:
        for k, v in env_before.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    t0 = min(r[0] for r in res)
    t1 = max(r[1] for r in res)
    counts = {}
    for p, r in zip(parts, res):
        for s, c in zip(p, r[2]):
            counts[s] = c
    return len(shifts) / (t1 - t0), t1 - t0, counts


def reference_arm(args, rank, world, dist):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    from oracle import dense
    X = W.uniform_cube(WORKLOAD["n"], WORKLOAD["d"], WORKLOAD["seed"])
    A = dense.kernel_matrix(WORKLOAD["kernel"], WORKLOAD["kparams"], X)
    lo, hi = dense.gershgorin(A)
    per_step = cores                      # one shift per core per step
    total = args.warmup + args.steps
    batches = _shift_batches(lo, hi, per_step, total, seed=11)
    rate, secs, _ = oracle_throughput(list(batches[args.warmup:].ravel()), cores,
                                      warm=list(batches[:args.warmup].ravel()))
    ms_step = secs / args.steps * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "shifts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "leaf": 64, "rank": 16, "eta": 1.0,
                       "shifts_per_step": per_step},
            "cpu_baseline": {"value": rate, "unit": "shifts/s", "cores": cores, "kind": "oracle",
                             "sample": "%d shifts of the %s workload, one process per core"
                                       % (per_step * args.steps, WORKLOAD["name"])},
            "e2e": {"value": rate, "unit": "shifts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- our path --
def ours(args, rank, world, local, dist):
    import torch
    import paper_2311_08618_gb300 as pkg
    from paper_2311_08618_gb300 import build
    if rank == 0:
        build.build()
    _barrier(dist)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    # a dedicated stream: the library and the CUDA events both use it
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        _ours_on_stream(args, rank, world, local, dist, pkg, dev, stream)


def _finish_short(args, rank, world, M, info, value, e2e_value, lanes, ms_max, clocks, build_s, same):
    """Line for a workload measured without the k-th solves (large configurations)."""
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "shifts/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == 0 else "f64+f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD["name"], "n": WORKLOAD["n"], "leaf": WORKLOAD["leaf"],
                           "rank": WORKLOAD["rank"], "eta": WORKLOAD["eta"], "shifts_per_step": lanes,
                           "precision": ["fp64", "mixed"][args.precision],
                           "workspace_gb": info["workspace_bytes"] / 1e9},
                "e2e": {"value": e2e_value, "unit": "shifts/s", "h2d_bytes_per_step": 8 * lanes,
                        "d2h_bytes_per_step": 8 * lanes, "counts_match_device_path": same},
                "gpu_launches": info["kernels_per_batch"] * args.steps, "build_s": build_s, "clocks": clocks,
                "info": {k: info[k] for k in ("levels", "leaves", "max_rank", "near_pairs", "fill_pairs",
                                              "norm_inf", "kernels_per_batch")}}
        print(json.dumps(line), flush=True)
    M.close()


def _ours_on_stream(args, rank, world, local, dist, pkg, dev, stream):
    import torch
    lanes = args.lanes
    X = _points(WORKLOAD)
    t0 = time.time()
    M = pkg.H2Matrix(X, WORKLOAD["kernel"], WORKLOAD["kparams"], leaf=WORKLOAD["leaf"], rank=WORKLOAD["rank"],
                     eta=WORKLOAD["eta"], max_lanes=lanes, stream=stream.cuda_stream, precision=args.precision,
                     autotune=1)
    torch.cuda.synchronize()
    build_s = time.time() - t0
    info = M.h2_info()
    lo, hi = info["gershgorin_lo"], info["gershgorin_hi"]
    total = args.warmup + args.steps
    sh = _shift_batches(lo, hi, lanes, total, seed=7 + rank)
    d_sh = torch.tensor(sh, dtype=torch.float64, device=dev)
    d_cnt = torch.zeros((total, lanes), dtype=torch.int64, device=dev)
    d_mp = torch.zeros((total, lanes), dtype=torch.float64, device=dev)
    assert stream.cuda_stream != 0
    # ---- device-resident timed region
    for i in range(args.warmup):
        M.h2_inertia_device(d_sh[i], lanes, d_cnt[i], d_mp[i])
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    _barrier(dist)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.warmup, total):
        M.h2_inertia_device(d_sh[i], lanes, d_cnt[i], d_mp[i])
    e1.record(stream)
    torch.cuda.synchronize()
    _barrier(dist)
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    ms_max = _max_over_ranks(ms, dist, dev)
    value = world * args.steps * lanes / (ms_max / 1e3)
    cnt_fp64 = d_cnt.clone()          # FP64 counts (the buffers are reused below)
    # ---- end to end: host (pinned) shifts in, host counts out, every step
    h_sh = torch.tensor(sh, dtype=torch.float64).pin_memory()
    h_cnt = torch.zeros((total, lanes), dtype=torch.int64).pin_memory()
    L = pkg.lib()
    import ctypes as C

    def e2e_step(i):
        rc = L.h2_inertia(M._h, C.c_void_p(h_sh[i].data_ptr()), lanes, C.c_void_p(h_cnt[i].data_ptr()), None)
        if rc != 0:
            raise RuntimeError(L.h2_last_error().decode())

    for i in range(args.warmup):
        e2e_step(i)
    _barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.warmup, total):
        e2e_step(i)
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks(time.perf_counter() - t0, dist, dev)
    _barrier(dist)
    e2e_value = world * args.steps * lanes / e2e_s
    same = bool(torch.equal(d_cnt.cpu(), h_cnt))
    info = M.h2_info()
    # ---- k-th eigenvalue solves (all of the path incl. the bisection driver),
    # on a handle with eig_lanes lanes (latency: fewer lanes per round)
    if args.eig_solves <= 0:
        return _finish_short(args, rank, world, M, info, value, e2e_value, lanes, ms_max, clocks, build_s, same)
    Me = pkg.H2Matrix(X, WORKLOAD["kernel"], WORKLOAD["kparams"], leaf=WORKLOAD["leaf"], rank=WORKLOAD["rank"],
                      eta=WORKLOAD["eta"], max_lanes=args.eig_lanes, stream=stream.cuda_stream)
    lat = []
    lam = None
    for i in range(args.eig_solves + 2):
        torch.cuda.synchronize()
        t = time.perf_counter()
        out, eb = Me.h2_kth_eig([WORKLOAD["k"]], WORKLOAD["tol"])
        lat.append(time.perf_counter() - t)
        lam = (out[0], eb[0])
    lat = np.array(lat[2:])
    info2 = Me.h2_info()
    Me.close()
    # latency of one k-th solve against the lanes per round: (q+1)-section
    # needs fewer rounds with more lanes, but each round's batch takes longer
    eig_sweep = []
    for ln in (8, 16, 32, 64):
        Ms = pkg.H2Matrix(X, WORKLOAD["kernel"], WORKLOAD["kparams"], leaf=WORKLOAD["leaf"], rank=WORKLOAD["rank"],
                          eta=WORKLOAD["eta"], max_lanes=ln, stream=stream.cuda_stream)
        ls = []
        for i in range(5):
            torch.cuda.synchronize()
            t = time.perf_counter()
            Ms.h2_kth_eig([WORKLOAD["k"]], WORKLOAD["tol"])
            ls.append(time.perf_counter() - t)
        inf_s = Ms.h2_info()
        eig_sweep.append({"lanes": ln, "p50_ms": float(np.percentile(ls[2:], 50) * 1e3),
                          "rounds": inf_s["last_rounds"], "shifts": inf_s["last_shifts"]})
        Ms.close()
    # ---- all n eigenvalues in one call (spectrum slicing with the reuse of
    # every (mu, nu) for every k, Sec. 4.2), on the throughput handle
    all_eigs = None
    if args.all_eigs and WORKLOAD["n"] <= 8192:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lam_all, eb_all = M.h2_kth_eig(np.arange(1, WORKLOAD["n"] + 1), WORKLOAD["tol"])
        t_all = time.perf_counter() - t0
        inf_all = M.h2_info()
        all_eigs = {"k": "1..%d" % WORKLOAD["n"], "tol": WORKLOAD["tol"], "lanes": lanes, "seconds": t_all,
                    "eigs_per_s": WORKLOAD["n"] / t_all, "rounds": inf_all["last_rounds"],
                    "shifts": inf_all["last_shifts"], "max_err_bound": float(eb_all.max()),
                    "sorted": bool(np.all(np.diff(lam_all) >= 0))}
    # ---- roofline of the dominant kernel: profiled batches (events per launch)
    prof = None
    for i in range(args.warmup, min(total, args.warmup + 5)):
        p = M.h2_profile_batch(d_sh[i], lanes, d_cnt[i])
        if prof is None:
            prof = p
        else:
            for k in prof:
                for f in ("ms", "flops", "bytes"):
                    prof[k][f] += p[k][f]
                prof[k]["launches"] += p[k]["launches"]
    dom = max((k for k in prof if k != "other" and prof[k]["launches"] > 0), key=lambda k: prof[k]["ms"])
    tot_ms = sum(v["ms"] for v in prof.values())
    pk = prof[dom]
    per_launch_ms = pk["ms"] / pk["launches"]
    flops_launch = pk["flops"] / pk["launches"]
    bytes_launch = pk["bytes"] / pk["launches"]
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6746.0)
    try:
        fp64_gf = _fp64_peak_gflops(dev)
        fp64_src = "measured in this run: cuBLAS DGEMM 8192^3 (torch.matmul float64), best of 3"
    except Exception as ex:  # noqa: BLE001
        fp64_gf = FP64_PEAK_GFLOPS
        fp64_src = "nominal FP64 (recipe table); DGEMM measurement failed: %s" % ex
    ai = flops_launch / max(bytes_launch, 1.0)
    if ai > fp64_gf / hbm:
        achieved = flops_launch / (per_launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_gf / 1e3, "unit": "TFLOP/s",
                "frac": achieved / (fp64_gf / 1e3), "peak_source": fp64_src,
                "frac_of_nominal_1250": achieved / 1.25}
    else:
        achieved = bytes_launch / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_source": "measured hbm_gbs"}
    traffic = None
    if NCU_TRAFFIC["bytes_per_launch"] and NCU_TRAFFIC["kernel"] == "k_" + dom and \
            NCU_TRAFFIC["workload"] == WORKLOAD["name"] and NCU_TRAFFIC["lanes"] == lanes and \
            NCU_TRAFFIC["source_sha"] == _kernel_sha(NCU_TRAFFIC["kernel"]):
        traffic = NCU_TRAFFIC["bytes_per_launch"]
    roof.update({"kernel": "k_" + dom, "traffic": traffic, "flops_per_launch": flops_launch,
                 "bytes_per_launch": bytes_launch, "launch_ms": per_launch_ms,
                 "share_of_batch": pk["ms"] / tot_ms,
                 "kernel_shares": {k: v["ms"] / tot_ms for k, v in prof.items()}})
    # ---- precision variant: FP32 Schur/rotation products, FP64 pivots/counts
    Mx = pkg.H2Matrix(X, WORKLOAD["kernel"], WORKLOAD["kparams"], leaf=WORKLOAD["leaf"], rank=WORKLOAD["rank"],
                      eta=WORKLOAD["eta"], max_lanes=lanes, stream=stream.cuda_stream,
                      precision=pkg.H2_PREC_MIXED)
    Mxe = pkg.H2Matrix(X, WORKLOAD["kernel"], WORKLOAD["kparams"], leaf=WORKLOAD["leaf"], rank=WORKLOAD["rank"],
                       eta=WORKLOAD["eta"], max_lanes=args.eig_lanes, stream=stream.cuda_stream,
                       precision=pkg.H2_PREC_MIXED)
    for i in range(args.warmup):
        Mx.h2_inertia_device(d_sh[i], lanes, d_cnt[i], d_mp[i])
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(args.warmup, total):
        Mx.h2_inertia_device(d_sh[i], lanes, d_cnt[i], d_mp[i])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_mix = _max_over_ranks(e0.elapsed_time(e1), dist, dev)
    latm = []
    for i in range(args.eig_solves + 2):
        torch.cuda.synchronize()
        t = time.perf_counter()
        outm, ebm = Mxe.h2_kth_eig([WORKLOAD["k"]], WORKLOAD["tol"])
        latm.append(time.perf_counter() - t)
    latm = np.array(latm[2:])
    infm = Mxe.h2_info()
    Mxe.close()
    ginfo = Mx.h2_info()
    precision = {"mode": "fp32 products, fp64 storage/pivots/counts; every count certified: mixed "
                         "factorizations at mu -/+ Delta (Delta = 64 2^-24 ||A||_inf), FP64 re-run of the "
                         "shifts whose pair disagrees or whose min |pivot| < 1e-3 ||A||_inf, all inside the "
                         "timed region",
                 "value": world * args.steps * lanes / (ms_mix / 1e3), "unit": "shifts/s",
                 "counts_equal_to_fp64": bool(torch.equal(d_cnt, cnt_fp64)),
                 "guard_checked": ginfo["guard_checked"], "guard_reruns": ginfo["guard_reruns"],
                 "guard_rerun_rate": ginfo["guard_reruns"] / max(1, ginfo["guard_checked"]),
                 "eigs_per_s": float(1.0 / np.mean(latm)), "p50_ms": float(np.percentile(latm, 50) * 1e3),
                 "p99_ms": float(np.percentile(latm, 99) * 1e3), "rounds": infm["last_rounds"],
                 "mixed_rounds": infm["last_mixed_rounds"], "bracket_resets": infm["bracket_resets"],
                 "lambda": float(outm[0]), "abs_diff_vs_fp64": float(abs(outm[0] - lam[0]))}
    Mx.close()
    # ---- FP64 with the Schur-update products on the tensor cores (exact
    # BF16 products of 7-bit digits, integer accumulation, one FP64 rounding)
    Mt = pkg.H2Matrix(X, WORKLOAD["kernel"], WORKLOAD["kparams"], leaf=WORKLOAD["leaf"], rank=WORKLOAD["rank"],
                      eta=WORKLOAD["eta"], max_lanes=lanes, stream=stream.cuda_stream,
                      precision=pkg.H2_PREC_FP64_TC)
    for i in range(args.warmup):
        Mt.h2_inertia_device(d_sh[i], lanes, d_cnt[i], d_mp[i])
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(args.warmup, total):
        Mt.h2_inertia_device(d_sh[i], lanes, d_cnt[i], d_mp[i])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_tc = _max_over_ranks(e0.elapsed_time(e1), dist, dev)
    tc_same = bool(torch.equal(d_cnt, cnt_fp64))
    ptc = Mt.h2_profile_batch(d_sh[args.warmup], lanes, d_cnt[args.warmup])
    Mt.close()
    Mte = pkg.H2Matrix(X, WORKLOAD["kernel"], WORKLOAD["kparams"], leaf=WORKLOAD["leaf"], rank=WORKLOAD["rank"],
                       eta=WORKLOAD["eta"], max_lanes=args.eig_lanes, stream=stream.cuda_stream,
                       precision=pkg.H2_PREC_FP64_TC)
    latt = []
    for i in range(args.eig_solves + 2):
        torch.cuda.synchronize()
        t = time.perf_counter()
        outt, ebt = Mte.h2_kth_eig([WORKLOAD["k"]], WORKLOAD["tol"])
        latt.append(time.perf_counter() - t)
    latt = np.array(latt[2:])
    Mte.close()
    tot_tc = sum(v["ms"] for v in ptc.values())
    fp64_tc = {"mode": "FP64; Schur-update products on the tensor cores (8 exact 7-bit digits per entry, "
                       "BF16 digit products summed exactly, one FP64 rounding per entry)",
               "value": world * args.steps * lanes / (ms_tc / 1e3), "unit": "shifts/s",
               "counts_equal_to_fp64": tc_same,
               "eigs_per_s": float(1.0 / np.mean(latt)), "p50_ms": float(np.percentile(latt, 50) * 1e3),
               "p99_ms": float(np.percentile(latt, 99) * 1e3), "lambda": float(outt[0]),
               "abs_diff_vs_fp64": float(abs(outt[0] - lam[0])),
               "schur_ms_per_launch": ptc["schur"]["ms"] / max(1, ptc["schur"]["launches"]),
               "kernel_shares": {k: v["ms"] / tot_tc for k, v in ptc.items()}}
    # ---- the plain FP64 path: one shift per launch sequence (1 lane), kernels
    # launched one by one (no graph, no batching)
    Mp = pkg.H2Matrix(X, WORKLOAD["kernel"], WORKLOAD["kparams"], leaf=WORKLOAD["leaf"], rank=WORKLOAD["rank"],
                      eta=WORKLOAD["eta"], max_lanes=1, stream=stream.cuda_stream, graphs=0)
    nplain = min(64, lanes)
    p_cnt = torch.zeros(nplain, dtype=torch.int64, device=dev)
    src = d_sh[args.warmup]
    for j in range(3):
        Mp.h2_inertia_device(src[j:j + 1], 1, p_cnt[j:j + 1])
    torch.cuda.synchronize()
    e0.record(stream)
    for j in range(nplain):
        Mp.h2_inertia_device(src[j:j + 1], 1, p_cnt[j:j + 1])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    plain_rate = nplain / (ms_plain / 1e3)
    plain_same = bool(torch.equal(p_cnt, cnt_fp64[args.warmup][:nplain]))
    Mp.close()
    plain = {"mode": "FP64, 1 lane, kernels launched one by one (no graph, no batching)", "value": plain_rate,
             "unit": "shifts/s", "shifts": nplain, "counts_equal_to_batched": plain_same,
             "batched_fp64_over_plain": value / plain_rate,
             "batched_mixed_over_plain": precision["value"] / plain_rate}
    compression = _compression(args, X, dev, stream, e0, e1, d_sh, total, lanes) if args.compression else None
    e2 = _e2_sweep(args) if args.e2_sweep and world == 1 else None
    large = _large_configs(args) if args.large_configs and world == 1 else None
    serving_res = _serving(args) if args.serving_s > 0 and world == 1 else None
    batching_res = _batching(args) if args.batch_count > 0 and world == 1 else None
    ws_mb = info["workspace_bytes"] / 1e6
    line = {"metric": METRIC, "value": value, "unit": "shifts/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "n": WORKLOAD["n"], "leaf": WORKLOAD["leaf"],
                       "rank": WORKLOAD["rank"], "eta": WORKLOAD["eta"], "admissibility": "box",
                       "shifts_per_step": lanes, "parallelism": "replica per GPU",
                       "autotuned_levels": [list(M.h2_autotune_choice(l)) for l in range(info["levels"])],
                       "l2": "per-step working set %.0f MB > 129 MB L2" % ws_mb},
            "e2e": {"value": e2e_value, "unit": "shifts/s", "h2d_bytes_per_step": 8 * lanes,
                    "d2h_bytes_per_step": 8 * lanes, "counts_match_device_path": same},
            "gpu_launches": info["kernels_per_batch"] * args.steps,
            "eigs": {"k": WORKLOAD["k"], "tol": WORKLOAD["tol"], "lanes": args.eig_lanes,
                     "eigs_per_s": float(1.0 / np.mean(lat)),
                     "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                     "rounds": info2["last_rounds"], "shifts_per_solve": info2["last_shifts"],
                     "lambda": lam[0], "err_bound": lam[1], "by_lanes": eig_sweep},
            "build_s": build_s, "roofline": roof, "clocks": clocks, "precision": precision,
            "all_eigs": all_eigs, "fp64_tc": fp64_tc, "plain_fp64": plain, "compression": compression,
            "e2_sweep": e2, "large_configs": large,
            "serving": serving_res,
            "batching": batching_res}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        # up to 16 shifts per core (all 256 shifts of the step on 16 cores): about
        # 10-30 s of CPU work, a couple of seconds of wall time
        sample = list(sh[args.warmup][:: max(1, lanes // (16 * cores))][:16 * cores])
        rate, secs, ocounts = oracle_throughput(sample, cores)
        got = {s: int(c) for s, c in zip(sh[args.warmup], cnt_fp64[args.warmup].cpu().numpy())}
        agree = sum(int(got[s] == ocounts[s]) for s in sample)
        line["cpu_baseline"] = {"value": rate, "unit": "shifts/s", "cores": cores, "kind": "oracle",
                                "sample": "%d shifts of step 1 (%.1f s wall, about %.0f s of CPU work, "
                                          "one process per core)" % (len(sample), secs, secs * cores),
                                "counts_equal_to_gpu": "%d/%d" % (agree, len(sample)),
                                "seconds_per_shift_one_core": secs * cores / max(1, len(sample))}
    if rank == 0:
        print(json.dumps(line), flush=True)
    M.close()


def _compression(args, X, dev, stream, e0, e1, d_sh, total, lanes):
    """||A - A~||_2 / ||A||_2 of the GPU's own A~ (h2_compression_error: power
    iteration on the device) at the configured rank cap and at the cap that
    meets the 1e-8 criterion, with the FP64 step throughput at each."""
    import torch
    import paper_2311_08618_gb300 as pkg
    out = {}
    for rank in (WORKLOAD["rank"], WORKLOAD["rank"] + 1):
        M = pkg.H2Matrix(X, WORKLOAD["kernel"], WORKLOAD["kparams"], leaf=WORKLOAD["leaf"], rank=rank,
                         eta=WORKLOAD["eta"], max_lanes=lanes, stream=stream.cuda_stream)
        err, nrm = M.h2_compression_error(40)
        info = M.h2_info()
        d_c = torch.zeros(lanes, dtype=torch.int64, device=dev)
        for i in range(args.warmup):
            M.h2_inertia_device(d_sh[i], lanes, d_c)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(args.warmup, total):
            M.h2_inertia_device(d_sh[i], lanes, d_c)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out["rank_cap_%d" % rank] = {"err2": err, "norm2": nrm, "rel": err / nrm, "meets_1e-8": err / nrm <= 1e-8,
                                     "cap_bound_clusters": info["cap_bound"], "max_rank": info["max_rank"],
                                     "fp64_shifts_per_s": args.steps * lanes / (ms / 1e3)}
        M.close()
    return out


def _large_configs(args):
    """The two large configurations at the lane counts one GB300 holds: the 3D
    Yukawa n = 65536 matrix (leaf 256, rank 32), one batch in FP64_TC and one
    in certified mixed precision, and the n = 262144 cylindrical lattice (leaf
    256, rank 48; the precision configuration), one batch in certified mixed
    precision.  Build time, workspace, shifts at 10..90 % of the Gershgorin
    interval; batches of several seconds, timed without a warm-up batch."""
    import torch
    import paper_2311_08618_gb300 as pkg
    out = {}
    plan = (("yukawa3d_n65536", args.large_lanes_c2, ((pkg.H2_PREC_FP64_TC, "fp64_tc"), (pkg.H2_PREC_MIXED, "mixed"))),
            ("cylinder_n262144", args.large_lanes_cyl, ((pkg.H2_PREC_MIXED, "mixed"),)))
    for name, lanes, precs in plan:
        wl = WORKLOADS[name]
        X = _points(wl)
        st = torch.cuda.Stream()
        rec = {"lanes": lanes}
        counts = {}
        for prec, key in precs:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            M = pkg.H2Matrix(X, wl["kernel"], wl["kparams"], leaf=wl["leaf"], rank=wl["rank"], eta=wl["eta"],
                             max_lanes=lanes, stream=st.cuda_stream, precision=prec)
            torch.cuda.synchronize()
            build_s = time.perf_counter() - t0
            info = M.h2_info()
            lo, hi = info["gershgorin_lo"], info["gershgorin_hi"]
            sh = torch.tensor(lo + (hi - lo) * (0.1 + 0.8 * (np.arange(lanes) + 0.5) / lanes), dtype=torch.float64,
                              device="cuda")
            c = torch.zeros(lanes, dtype=torch.int64, device="cuda")
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            M.h2_inertia_device(sh, lanes, c)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            counts[key] = c.cpu().numpy().tolist()
            rec[key] = {"build_s": build_s, "batch_s": ms / 1e3, "shifts_per_s": lanes / (ms / 1e3),
                        "workspace_GB": info["workspace_bytes"] / 1e9, "max_rank": info["max_rank"],
                        "levels": info["levels"], "near_pairs_leaf": info["near_pairs"],
                        "fill_pairs_leaf": info["fill_pairs"]}
            if prec == pkg.H2_PREC_MIXED:
                g = M.h2_info()
                rec[key]["guard_reruns"] = g["guard_reruns"]
                rec[key]["guard_checked"] = g["guard_checked"]
            M.close()
            torch.cuda.empty_cache()
        rec["counts"] = counts[precs[0][1]]
        if len(counts) == 2:
            rec["counts_equal_fp64_tc_mixed"] = counts["fp64_tc"] == counts["mixed"]
        out[name] = rec
    return out


def _e2_sweep(args):
    """Sec. 5.1's second accuracy experiment: all n = 1024 eigenvalues of the
    unit-circle Laplace matrix at decreasing eps_ev (eps_H2 = 1e-2 eps_ev,
    leaf 64, rank cap 48); the largest error against the dense eigenvalues
    (cuSOLVER eigvalsh in FP64 on the kernel matrix built with torch, a
    reference outside the library's path) and ||A - A~||_2 from
    h2_compression_error."""
    import torch
    import paper_2311_08618_gb300 as pkg
    n = 1024
    X = W.unit_circle(n, 5)
    Xt = torch.tensor(X, dtype=torch.float64, device="cuda")
    r = torch.cdist(Xt, Xt, compute_mode="donot_use_mm_for_euclid_dist")   # exact differences: r_ii = 0
    ev = torch.linalg.eigvalsh(1.0 / (r + 1e-3)).cpu().numpy()
    del Xt, r
    st = torch.cuda.Stream()
    rows = []
    for eps in (1e-2, 1e-4, 1e-6, 1e-8, 1e-10):
        M = pkg.H2Matrix(X, W.LAPLACE_EPS, (1e-3, 0, 0, 0), leaf=64, rank=48, eta=1.0, eps_h2=1e-2 * eps,
                         max_lanes=256, stream=st.cuda_stream)
        err, nrm = M.h2_compression_error(40)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lam, eb = M.h2_kth_eig(np.arange(1, n + 1), eps)
        sec = time.perf_counter() - t0
        info = M.h2_info()
        e = np.abs(lam - ev)
        rows.append({"eps_ev": eps, "max_err": float(e.max()), "max_err_over_half_eps": float(e.max() / (0.5 * eps)),
                     "below_half_eps": int(np.sum(e < 0.5 * eps)), "h2_err2": err, "max_rank": info["max_rank"],
                     "seconds": sec, "rounds": info["last_rounds"], "shifts": info["last_shifts"]})
        M.close()
    return {"workload": "unit circle n=1024, 1/(r+1e-3), all 1024 eigenvalues, FP64, 256 lanes", "rows": rows}


SERVING_SIZES = (1024, 2048, 4096, 8192)


def _circle_sweep(args):
    """The paper's scaling experiment (Sec. 5.1): A_ij = 1/(|x_i - x_j| + 1e-3)
    on n points uniformly distributed on the unit circle, the k = n/2
    eigenvalue to eps_ev = 1e-5 from the constant starting interval [0, 2048]
    (checked: nu(0) < k <= nu(2048)), eps_H2 = 1e-2 eps_ev (relative to
    ||A||_inf), leaf 64, rank cap 32, FP64, --circle-lanes shifts per round.
    Prints one JSON line per run (not the bench line)."""
    import torch
    import paper_2311_08618_gb300 as pkg
    from paper_2311_08618_gb300 import batching
    st = torch.cuda.Stream()
    out = []
    for n in [int(v) for v in args.circle_sweep.split(",")]:
        X = W.unit_circle(n, 5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        M = pkg.H2Matrix(X, W.LAPLACE_EPS, (1e-3, 0, 0, 0), leaf=64, rank=32, eta=1.0, eps_h2=1e-7,
                         max_lanes=args.circle_lanes, stream=st.cuda_stream)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        info = M.h2_info()
        k = n // 2
        c, _ = M.h2_inertia([0.0, 2048.0])
        rec = {"n": n, "build_s": build_s, "workspace_GB": info["workspace_bytes"] / 1e9,
               "max_rank": info["max_rank"], "levels": info["levels"], "nu_0": int(c[0]), "nu_2048": int(c[1])}
        if c[0] < k <= c[1]:
            G = pkg.H2Group([M])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lam, rounds, shifts = batching.kth_group([M], [k], 1e-5, st, G, start=([0.0], [2048.0]))
            sec = time.perf_counter() - t0
            rec.update({"lambda_k": float(lam[0]), "seconds": sec, "rounds": rounds, "shifts": shifts,
                        "ms_per_shift": 1e3 * sec / shifts})
            G.close()
        M.close()
        out.append(rec)
        print(json.dumps({"circle_sweep_point": rec}), flush=True)
    return out


def _tune_summary(mats):
    """Levels per Bunch-Kaufman kernel (one warp, 128- or 256-thread CTA per
    block) and levels with a clustered recompression, over all handles."""
    n = clu = 0
    per = {32: 0, 128: 0, 256: 0}
    for M in mats:
        for l in range(M.h2_info()["levels"]):
            t, c = M.h2_autotune_choice(l)
            n += 1
            per[int(t)] = per.get(int(t), 0) + 1
            clu += c
    return "%d/%d/%d of %d, %d/%d" % (per[32], per[128], per[256], n, clu, n)


def _batching(args):
    """The many-matrix configuration on a bounded sample: the first
    --batch-count members of the seeded 512-matrix list (workloads.batch_members)
    with n <= --batch-nmax, FP64, --batch-lanes lanes each, their own random k,
    tol 1e-8.  All k-th eigenvalues through group batches (one launch per tree
    level and colour over all matrices), against the same handles solved one
    after another with h2_kth_eig."""
    import torch
    import paper_2311_08618_gb300 as pkg
    from paper_2311_08618_gb300 import batching
    members = [w for w in W.batch_members(512) if w.points.shape[0] <= args.batch_nmax][:args.batch_count]
    st = torch.cuda.Stream()
    t0 = time.perf_counter()
    mats = [pkg.H2Matrix(w.points, w.kernel, w.kparams, leaf=w.leaf, rank=w.rank, eta=w.eta,
                         max_lanes=args.batch_lanes, stream=st.cuda_stream, autotune=1) for w in members]
    G = pkg.H2Group(mats)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    ks = [w.ks[0] for w in members]
    tol = 1e-8
    batching.kth_group(mats, ks, 1e3, st, G)          # warm-up rounds
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam_g, rounds, shifts = batching.kth_group(mats, ks, tol, st, G)
    tg = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam_s = np.array([M.h2_kth_eig([k], tol)[0][0] for M, k in zip(mats, ks)])
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    ns = [w.points.shape[0] for w in members]
    res = {"sample": "first %d of the 512-matrix list with n <= %d (n %d..%d, %d in 3D); FP64, %d lanes each"
                     % (len(members), args.batch_nmax, min(ns), max(ns),
                        sum(w.points.shape[1] == 3 for w in members), args.batch_lanes),
           "eigs_per_s": len(members) / tg, "sequential_eigs_per_s": len(members) / ts,
           "speedup_vs_sequential": ts / tg, "rounds": rounds, "shifts": shifts,
           "launches_per_group_batch": G.launches(),
           "launches_per_sequential_round": int(sum(M.h2_info()["kernels_per_batch"] for M in mats)),
           "max_abs_diff_vs_sequential": float(np.max(np.abs(lam_g - lam_s))), "tol": tol,
           "build_s": build_s, "autotune": "per level: Bunch-Kaufman on one warp or one CTA per block, "
                                            "recompression on one CTA or an 8-CTA cluster, timed at build; "
                                            "levels choosing (warp/128/256 threads, clustered): %s" % _tune_summary(mats)}
    G.close()
    for M in mats:
        M.close()
    return res


def _serving_run(args, rate, seconds, seed, mats=None, lanes=None, grace_s=25.0):
    """One open-loop run on freshly built resident matrices (cold (mu, nu)
    tables): Poisson arrivals at `rate` for `seconds`.  mats: (n, d, leaf,
    rank) per matrix, the 2D stand-in by default."""
    import paper_2311_08618_gb300 as pkg
    from paper_2311_08618_gb300 import serving
    srv = serving.Server()
    mats = mats or [(n, 2, 64, 16) for n in SERVING_SIZES]
    for i, (n, d, leaf, rank) in enumerate(mats):
        srv.add_matrix("m%d" % i, W.uniform_cube(n, d, 100 + i), W.LAPLACE_EPS, (1e-3, 0, 0, 0), leaf, rank,
                       lanes=lanes or args.serving_lanes, precision=pkg.H2_PREC_FP64_TC)
    sizes = [m[0] for m in mats]
    u = W.uniform(seed, 4 * 100000)
    arr, t, j = [], 0.0, 0
    while True:
        t += -math.log(1.0 - u[j]) / rate
        j += 1
        if t > seconds:
            break
        mi = int(u[j] * len(sizes))
        k = 1 + int(u[j + 1] * sizes[mi])
        tol = 10.0 ** (-10.0 + 4.0 * u[j + 2])
        j += 3
        arr.append((t, "m%d" % mi, k, tol))
    t0 = time.perf_counter()
    done, unfinished = serving.run_open_loop(srv, arr, seconds, deadline_s=seconds + grace_s)
    wall = time.perf_counter() - t0
    res = {"arrivals": "Poisson %g q/s for %g s" % (rate, seconds), "offered": len(arr),
           "completed": len(done), "unfinished": unfinished, "wall_s": wall,
           "eigs_per_s": len(done) / wall, "shifts_per_s": srv.shifts_evaluated / wall, "ticks": srv.ticks,
           "ms_per_tick": 1e3 * srv.host_s / max(1, srv.ticks),
           "device_wait_ms_per_tick": 1e3 * srv.wait_s / max(1, srv.ticks),
           "host_ms_per_tick": 1e3 * (srv.host_s - srv.wait_s) / max(1, srv.ticks)}
    res.update(serving.latency_stats(done))
    srv.close()
    return res


def _serving(args):
    """Open-loop serving: Poisson arrivals of k-th eigenvalue queries (k uniform,
    tol log-uniform in [1e-10, 1e-6]) over resident 2D Laplace H^2 matrices of
    different sizes; continuous batching (paper_2311_08618_gb300.serving).  One
    run at the offered (overload) rate and one at a sustainable rate."""
    res = {"matrices": "4 resident 2D Laplace H2 matrices n=%s (leaf 64, rank 16), %d lanes each, FP64_TC"
                       % (list(SERVING_SIZES), args.serving_lanes),
           "stand_in": "the 64-matrix 3D n<=131072 configuration needs ~16-70 GB per lane under eta=1 box "
                       "admissibility and does not fit one GPU"}
    res.update(_serving_run(args, args.serving_rate, args.serving_s, 4242))
    if args.serving_sustain_rate > 0:
        res["sustainable"] = _serving_run(args, args.serving_sustain_rate, args.serving_sustain_s, 4343)
    res["plain_fp64_same_matrices"] = _plain_on_serving_mix()
    res["served_over_plain"] = res["shifts_per_s"] / res["plain_fp64_same_matrices"]["shifts_per_s"]
    if args.serving_3d_s > 0:
        r3 = {"matrices": "2 resident 3D 1/(r+1e-3) H2 matrices n=16384 (leaf 256, rank 32: the serving "
                          "configuration's shape), 8 lanes each, FP64_TC"}
        r3.update(_serving_run(args, args.serving_3d_rate, args.serving_3d_s, 4444,
                               mats=[(16384, 3, 256, 32), (16384, 3, 256, 32)], lanes=8, grace_s=60.0))
        res["serving_3d"] = r3
    return res


def _plain_on_serving_mix():
    """The plain FP64 path (one shift per launch sequence, 1 lane, no graph,
    no batching) on the serving matrices: shifts/s with the shifts spread
    evenly over the four matrices, the baseline of the served rate."""
    import torch
    import paper_2311_08618_gb300 as pkg
    st = torch.cuda.Stream()
    per = []
    for i, n in enumerate(SERVING_SIZES):
        M = pkg.H2Matrix(W.uniform_cube(n, 2, 100 + i), W.LAPLACE_EPS, (1e-3, 0, 0, 0), leaf=64, rank=16,
                         max_lanes=1, stream=st.cuda_stream, graphs=0)
        info = M.h2_info()
        sh = torch.tensor([0.5 * (info["gershgorin_lo"] + info["gershgorin_hi"])], dtype=torch.float64, device="cuda")
        c = torch.zeros(1, dtype=torch.int64, device="cuda")
        for _ in range(2):
            M.h2_inertia_device(sh, 1, c)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(4):
            M.h2_inertia_device(sh, 1, c)
        e1.record(st)
        torch.cuda.synchronize()
        per.append(e0.elapsed_time(e1) / 4)
        M.close()
    mean_ms = sum(per) / len(per)
    return {"ms_per_shift": dict(zip([str(n) for n in SERVING_SIZES], per)), "shifts_per_s": 1e3 / mean_ms}


def _ncu_case(args):
    """A small, fixed workload for ncu captures: one handle of the bench
    configuration in the given precision with --lanes lanes, --warmup +
    --steps device-resident batches, one line of output."""
    import torch
    import paper_2311_08618_gb300 as pkg
    from paper_2311_08618_gb300 import build
    build.build()
    prec = {"fp64": pkg.H2_PREC_FP64, "mixed": pkg.H2_PREC_MIXED, "fp64_tc": pkg.H2_PREC_FP64_TC,
            "fp64_tc_tcgen05": pkg.H2_PREC_FP64_TC}[args.ncu_case]
    st = torch.cuda.Stream()
    X = _points(WORKLOAD)
    M = pkg.H2Matrix(X, WORKLOAD["kernel"], WORKLOAD["kparams"], leaf=WORKLOAD["leaf"], rank=WORKLOAD["rank"],
                     eta=WORKLOAD["eta"], max_lanes=args.lanes, stream=st.cuda_stream, precision=prec,
                     tc_schur=1 if args.ncu_case == "fp64_tc_tcgen05" else 0)
    info = M.h2_info()
    sh = torch.tensor(_shift_batches(info["gershgorin_lo"], info["gershgorin_hi"], args.lanes, 1)[0],
                      dtype=torch.float64, device="cuda")
    c = torch.zeros(args.lanes, dtype=torch.int64, device="cuda")
    for _ in range(args.warmup + args.steps):
        M.h2_inertia_device(sh, args.lanes, c)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": args.ncu_case, "lanes": args.lanes, "batches": args.warmup + args.steps,
                      "kernels_per_batch": info["kernels_per_batch"], "negative_counts_sum": int(c.sum())}))
    M.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lanes", type=int, default=256, help="shifts per step (throughput)")
    ap.add_argument("--eig-lanes", type=int, default=64, help="lanes of the k-th eigenvalue solves")
    ap.add_argument("--eig-solves", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-s", type=float, default=3.0, help="seconds of arrivals (0: skip)")
    ap.add_argument("--serving-rate", type=float, default=40.0)
    ap.add_argument("--serving-sustain-rate", type=float, default=2.0, help="second, sustainable rate (0: skip)")
    ap.add_argument("--serving-sustain-s", type=float, default=5.0)
    ap.add_argument("--batch-count", type=int, default=24, help="matrices of the batching sample (0: skip)")
    ap.add_argument("--all-eigs", type=int, default=1, help="1: also solve for all n eigenvalues (n <= 8192)")
    ap.add_argument("--compression", type=int, default=1, help="1: measure ||A - A~|| at rank caps r and r + 1")
    ap.add_argument("--e2-sweep", type=int, default=1, help="1: all-eigenvalue error sweep over eps_ev (Sec. 5.1)")
    ap.add_argument("--large-configs", type=int, default=1,
                    help="1: one timed batch of the 3D n=65536 and the n=262144 cylinder configurations")
    ap.add_argument("--large-lanes-c2", type=int, default=8)
    ap.add_argument("--large-lanes-cyl", type=int, default=4)
    ap.add_argument("--circle-sweep", default="", help="comma-separated n: run the unit-circle scaling sweep only")
    ap.add_argument("--circle-lanes", type=int, default=4)
    ap.add_argument("--batch-nmax", type=int, default=8192)
    ap.add_argument("--batch-lanes", type=int, default=4)
    ap.add_argument("--serving-lanes", type=int, default=16)
    ap.add_argument("--serving-3d-s", type=float, default=10.0, help="seconds of arrivals, 3D serving (0: skip)")
    ap.add_argument("--serving-3d-rate", type=float, default=0.5)
    ap.add_argument("--workload", default="laplace2d_n1024", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1], help="0 FP64, 1 mixed (main handle)")
    ap.add_argument("--ncu-case", default="", choices=["", "fp64", "mixed", "fp64_tc", "fp64_tc_tcgen05"],
                    help="run only a small fixed workload for ncu captures")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    global WORKLOAD
    WORKLOAD = WORKLOADS[args.workload]
    rank, world, local, dist = _dist()
    try:
        if args.impl == "reference":
            reference_arm(args, rank, world, dist)
        elif args.ncu_case:
            _ncu_case(args)
        elif args.circle_sweep:
            _circle_sweep(args)
        else:
            ours(args, rank, world, local, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
