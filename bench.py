#!/usr/bin/env python
"""Benchmark of the gamblet setup + solve hot path on GB300.

Metric: fine DOFs per second of one full pass (gamblet_setup + gamblet_solve
with float64 refinement to the stated tolerance) on the 1024 x 1024 Q1
rough-coefficient problem (1,046,529 unknowns, q = 10, rho = 3, contrast
1e4, seed = rank).  The headline value is the mixed-precision path; the plain
float64 path is measured beside it, and both must reach a relative error
<= 1e-8 against the refined direct solve of the CPU oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gamblet|reference]

Under torchrun (N > 1) every rank solves its own independent problem (weak
scaling, no data-path collective); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fine DOFs/s setup+solve at 2^20 DOF: batched/mixed vs plain FP64, rel err <=1e-8"
UNIT = "DOF/s"
REL_ERR_BAR = 1e-8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gamblet", choices=["gamblet", "reference"])
    ap.add_argument("--size", type=int, default=1024, help="cells per side (power of two)")
    ap.add_argument("--contrast", type=float, default=1e4)
    ap.add_argument("--rho", type=float, default=3.0)
    ap.add_argument("--level-tol", type=float, default=0.05)
    ap.add_argument("--refine-tol", type=float, default=1e-9)
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="end-to-end steps (0: the same as --steps)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain float64 arm")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-gradient timing")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the many-problem (48 x {128,256,512}^2) timing")
    ap.add_argument("--batch-problems", type=int, default=48)
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--no-localization", action="store_true",
                    help="skip the one-pass localization error per patch radius")
    ap.add_argument("--no-mass", action="store_true",
                    help="skip the mass-matrix initialisation timings")
    ap.add_argument("--no-3d", action="store_true",
                    help="skip the three-dimensional (64^3) timing")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_name(a):
    return (f"{a.size}x{a.size} Q1 rough coefficient, q={int(np.log2(a.size))}, rho={a.rho:g} "
            f"(Euclidean), contrast {a.contrast:g}, g~N(0,1)")


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except OSError:
            rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if self.path:
            os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        load = [v for v in sm if v > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def ncu_traffic(kernel: str, mixed: bool = True):
    """Per-launch DRAM traffic of `kernel` from the committed ncu summary, or
    None when absent, taken on a different version of the kernel source, or
    taken in the other working precision (float vs double instantiation)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        rec = json.load(open(path)).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    prec = rec.get("precision")
    if prec is None:
        prec = "f32" if "<float" in rec.get("kernel", "") else "f64"
    if (prec == "f32") != mixed:
        return None
    src = os.path.join(ROOT, rec["source"])
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if sha != rec.get("source_sha"):
        return None
    return rec.get("bytes_per_launch")


def make_inputs(a, rank):
    from workloads import make_problem
    p = make_problem(a.size, a.contrast, seed=rank)
    A = p.A.tocsr()
    A.sort_indices()
    host = {
        "rowptr": np.ascontiguousarray(A.indptr, dtype=np.int32),
        "colind": np.ascontiguousarray(A.indices, dtype=np.int32),
        "val": np.ascontiguousarray(A.data, dtype=np.float64),
        "cells": np.ascontiguousarray(p.cells, dtype=np.int32),
        "g": np.ascontiguousarray(p.g, dtype=np.float64),
    }
    return p, host


def opts_for(nv, a, precision, stream_ptr, profile):
    o = nv.gamblet_default_opts()
    o.rho = a.rho
    o.nbr_rule = 0
    o.precision = precision
    o.level_tol = a.level_tol
    o.level_max_iter = 2000
    o.refine_tol = a.refine_tol
    o.refine_max_iter = 100
    o.patch_tol = getattr(a, "patch_tol", 0.0)
    o.profile = profile
    o.stream = stream_ptr
    return o


def run_arm(nv, torch, a, dev_in, precision, steps, warmup, stream, flush, clocks_dev=None,
            profile=0):
    """Times `steps` setup+solve passes on device-resident inputs.  With
    profile = 1 the library also brackets every kernel phase with CUDA
    events (per-kernel times for the roofline); the headline pass runs with
    profile = 0."""
    ndof = int(dev_in["g"].shape[0])
    q = int(np.log2(a.size))
    o = opts_for(nv, a, precision, stream.cuda_stream, profile)
    u = torch.zeros(ndof, dtype=torch.float64, device=dev_in["g"].device)
    times, setup_ms, solve_ms, infos, stats = [], [], [], [], {}
    clk = None
    launches0 = None
    for it in range(warmup + steps):
        timed = it >= warmup
        if timed and it == warmup and clocks_dev is not None:
            clk = Clocks(clocks_dev).__enter__()
        if timed and launches0 is None:
            launches0 = nv.gamblet_kernel_launches()
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            h = nv.gamblet_setup(dev_in["rowptr"], dev_in["colind"], dev_in["val"], q,
                                 dev_in["cells"], o)
            info = nv.Info()
            nv.gamblet_solve(h, dev_in["g"], u, None, info)
            e1.record(stream)
        e1.synchronize()
        if timed:
            times.append(e0.elapsed_time(e1))
            setup_ms.append(info.setup_ms)
            solve_ms.append(info.solve_ms)
            infos.append(info.as_dict())
            for st in (nv.gamblet_kernel_stats(h) if profile else []):
                acc = stats.setdefault(st["name"], {"launches": 0, "ms": 0.0, "bytes": 0.0,
                                                    "flops": 0.0})
                for key in ("launches", "ms", "bytes", "flops"):
                    acc[key] += st[key]
        nv.gamblet_destroy(h)
    launches = nv.gamblet_kernel_launches() - launches0
    clocks = None
    if clk is not None:
        clk.__exit__(None, None, None)
        clocks = clk.summary()
    return {"times_ms": times, "setup_ms": setup_ms, "solve_ms": solve_ms, "infos": infos,
            "stats": stats, "u": u.cpu().numpy(), "launches": launches, "clocks": clocks}


def pinned_copy(torch, arr):
    """A copy of a host array in page-locked memory (the numpy view and the
    tensor that owns the memory)."""
    t = torch.empty(arr.shape, dtype=torch.from_numpy(arr[:0]).dtype, pin_memory=True)
    view = t.numpy()
    view[...] = arr
    return view, t


def run_e2e(nv, a, host, precision, steps):
    """setup + solve through the C ABI with host buffers: every step copies
    the inputs from page-locked host memory to the device and reads the
    solution back into page-locked host memory (both inside the timed
    region); the buffers are filled before the clock starts."""
    import torch
    q = int(np.log2(a.size))
    o = opts_for(nv, a, precision, None, 0)
    keep = []
    pin = {}
    for k in ("rowptr", "colind", "val", "cells", "g"):
        pin[k], t = pinned_copy(torch, host[k])
        keep.append(t)
    u, t = pinned_copy(torch, np.zeros_like(host["g"]))
    keep.append(t)
    times = []
    for it in range(steps + 1):
        t0 = time.perf_counter()
        h = nv.gamblet_setup(pin["rowptr"], pin["colind"], pin["val"], q, pin["cells"], o)
        nv.gamblet_solve(h, pin["g"], u)
        t1 = time.perf_counter()
        nv.gamblet_destroy(h)
        if it > 0:
            times.append((t1 - t0) * 1e3)
    h2d = sum(pin[k].nbytes for k in ("rowptr", "colind", "val", "cells", "g"))
    return {"ms": statistics.mean(times), "h2d": h2d, "d2h": u.nbytes, "u": np.array(u)}


def cold_start(a, dev_index):
    """First setup + solve in a fresh process: the process-wide symbolic plan,
    the autotuner's choices and the library's memory pool are all empty, so
    this includes building the plan, tuning the launch shapes and the first
    device allocations (the CUDA context is created before the clock
    starts).  The timed steps of the headline reuse all three, the way a
    repeated solve on the same geometry would."""
    cmd = [sys.executable, "-m", "paper_1503_03467_gb300", "--size", str(a.size),
           "--precision", "mixed", "--rho", f"{a.rho:g}", "--contrast", f"{a.contrast:g}",
           "--level-tol", f"{a.level_tol:g}", "--refine-tol", f"{a.refine_tol:g}", "--wall"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES=os.environ.get("CUDA_VISIBLE_DEVICES",
                                                               str(dev_index)))
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
        out = json.loads(r.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError) as e:
        return {"error": f"{type(e).__name__}: {e}"}
    return {"wall_ms": out.get("wall_ms"), "setup_ms": out.get("setup_ms"),
            "solve_ms": out.get("solve_ms"),
            "what": "first setup + solve in a fresh process (plan, tuner and memory pool "
                    "empty; CUDA context created beforehand)"}


def measured_alu_peaks(torch, dev):
    """Dense GEMM throughput of this GPU through torch.matmul (cuBLAS), the
    way the HBM and bf16 figures of MEASURED_PEAKS.json are taken: float32
    with IEEE products (SIMT FMA lanes), TF32 tensor cores, float64.  Best of
    five, CUDA events; no clock or power setting is touched."""
    out = {}
    prev = torch.get_float32_matmul_precision()
    try:
        for name, dtype, prec, n in (("fp32_simt_tflops", torch.float32, "highest", 8192),
                                     ("tf32_tflops", torch.float32, "high", 8192),
                                     ("fp64_tflops", torch.float64, "highest", 4096)):
            torch.set_float32_matmul_precision(prec)
            x = torch.randn(n, n, device=dev, dtype=dtype)
            y = torch.randn(n, n, device=dev, dtype=dtype)
            torch.matmul(x, y)
            best = float("inf")
            for _ in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(x, y)
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[name] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            del x, y
    finally:
        torch.set_float32_matmul_precision(prev)
    torch.cuda.empty_cache()
    out["how"] = ("torch.matmul n^3 (2 n^3 flop), best of 5, CUDA events: float32 with "
                  "precision 'highest' (8192), TF32 with precision 'high' (8192), float64 (4096)")
    return out


def adjoint_timing(nv, torch, dev, steps=3):
    """Gradient of J = 1/2 |u - u_obs|^2 with respect to log a on the 256 x 256
    problem (q = 8, contrast 1e3, u_obs from the field of seed 7): forward
    (assembly + setup + solve) and backward through the autograd wrapper,
    timed with CUDA events, checked against the CPU oracle's direct-solve
    adjoint.  The headline backward recomputes the hierarchy level by level
    (released after the forward solve); grad_ms_kept keeps it alive."""
    from oracle import adjoint, direct
    from paper_1503_03467_gb300.solver import Q1Mesh, gamblet_solve
    from workloads import cell_corner_dofs, make_problem
    from workloads.rough import K_REF
    n = 256
    p = make_problem(n, 1e3, 0)
    obs = make_problem(n, 1e3, 7)
    u_obs_np, _ = direct.solve(obs.A, p.g)
    A = p.A.tocsr()
    mesh = Q1Mesh(A.indptr, A.indices, p.cells, cell_corner_dofs(n), K_REF, p.q, dev)
    o = nv.gamblet_default_opts()
    o.precision = nv.MIXED
    o.level_tol = 0.1
    o.refine_tol = 1e-12
    o.refine_max_iter = 100
    g = torch.tensor(p.g, device=dev)
    u_obs = torch.tensor(u_obs_np, device=dev)

    def run(keep):
        fwd, bwd = [], []
        for it in range(steps + 1):
            log_a = torch.tensor(p.log_a.ravel(), dtype=torch.float64, device=dev,
                                 requires_grad=True)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            torch.cuda.synchronize()
            e0.record()
            u = gamblet_solve(log_a, g, mesh, o, keep_hierarchy=keep)
            J = 0.5 * ((u - u_obs) ** 2).sum()
            e1.record()
            J.backward()
            e2.record()
            e2.synchronize()
            if it > 0:
                fwd.append(e0.elapsed_time(e1))
                bwd.append(e1.elapsed_time(e2))
        return statistics.mean(fwd), statistics.mean(bwd), log_a.grad.cpu().numpy()

    f, b, gr = run(False)
    fk, bk, grk = run(True)
    _, grad_ref, _ = adjoint.gradient(p.A, p.g, u_obs_np, n, np.exp(p.log_a), K_REF)
    err = float(np.linalg.norm(gr - grad_ref) / np.linalg.norm(grad_ref))
    errk = float(np.linalg.norm(grk - grad_ref) / np.linalg.norm(grad_ref))
    return {"workload": "256x256 Q1, q=8, contrast 1e3, 65,536 cells", "forward_ms": f,
            "grad_ms": b, "grad_over_forward": b / f,
            "backward": "hierarchy released after the forward solve, recomputed level by level",
            "rel_err_vs_oracle_adjoint": err, "grad_ms_kept": bk,
            "grad_over_forward_kept": bk / fk, "rel_err_vs_oracle_adjoint_kept": errk}


def onepass_grad_timing(nv, torch, dev, steps=3):
    """Gradient through the one-pass localized transform (gamblet_one_pass
    autograd wrapper -> gamblet_grad_onepass) on the 256 x 256 problem of the
    adjoint entry, float64 with patch and level solves to 1e-10: forward
    (assembly + setup + one-pass solve) and backward (the misfit's pass and
    the reverse pass over the setup), CUDA events; checked against central
    differences of J through the same one-pass map along a random direction;
    per-kernel times of one profiled reverse pass."""
    from oracle import direct
    from paper_1503_03467_gb300.solver import Q1Mesh, gamblet_one_pass
    from workloads import assemble_q1, cell_corner_dofs, make_problem
    from workloads.rough import K_REF
    n = 256
    p = make_problem(n, 1e3, 0)
    obs = make_problem(n, 1e3, 7)
    u_obs_np, _ = direct.solve(obs.A, p.g)
    A = p.A.tocsr()
    mesh = Q1Mesh(A.indptr, A.indices, p.cells, cell_corner_dofs(n), K_REF, p.q, dev)

    def opts(profile=0, precision=0):
        o = nv.gamblet_default_opts()
        o.precision = precision
        o.patch_tol = 1e-10 if precision == 0 else 1e-6
        o.level_tol = 1e-10 if precision == 0 else 1e-6
        o.level_max_iter = 5000
        o.profile = profile
        return o

    g = torch.tensor(p.g, device=dev)
    u_obs = torch.tensor(u_obs_np, device=dev)

    def run(precision):
        fwd, bwd = [], []
        for it in range(steps + 1):
            log_a = torch.tensor(p.log_a.ravel(), dtype=torch.float64, device=dev,
                                 requires_grad=True)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            torch.cuda.synchronize()
            e0.record()
            u = gamblet_one_pass(log_a, g, mesh, opts(precision=precision))
            J = 0.5 * ((u - u_obs) ** 2).sum()
            e1.record()
            J.backward()
            e2.record()
            e2.synchronize()
            if it > 0:
                fwd.append(e0.elapsed_time(e1))
                bwd.append(e1.elapsed_time(e2))
        return statistics.mean(fwd), statistics.mean(bwd), log_a.grad.cpu().numpy()

    f, b, grad = run(0)
    fm, bm, gradm = run(nv.MIXED)
    # central differences of J(log a) through the same map
    d = np.random.default_rng(5).standard_normal(n * n)
    hstep = 1e-5
    Js = []
    for sgn in (1.0, -1.0):
        la = torch.tensor(p.log_a.ravel() + sgn * hstep * d, dtype=torch.float64, device=dev)
        with torch.no_grad():
            us = gamblet_one_pass(la, g, mesh, opts())
        Js.append(0.5 * float(((us - u_obs) ** 2).sum()))
    fd = (Js[0] - Js[1]) / (2 * hstep)
    # per-kernel times of one reverse pass
    cn = torch.tensor(cell_corner_dofs(n), device=dev)
    a_dev = torch.tensor(np.exp(p.log_a.ravel()), device=dev)
    kr = torch.tensor(K_REF.ravel(), device=dev)
    h = nv.gamblet_setup(A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data, p.q,
                         p.cells, opts(1))
    try:
        nv.gamblet_reset_kernel_stats(h)
        dJ = torch.empty(n * n, dtype=torch.float64, device=dev)
        nv.gamblet_grad_onepass(h, cn, a_dev, kr, g, u_obs, dJ)
        ks = {s_["name"]: round(s_["ms"], 4) for s_ in nv.gamblet_kernel_stats(h)
              if s_["name"].startswith("grad_") or s_["name"] in ("level_cg", "restrict",
                                                                   "prolong")}
    finally:
        nv.gamblet_destroy(h)
    return {"workload": "256x256 Q1, q=8, contrast 1e3, 65,536 cells, rho 3, float64, patch and "
                        "level solves to 1e-10",
            "forward_ms": f, "grad_ms": b, "grad_over_forward": b / f,
            "fd_directional_rel_err": abs(fd - float(grad @ d)) / abs(fd),
            "reverse_kernels_ms": ks,
            "mixed": {"precision": "float32 hierarchy and reverse pass, patch and level solves "
                                   "to 1e-6",
                      "forward_ms": fm, "grad_ms": bm, "grad_over_forward": bm / fm,
                      "rel_diff_vs_float64_grad": float(np.linalg.norm(gradm - grad)
                                                        / np.linalg.norm(grad))}}


def rank_share(items, ws, rank):
    """The items of one rank: round-robin, so sizes mix evenly; every item
    belongs to exactly one rank."""
    return list(items)[rank::ws]


def reduce_over_ranks(torch, dev, ms, count):
    """(max of ms, sum of count) over the ranks of the default process group
    (one all-reduce each, on a tensor of `dev`); identity without one."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), int(count)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    c = torch.tensor([float(count)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())


def batched_timing(nv, torch, dev, a, stream, flush, ws=1, rank=0):
    """Many independent problems (seeds 1..P, sides drawn from {128, 256, 512},
    contrast log-uniform in [1e2, 1e6]) set up and solved as one hierarchy by
    gamblet_setup_batched, against the same problems one by one through
    gamblet_setup.  Accuracy: relative residual of every problem (float64,
    torch sparse product, validation only) and the oracle's direct solve for
    the first problem of each side."""
    from workloads import make_batch
    # with several ranks the problems are partitioned round-robin (no
    # collective on the data path); each rank sets up its share as one batch
    probs = rank_share(make_batch(a.batch_problems, first_seed=1), ws, rank)
    items, gs = [], []
    for p in probs:
        A = p.A.tocsr()
        A.sort_indices()
        items.append((torch.from_numpy(A.indptr.astype(np.int32)).to(dev),
                      torch.from_numpy(A.indices.astype(np.int32)).to(dev),
                      torch.from_numpy(A.data.astype(np.float64)).to(dev), p.q,
                      torch.from_numpy(np.ascontiguousarray(p.cells, dtype=np.int32)).to(dev)))
        gs.append(torch.from_numpy(p.g).to(dev))
    g = torch.cat(gs)
    ndof = int(g.shape[0])
    u = torch.zeros_like(g)
    o = opts_for(nv, a, nv.MIXED, stream.cuda_stream, 0)
    times, setup, solve, outer = [], [], [], []
    off = None
    for it in range(1 + a.batch_steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            h, off = nv.gamblet_setup_batched(items, o)
            info = nv.Info()
            nv.gamblet_solve(h, g, u, None, info)
            e1.record(stream)
        e1.synchronize()
        nv.gamblet_destroy(h)
        if it > 0:
            times.append(e0.elapsed_time(e1))
            setup.append(info.setup_ms)
            solve.append(info.solve_ms)
            outer.append(info.outer_iters)
    ms = statistics.mean(times)
    ms, total_dofs = reduce_over_ranks(torch, dev, ms, ndof)
    # accuracy per problem
    res = []
    for p, (rp, ci, va, q, _), gp in zip(range(len(probs)), items, gs):
        A = torch.sparse_csr_tensor(rp.long(), ci.long(), va, size=(gp.shape[0],) * 2)
        up = u[int(off[p]):int(off[p + 1])]
        res.append(float(torch.linalg.norm(gp - A @ up) / torch.linalg.norm(gp)))
    ub = u.cpu().numpy()
    err = {}
    for p, pr in enumerate(probs):
        if pr.n in err:
            continue
        ud, _ = cpu_oracle(pr)
        err[pr.n] = rel_err(ub[int(off[p]):int(off[p + 1])], ud)
    # the same problems one at a time (plans of each size warmed first)
    seq = []
    seen = set()
    for p, it in enumerate(items):
        if probs[p].n not in seen:
            seen.add(probs[p].n)
            with torch.cuda.stream(stream):
                h = nv.gamblet_setup(it[0], it[1], it[2], it[3], it[4], o)
                nv.gamblet_solve(h, gs[p], torch.zeros_like(gs[p]))
            nv.gamblet_destroy(h)
    for p, it in enumerate(items):
        up = torch.zeros_like(gs[p])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            h = nv.gamblet_setup(it[0], it[1], it[2], it[3], it[4], o)
            nv.gamblet_solve(h, gs[p], up)
            e1.record(stream)
        e1.synchronize()
        nv.gamblet_destroy(h)
        seq.append(e0.elapsed_time(e1))
    seq_total = sum(seq)
    sides = [pr.n for pr in probs]
    return {
        "workload": f"{a.batch_problems} problems, seeds 1..{a.batch_problems}, sides 128/256/512 "
                    f"(this rank: {len(probs)} problems, {sides.count(128)}/{sides.count(256)}/"
                    f"{sides.count(512)}), contrast log-uniform [1e2, 1e6], rho 3, mixed precision",
        "dofs": total_dofs, "value": total_dofs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
        "ranks": ws, "partition": "problems round-robin over ranks, max time over ranks",
        "setup_ms": statistics.mean(setup), "solve_ms": statistics.mean(solve),
        "outer_iters": max(outer), "max_rel_residual": max(res),
        "rel_err_vs_oracle": {str(k): v for k, v in sorted(err.items())},
        "batched_problem_latency_ms": ms,
        "one_by_one": {"value": ndof / (seq_total * 1e-3), "ms_total": seq_total,
                       "p50_ms": float(np.percentile(seq, 50)),
                       "p99_ms": float(np.percentile(seq, 99))},
        "speedup_vs_one_by_one": seq_total / ms,
    }


def localization_errors(nv, a, dev_in, ud, radii=(1.0, 2.0, 3.0, 4.0, 5.0, 6.0)):
    """One-pass (no outer iteration) relative error against the direct
    solution for each patch radius rho: the localization error of the
    transform of Definition defb.  Float64 with patch and level solves to
    1e-12, so that localization, not rounding, is measured (in float32 the
    one-pass result carries rounding errors near 1e-3 at contrast 1e4).  From
    rho = 4 on, the float64 patch blocks exceed one CTA's shared memory and
    the patch CG runs over thread-block clusters."""
    import torch
    q = int(np.log2(a.size))
    out = {}
    for rho in radii:
        o = nv.gamblet_default_opts()
        o.rho = rho
        o.precision = nv.FP64
        o.level_tol = 1e-12
        o.level_max_iter = 5000
        o.patch_tol = 1e-12
        o.refine_max_iter = 0
        h = nv.gamblet_setup(dev_in["rowptr"], dev_in["colind"], dev_in["val"], q,
                             dev_in["cells"], o)
        try:
            u = torch.zeros_like(dev_in["g"])
            nv.gamblet_solve(h, dev_in["g"], u)
            out[str(int(rho))] = rel_err(u.cpu().numpy(), ud)
        finally:
            nv.gamblet_destroy(h)
    return out


def mixed_by_rho(nv, torch, a, dev_in, stream, flush, ud, radii=(3.0, 4.0), steps=3):
    """The headline mixed arm (setup + refined solve, the same tolerances) at
    patch radii 3 and 4: device time per step, DOF/s, outer iterations and
    the error against the direct solution.  A larger radius makes the
    one-pass transform more accurate (fewer outer iterations) and the setup
    heavier."""
    import copy
    out = {}
    for rho in radii:
        b = copy.copy(a)
        b.rho = rho
        r = run_arm(nv, torch, b, dev_in, nv.MIXED, steps, 2, stream, flush)
        ms = statistics.mean(r["times_ms"])
        out[str(int(rho))] = {"ms_per_step": ms, "value": int(dev_in["g"].shape[0]) / (ms * 1e-3),
                              "unit": UNIT, "setup_ms": statistics.mean(r["setup_ms"]),
                              "solve_ms": statistics.mean(r["solve_ms"]),
                              "outer_iters": r["infos"][-1]["outer_iters"],
                              "rel_err": rel_err(r["u"], ud)}
    return out


def mass_init_timing(nv, torch, dev, a, stream):
    """Setup with the mass-matrix initialisation (Algorithm 2 lines 2a-5,
    rho_q = 2) and refined solve: the paper's Example 1 (q = 6, float64,
    error against the oracle's direct solve of the initialised system) and
    the 1024 x 1024 rough problem (mixed, relative residual of A^(q) U = g)."""
    import scipy.sparse.linalg as spla
    from oracle.massinit import mass_initialised_operator
    from workloads import assemble_q1_mass, make_example1, make_problem
    out = {}
    for name, p, prec in (("example1_q6", make_example1(6), nv.FP64),
                          (f"rough_{a.size}x{a.size}", make_problem(a.size, a.contrast, 0), nv.MIXED)):
        M = assemble_q1_mass(p.n)
        dev_arrays = []
        for X in (p.A, M):
            X = X.tocsr()
            X.sort_indices()
            dev_arrays.append(tuple(torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in
                                    (X.indptr.astype(np.int32), X.indices.astype(np.int32),
                                     X.data.astype(np.float64))))
        cells = torch.from_numpy(np.ascontiguousarray(p.cells, dtype=np.int32)).to(dev)
        g = torch.from_numpy(p.g).to(dev)
        o = opts_for(nv, a, prec, stream.cuda_stream, 0)
        o.refine_tol = 1e-12 if prec == nv.FP64 else a.refine_tol
        times = []
        for it in range(3):
            u = torch.zeros_like(g)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                h = nv.gamblet_setup_mass(dev_arrays[0], dev_arrays[1], p.q, cells, 2.0, o)
                info = nv.Info()
                nv.gamblet_solve(h, g, u, None, info)
                e1.record(stream)
            e1.synchronize()
            nv.gamblet_destroy(h)
            if it > 0:
                times.append(e0.elapsed_time(e1))
        ms = statistics.mean(times)
        rec = {"dofs": p.ndof, "rho": a.rho, "rho_q": 2.0, "ms_per_step": ms,
               "value": p.ndof / (ms * 1e-3), "unit": UNIT, "setup_ms": info.setup_ms,
               "solve_ms": info.solve_ms, "outer_iters": info.outer_iters,
               "rel_residual": info.rel_residual,
               "precision": "f64" if prec == nv.FP64 else "f32+f64"}
        if p.ndof <= 20000:
            Aq, Minv = mass_initialised_operator(p.A, M, p.cells, p.q, 2.0)
            u_ref = Minv @ spla.spsolve(Aq.tocsc(), p.g)
            rec["rel_err_vs_oracle"] = rel_err(u.cpu().numpy(), u_ref)
        out[name] = rec
    return out


def three_d_timing(nv, torch, dev, peaks, alu, steps=3):
    """The three-dimensional path (include/gamblet3d.h, float64 throughout):
    setup + refined solve to a relative residual of 1e-9 on the 64^3
    trilinear rough-coefficient problem (250,047 unknowns, contrast 1e4,
    seed 0) with patch radius 1 under both neighbourhood rules, inputs
    resident on the device; the error against the oracle's direct solve on
    the 32^3 problem (29,791 unknowns); per-kernel device times and the
    roofline of the three largest kernels from a separate profiled pass."""
    from oracle import direct
    from workloads import make_problem3

    def dev_csr(p):
        A = p.A.tocsr()
        A.sort_indices()
        return [torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in
                (A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64))]

    def opts(rho, rule, profile):
        o = nv.gamblet_default_opts()
        o.rho, o.nbr_rule, o.profile = rho, rule, profile
        o.level_tol, o.patch_tol = 0.05, 1e-3
        o.refine_tol, o.refine_max_iter = 1e-9, 200
        return o

    out = {"workload": "64^3 Q1 trilinear rough coefficient, q=6, contrast 10000, g~N(0,1), "
                       "float64", "l2": "inputs and operators (about 1 GB) exceed L2"}
    p = make_problem3(64, 1e4, 0)
    rp, ci, va = dev_csr(p)
    cells = torch.from_numpy(np.ascontiguousarray(p.cells)).to(dev)
    g = torch.from_numpy(p.g).to(dev)
    u = torch.zeros_like(g)
    for rule, rname in ((1, "cheb"), (0, "euclid")):
        o = opts(1.0, rule, 0)
        times, infos = [], []
        for rep in range(steps + 1):
            torch.cuda.synchronize()
            h = nv.gamblet3d_setup(rp, ci, va, p.q, cells, o)
            info = nv.Info()
            nv.gamblet3d_solve(h, g, u, None, info)
            nv.gamblet3d_destroy(h)
            if rep:
                times.append(info.setup_ms + info.solve_ms)
                infos.append(info.as_dict())
        ms = statistics.mean(times)
        row = {"rho": 1, "rule": rname, "dofs": p.ndof, "ms_per_step": ms,
               "value": p.ndof / (ms * 1e-3), "unit": UNIT,
               "setup_ms": statistics.mean(i["setup_ms"] for i in infos),
               "solve_ms": statistics.mean(i["solve_ms"] for i in infos),
               "outer_iters": infos[-1]["outer_iters"], "rel_residual": infos[-1]["rel_residual"],
               "patch_iters_mean": infos[-1]["patch_iters_mean"]}
        # profiled pass: per-kernel times and the roofline of the largest kernels
        h = nv.gamblet3d_setup(rp, ci, va, p.q, cells, opts(1.0, rule, 1))
        nv.gamblet3d_solve(h, g, u, None, nv.Info())
        st = nv.gamblet3d_kernel_stats(h)
        nv.gamblet3d_destroy(h)
        tot = sum(x["ms"] for x in st)
        top = sorted(st, key=lambda x: -x["ms"])[:3]
        rl = {}
        for x in top:
            e = {"ms": x["ms"], "share": x["ms"] / tot, "launches": x["launches"]}
            if x["ms"] > 0 and x["bytes"] > 0:
                gbs = x["bytes"] / (x["ms"] * 1e-3) / 1e9
                e["hbm"] = {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": gbs / peaks["hbm_gbs"]}
            if x["ms"] > 0 and x["flops"] > 0 and alu.get("fp64_tflops"):
                tf = x["flops"] / (x["ms"] * 1e-3) / 1e12
                e["fp64"] = {"achieved": tf, "peak": alu["fp64_tflops"], "unit": "TFLOP/s",
                             "frac": tf / alu["fp64_tflops"]}
            rl[x["name"]] = e
        row["kernels_top"] = rl
        out[rname] = row
    # error against the oracle's direct solve (32^3)
    p = make_problem3(32, 1e4, 0)
    rp, ci, va = dev_csr(p)
    cells = torch.from_numpy(np.ascontiguousarray(p.cells)).to(dev)
    g = torch.from_numpy(p.g).to(dev)
    u = torch.zeros_like(g)
    h = nv.gamblet3d_setup(rp, ci, va, p.q, cells, opts(1.0, 1, 0))
    info = nv.Info()
    nv.gamblet3d_solve(h, g, u, None, info)
    nv.gamblet3d_destroy(h)
    ud, _ = direct.solve(p.A, p.g)
    out["rel_err_vs_oracle_32x32x32"] = rel_err(u.cpu().numpy(), ud)
    out["peaks"] = "HBM: MEASURED_PEAKS.json hbm_gbs; float64: torch.matmul float64 (alu_peaks)"
    return out


def level_conditions(nv, a, dev_in, steps=60):
    """cond(B^(k)) estimates (Lanczos, float64 level operators) per level, for
    W of Construction const2 (the stored basis) and const1: the paper bounds
    them uniformly in k (Theorem thmodhehiudhehd) and finds const2 the better
    conditioned."""
    q = int(np.log2(a.size))
    o = opts_for(nv, a, nv.FP64, None, 0)
    o.refine_max_iter = 0
    h = nv.gamblet_setup(dev_in["rowptr"], dev_in["colind"], dev_in["val"], q, dev_in["cells"], o)
    try:
        out = {}
        for k in range(2, q + 1):
            lo, hi = nv.gamblet_level_condition(h, k, steps, 2)
            lo1, hi1 = nv.gamblet_level_condition(h, k, steps, 1)
            out[str(k)] = {"lmin": lo, "lmax": hi, "cond": hi / lo, "cond_const1": hi1 / lo1}
        return out
    finally:
        nv.gamblet_destroy(h)


def multi_rhs_timing(nv, torch, a, dev_in, stream, nrhs=4, steps=3):
    """Solve phase only: nrhs right-hand sides through gamblet_solve_many
    (matrices read once per group) against nrhs calls of gamblet_solve, on
    one mixed-precision hierarchy of the bench problem."""
    q = int(np.log2(a.size))
    o = opts_for(nv, a, nv.MIXED, stream.cuda_stream, 0)
    h = nv.gamblet_setup(dev_in["rowptr"], dev_in["colind"], dev_in["val"], q, dev_in["cells"], o)
    try:
        n = int(dev_in["g"].shape[0])
        gen = torch.Generator(device="cpu").manual_seed(11)
        G = torch.randn(nrhs, n, generator=gen, dtype=torch.float64).to(dev_in["g"].device)
        U = torch.zeros_like(G)
        u1 = torch.zeros(n, dtype=torch.float64, device=G.device)

        def timed(fn):
            ts = []
            for it in range(steps + 1):
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    e0.record(stream)
                    fn()
                    e1.record(stream)
                e1.synchronize()
                if it > 0:
                    ts.append(e0.elapsed_time(e1))
            return statistics.mean(ts)

        info = nv.Info()
        many_ms = timed(lambda: nv.gamblet_solve_many(h, G, U, info))
        worst = info.rel_residual
        single_ms = timed(lambda: [nv.gamblet_solve(h, G[r], u1) for r in range(nrhs)])
        return {"nrhs": nrhs, "dofs": n, "solve_many_ms": many_ms, "single_solves_ms": single_ms,
                "speedup": single_ms / many_ms, "value": nrhs * n / (many_ms * 1e-3),
                "unit": "DOF/s (solve phase, all right-hand sides)", "worst_rel_residual": worst}
    finally:
        nv.gamblet_destroy(h)


def cpu_oracle(p):
    """The oracle's direct solve (SuperLU + extended-precision refinement)."""
    from oracle import direct
    t0 = time.perf_counter()
    u, _ = direct.solve(p.A, p.g)
    return u, time.perf_counter() - t0


def cpu_oracle_other():
    """The other CPU baselines: the oracle's exact (non-localized)
    decomposition at 32 x 32 cells (q = 5, C = 100), its localized setup +
    one-pass solve at 128 x 128 (q = 7, C = 1e4, rho = 3), and its gradient
    through the one-pass transform at 32 x 32 (rho = 3), in fine DOFs/s.
    All run numpy/scipy, whose BLAS uses the host's cores."""
    from workloads import make_problem
    from oracle.exact import gamblet_exact
    from oracle.local import gamblet_local_setup, gamblet_local_solve
    out = {}
    p = make_problem(32, 100.0, 0)
    t0 = time.perf_counter()
    gamblet_exact(p.A, p.g, p.cells, p.q)
    t = time.perf_counter() - t0
    out["exact_32x32"] = {"value": p.ndof / t, "unit": UNIT, "seconds": t,
                          "sample": "exact decomposition, Algorithm 1 with dense level solves, "
                                    "961 unknowns"}
    p = make_problem(128, 1e4, 0)
    t0 = time.perf_counter()
    st = gamblet_local_setup(p.A, p.cells, p.q, 3.0)
    t1 = time.perf_counter()
    gamblet_local_solve(st, p.g)
    t2 = time.perf_counter()
    out["localized_128x128"] = {"value": p.ndof / (t2 - t0), "unit": UNIT,
                                "setup_s": t1 - t0, "solve_s": t2 - t1,
                                "sample": "localized setup (dense patch solves, rho = 3) and "
                                          "one-pass solve, 16,129 unknowns"}
    # the gradient through the one-pass transform (dense reverse pass)
    from oracle import direct
    from oracle.local_adjoint import gradient_one_pass
    from workloads.rough import K_REF
    p = make_problem(32, 1e4, 0)
    u_obs, _ = direct.solve(make_problem(32, 1e4, 7).A, p.g)
    t0 = time.perf_counter()
    gradient_one_pass(p.A, p.g, u_obs, 32, np.exp(p.log_a), K_REF, p.cells, p.q, 3.0)
    t = time.perf_counter() - t0
    out["one_pass_gradient_32x32"] = {"value": p.ndof / t, "unit": UNIT, "seconds": t,
                                      "sample": "localized setup, one-pass solve and the reverse "
                                                "pass through both (dense), rho = 3, 961 "
                                                "unknowns"}
    out["cores"] = os.cpu_count()
    out["kind"] = "oracle"
    return out


def rel_err(u, ud):
    return float(np.linalg.norm(u - ud) / np.linalg.norm(ud))


def families(stats):
    """Per-level entries (name_kN) summed into kernel families."""
    out = {}
    for k, v in stats.items():
        base = k.rsplit("_k", 1)[0] if "_k" in k and k.rsplit("_k", 1)[1].isdigit() else k
        acc = out.setdefault(base, {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0})
        for key in acc:
            acc[key] += v[key]
    return out


# CUDA graphs of several kernels (the level CG's device-side loop) are timed
# as one entry; the contract's roofline is for a single kernel
COMPOSITE = ("level_cg",)


def roofline(stats, peaks, alu, mixed, name=None):
    """Roofline entry of one kernel (kernel family and level): by default the
    single kernel with the largest share of device time; per-launch figures
    are its own averages.  `alu` holds the measured GEMM throughputs
    (measured_alu_peaks)."""
    if name is None:
        single = {k: v for k, v in stats.items() if k not in COMPOSITE} or stats
        name = max(single.items(), key=lambda kv: kv[1]["ms"])[0]
    st = stats[name]
    family = name.rsplit("_k", 1)[0] if "_k" in name and name.rsplit("_k", 1)[1].isdigit() else name
    launches = max(st["launches"], 1)
    avg_ms = st["ms"] / launches
    per_launch_bytes = st["bytes"] / launches
    per_launch_flops = st["flops"] / launches
    total_ms = sum(s["ms"] for s in stats.values())
    common = {"kernel": name, "launches": st["launches"], "avg_launch_ms": avg_ms,
              "share_of_device_time": st["ms"] / total_ms, "traffic": ncu_traffic(name, mixed),
              "timing": "CUDA events around every launch of the kernel, over a second pass of "
                        "the timed steps with the library's per-kernel events on"}
    if family in ("patch_pcg", "patch_cholesky", "patch_mma", "patch_cluster"):
        tensor = family == "patch_mma"
        if tensor:
            # kind::f16 products: the dense float16 rate equals the bf16 rate
            peak = peaks.get("bf16_tflops")
            what = "dense bf16/fp16 tensor-core GEMM, MEASURED_PEAKS.json bf16_tflops (of measured)"
        elif mixed:
            peak = alu.get("fp32_simt_tflops")
            what = "float32 SIMT GEMM (torch.matmul, of measured)"
        else:
            peak = alu.get("fp64_tflops")
            what = "float64 GEMM (torch.matmul, of measured)"
        achieved = per_launch_flops / (avg_ms * 1e-3) / 1e12
        out = {**common, "bound": "tensor" if tensor else "alu", "achieved": achieved,
               "peak": peak, "unit": "TFLOP/s",
               "frac": achieved / peak if peak else None, "peak_source": what,
               "algorithmic": f"{per_launch_flops:.4g} flop per launch" + (
                   " (tensor-core products issued: windows x iterations x M-tiles x "
                   "2 x 128 x 16 x K)" if tensor else "")}
        if tensor:
            out["binding_unit"] = ("per-iteration latency of the window CG (block reductions, "
                                   "barriers, product issue); N = 16 products use a fraction "
                                   "of the pipe by construction (ncu: tensor pipe 3 % active)")
        if mixed and not tensor:
            # the lanes are not what binds this kernel: its shared-memory block
            # products are (ncu summary of the patch CG kernel)
            out["binding_unit"] = "shared-memory load pipe, L1/TEX 81-85% of peak (ncu)"
        return out
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = per_launch_bytes / (avg_ms * 1e-3) / 1e9
    out = {**common, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks
           else "fallback 6.8 TB/s", "algorithmic": f"{per_launch_bytes:.4g} byte per launch"}
    if per_launch_flops > 0:
        fp = alu.get("fp32_simt_tflops" if mixed else "fp64_tflops")
        tf = per_launch_flops / (avg_ms * 1e-3) / 1e12
        out["alu"] = {"achieved": tf, "peak": fp, "unit": "TFLOP/s",
                      "frac": tf / fp if fp else None,
                      "algorithmic": f"{per_launch_flops:.4g} flop per launch"}
    if name in COMPOSITE:
        out["composite"] = ("one CUDA graph per launch: SpMV, update, scalar and direction "
                            "kernels repeated by a device-side while loop; ncu lists none of "
                            "them, so traffic is not measured")
    return out


def bench_config(a, ndof):
    """The workload description shared by both arms of the bench."""
    return {"workload": workload_name(a), "dofs": ndof, "per_rank_problems": 1,
            "l2": "flushed between timed steps (256 MiB device write)",
            "level_tol": a.level_tol, "refine_tol": a.refine_tol,
            "precision": "mixed: float32 patch solves (block-Jacobi CG to 1e-3), Galerkin "
                         "products and level-CG SpMV; float64 dot products, coarsest solve and "
                         "outer refinement",
            "caches": "the symbolic plan, the autotuner's launch shapes and the library's "
                      "memory pool are process-wide and warm in the timed steps (filled "
                      "during warm-up); the cold first call is reported as setup_cold"}


def reference_main(a, ws, rank):
    """--impl reference: the CPU oracle (direct solve) timed on host cores."""
    if rank != 0:
        return 0
    from workloads import make_problem
    p = make_problem(a.size, a.contrast, seed=0)
    times = []
    for it in range(a.warmup + a.steps):
        _, t = cpu_oracle(p)
        if it >= a.warmup:
            times.append(t)
    ms = statistics.mean(times) * 1e3
    value = p.ndof / (ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": bench_config(a, p.ndof),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "full 2^20-class problem: SuperLU factor + solve + 3 "
                                   "extended-precision refinement steps, per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    a = parse()
    ws, rank, local = dist_env()
    if a.impl == "reference":
        return reference_main(a, ws, rank)
    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1503_03467_gb300 import build as _b
    _b.build()
    from paper_1503_03467_gb300 import native as nv

    dev = torch.device("cuda", torch.cuda.current_device())
    p, host = make_inputs(a, rank)
    ndof = p.ndof
    # oracle solution for the error bar (and the CPU baseline on rank 0, N = 1)
    ud, cpu_s = cpu_oracle(p)
    cold = cold_start(a, torch.cuda.current_device()) if rank == 0 else None
    dev_in = {k: torch.from_numpy(v).to(dev) for k, v in host.items()}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    if ws > 1:
        dist.barrier()
    mixed = run_arm(nv, torch, a, dev_in, nv.MIXED, a.steps, a.warmup, stream, flush,
                    clocks_dev=torch.cuda.current_device())
    plain = None
    if not a.no_plain:
        plain = run_arm(nv, torch, a, dev_in, nv.FP64, max(2, a.steps // 2), max(1, a.warmup // 2),
                        stream, flush, profile=1)
    e2e = run_e2e(nv, a, host, nv.MIXED, a.e2e_steps or a.steps)
    # per-kernel CUDA-event times for the roofline: the same K steps again with
    # the library's per-phase events on (the headline pass above runs without)
    prof = run_arm(nv, torch, a, dev_in, nv.MIXED, a.steps, 1, stream, flush, profile=1)
    ms = statistics.mean(mixed["times_ms"])
    ms_max, _ = reduce_over_ranks(torch, dev, ms, ndof)
    if ws > 1:
        dist.barrier()
    err_mixed = rel_err(mixed["u"], ud)
    err_e2e = rel_err(e2e["u"], ud)
    value = ws * ndof / (ms_max * 1e-3)
    peaks = load_peaks()
    alu = measured_alu_peaks(torch, dev)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": bench_config(a, ndof),
        "rel_err": err_mixed, "rel_err_ok": err_mixed <= REL_ERR_BAR,
        "setup_ms": statistics.mean(mixed["setup_ms"]),
        "solve_ms": statistics.mean(mixed["solve_ms"]),
        "outer_iters": mixed["infos"][-1]["outer_iters"],
        "level_iters": mixed["infos"][-1]["level_iters"],
        "gpu_launches": int(mixed["launches"]),
        "e2e": {"value": ws * ndof / (e2e["ms"] * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(e2e["h2d"]), "d2h_bytes_per_step": int(e2e["d2h"]),
                "rel_err": err_e2e},
        "roofline": roofline(prof["stats"], peaks, alu, True),
        "roofline_others": {n: roofline(prof["stats"], peaks, alu, True, name=n)
                            for n in ("level_cg", "patch_mma_k9", "galerkin_k9", "galerkin_k10",
                                      "patch_pcg_k10", "restrict", "prolong")
                            if n in prof["stats"]},
        "clocks": mixed["clocks"],
        "alu_peaks": alu,
        "setup_cold": cold,
        "kernels": {k: {"share": v["ms"] / sum(s["ms"] for s in families(prof["stats"]).values()),
                        "ms_per_step": v["ms"] / a.steps, "launches_per_step": v["launches"] / a.steps}
                    for k, v in sorted(families(prof["stats"]).items(), key=lambda kv: -kv[1]["ms"])},
    }
    if plain is not None:
        pms = statistics.mean(plain["times_ms"])
        line["plain_fp64"] = {
            "value": ndof / (pms * 1e-3), "ms_per_step": pms,
            "setup_ms": statistics.mean(plain["setup_ms"]),
            "solve_ms": statistics.mean(plain["solve_ms"]),
            "rel_err": rel_err(plain["u"], ud), "outer_iters": plain["infos"][-1]["outer_iters"],
            "roofline": roofline(plain["stats"], peaks, alu, False)}
        line["speedup_mixed_vs_plain"] = line["plain_fp64"]["ms_per_step"] / ms
    if not a.no_adjoint:
        line["adjoint"] = adjoint_timing(nv, torch, dev)
        line["adjoint_one_pass"] = onepass_grad_timing(nv, torch, dev)
    if not a.no_batched:
        line["batched"] = batched_timing(nv, torch, dev, a, stream, flush, ws, rank)
    if not a.no_localization:
        line["localization_error_one_pass"] = localization_errors(nv, a, dev_in, ud)
        line["mixed_by_rho"] = mixed_by_rho(nv, torch, a, dev_in, stream, flush, ud)
    if not a.no_mass:
        line["mass_init"] = mass_init_timing(nv, torch, dev, a, stream)
    if not a.no_localization:
        line["level_condition"] = level_conditions(nv, a, dev_in)
    if not a.no_3d:
        line["three_d"] = three_d_timing(nv, torch, dev, peaks, alu)
    if not a.no_mass:
        line["multi_rhs"] = multi_rhs_timing(nv, torch, a, dev_in, stream)
    if rank == 0 and ws == 1 and not a.no_cpu:
        line["cpu_baseline"] = {"value": ndof / cpu_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "one full solve of the same problem: SuperLU factor + "
                                          "solve + 3 extended-precision refinement steps"}
        line["cpu_oracle_other"] = cpu_oracle_other()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
