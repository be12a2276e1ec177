#!/usr/bin/env python
"""Benchmark of the contour-integral overlap path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--mode MODE]
    python bench.py --impl reference ...

A step is one pass of the hot path over one batch of synthetic sources:
D_ov(m_q) b = (1+m_q)/2 b + (1-m_q)/2 gamma5 S_N b for every source of the batch,
S_N b = c0 b + sum_j c_j (z_j - H_W)^-1 b from one shifted Krylov solve (Eqs. 1, 5-7).
The default workload is 16^3 x 32 (eps 0.6, m_q 0.01), N_q = 64, the 12 spin-colour point
sources, in the FP64 coefficient-space form; the contour is one explicit ellipse shared
with the reference arm.  The metric is source applies per second.  The same line carries
the double-float and FP32-refinement forms on the same step (speed-up and difference),
the FP32 stencil's HBM bandwidth on 12 right-hand sides, the dominant kernel's roofline
and the CPU oracle's throughput.  Prints ONE JSON line on rank 0.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on
the launching stream; a 256 MiB buffer is written between timed steps to flush
L2; barrier + synchronize on both sides; max over ranks.  The end-to-end figure
repeats the K steps through the same C-ABI call with pinned HOST buffers (copies
inside the timed region).  Kernel durations for the roofline come from the
library's per-launch CUDA events on the same stream (a separate pass of a few steps,
because the timed pass replays CUDA graphs that cannot hold those events).

--impl reference times the FP64 CPU oracle (per-node CGNR solves and the weighted
sum) on the host cores, on bounded slices of the same workload (see OracleSample).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "sgn(H_W)·b applies/s and dslash HBM GB/s vs roofline; batched-mixed vs FP64"
UNIT = "applies/s"

# FP64 arithmetic peak of one GB300 (profiling recipe's nominal table); HBM from MEASURED_PEAKS.json
FP64_PEAK_TFLOPS = 1.25
HBM_FALLBACK_GBS = 6800.0

# The contour of the sign workloads: one explicit single ellipse, the same for both arms
# (recorded in the line's config).  ||H_W|| <= |4 - m0| + 4 = 6.4 for every SU(3) field at
# r = 1 (each of the eight hops has norm 1/2), so the ellipse from 0 to 1.05 x 6.4 encloses
# the whole positive spectrum; alpha = 0.25 minimises max |r_N - sgn| over +-[0.3, 6.4] at
# 64 nodes (4.4e-7).  The library's Lanczos placement runs too, untimed, for the spectrum.
ELLIPSE = dict(gamma=3.36, rho=3.36, alpha=0.25)

WORKLOADS = {
    # name: lattice, link roughness, quark mass, nodes, sources, source kind, tolerance, solver mode
    "16^3x32-nq64-12pt": dict(dims=(16, 16, 16, 32), eps=0.6, m_q=0.01, n_q=64, nsrc=12, src="point", tol=1e-12,
                              mode="fp64_2pass", compare=("f32x2", "mixed"), dslash=True, ellipse=ELLIPSE),
    "16^4-nq64-12pt": dict(dims=(16, 16, 16, 16), eps=0.5, m_q=0.05, n_q=64, nsrc=12, src="point", tol=1e-12,
                           mode="fp64_2pass", compare=("f32x2",), dslash=True, ellipse=ELLIPSE),
    "8^4-fp64-nq64-4src": dict(dims=(8, 8, 8, 8), eps=0.5, m_q=0.05, n_q=64, nsrc=4, src="gauss", tol=1e-12,
                               mode="fp64_2pass", compare=("f32x2",), ellipse=ELLIPSE),
    "4^4-fp64-nq32-1src": dict(dims=(4, 4, 4, 4), eps=0.3, m_q=0.1, n_q=32, nsrc=1, src="gauss", tol=1e-12,
                               mode="fp64", ellipse=ELLIPSE),
    # stencil only: H_W on 12 right-hand sides (diagnostic of the HBM roofline)
    "dslash-16^3x32-fp32-12rhs": dict(dims=(16, 16, 16, 32), eps=0.6, nsrc=12, kind="dslash", prec="fp32"),
    "dslash-16^3x32-fp64-12rhs": dict(dims=(16, 16, 16, 32), eps=0.6, nsrc=12, kind="dslash", prec="fp64"),
    "dslash-16^4-fp32-12rhs": dict(dims=(16, 16, 16, 16), eps=0.5, nsrc=12, kind="dslash", prec="fp32"),
    # overlap solve x = D_ov^-1 b (CG on the normal equations, double-float inner solves)
    "ovsolve-8^4-mq0.05-4src": dict(dims=(8, 8, 8, 8), eps=0.5, m_q=0.05, n_q=64, nsrc=4, src="gauss", tol=1e-10,
                                    inner_tol=1e-12, mode="f32x2", kind="ovsolve"),
    # gradient of Re<eta, sgn(H_W) b> w.r.t. b and the links (adjoint solves + fused force)
    "vjp-8^4-nq48": dict(dims=(8, 8, 8, 8), eps=0.4, n_q=48, nsrc=1, src="gauss", tol=1e-12, kind="vjp",
                         mode="f32x2"),
    # the same measure with Zolotarev's optimal node set (n pole pairs = 2n nodes) from Lanczos bounds
    "sigma-8^4-zolotarev": dict(dims=(8, 8, 8, 8), eps=0.5, nsrc=4, src="gauss", kind="sigma", rule="zolotarev",
                                n_list=(4, 8, 12, 16, 20)),
    # sigma vs nodes per contour with the paper's two-ellipse contour (rescaled), 8^4
    "sigma-8^4-paper-contour": dict(dims=(8, 8, 8, 8), eps=0.5, nsrc=4, src="gauss", kind="sigma",
                                    n_list=(100, 250, 500, 1000)),
}
DEFAULT_WORKLOAD = "16^3x32-nq64-12pt"
# arithmetic type of the vector work per solver mode (scalars, inner products and the sum stay f64)
DTYPES = {"fp64": "f64", "fp64_2pass": "f64", "fp64_regen": "f64", "mixed": "f32+f64", "f32x2": "f32x2"}
M0 = 1.6
# the oracle's resolvent tolerance (per-node CGNR, true relative residual)
ORACLE_TOL = 1e-13


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default=None, choices=[None, "fp64", "fp64_2pass", "fp64_regen", "mixed", "f32x2"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--variant", type=int, default=None, help="dslash workloads: time only this FP32 stencil variant")
    ap.add_argument("--compare-steps", type=int, default=2,
                    help="steps of each comparison mode (the workload's 'compare' list) timed beside the line")
    ap.add_argument("--no-dslash", action="store_true", help="skip the FP32 stencil measurement")
    ap.add_argument("--parallel", default="sources", choices=["sources", "nodes"],
                    help="N > 1: independent sources per GPU (weak), or the contour nodes split over the GPUs "
                         "with one sum-allreduce per step (strong)")
    ap.add_argument("--nsrc", type=int, default=None, help="use only the first N sources (profiling cases)")
    ap.add_argument("--max-iter", type=int, default=None,
                    help="cap the Krylov iterations (profiling cases; the line is then not a valid measurement)")
    ap.add_argument("--concurrency", type=int, default=0, help="source groups replayed as parallel graph branches")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload_inputs(wl, rank):
    import synthetic as S

    dims = wl["dims"]
    U = S.su3_links(dims, wl["eps"], S.seed_for("gauge:" + "x".join(map(str, dims))))
    if wl["src"] == "gauss":
        b = S.gaussian_spinor(dims, S.seed_for(f"src:{rank}"), n=wl["nsrc"])
    else:
        b = S.point_sources(dims)[: wl["nsrc"]]
    return U, b


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- oracle (CPU)

def workload_contour(wl):
    """(gamma, rho, alpha) of the workload's explicit single ellipse (both arms)."""
    e = wl["ellipse"]
    return e["gamma"], e["rho"], e["alpha"]


def oracle_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


class OracleSample:
    """Bounded timing of the FP64 CPU oracle (per-node CGNR to 1e-13 on (z_j - H_W) y = b,
    Eq. 6, then the weighted sum of Eqs. 5-7) on one source of the workload.

    One apply solves every node to 1e-13, which at 16^3 x 32 takes hours on the host.  The
    sample runs every `stride`-th node (as many as the host has cores, at most 16) for a
    capped number of CGNR iterations, in parallel over nodes.  From the true residual each
    node reaches, its iterations to 1e-13 are extrapolated geometrically (a node that
    converged inside the sample counts its own iterations); the sampled nodes stand for
    all of them.  CG slows down as it meets the small eigenvalues of the normal
    equations, so the extrapolated count is low and the estimate favours the oracle.
    Work of one apply = node-iterations; throughput = node-iterations per second of
    the sample."""

    def __init__(self, U, b0, z, c, c0, k_iter):
        from oracle import cimpl

        cimpl.build()
        n = len(z)
        self.threads = oracle_threads()
        nsamp = max(1, min(16, self.threads, n))
        self.stride = max(1, n // nsamp)
        self.idx = np.arange(0, n, self.stride)[:nsamp]
        self.U, self.b0, self.z, self.c, self.c0, self.n = U, b0, z, c, c0, n
        dt, iters, res = self.run(k_iter)
        need = []
        for it, r in zip(iters, res):
            if it < k_iter or r <= ORACLE_TOL:
                need.append(float(it))
            else:
                need.append(it * np.log(ORACLE_TOL) / np.log(max(min(r, 0.999999), 1e-300)))
        self.k_iter = k_iter
        self.work = float(np.sum(need)) * n / len(self.idx)  # node-iterations of one apply
        self.rate = float(np.sum(iters)) / dt                 # node-iterations per second
        self.setup_s = dt
        self.need = need

    def run(self, k_iter):
        from oracle import cimpl

        t0 = time.perf_counter()
        _, iters, res = cimpl.sign_apply(self.U, self.b0, self.z[self.idx], self.c[self.idx], 0.0, M0,
                                         tol=ORACLE_TOL, maxiter=int(k_iter), strict=False)
        return time.perf_counter() - t0, iters, res

    def applies_per_s(self):
        return self.rate / self.work

    def describe(self):
        return {
            "cores": int(min(self.threads, len(self.idx))), "host_cpu_count": os.cpu_count(),
            "sampled_nodes": int(len(self.idx)), "nodes": int(self.n),
            "cgnr_iterations_sampled": int(self.k_iter),
            "extrapolated_iterations_per_node": [int(round(x)) for x in self.need],
            "sample": (f"source 0, {len(self.idx)} of {self.n} nodes (every {self.stride}th), per-node CGNR "
                       f"(oracle, FP64) capped at {self.k_iter} iterations in parallel over nodes; iterations "
                       f"to {ORACLE_TOL:g} extrapolated per node from its residual reduction (geometric; "
                       f"favours the oracle), scaled to all {self.n} nodes: EXTRAPOLATED, not a full apply"),
        }


def oracle_iteration_seconds(U, b0):
    """Seconds of one CGNR iteration of the C oracle (two H_W applies and the vector
    updates), from one timed H_W apply; sizes the bounded samples."""
    from oracle import cimpl

    cimpl.build()
    cimpl.hw_apply(U, b0, M0)
    t0 = time.perf_counter()
    cimpl.hw_apply(U, b0, M0)
    return 2.3 * (time.perf_counter() - t0)


def run_reference(args, wl):
    """The oracle as it stands, timed on the host cores on the workload's explicit contour
    (the same nodes as the GPU arm), each step a bounded slice of one apply: every sampled
    node advances `k_step` CGNR iterations.  The fraction of one apply a step covers comes
    from the untimed setup sample (OracleSample), so value = fraction / step time."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import contour

    U, b = workload_inputs(wl, 0)
    g, r, a = workload_contour(wl)
    z, c, c0 = contour.single_contour(wl["n_q"], g, r, a)
    t_it = oracle_iteration_seconds(U, b[0])
    k_setup = int(np.clip(15.0 / t_it, 10, 4000))
    k_step = int(np.clip(3.0 / t_it, 2, 1000))
    samp = OracleSample(U, b[0], z, c, c0, k_setup)
    for _ in range(args.warmup):
        samp.run(k_step)
    times, iters_done = [], 0
    for _ in range(args.steps):
        dt, iters, _ = samp.run(k_step)
        times.append(dt)
        iters_done += int(np.sum(iters))
    total = sum(times)
    applies = iters_done / samp.work  # fraction of one source apply covered by the timed steps
    value = applies / total
    cb = samp.describe()
    cb.update({"value": value, "unit": UNIT, "kind": "oracle",
               "timed_steps": f"{args.steps} steps, each every sampled node advancing {k_step} CGNR iterations "
                              f"({applies / args.steps:.3g} of one source apply per step)"})
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
        "applies_per_step": applies / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args, wl, "oracle: per-node CGNR, FP64"),
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_dict(args, wl, mode):
    g, r, a = workload_contour(wl)
    c = {
        "workload": args.workload, "lattice": "x".join(map(str, wl["dims"])), "link_eps": wl["eps"], "m0": M0,
        "r": 1.0, "bc_t": "antiperiodic", "m_q": wl["m_q"], "N_q": wl["n_q"],
        "sources_per_gpu": args.nsrc or wl["nsrc"],
        "source": "complex Gaussian" if wl["src"] == "gauss" else "12 spin-colour point sources at the origin",
        "tol": wl["tol"], "mode": mode,
        "contour": {"form": "single ellipse (sgn = 2 P - 1), trapezoid rule of Eq. 7", "n_q": wl["n_q"],
                    "gamma": g, "rho": r, "alpha": a,
                    "why": "explicit and shared by both arms; encloses (0, 6.72], and |lambda| <= 6.4 for any "
                           "SU(3) field at m0 = 1.6"},
        "l2": "256 MiB buffer written between timed steps", "graph_branches": args.concurrency or "auto",
        "parallelism": (f"contour nodes split over {args.gpus} GPUs, one sum-allreduce per step"
                        if getattr(args, "parallel", "sources") == "nodes"
                        else f"independent sources per GPU x{args.gpus}"),
    }
    if args.max_iter is not None:
        c["profiling_case"] = f"Krylov iterations capped at {args.max_iter}: not a measurement of the workload"
    return c


# ------------------------------------------------------------------ ours

def kernel_src_hash(files=None):
    """sha256 (16 hex digits) of the named source files (paths relative to the package's
    csrc/), or of every file there."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2204_01583_gb300", "csrc")
    for f in sorted(files if files is not None else os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def stored_traffic(kernel, workload):
    """DRAM bytes per launch from profiles/dram_traffic.json, or None once any source file
    the capture depended on has changed."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
        e = t.get(f"{kernel}@{workload}")
        if e and e.get("src_hash") == kernel_src_hash(e.get("files")):
            return e.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def timed_steps(step, steps, stream, flush):
    """Device time (ms) of each step: CUDA events on the launching stream, L2 flushed first."""
    import torch

    ts, out = [], []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out.append(step())
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return ts, out


def run_ours(args, wl):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2204_01583_gb300 import build as build_lib

    build_lib()
    from paper_2204_01583_gb300 import lib, parallel

    mode = args.mode or wl["mode"]
    nodes_split = args.parallel == "nodes"
    U, b = workload_inputs(wl, 0 if nodes_split else rank)
    if args.nsrc:
        b = b[: args.nsrc]
    nsrc = b.shape[0]
    dev = torch.device("cuda", local)
    ctx = lib.Context(wl["dims"], bc_t=-1, m0=M0, device=local)
    ctx.set_gauge(torch.from_numpy(U).to(dev))
    spec = ctx.place_contour(wl["n_q"], steps=150)  # spectrum report (untimed); the solve uses the explicit ellipse
    g, r, a = workload_contour(wl)
    ctx.set_contour_ellipse(wl["n_q"], g, r, a)
    if nodes_split:
        z, c, c0 = ctx.get_contour()
        zr, cr, c0r = parallel.node_shard(z, c, c0, rank, world)
        ctx.set_contour(zr, cr, c0r)
    bd = torch.from_numpy(b).to(dev)
    out = torch.empty_like(bd)
    capped = args.max_iter is not None
    max_iter = args.max_iter or 20000
    opts = ctx.opts(mode=mode, tol=wl["tol"], max_iter=max_iter)
    ctx.set_concurrency(args.concurrency)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(o=opts, src=bd, dst=out, s=None):
        if nodes_split:  # partial sum over this rank's nodes, then the sum over ranks
            st = ctx.sgn(src, dst, nsrc, o, stream=s, allow_not_converged=capped)
            if world > 1:
                parallel.allreduce_sum(dst)
            return st
        return ctx.overlap(wl["m_q"], src, dst, nsrc, o, stream=s, allow_not_converged=capped)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if world > 1:
            import torch.distributed as dist

            t = torch.tensor([x], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())
        return x

    for _ in range(args.warmup):
        step()
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    t_steps, stats = timed_steps(step, args.steps, stream, flush)
    barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(t_steps))
    applies = nsrc * args.steps * (1 if nodes_split else world)
    value = applies / (total_ms / 1e3)

    # end to end: the same call with pinned host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e and not nodes_split:
        hb = torch.from_numpy(b).pin_memory()
        ho = torch.empty_like(hb).pin_memory()
        ho_opts = ctx.opts(mode=mode, tol=wl["tol"], host_io=True, max_iter=max_iter)
        step(ho_opts, hb, ho, stream)
        barrier()
        esampler = ClockSampler(local)
        esampler.start()
        te, est = timed_steps(lambda: step(ho_opts, hb, ho, stream), args.steps, stream, flush)
        barrier()
        eclocks = esampler.stop()
        tot = max_over_ranks(sum(te))
        nbytes = int(b.nbytes)
        e2e = {"value": applies / (tot / 1e3), "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "ms_per_step": tot / args.steps, "clocks": eclocks, "launches_per_step": est[-1]["launches"],
               "library_ms_per_step": sum(x["ms"] for x in est) / len(est),
               "step_ms_min_median_max": [min(te), float(np.median(te)), max(te)]}

    # per-kernel durations (library events on the launching stream), a few more steps
    ctx.set_kernel_timing(True)
    kstats = []
    for _ in range(min(args.steps, 3)):
        flush.zero_()
        kstats.append(step())
    torch.cuda.synchronize()
    ktimes = ctx.kernel_times()
    ctx.set_kernel_timing(False)
    roof, kernels = roofline(wl, mode, ktimes, kstats, nsrc)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if nodes_split else "weak",
        "vs_baseline": None, "dtype": DTYPES[mode], "data": "synthetic",
        "config": config_dict(args, wl, mode), "clocks": clocks, "e2e": e2e,
        "gpu_launches": int(sum(s["launches"] for s in stats)), "roofline": roof, "kernels": kernels,
        "solver": {"iterations": stats[-1]["iterations"], "max_residual": stats[-1]["max_residual"],
                   "error_bound": stats[-1]["error_bound"], "converged": stats[-1]["converged"],
                   "launches_per_step": stats[-1]["launches"],
                   "library_ms_per_step": sum(x["ms"] for x in stats) / len(stats),
                   "step_ms_min_median_max": [min(t_steps), float(np.median(t_steps)), max(t_steps)],
                   "lanczos_spectrum": spec},
    }
    if not capped and not nodes_split and args.compare_steps > 0:
        for other in wl.get("compare", ()):
            if other != mode:
                # the refinement form takes several seconds per step at full size: one timed step
                k = 1 if other == "mixed" else args.compare_steps
                line[f"{other}_vs_{mode}"] = compare_mode(ctx, wl, other, bd, out, nsrc, stream, flush, k,
                                                         total_ms / args.steps, max_iter)
    if wl.get("dslash") and not args.no_dslash:
        line["dslash_fp32"] = measure_dslash_fp32(ctx, wl, nsrc, args.steps, flush, args.warmup)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        z, c, c0 = ctx.get_contour()
        t_it = oracle_iteration_seconds(U, b[0])
        samp = OracleSample(U, b[0], z, c, c0, int(np.clip(15.0 / t_it, 10, 4000)))
        cb = samp.describe()
        cb.update({"value": samp.applies_per_s(), "unit": UNIT, "kind": "oracle"})
        line["cpu_baseline"] = cb
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


# Algorithmic work per unit for each kernel class (FP64): (flops, bytes).
# Units: "si" = source-iteration x site, "nu" = node-update x site, "ls" = launch x site.
#   lanczos_hw_kernel:     H_W stencil 1368 flop + epilogue 72 flop; U_i, U_{i-1} read and
#                          w written (3 x 192 B)                               per si
#                          + the links, 576 B, once for all sources of a launch   per ls
#   lanczos_update_kernel: U_{i+1} = w - alpha v (12 x 10 flop; 3 x 192 B)    per si
#                          + p = v - l p and s += c zeta p (12 x 16 flop; p read+write 384 B) per nu
#   lanczos_regen_kernel:  stencil + Lanczos update + s += g v (1368 + 12 x 24 flop;
#                          576 + 4 x 192 B + sum read+write 384 B)            per si
#   lanczos_coop_kernel:   the two above for every iteration in one persistent launch  per si
#   basis_sum_kernel:      s += g_i v_i over the stored basis, one basis vector per
#                          source-iteration (12 x 8 flop; the vector read, 192 B)  per si
FP64_WORK = {
    "basis_sum_kernel": {"si": (96.0, 192.0)},
    "lanczos_coop_kernel": {"si": (1560.0, 1728.0)},
    "lanczos_hw_kernel": {"si": (1440.0, 576.0), "ls": (0.0, 576.0)},
    "lanczos_update_kernel": {"si": (120.0, 576.0), "nu": (192.0, 384.0)},
    "lanczos_regen_kernel": {"si": (1656.0, 1728.0)},
}


def compare_mode(ctx, wl, other, bd, out_ref, nsrc, stream, flush, steps, ref_ms, max_iter):
    """The same step in another solver mode: device time per step, speed-up of that mode
    over the line's mode, and the largest difference per source from the line's result
    (element-wise, max |a - b| / max |b|, and in norm)."""
    import torch

    o = ctx.opts(mode=other, tol=wl["tol"], max_iter=max_iter)
    ob = torch.empty_like(bd)
    ctx.overlap(wl["m_q"], bd, ob, nsrc, o)  # warm-up (layouts, graphs, autotuning)
    ts, st = timed_steps(lambda: ctx.overlap(wl["m_q"], bd, ob, nsrc, o), steps, stream, flush)
    ms = sum(ts) / len(ts)
    d = (ob - out_ref).reshape(nsrc, -1)
    ref = out_ref.reshape(nsrc, -1)
    elem = (d.abs().amax(dim=1) / ref.abs().amax(dim=1)).max().item()
    norm = (d.norm(dim=1) / ref.norm(dim=1)).max().item()
    return {"mode": other, "dtype": DTYPES[other], "ms_per_step": ms, "steps": steps,
            "speedup": ref_ms / ms, "max_rel_diff_elementwise": elem, "max_rel_diff_norm": norm,
            "iterations": st[-1]["iterations"], "converged": st[-1]["converged"]}


def measure_dslash_fp32(ctx, wl, nrhs, steps, flush, warmup):
    """H_W on nrhs FP32 right-hand sides with the autotuned stencil (ov_apply_HW, OV_FP32):
    device time per stencil launch from the library's events on the launching stream, and
    algorithmic bytes (12-real links once, each RHS read and written once) over it."""
    import torch

    from paper_2204_01583_gb300 import lib
    import synthetic as S

    dims = wl["dims"]
    V = int(np.prod(dims))
    psi = torch.from_numpy(S.gaussian_spinor(dims, 5, n=nrhs).astype(np.complex64)).cuda()
    o = torch.empty_like(psi)
    ctx.set_hw32_variant(-1)
    for _ in range(max(warmup, 1)):
        ctx.apply_HW(psi, o, nrhs, lib.OV_FP32)  # the first call autotunes
    torch.cuda.synchronize()
    ctx.set_kernel_timing(True)
    for _ in range(steps):
        flush.zero_()
        ctx.apply_HW(psi, o, nrhs, lib.OV_FP32)
    torch.cuda.synchronize()
    n, ms = ctx.kernel_times()["hw_kernel"]
    ctx.set_kernel_timing(False)
    per = ms / n / 1e3
    by = V * (48 * 4 + nrhs * 48 * 4)
    hbm, src = hbm_peak()
    return {"rhs": nrhs, "us_per_launch": per * 1e6, "bytes_per_launch": by, "gbs": by / per / 1e9,
            "peak_gbs": hbm, "peak_source": src, "frac": by / per / 1e9 / hbm,
            "bytes": "12-real FP32 links once (48 reals/site) + 48 FP32 reals/site per RHS in and out",
            "l2": "256 MiB buffer written between launches"}


def roofline(wl, mode, ktimes, kstats, nsrc):
    """Achieved rate of each kernel class from algorithmic work and measured durations."""
    V = int(np.prod(wl["dims"]))
    units = {"nu": sum(s["node_updates"] for s in kstats) * V,
             "si": sum(s["iterations"] for s in kstats) * nsrc * V}  # source-iterations (upper bound)
    hbm, hbm_src = hbm_peak()
    out = {}
    for k, (n, ms) in ktimes.items():
        if not n:
            continue
        d = {"launches": n, "ms": ms, "avg_us": ms / n * 1e3}
        if mode in ("fp64", "fp64_2pass", "fp64_regen", "f32x2") and k in FP64_WORK:
            uk = dict(units, ls=n * V)
            fl = sum(uk[u] * w[0] for u, w in FP64_WORK[k].items())
            by = sum(uk[u] * w[1] for u, w in FP64_WORK[k].items())
            d["tflops"] = fl / (ms / 1e3) / 1e12
            d["gbs"] = by / (ms / 1e3) / 1e9
        out[k] = d
    if not out:
        return None, out
    dom = max(out, key=lambda k: out[k]["ms"])
    d = out[dom]
    if "tflops" in d and mode == "f32x2":
        # double-float vectors occupy 16 B per complex like FP64: the same algorithmic bytes;
        # the kernel itself is bound by the FP32 issue rate (about 10 FP32 instructions per
        # FP64-equivalent flop), so the HBM fraction says how far it is from streaming
        roof = {"bound": "hbm", "achieved": d["gbs"], "peak": hbm, "unit": "GB/s", "frac": d["gbs"] / hbm,
                "traffic": stored_traffic(dom, wl_name_of(wl)), "kernel": dom, "peak_source": hbm_src,
                "fp64_equivalent_tflops": d["tflops"], "launch_avg_us": d["avg_us"]}
    elif "tflops" in d:
        roof = {"bound": "alu", "achieved": d["tflops"], "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": d["tflops"] / FP64_PEAK_TFLOPS, "traffic": stored_traffic(dom, wl_name_of(wl)),
                "kernel": dom, "peak_source": "nominal FP64 of GB300 (profiling recipe); an FMA loop measures 1.20",
                "hbm_gbs_algorithmic": d["gbs"], "hbm_frac_of_measured": d["gbs"] / hbm,
                "launch_avg_us": d["avg_us"]}
    else:
        roof = {"bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None, "traffic": None,
                "kernel": dom, "peak_source": hbm_src}
    return roof, out


def wl_name_of(wl):
    for k, v in WORKLOADS.items():
        if v is wl:
            return k
    return "?"


def run_dslash(args, wl):
    """H_W on nsrc right-hand sides: device time of the stencil kernel per launch (library
    events on the launching stream), achieved algorithmic GB/s against the measured HBM
    copy bandwidth.  FP32: every stencil variant is timed; the line reports the fastest
    (the one the autotuner keeps) and lists all of them."""
    import torch

    from paper_2204_01583_gb300 import build as build_lib

    build_lib()
    from paper_2204_01583_gb300 import lib
    import synthetic as S

    dims = wl["dims"]
    V = int(np.prod(dims))
    nrhs = wl["nsrc"]
    U = S.su3_links(dims, wl["eps"], S.seed_for("gauge:" + "x".join(map(str, dims))))
    ctx = lib.Context(dims, bc_t=-1, m0=M0)
    ctx.set_gauge(torch.from_numpy(U).cuda())
    fp32 = wl["prec"] == "fp32"
    dt = np.complex64 if fp32 else np.complex128
    psi = torch.from_numpy(S.gaussian_spinor(dims, 5, n=nrhs).astype(dt)).cuda()
    out = torch.empty_like(psi)
    prec = lib.OV_FP32 if fp32 else lib.OV_FP64
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    s_real = 4 if fp32 else 8
    variants = list(enumerate(lib.hw32_variants())) if fp32 else [(None, (1, 0, 128))]
    if fp32 and args.variant is not None:
        variants = [variants[args.variant]]
    hbm, src = hbm_peak()
    rows = []
    sampler = ClockSampler(0)
    sampler.start()
    for k, (rt, comp, nt) in variants:
        if k is not None:
            ctx.set_hw32_variant(k)
        for _ in range(args.warmup):
            ctx.apply_HW(psi, out, nrhs, prec)
        torch.cuda.synchronize()
        ctx.set_kernel_timing(True)
        for _ in range(args.steps):
            flush.zero_()
            ctx.apply_HW(psi, out, nrhs, prec)
        torch.cuda.synchronize()
        n, ms = ctx.kernel_times()["hw_kernel"]
        ctx.set_kernel_timing(False)
        # algorithmic link reals: 72 for the plain links (all 9 elements), 48 for the
        # 12-real forms; duplicated lanes are not counted
        link_reals = 48 if comp in (1, 8, 9, 12) else 72
        by = V * (link_reals * s_real + nrhs * 48 * s_real)  # links once per launch; each RHS in + out
        per = ms / n / 1e3
        rows.append({"variant": k, "rhs_tile": rt, "compressed_links": bool(comp), "threads": nt,
                     "us": per * 1e6, "bytes_per_launch": by, "gbs": by / per / 1e9,
                     "tflops": 1368.0 * V * nrhs / per / 1e12})
    clocks = sampler.stop()
    best = min(rows, key=lambda r: r["us"])  # the variant the autotuner keeps
    if fp32:
        code = variants[[r["variant"] for r in rows].index(best["variant"])][1][1]
        kern = {0: "hw32_tile_kernel", 1: "hw32_tile_kernel", 8: "hw32_s4_kernel"}.get(code, "hw_pair12_kernel")
        if code in (0, 1) and best["rhs_tile"] == 0:
            kern = "hw32_split_kernel"
    else:
        kern = "hw_kernel"
    if fp32:
        roof = {"bound": "hbm", "achieved": best["gbs"], "peak": hbm, "unit": "GB/s", "frac": best["gbs"] / hbm,
                "traffic": stored_traffic(kern, args.workload), "kernel": kern, "peak_source": src}
    else:
        roof = {"bound": "alu", "achieved": best["tflops"], "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": best["tflops"] / FP64_PEAK_TFLOPS, "traffic": stored_traffic(kern, args.workload),
                "kernel": kern, "peak_source": "nominal FP64 of GB300 (profiling recipe)", "gbs": best["gbs"]}
    line = {"metric": "H_W stencil algorithmic GB/s", "value": best["gbs"], "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["us"] / 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "lattice": "x".join(map(str, dims)), "rhs": nrhs,
                       "l2": "256 MiB buffer written between launches",
                       "bytes": "links once per launch (72 reals/site when all 9 elements are read, "
                                "48 for 12-real links; duplicated lanes and padding not counted) + "
                                "48 reals/site per RHS in and out"},
            "clocks": clocks, "roofline": roof, "variants": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_sigma(args, wl):
    """sigma = |s's - b'b| / b'b and device time per source apply versus the nodes per
    contour, with the paper's contour form (alpha 0.1, rho 1.1999, centres +-1.2) scaled by
    the Lanczos bound of |lambda|; FP64 coefficient-space solve, tol 1e-13."""
    import torch

    from paper_2204_01583_gb300 import build as build_lib

    build_lib()
    from paper_2204_01583_gb300 import lib

    dims = wl["dims"]
    U, b = workload_inputs(wl, 0)
    ctx = lib.Context(dims, bc_t=-1, m0=M0)
    ctx.set_gauge(torch.from_numpy(U).cuda())
    spec = ctx.place_contour(16, steps=150)
    scale = spec["abs_max_bound"] / 2.35
    bd = torch.from_numpy(b).cuda()
    out = torch.empty_like(bd)
    nsrc = b.shape[0]
    zolo = wl.get("rule") == "zolotarev"
    rows = []
    for n in wl["n_list"]:
        if zolo:
            zs = ctx.place_zolotarev(n, steps=150)
        else:
            ctx.set_contour_ellipse(n, 1.2 * scale, 1.1999 * scale, 0.1, lib.OV_CONTOUR_PAIR)
        o = ctx.opts(mode="fp64_2pass", tol=1e-13)
        for _ in range(args.warmup):
            ctx.sgn(bd, out, nsrc, o)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            st = ctx.sgn(bd, out, nsrc, o)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        s = out.reshape(nsrc, -1)
        bb = bd.reshape(nsrc, -1)
        sig = ((s.abs() ** 2).sum(1) - (bb.abs() ** 2).sum(1)).abs() / (bb.abs() ** 2).sum(1)
        row = {"nodes_per_contour": n, "total_nodes": 2 * n, "sigma_max": float(sig.max()),
               "sigma_mean": float(sig.mean()), "ms_per_apply": ms / nsrc, "iterations": st["iterations"]}
        if zolo:
            row = {"pole_pairs": n, "total_nodes": 2 * n, "predicted_error": zs["predicted_error"],
                   "interval": [zs["gap"], zs["abs_max_bound"]], **{k: row[k] for k in row if k not in
                                                                     ("nodes_per_contour", "total_nodes")}}
        rows.append(row)
    line = {"metric": "sigma vs N_q (" + ("Zolotarev node set" if zolo else "paper contour form") + ")",
            "value": rows[-1]["sigma_max"], "unit": "sigma",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "lattice": "x".join(map(str, dims)), "link_eps": wl["eps"],
                       "sources": nsrc,
                       "contour": ("Zolotarev on [Lanczos gap lowered by its residual bound, |lambda| bound]" if zolo
                                   else "alpha 0.1, rho 1.1999 s, centres +-1.2 s, s = bound/2.35"),
                       "scale": scale, "spectrum": spec},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_vjp(args, wl):
    """Gradients per second: ov_sgn_vjp (grad_b = S_N^dag eta and the su(3) link force of
    L = Re<eta, S_N b>) for one source, L2 flushed between timed evaluations."""
    import torch

    from paper_2204_01583_gb300 import build as build_lib

    build_lib()
    from paper_2204_01583_gb300 import lib
    import synthetic as S

    dims = wl["dims"]
    U = S.su3_links(dims, wl["eps"], S.seed_for("config4"))
    ctx = lib.Context(dims, bc_t=-1, m0=M0)
    ctx.set_gauge(torch.from_numpy(U).cuda())
    spec = ctx.place_contour(wl["n_q"], steps=150)
    b = torch.from_numpy(S.gaussian_spinor(dims, S.seed_for("config4.b"))).cuda()
    eta = torch.from_numpy(S.gaussian_spinor(dims, S.seed_for("config4.eta"))).cuda()
    gb = torch.empty_like(b)
    F = torch.empty((4,) + tuple(b.shape[:4]) + (8,), dtype=torch.float64, device="cuda")
    mode = args.mode or wl["mode"]
    o = ctx.opts(mode=mode, tol=wl["tol"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        ctx.sgn_vjp(eta, b, gb, F, o)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    ts, st = [], None
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = ctx.sgn_vjp(eta, b, gb, F, o)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    ctx.set_kernel_timing(True)
    ctx.sgn_vjp(eta, b, gb, F, o)
    torch.cuda.synchronize()
    kt = {k: {"launches": n, "ms": ms} for k, (n, ms) in ctx.kernel_times().items() if n}
    ctx.set_kernel_timing(False)
    ms = sum(ts) / len(ts)
    line = {"metric": "gradients/s of Re<eta, sgn(H_W) b> (b and link force)", "value": 1e3 / ms,
            "unit": "gradients/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[mode],
            "data": "synthetic",
            "config": {"workload": args.workload, "lattice": "x".join(map(str, dims)), "link_eps": wl["eps"],
                       "N_q": wl["n_q"], "tol": wl["tol"], "mode": mode,
                       "l2": "256 MiB buffer written between timed steps"},
            "clocks": clocks, "kernels_one_step": kt,
            "solver": {"iterations": st["iterations"], "converged": st["converged"], "spectrum": spec}}
    ctx.close()
    print(json.dumps(line), flush=True)
    return 0


def run_ovsolve(args, wl):
    """Overlap solves per second: x = D_ov(m_q)^-1 b for all sources in one call, L2 flushed
    between timed solves; the line carries the CG iteration count, the D applies and the
    true residual ||b - D x|| / ||b||."""
    import torch

    from paper_2204_01583_gb300 import build as build_lib

    build_lib()
    from paper_2204_01583_gb300 import lib

    dims = wl["dims"]
    U, b = workload_inputs(wl, 0)
    nsrc = b.shape[0]
    ctx = lib.Context(dims, bc_t=-1, m0=M0)
    ctx.set_gauge(torch.from_numpy(U).cuda())
    spec = ctx.place_contour(wl["n_q"], steps=150)
    bd = torch.from_numpy(b).cuda()
    x = torch.empty_like(bd)
    inner = ctx.opts(mode=wl["mode"], tol=wl["inner_tol"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        ctx.overlap_solve(wl["m_q"], bd, x, nsrc, inner, tol=wl["tol"])
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    ts, st = [], None
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = ctx.overlap_solve(wl["m_q"], bd, x, nsrc, inner, tol=wl["tol"])
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    ms = sum(ts) / len(ts)
    line = {"metric": "overlap solves/s (CG on D_ov^dag D_ov)", "value": nsrc / (ms / 1e3), "unit": "solves/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[wl["mode"]], "data": "synthetic",
            "config": {"workload": args.workload, "lattice": "x".join(map(str, dims)), "link_eps": wl["eps"],
                       "m_q": wl["m_q"], "N_q": wl["n_q"], "sources": nsrc, "tol": wl["tol"],
                       "inner": {"mode": wl["mode"], "tol": wl["inner_tol"]},
                       "l2": "256 MiB buffer written between timed solves"},
            "clocks": clocks,
            "solver": {"cg_iterations": st["iterations"], "overlap_applies": st["refine_rounds"],
                       "krylov_iterations": st["inner_iterations"], "true_residual": st["max_residual"],
                       "normal_residual": st["error_bound"], "converged": st["converged"], "spectrum": spec}}
    ctx.close()
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    if wl.get("kind") == "dslash":
        return run_dslash(args, wl)
    if wl.get("kind") == "vjp":
        return run_vjp(args, wl)
    if wl.get("kind") == "ovsolve":
        return run_ovsolve(args, wl)
    if wl.get("kind") == "sigma":
        return run_sigma(args, wl)
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
