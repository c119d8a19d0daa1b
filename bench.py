#!/usr/bin/env python3
"""Benchmark: DOF/s solved to a 1e-8 relative residual on the 128^3 workload.

A step is one pass of the whole method on one synthetic problem: amg_setup on
the device-resident graph (validation, matching, Galerkin, smoother data,
coarsest pseudo-inverse) followed by amg_solve (flexible CG + K-cycle with the
polynomial smoother) to ||r|| <= 1e-8 ||b||, then amg_free.  value = DOF of
all ranks per step / step time; solve_dof_per_s divides by the solve phase
alone (setup timed and reported beside it).  Workload: 3D 7-point graph
Laplacian on a 128^3 grid (2,097,152 vertices, unit weights, d_i = 1 on
boundary-face vertices), degree-5 smoother, three matching passes per level,
nu = 2 inner flexible-CG steps, seeded uniform[-1,1] right-hand side.

The default run also reports, under "variants", the other configurations of
the measurement plan, each with its own bounded oracle sample: the fp32
preconditioner on the same workload, the 64^2 case (us per solve), the
2048^2 random-diagonal case (fp64 and fp32 preconditioner, error against the
oracle), the 96^3 x 32 batched case and the serving run (solves/s, p50/p99).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--variants all|none|fp32,c1,c3,c4,c5] [--workload NAME]

Multi-GPU runs (torchrun) solve independent replicas, one per rank (weak
scaling, no data-path collective); the reference arm runs the CPU oracle.
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
import traceback

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

WORKLOADS = {
    "grid3d_128": ("128^3 7-point graph Laplacian, w=1, d=1 on boundary faces; degree-5 polynomial "
                   "smoother, 3 matching passes/level, K-cycle nu=2, FCG restart 5, tol 1e-8 (fp64)"),
    "grid2d_64": ("64^2 5-point pure graph Laplacian; degree-3 smoother, 2 matching passes/level, K-cycle nu=2, "
                  "coarsest <= 64 vertices, tol 1e-8 (fp64)"),
    "rdiag2d_2048": ("2048^2 grid, each square split along a seeded random diagonal (4,194,304 vertices), pure "
                     "Laplacian; degree-4 smoother, 3 passes/level, K-cycle nu=2, tol 1e-8"),
    "grid3d_128_neumann_mis": ("128^3 7-point pure (Neumann) graph Laplacian; degree-4 polynomial smoother, "
                               "aggregation by the maximal independent set of the graph of A^4 (one pass per "
                               "level), K-cycle nu=2, FCG restart 5, tol 1e-8 (fp64): the setting of the paper's "
                               "Table (matrix and right-hand side synthetic)"),
    "delaunay3d_64_mis": ("64^3-vertex unstructured tetrahedral mesh of the unit cube (grid vertices moved by "
                          "random vectors of length h/2, then Delaunay), pure Laplacian of the mesh graph; "
                          "degree-4 smoother, aggregation by the maximal independent set of the graph of A^4, "
                          "K-cycle nu=2, tol 1e-8 (fp64): the paper's unstructured setting (synthetic mesh)"),
    "grid3d_96x32": ("96^3 7-point graph Laplacian, d=1 on boundary faces, 32 right-hand sides solved in one "
                     "batched call; degree-5 smoother, 3 passes/level, fp32 preconditioner / fp64 FCG, tol 1e-8"),
    "serve": ("continuous-batching server: Poisson arrivals of solve requests over a pool of 48 graphs (half "
              "random geometric graphs in the unit square with mean degree 8, a quarter each 2D/3D grids), sizes "
              "log-uniform in [1e4, 1e6], hierarchies set up on first arrival and kept resident, same-graph "
              "requests batched (up to 8 per solve), 8 slots, 60 GB cap; degree-4 smoother, 3 passes, fp32 "
              "preconditioner / fp64 FCG, tol 1e-8"),
}

METRIC = "DOF/s solved to 1e-8 rel. residual (setup + solve per step)"
UNIT = "DOF/s"
L2_BYTES = 129 * 2 ** 20
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
PROFILE = os.path.join(ROOT, "profiles", "cheb_step_grid3d_128.txt")
VARIANTS = ("fp32", "c1", "c3", "c4", "c5")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time: every rank solves its own replica (no
    data-path collective), the job is as fast as its slowest rank."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed per second of the
    slowest rank (weak scaling: each rank has the same workload)."""
    return units_per_rank * world / (ms / 1e3)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash() -> str:
    src = open(os.path.join(ROOT, "paper_1307_6305_gb300", "csrc", "sell_kernels.cuh"), "rb").read()
    return hashlib.sha256(src).hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the fused smoother step from the committed ncu
    summary, if it was taken on the current kernel source."""
    if not os.path.exists(PROFILE):
        return None
    kv = {}
    for line in open(PROFILE):
        if ":" in line and not line.startswith(" "):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def workload_config(name: str, g, nrhs: int, world: int, cycle: int = 0) -> dict:
    """The `config` object of the JSON line; both arms print the same one."""
    in_bytes = g.rowptr.nbytes + g.col.nbytes + g.w.nbytes + (0 if g.d is None else g.d.nbytes) + 8 * g.n * nrhs
    return {"workload": WORKLOADS[name] + ("" if cycle == 0 else "; stationary AMLI W-cycle instead of the K-cycle"),
            "n": int(g.n), "nrhs": int(nrhs), "nnz_offdiag": int(g.nnz),
            "l2": f"inputs {in_bytes / 2**20:.0f} MiB vs 129 MiB L2 (no flush)",
            "parallelism": f"replicas x{world}"}


class ClockSampler:
    """nvidia-smi clock/throttle sampling in the background during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_oracle_step(g, p, b, ncols=None, cycle=0, want_x=False):
    """Oracle setup + solve of the first `ncols` right-hand sides (all by default)."""
    import oracle

    nr = b.size // g.n
    ncols = nr if ncols is None else min(ncols, nr)
    t0 = time.perf_counter()
    h = oracle.Hierarchy(g, degree=p["degree"], passes=p["passes"], cycle=cycle,
                         aggregation=p.get("aggregation", 0))
    r = None
    for j in range(ncols):
        r = h.solve(b[j * g.n:(j + 1) * g.n], tol=1e-8)
        assert r.status == 0, r.status
    dt = time.perf_counter() - t0
    assert h.status == 0
    return dt, r, ncols


def guarded(name, fn):
    """Run one variant; a failure is reported in its entry, not raised."""
    t0 = time.perf_counter()
    try:
        out = fn()
    except Exception as e:  # noqa: BLE001 -- reported in the JSON line
        out = {"error": f"{type(e).__name__}: {e}", "trace": traceback.format_exc(limit=3)[-600:]}
    out["wall_s"] = round(time.perf_counter() - t0, 2)
    return out


# ---------------------------------------------------------------------------
# GPU helpers (imported lazily: the reference arm needs no torch.cuda)
# ---------------------------------------------------------------------------
class Problem:
    """A workload resident on the device, with pinned host copies for e2e."""

    def __init__(self, name, dev):
        import torch

        self.name = name
        self.g, self.p = gg.workload(name)
        g = self.g
        self.nrhs = len(self.p["rhs_seeds"])
        self.b = np.concatenate([gg.rhs(g.n, sd, gg.is_pure_laplacian(g)) for sd in self.p["rhs_seeds"]])
        self.rp = torch.as_tensor(g.rowptr, device=dev)
        self.col = torch.as_tensor(g.col, device=dev)
        self.w = torch.as_tensor(g.w, device=dev)
        self.d = None if g.d is None else torch.as_tensor(g.d, device=dev)
        self.bd = torch.as_tensor(self.b, device=dev)
        self.xd = torch.zeros_like(self.bd)


def make_opts(amg, p, precision, cycle=0):
    return amg.amg_default_options(degree=p["degree"], passes=p["passes"], precision=precision, cycle=cycle,
                                   aggregation=p.get("aggregation", 0))


def timed_steps(amg, P, opts, sp, stream, steps, warmup):
    """`warmup` untimed then `steps` timed steps (setup + solve + free) on the
    device-resident problem.  CUDA events on the library's stream bracket the
    steps and split each step into setup and solve."""
    import torch

    def one(evs=None):
        if evs:
            evs[0].record(stream)
        st, h = amg.amg_setup(P.g.n, P.rp, P.col, P.w, P.d, opts, amg.AMG_MEM_DEVICE, sp)
        assert st == 0, amg.amg_last_error(None)
        launches = amg.lib().amg_launch_count(h)
        if evs:
            evs[1].record(stream)
        info = amg.amg_info()
        st = amg.amg_solve(h, P.bd, P.xd, P.nrhs, P.g.n, 1e-8, info)
        assert st == 0, amg.amg_last_error(h)
        if evs:
            evs[2].record(stream)
        launches += amg.lib().amg_launch_count(h)
        amg.amg_free(h)
        return launches, info

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    marks = [[ev(), ev(), ev()] for _ in range(steps)]
    e0, e1 = ev(), ev()
    e0.record(stream)
    launches, infos = 0, []
    for k in range(steps):
        nl, info = one(marks[k])
        launches += nl
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    total = e0.elapsed_time(e1)
    setup = [m[0].elapsed_time(m[1]) for m in marks]
    solve = [m[1].elapsed_time(m[2]) for m in marks]
    return {"ms_per_step": total / steps, "setup_ms": statistics.median(setup),
            "solve_ms": statistics.median(solve), "launches": launches, "iterations": infos[-1].iterations,
            "n_levels": infos[-1].n_levels, "true_rel_residual": infos[-1].true_rel_residual}


def kernel_roofline(amg, P, opts, sp, precision, steps=2):
    """The dominant kernel (the level-0 fused smoother step) timed live with
    CUDA events in a separate pass, so that the headline's steps carry no
    timing nodes."""
    import ctypes as C

    acc = {kind: [0, 0.0, 0.0] for kind in (0, 1, 2)}   # launches, ms, bytes per launch
    for _ in range(steps):
        st, h = amg.amg_setup(P.g.n, P.rp, P.col, P.w, P.d, opts, amg.AMG_MEM_DEVICE, sp)
        assert st == 0, amg.amg_last_error(None)
        amg.lib().amg_kernel_timing(h, 1)
        assert amg.amg_solve(h, P.bd, P.xd, P.nrhs, P.g.n, 1e-8, None) == 0
        for kind in acc:
            nl, ms, b = C.c_int64(), C.c_double(), C.c_double()
            amg.lib().amg_kernel_timing_read_kind(h, kind, C.byref(nl), C.byref(ms), C.byref(b))
            acc[kind][0] += nl.value
            acc[kind][1] += ms.value
            acc[kind][2] = b.value
        amg.amg_free(h)
    nl_tot, ms_tot, bpl = acc[0]
    if nl_tot == 0:
        return None
    avg_ms = ms_tot / nl_tot
    gbs = bpl / (avg_ms * 1e-3) / 1e9
    # one step T_{j+1} = S T_j - T_{j-1}, x += c_j T_{j+1} with the smoother
    # form S = 2 t(A): 2 flops per stored off-diagonal, the diagonal product,
    # one subtraction and one FMA per row
    flops = 2.0 * P.g.nnz + 4.0 * P.g.n
    tflops = flops / (avg_ms * 1e-3) / 1e12
    hbm_peak, peak_kind = peaks()
    f64 = precision == 0
    kname = "k_cheb_step<%s> (level 0: SELL-32 SpMV + Chebyshev recurrence step)" % ("double" if f64 else "float")
    hbm_view = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy)"}
    alu_view = {"achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": tflops / FP64_PEAK_TFLOPS,
                "peak_kind": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (an FMA probe measured 1.198)"}
    traffic = profiled_traffic() if f64 else None
    if f64 and alu_view["frac"] > hbm_view["frac"]:
        roof = dict(bound="alu", traffic=traffic, hbm_view=hbm_view, **alu_view)
    else:
        roof = dict(bound="hbm", traffic=traffic, **hbm_view)
        if f64:
            roof["alu_view"] = alu_view
    roof.update({"kernel": kname, "launches_timed": nl_tot, "avg_launch_us": avg_ms * 1e3,
                 "algorithmic_bytes_per_launch": bpl, "algorithmic_flops_per_launch": flops})
    # the level-0 transfer kernels, timed in the same pass
    tr = {}
    for kind, name in ((1, "restriction r_H = P^T s (level 0)"), (2, "prolongation x = u + P e_H (level 0)")):
        nl, ms, b = acc[kind]
        if nl:
            us = ms / nl * 1e3
            gb = b / (us * 1e-6) / 1e9
            tr["restrict" if kind == 1 else "prolong"] = {
                "kernel": name, "launches_timed": nl, "avg_launch_us": us, "algorithmic_bytes_per_launch": b,
                "achieved": gb, "peak": hbm_peak, "unit": "GB/s", "frac": gb / hbm_peak}
    roof["transfers"] = tr or None
    return roof


# ---------------------------------------------------------------------------
# variants
# ---------------------------------------------------------------------------
def variant_fp32(amg, P, sp, stream, args, world, dev, cycle):
    opts32 = make_opts(amg, P.p, amg.AMG_PREC_FP32, cycle)
    r = timed_steps(amg, P, opts32, sp, stream, args.steps, args.warmup)
    ms = max_over_ranks(r["ms_per_step"], world, dev)
    return {"value": job_value(P.g.n * P.nrhs, world, ms), "unit": UNIT, "ms_per_step": ms,
            "solve_dof_per_s": P.g.n * P.nrhs / (r["solve_ms"] * 1e-3), "setup_ms": r["setup_ms"],
            "solve_ms": r["solve_ms"], "iterations": r["iterations"],
            "roofline": kernel_roofline(amg, P, opts32, sp, 1),
            "dtype": "f32 preconditioner / f64 outer CG, dots and coarsest solve"}


def variant_c1(amg, dev, sp, stream):
    """64^2 pure Laplacian: latency-bound, reported as us per solve."""
    import torch

    P = Problem("grid2d_64", dev)
    opts = make_opts(amg, P.p, amg.AMG_PREC_FP64)
    setups = []
    for _ in range(8):
        t0 = time.perf_counter()
        st, h = amg.amg_setup(P.g.n, P.rp, P.col, P.w, P.d, opts, amg.AMG_MEM_DEVICE, sp)
        setups.append((time.perf_counter() - t0) * 1e3)
        assert st == 0
        if _ < 7:
            amg.amg_free(h)
    info = amg.amg_info()
    for _ in range(5):
        assert amg.amg_solve(h, P.bd, P.xd, 1, P.g.n, 1e-8, info) == 0
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 50
    e0.record(stream)
    for _ in range(reps):
        amg.amg_solve(h, P.bd, P.xd, 1, P.g.n, 1e-8, info)
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / reps
    amg.amg_free(h)
    dt, ref, _ = run_oracle_step(P.g, P.p, P.b)
    return {"workload": WORKLOADS["grid2d_64"], "n": P.g.n, "us_per_solve": us,
            "solve_dof_per_s": P.g.n / (us * 1e-6), "setup_ms_host": statistics.median(setups[2:]),
            "iterations": info.iterations, "oracle_iterations": ref.iterations,
            "cpu_baseline": {"value": P.g.n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"oracle setup + solve in full, {dt * 1e3:.1f} ms single thread"}}


def variant_c3(amg, dev, sp, stream):
    """2048^2 random diagonals: fp64 GPU, fp32-preconditioner GPU, both against
    the fp64 oracle (final error and iterations)."""
    import torch

    P = Problem("rdiag2d_2048", dev)
    out = {"workload": WORKLOADS["rdiag2d_2048"], "n": P.g.n}
    xs = {}
    for prec, key in ((amg.AMG_PREC_FP64, "fp64"), (amg.AMG_PREC_FP32, "fp32_precond")):
        opts = make_opts(amg, P.p, prec)
        r = timed_steps(amg, P, opts, sp, stream, 3, 1)
        xs[key] = P.xd.cpu().numpy().copy()
        out[key] = {"value": P.g.n / (r["ms_per_step"] * 1e-3), "unit": UNIT, "ms_per_step": r["ms_per_step"],
                    "solve_dof_per_s": P.g.n / (r["solve_ms"] * 1e-3), "setup_ms": r["setup_ms"],
                    "solve_ms": r["solve_ms"], "iterations": r["iterations"],
                    "true_rel_residual": r["true_rel_residual"]}
    dt, ref, _ = run_oracle_step(P.g, P.p, P.b)
    nx = np.linalg.norm(ref.x)
    for key, x in xs.items():
        out[key]["rel_error_vs_oracle"] = float(np.linalg.norm(x - ref.x) / nx)
    out["oracle_iterations"] = ref.iterations
    out["cpu_baseline"] = {"value": P.g.n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                           "sample": f"oracle setup + solve in full ({ref.iterations} iterations), "
                                     f"{dt:.1f} s single thread"}
    del P
    torch.cuda.empty_cache()
    return out


def variant_c4(amg, dev, sp, stream):
    """96^3 x 32 right-hand sides in one batched call, fp32 preconditioner."""
    import torch

    P = Problem("grid3d_96x32", dev)
    opts = make_opts(amg, P.p, amg.AMG_PREC_FP32)
    r = timed_steps(amg, P, opts, sp, stream, 3, 2)
    units = P.g.n * P.nrhs
    dt, ref, nc = run_oracle_step(P.g, P.p, P.b, 2)
    out = {"workload": WORKLOADS["grid3d_96x32"], "n": P.g.n, "nrhs": P.nrhs,
           "value": units / (r["ms_per_step"] * 1e-3), "unit": UNIT, "ms_per_step": r["ms_per_step"],
           "solve_dof_per_s": units / (r["solve_ms"] * 1e-3), "setup_ms": r["setup_ms"], "solve_ms": r["solve_ms"],
           "iterations": r["iterations"], "oracle_iterations_col0": ref.iterations,
           "dtype": "f32 preconditioner / f64 outer CG",
           "cpu_baseline": {"value": P.g.n * nc / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"oracle setup + {nc} of {P.nrhs} right-hand sides, {dt:.1f} s single thread"}}
    del P
    torch.cuda.empty_cache()
    return out


def _build_serve_graph(spec):
    return gg.serve_graph(spec)


def serve_graphs(count):
    """The serving pool, built by a process pool of the host's cores (spawned,
    so that it is safe after CUDA initialisation)."""
    import multiprocessing as mp

    specs = gg.serve_graph_specs(count)
    workers = max(1, min(8, (os.cpu_count() or 2) - 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        return list(pool.map(_build_serve_graph, specs, chunksize=1))


def serve_bench(count_graphs=48, main_requests=2000, low_requests=600, oracle_requests=50):
    """Solves/s and p50/p99 latency of the server under Poisson arrivals at
    1.2x and 0.5x of its saturated throughput.  The main run starts cold: each
    graph's hierarchy is set up when its first request arrives, under load."""
    import paper_1307_6305_gb300 as amg

    graphs = serve_graphs(count_graphs)
    rng = np.random.default_rng(5)

    def new_server():
        srv = amg.Server(60 << 30, 8, batch_max=8, degree=4, passes=3, precision=amg.AMG_PREC_FP32)
        return srv, [srv.add_graph(g) for g in graphs]

    seed = [7000]

    def pick():
        gi = int(rng.integers(len(graphs)))
        seed[0] += 1
        return gi, gg.rhs(graphs[gi].n, seed[0], True)

    # saturated throughput, cold: everything queued at once
    srv, ids = new_server()
    burst = [pick() for _ in range(256)]
    t0 = time.perf_counter()
    tickets = [srv.submit(ids[gi], b) for gi, b in burst]
    for t in tickets:
        assert srv.wait(t)[0] == 0
    sat = len(burst) / (time.perf_counter() - t0)
    srv.close()
    srv, ids = new_server()
    runs, stream_main = [], None
    for load, count in ((1.2, main_requests), (0.5, low_requests)):
        before = srv.stats()
        rate = load * sat
        arrivals = np.cumsum(rng.exponential(1.0 / rate, count))
        reqs = [pick() for _ in range(count)]
        if stream_main is None:
            stream_main = reqs
        tickets = []
        t0 = time.perf_counter()
        for (gi, b), ta in zip(reqs, arrivals):
            delay = ta - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(ids[gi], b))
        lat, iters = [], []
        for t in tickets:
            st, x, info, ms = srv.wait(t)
            assert st == 0
            lat.append(ms)
            iters.append(info.iterations)
        wall = time.perf_counter() - t0
        after = srv.stats()
        solves = after.solves - before.solves
        runs.append({"offered_load": load, "offered_rate_per_s": rate, "requests": count,
                     "solves_per_s": count / wall, "p50_ms": float(np.percentile(lat, 50)),
                     "p99_ms": float(np.percentile(lat, 99)), "mean_iterations": float(np.mean(iters)),
                     "setups": int(after.setups - before.setups),
                     "mean_batch": count / max(solves, 1), "peak_active": int(after.peak_active)})
    stats = srv.stats()
    srv.close()
    # oracle on the first requests of the main stream: each graph set up once
    # (as the server keeps hierarchies resident), every request solved
    import oracle

    sub = stream_main[:oracle_requests]
    t0 = time.perf_counter()
    orc_h = {}
    for gi, b in sub:
        if gi not in orc_h:
            orc_h[gi] = oracle.Hierarchy(graphs[gi], degree=4, passes=3)
        assert orc_h[gi].solve(b, tol=1e-8).status == 0
    dt = time.perf_counter() - t0
    main = runs[0]
    return {"metric": "solves/s under Poisson arrivals at 1.2x saturated throughput (p50/p99 latency)",
            "value": main["solves_per_s"], "unit": "solves/s", "saturated_solves_per_s": sat,
            "latency_ms": {"p50": main["p50_ms"], "p99": main["p99_ms"]}, "runs": runs,
            "graphs": [int(g.n) for g in graphs],
            "server": {"setups": int(stats.setups), "solves": int(stats.solves), "completed": int(stats.completed),
                       "evictions": int(stats.evictions), "setup_retries": int(stats.setup_retries),
                       "peak_active": int(stats.peak_active),
                       "peak_resident_gb": stats.peak_resident_bytes / 2 ** 30},
            "cpu_baseline": {"value": len(sub) / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"the first {len(sub)} requests of the 1.2x stream, {len(orc_h)} graphs set "
                                       f"up once each, {dt:.1f} s single thread"}}


# ---------------------------------------------------------------------------
def reference_arm(args, name, cycle):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    g, p = gg.workload(name)
    nrhs = len(p["rhs_seeds"])
    b = np.concatenate([gg.rhs(g.n, sd, gg.is_pure_laplacian(g)) for sd in p["rhs_seeds"]])
    ncols = 1 if nrhs == 1 else 2          # bounded sample: two of the 32 columns
    for _ in range(args.warmup):
        run_oracle_step(g, p, b, ncols, cycle)
    times = [run_oracle_step(g, p, b, ncols, cycle)[0] for _ in range(args.steps)]
    ms = 1e3 * sum(times) / len(times)
    value = g.n * ncols / (ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(name, g, nrhs, world, cycle),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"oracle setup + {ncols} of {nrhs} right-hand sides per step, single thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-variant", action="store_true", help="same as --variants none")
    ap.add_argument("--variants", default="all", help="all, none, or a comma list of " + ",".join(VARIANTS))
    ap.add_argument("--workload", default="grid3d_128", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="fp32: the whole preconditioner in fp32 inside the fp64 outer CG")
    ap.add_argument("--cycle", default="k", choices=["k", "amli"],
                    help="k: nonlinear AMLI cycle (K-cycle, default); amli: stationary AMLI W-cycle")
    args = ap.parse_args()
    CYCLE = 1 if args.cycle == "amli" else 0
    rank, world, local = dist_env()
    if args.workload == "serve":
        if args.impl != "ours" or rank != 0:
            return 0
        import torch

        torch.cuda.set_device(0)
        r = serve_bench()
        r.update({"n_gpus": 1, "steps": r["runs"][0]["requests"], "warmup": 256,
                  "ms_per_step": 1e3 / r["value"], "higher_is_better": True, "scaling": "weak",
                  "vs_baseline": None, "dtype": "f32 preconditioner / f64 outer", "data": "synthetic",
                  "config": {"workload": WORKLOADS["serve"]}})
        print(json.dumps(r), flush=True)
        return 0
    if args.impl == "reference":
        return reference_arm(args, args.workload, CYCLE)

    import torch

    import paper_1307_6305_gb300 as amg

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    P = Problem(args.workload, dev)
    g, nrhs = P.g, P.nrhs
    if nrhs > 1:
        args.precision = "fp32" if P.p["precision"] else args.precision
    prec = amg.AMG_PREC_FP32 if args.precision == "fp32" else amg.AMG_PREC_FP64
    opts = make_opts(amg, P.p, prec, CYCLE)

    # ---- headline: setup + solve steps, nothing else on the stream ----
    for _ in range(args.warmup):
        timed_steps(amg, P, opts, sp, stream, 1, 0)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    head = timed_steps(amg, P, opts, sp, stream, args.steps, 0)
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    ms = max_over_ranks(head["ms_per_step"], world, dev)
    solve_ms = max_over_ranks(head["solve_ms"], world, dev)
    value = job_value(g.n * nrhs, world, ms)

    # ---- the dominant kernel, timed in its own pass ----
    roof = kernel_roofline(amg, P, opts, sp, prec) if nrhs == 1 else None

    # ---- end to end through the C ABI with pinned host buffers (H2D + D2H inside) ----
    e2e_steps = 0 if args.no_e2e else args.steps
    pin = lambda a: torch.as_tensor(a).pin_memory()
    hrp, hcol, hw = pin(g.rowptr), pin(g.col), pin(g.w)
    hd = None if g.d is None else pin(g.d)
    hb = pin(P.b)
    hx = torch.zeros_like(hb).pin_memory()
    in_bytes = g.rowptr.nbytes + g.col.nbytes + g.w.nbytes + (0 if g.d is None else g.d.nbytes) + P.b.nbytes
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        st, h = amg.amg_setup(g.n, hrp, hcol, hw, hd, opts, amg.AMG_MEM_HOST, sp)
        assert st == 0
        st = amg.amg_solve(h, hb, hx, nrhs, g.n, 1e-8, None)
        assert st == 0
        amg.amg_free(h)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / max(e2e_steps, 1) if e2e_steps else float("nan")
    e2e_ms = max_over_ranks(e2e_ms, world, dev)

    # ---- the other configurations (rank 0 of a single-GPU run only) ----
    want = set() if args.no_variant or args.variants == "none" else (
        set(VARIANTS) if args.variants == "all" else set(args.variants.split(",")))
    variants = {}
    if "fp32" in want and args.precision == "fp64" and nrhs == 1:
        variants["fp32_precond"] = guarded("fp32", lambda: variant_fp32(amg, P, sp, stream, args, world, dev, CYCLE))
    if world == 1 and args.workload == "grid3d_128" and CYCLE == 0:
        if "c1" in want:
            variants["c1_grid2d_64"] = guarded("c1", lambda: variant_c1(amg, dev, sp, stream))
        if "c3" in want:
            variants["c3_rdiag2d_2048"] = guarded("c3", lambda: variant_c3(amg, dev, sp, stream))
        if "c4" in want:
            variants["c4_grid3d_96x32"] = guarded("c4", lambda: variant_c4(amg, dev, sp, stream))
        if "c5" in want:
            variants["c5_serve"] = guarded("c5", serve_bench)
    if world > 1:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return 0

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        dt, r, nc = run_oracle_step(g, P.p, P.b, 1 if nrhs == 1 else 2, CYCLE)
        cpu = {"value": g.n * nc / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle setup + {nc} of {nrhs} right-hand sides ({r.iterations} iterations), "
                         f"{dt:.1f} s single thread"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32 preconditioner / f64 outer",
        "data": "synthetic", "config": workload_config(args.workload, g, nrhs, world, CYCLE),
        "solve_dof_per_s": job_value(g.n * nrhs, world, solve_ms),
        "iterations": head["iterations"], "n_levels": head["n_levels"],
        "setup_ms": head["setup_ms"], "solve_ms": head["solve_ms"],
        "e2e": {"value": job_value(g.n * nrhs, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": in_bytes,
                "d2h_bytes_per_step": P.b.nbytes, "ms_per_step": e2e_ms},
        "gpu_launches": head["launches"], "roofline": roof, "cpu_baseline": cpu, "clocks": ck,
        "variants": variants or None,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
