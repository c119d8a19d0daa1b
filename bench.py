#!/usr/bin/env python3
"""Benchmark: DOF/s solved to a 1e-8 relative residual on the 128^3 workload.

A step is one pass of the whole method on one synthetic problem: amg_setup on
the device-resident graph (validation, matching, Galerkin, smoother data,
coarsest pseudo-inverse) followed by amg_solve (flexible CG + K-cycle with the
polynomial smoother) to ||r|| <= 1e-8 ||b||, then amg_free.  value = DOF of
all ranks per step / step time.  Workload: 3D 7-point graph Laplacian on a
128^3 grid (2,097,152 vertices, unit weights, d_i = 1 on boundary-face
vertices), degree-5 smoother, three matching passes per level, nu = 2 inner
flexible-CG steps, seeded uniform[-1,1] right-hand side.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

WORKLOADS = {
    "grid3d_128": ("128^3 7-point graph Laplacian, w=1, d=1 on boundary faces; degree-5 polynomial "
                   "smoother, 3 matching passes/level, K-cycle nu=2, FCG restart 5, tol 1e-8 (fp64)"),
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
    "serve": ("continuous-batching server: pool of 16 graphs (8 random geometric, 4 2D and 4 3D grids), sizes "
              "log-uniform in [1e4, 1e6], resident hierarchies, 8 slots, 60 GB cap, Poisson arrivals; "
              "degree-4 smoother, 3 passes, fp32 preconditioner / fp64 FCG, tol 1e-8"),
}


def serve_bench(args):
    """Solves/s and p50/p99 latency of the server under Poisson arrivals at
    1.2x and 0.5x of its saturated throughput."""
    import torch

    import paper_1307_6305_gb300 as amg

    torch.cuda.set_device(0)
    rng = np.random.default_rng(5)
    sizes = np.exp(rng.uniform(np.log(1e4), np.log(1e6), 16))
    graphs = []
    for i, sz in enumerate(sizes):
        if i < 8:
            graphs.append(gg.random_geometric(int(sz), 500 + i))
        elif i < 12:
            graphs.append(gg.grid2d_5pt(int(round(np.sqrt(sz)))))
        else:
            graphs.append(gg.grid3d_7pt(int(round(sz ** (1.0 / 3.0))), None))
    rhs = [[gg.rhs(g.n, 7000 + 10 * gi + j, True) for j in range(4)] for gi, g in enumerate(graphs)]
    srv = amg.Server(60 << 30, 8, degree=4, passes=3, precision=amg.AMG_PREC_FP32)
    ids = [srv.add_graph(g) for g in graphs]
    for gi in range(len(graphs)):                      # hierarchies become resident
        st, _, _, _ = srv.wait(srv.submit(ids[gi], rhs[gi][0]))
        assert st == 0
    def pick():
        gi = int(rng.integers(len(graphs)))
        return gi, rhs[gi][int(rng.integers(4))]
    # saturated throughput: everything queued at once
    burst = [pick() for _ in range(256)]
    t0 = time.perf_counter()
    tickets = [srv.submit(ids[gi], b) for gi, b in burst]
    for t in tickets:
        assert srv.wait(t)[0] == 0
    sat = len(burst) / (time.perf_counter() - t0)
    runs = []
    for load, count in ((1.2, 2000), (0.5, 600)):
        rate = load * sat
        arrivals = np.cumsum(rng.exponential(1.0 / rate, count))
        reqs = [pick() for _ in range(count)]
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
        runs.append({"offered_load": load, "requests": count, "solves_per_s": count / wall,
                     "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "mean_iterations": float(np.mean(iters))})
    stats = srv.stats()
    srv.close()
    main = runs[0]
    line = {"metric": "solves/s under Poisson arrivals at 1.2x saturated throughput (p50/p99 latency)",
            "value": main["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": main["requests"],
            "warmup": len(graphs), "ms_per_step": 1e3 / main["solves_per_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 preconditioner / f64 outer", "data": "synthetic",
            "config": {"workload": WORKLOADS["serve"], "graphs": [int(g.n) for g in graphs]},
            "saturated_solves_per_s": sat, "latency_ms": {"p50": main["p50_ms"], "p99": main["p99_ms"]},
            "runs": runs, "server": {"peak_active": stats.peak_active, "setups": int(stats.setups),
                                      "evictions": int(stats.evictions),
                                      "peak_resident_gb": stats.peak_resident_bytes / 2 ** 30}}
    print(json.dumps(line), flush=True)
    return 0


METRIC = "DOF/s solved to 1e-8 rel. residual (setup + solve per step)"
UNIT = "DOF/s"
L2_BYTES = 129 * 2 ** 20
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
PROFILE = os.path.join(ROOT, "profiles", "cheb_step_grid3d_128.txt")


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


def run_oracle_step(g, p, b, ncols=None, cycle=0):
    """Oracle setup + solve of the first `ncols` right-hand sides (all by default)."""
    import oracle

    nr = b.size // g.n
    ncols = nr if ncols is None else min(ncols, nr)
    t0 = time.perf_counter()
    h = oracle.Hierarchy(g, degree=p["degree"], passes=p["passes"], cycle=cycle,
                         aggregation=p.get("aggregation", 0))
    for j in range(ncols):
        r = h.solve(b[j * g.n:(j + 1) * g.n], tol=1e-8)
        assert r.status == 0, r.status
    dt = time.perf_counter() - t0
    assert h.status == 0
    return dt, r, ncols


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-variant", action="store_true", help="skip the fp32-preconditioner variant")
    ap.add_argument("--workload", default="grid3d_128", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="fp32: the whole preconditioner in fp32 inside the fp64 outer CG")
    ap.add_argument("--cycle", default="k", choices=["k", "amli"],
                    help="k: nonlinear AMLI cycle (K-cycle, default); amli: stationary AMLI W-cycle")
    args = ap.parse_args()
    CYCLE = 1 if args.cycle == "amli" else 0
    rank, world, local = dist_env()
    if args.workload == "serve":
        return serve_bench(args) if args.impl == "ours" and rank == 0 else 0
    WORKLOAD, WORKLOAD_DESC = args.workload, WORKLOADS[args.workload]
    g, p = gg.workload(WORKLOAD)
    nrhs = len(p["rhs_seeds"])
    if nrhs > 1:
        args.precision = "fp32" if p["precision"] else args.precision
    b = np.concatenate([gg.rhs(g.n, sd, gg.is_pure_laplacian(g)) for sd in p["rhs_seeds"]])

    if args.impl == "reference":
        if rank != 0:
            return 0
        ncols = 1 if nrhs == 1 else 2          # bounded sample: two of the 32 columns
        for _ in range(args.warmup):
            run_oracle_step(g, p, b, ncols, CYCLE)
        times = [run_oracle_step(g, p, b, ncols, CYCLE)[0] for _ in range(args.steps)]
        ms = 1e3 * sum(times) / len(times)
        value = g.n * ncols / (ms / 1e3)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": WORKLOAD_DESC + ("" if CYCLE == 0 else "; stationary AMLI W-cycle"),
                           "n": g.n, "nrhs": nrhs},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"oracle setup + {ncols} of {nrhs} right-hand sides per step, single thread"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import torch

    import paper_1307_6305_gb300 as amg

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    rp = torch.as_tensor(g.rowptr, device=dev)
    col = torch.as_tensor(g.col, device=dev)
    w = torch.as_tensor(g.w, device=dev)
    d = None if g.d is None else torch.as_tensor(g.d, device=dev)
    bd = torch.as_tensor(b, device=dev)          # column j at bd[j*n:(j+1)*n]
    xd = torch.zeros_like(bd)
    in_bytes = g.rowptr.nbytes + g.col.nbytes + g.w.nbytes + (0 if g.d is None else g.d.nbytes) + b.nbytes
    prec = amg.AMG_PREC_FP32 if args.precision == "fp32" else amg.AMG_PREC_FP64
    opts = amg.amg_default_options(degree=p["degree"], passes=p["passes"], precision=prec, cycle=CYCLE,
                                   aggregation=p.get("aggregation", 0))
    state = {"launches": 0, "iters": [], "setup_ms": [], "solve_ms": [], "kt": [0, 0.0, 0.0]}

    def step(timed_kernel: bool):
        st, h = amg.amg_setup(g.n, rp, col, w, d, opts, amg.AMG_MEM_DEVICE, sp)
        assert st == 0, amg.amg_last_error(None)
        launches = amg.lib().amg_launch_count(h)
        if timed_kernel:
            amg.lib().amg_kernel_timing(h, 1)
        info = amg.amg_info()
        st = amg.amg_solve(h, bd, xd, nrhs, g.n, 1e-8, info)
        assert st == 0, amg.amg_last_error(h)
        launches += amg.lib().amg_launch_count(h)
        if timed_kernel:
            import ctypes as C

            nl, ms, bpl = C.c_int64(), C.c_double(), C.c_double()
            amg.lib().amg_kernel_timing_read(h, C.byref(nl), C.byref(ms), C.byref(bpl))
            state["kt"][0] += nl.value
            state["kt"][1] += ms.value
            state["kt"][2] = bpl.value
        amg.amg_free(h)
        return launches, info

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    last_info = None
    for _ in range(args.steps):
        nl, last_info = step(True)
        launches += nl
        state["iters"].append(last_info.iterations)
        state["setup_ms"].append(last_info.setup_ms)
        state["solve_ms"].append(last_info.solve_ms)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    value = job_value(g.n * nrhs, world, ms)

    # the fp32-preconditioner form on the same workload (the metric compares both)
    variant = None
    if args.precision == "fp64" and nrhs == 1 and not args.no_variant:
        opts32 = amg.amg_default_options(degree=p["degree"], passes=p["passes"], precision=amg.AMG_PREC_FP32,
                                         cycle=CYCLE, aggregation=p.get("aggregation", 0))
        its = []

        def step32():
            st, h = amg.amg_setup(g.n, rp, col, w, d, opts32, amg.AMG_MEM_DEVICE, sp)
            assert st == 0
            info = amg.amg_info()
            assert amg.amg_solve(h, bd, xd, nrhs, g.n, 1e-8, info) == 0
            its.append(info.iterations)
            amg.amg_free(h)

        for _ in range(args.warmup):
            step32()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step32()
        e1.record(stream)
        torch.cuda.synchronize()
        ms32 = e0.elapsed_time(e1) / args.steps
        ms32 = max_over_ranks(ms32, world, dev)
        variant = {"fp32_precond": {"value": job_value(g.n * nrhs, world, ms32), "unit": UNIT, "ms_per_step": ms32,
                                    "iterations": its[-1],
                                    "dtype": "f32 preconditioner / f64 outer CG, dots and coarsest solve"}}

    # end to end through the C ABI with pinned host buffers (H2D + D2H inside)
    e2e_steps = 0 if args.no_e2e else args.steps
    pin = lambda a: torch.as_tensor(a).pin_memory()
    hrp, hcol, hw = pin(g.rowptr), pin(g.col), pin(g.w)
    hd = None if g.d is None else pin(g.d)
    hb = pin(b)
    hx = torch.zeros_like(hb).pin_memory()
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
    if world > 1:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return 0

    nl, kms, bpl = state["kt"]
    avg_ms = kms / max(nl, 1)
    gbs = bpl / (avg_ms * 1e-3) / 1e9 if nl else None
    # one step T_{j+1} = S T_j - T_{j-1}, x += c_j T_{j+1} with the smoother form
    # S = 2 t(A): 2 flops per stored off-diagonal, the diagonal product, one
    # subtraction and one FMA per row
    flops = 2.0 * g.nnz + 4.0 * g.n
    tflops = flops / (avg_ms * 1e-3) / 1e12 if nl else None
    hbm_peak, peak_kind = peaks()
    kname = "k_cheb_step<%s> (level 0: SELL-32 SpMV + Chebyshev recurrence step)" % (
        "double" if args.precision == "fp64" else "float")
    hbm_view = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak if gbs else None,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy)"}
    alu_view = {"achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tflops / FP64_PEAK_TFLOPS if tflops else None,
                "peak_kind": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (an FMA probe measured 1.198)"}
    if args.precision == "fp64" and (alu_view["frac"] or 0) > (hbm_view["frac"] or 0):
        # the FP64 pipe (2 lanes/clk/SM on this part) is the closer ceiling
        roof = dict(bound="alu", traffic=profiled_traffic(), hbm_view=hbm_view, **alu_view)
    else:
        roof = dict(bound="hbm", traffic=profiled_traffic() if args.precision == "fp64" else None,
                    **{k: v for k, v in hbm_view.items()})
        if args.precision == "fp64":
            roof["alu_view"] = alu_view
    roof.update({"kernel": kname, "launches_timed": nl, "avg_launch_us": avg_ms * 1e3,
                 "algorithmic_bytes_per_launch": bpl, "algorithmic_flops_per_launch": flops})
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        dt, r, nc = run_oracle_step(g, p, b, 1 if nrhs == 1 else 2, CYCLE)
        cpu = {"value": g.n * nc / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle setup + {nc} of {nrhs} right-hand sides ({r.iterations} iterations), "
                         f"{dt:.1f} s single thread"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32 preconditioner / f64 outer",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC + ("" if CYCLE == 0 else "; stationary AMLI W-cycle instead of the K-cycle"),
                   "n": g.n, "nrhs": nrhs, "nnz_offdiag": g.nnz,
                   "l2": f"inputs {in_bytes / 2**20:.0f} MiB > 129 MiB L2 (no flush)",
                   "parallelism": f"replicas x{world}"},
        "iterations": state["iters"][-1], "setup_ms_host": statistics.median(state["setup_ms"]),
        "solve_ms_host": statistics.median(state["solve_ms"]),
        "e2e": {"value": job_value(g.n * nrhs, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": in_bytes,
                "d2h_bytes_per_step": b.nbytes, "ms_per_step": e2e_ms},
        "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": ck,
        "variants": variant,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
