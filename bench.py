#!/usr/bin/env python3
"""Throughput of the tensor-representation hot path on one GB300 (or N replicas).

Workload: unit cube, 48^3 hexes x 6 Kuhn tetrahedra (663,552 cells, 117,649
vertices), interior vertices jittered by +-0.15h (seed 2); the mass and Poisson
forms with scalar Lagrange P1..P4 -- eight (form, degree) problems.

One step = every one of the eight CSR matrices assembled from scratch (Algorithm 2
with the tensor representation, geometry G_K -> contraction A0:G_K -> insertion):

* P3 and P4 (--rows-degrees): row-owner assembly, mass and Poisson in one
  ffc_assemble_rows_pair launch per degree; each CSR value is summed in fixed point in
  shared memory and written once, so nothing is zeroed or read back;
* P1 and P2: the fused atomic assembly, mass and Poisson in one ffc_assemble_pair
  launch per degree, into values zeroed on a second stream ahead of it.

The row plans and the CSR patterns are set up once per mesh, outside the timed step.
The headline `value` is element tensors computed and inserted per second over the
whole step (8 x 663,552 per step); `nnz_per_s` is the assembled CSR entries per second.
The top-level `fp64` block times the same step in FP64 arithmetic.

Also measured (under "detail"): ffc_tabulate alone (A_K written to HBM) for each
problem in FP64 and in the mixed-precision path, both assembly paths per degree, the
other four workloads (P1 triangles, vector-P2 convection, the 32-mesh batch, the P2
adjoint, the P4 source form) each with its own roofline, clocks and CPU baseline, and
the compute ceilings of the GPU measured by ffc_diag_peak.

The oracle (a plain CPU quadrature evaluator) is timed as the CPU baseline on a
bounded sample of the same workload, using the host cores of this machine.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "tet_scalar_48"
FORMS = (0, 1)  # mass, Poisson
DEGREES = (1, 2, 3, 4)
FORM_NAME = {0: "mass", 1: "poisson"}
METRIC = "element tensors/s (assembled, mass+Poisson P1..P4 on 48^3x6 tets)"
REF_FRACTION = 1.0 / 16   # share of each problem's cells in one sampled oracle step


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["tet_scalar", "tri_p1", "ns_vp2", "batched", "adjoint", "source", "rows",
                                           "quad_curved"],
                    default="tet_scalar",
                    help="tet_scalar is the headline; the others print their own line")
    ap.add_argument("--precision", default="fp32", help="contraction arithmetic of the headline step")
    ap.add_argument("--n", type=int, default=48, help="hexes per axis")
    ap.add_argument("--scale", type=float, default=1.0, help="batched workload: mesh size scale")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-detail", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads' sub-records")
    ap.add_argument("--rows-degrees", default="3,4",
                    help="degrees assembled by the row-owner kernels (one ffc_assemble_rows_pair launch)")
    ap.add_argument("--pair-degrees", default="1,2,3",
                    help="atomic degrees whose mass and Poisson matrices share one ffc_assemble_pair launch "
                         "(others: one launch per matrix); empty for none")
    ap.add_argument("--fp64-rows-degrees", default="",
                    help="degrees of the FP64 step assembled by the row-owner kernels (default: none; the "
                         "FP64 contraction bounds both paths and the atomic one is faster)")
    return ap.parse_args()


def _degrees(text: str) -> set[int]:
    return {int(q) for q in text.split(",") if q.strip()}


# ------------------------------------------------------------------ ranks
def dist_env():
    """(world, rank, local_rank) from the launcher's environment (1, 0, 0 without one)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_units: int, rank: int, world: int) -> list[int]:
    """Independent units (meshes, problems) of this rank: round-robin, no data exchange."""
    return list(range(rank, n_units, world))


def max_over_ranks(seconds: float, world: int, device=None) -> float:
    """Slowest rank's time (the job's time); a no-op with one rank."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist

    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if self.bus_id:
            mine = [r for r in rows if r[0].strip().lower().endswith(self.bus_id[-12:])]
            rows = mine or rows
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(name)
        power = [float(r[3]) for r in rows if r[3].strip().replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ workload
def build_workload(F, n, device, rows_degrees=(3, 4)):
    import torch

    from synthetic import workloads as W

    mesh = W.tet_scalar_mesh(n)
    ctx = {"mesh": mesh, "cells": torch.as_tensor(mesh.cells, device=device),
           "verts": torch.as_tensor(mesh.vertices, device=device), "problems": [], "plans": {}}
    for q in DEGREES:
        p = W.make_problem(mesh, W.POISSON, q)
        row_ptr, col, slot = F.csr_pattern(p.dofmap, p.n_dof)
        slot_d = torch.as_tensor(slot, device=device)
        del slot
        # host copy of the pattern: the full-size tests use it
        ctx.setdefault("patterns", {})[q] = {"dofmap": p.dofmap, "n_dof": p.n_dof, "row_ptr": row_ptr, "col": col}
        if q in rows_degrees:
            ctx["plans"][q] = F.RowPlan(torch.as_tensor(p.dofmap, device=device), p.n_dof,
                                        torch.as_tensor(row_ptr, device=device), torch.as_tensor(col, device=device))
        for form in FORMS:
            ctx["problems"].append({
                "form": form, "q": q, "F": F.Form(form, F.TETRAHEDRON, q), "n_local": p.n_local,
                "nnz": int(col.size), "n_dof": p.n_dof, "slot": slot_d,
                "val": torch.zeros(int(col.size), dtype=torch.float64, device=device)})
    return ctx


def launch_list(ctx, pair_degrees, rows_degrees=()):
    """The step's launches: (label, problem indices, kind). A degree in `rows_degrees` (it
    needs a row plan) is one row-owner launch for its mass and Poisson matrices ("rows");
    an atomic degree in `pair_degrees` shares one ffc_assemble_pair launch ("pair"), any
    other atomic problem is one ffc_assemble launch ("single"). The launches alternate
    between the smallest and the largest remaining, so the zeroing that runs on the side
    stream (in launch order) overlaps long assemblies."""
    probs = ctx["problems"]
    out = []
    k = 0
    while k < len(probs):
        a = probs[k]
        paired = k + 1 < len(probs) and probs[k + 1]["q"] == a["q"]
        if a["q"] in rows_degrees and paired:
            out.append((f"rows_mass+poisson_p{a['q']}", [k, k + 1], "rows"))
            k += 2
        elif a["q"] in pair_degrees and paired:
            b = probs[k + 1]
            assert (a["form"], b["form"]) == (0, 1)
            out.append((f"mass+poisson_p{a['q']}", [k, k + 1], "pair"))
            k += 2
        else:
            out.append((f"{FORM_NAME[a['form']]}_p{a['q']}", [k], "single"))
            k += 1
    rest = sorted(out, key=lambda lk: sum(probs[k]["nnz"] for k in lk[1]))
    order = []
    while rest:
        order.append(rest.pop(0))
        if rest:
            order.append(rest.pop())
    return order


def kernels_of(entry, precision):
    """Kernels of this library one launch-list entry starts: a row-owner call runs its
    geometry pass and the assembly (twice for FP64, which takes the forms one at a time);
    a fused atomic call is one kernel per launch (two for an FP64 pair)."""
    kind = entry[2]
    if kind == "rows":
        return 2 if precision != "fp64" else 4
    if kind == "pair":
        return 1 if precision != "fp64" else 2
    return 1


def assemble_step(F, ctx, precision, events=None, launches=None):
    """Assemble every CSR matrix from scratch. The atomic launches' matrices are zeroed
    (bandwidth bound) on a side stream, ahead of the assemblies that wait for them; the
    row-owner launches overwrite their matrices and wait for nothing."""
    import torch

    launches = ctx["launches"] if launches is None else launches
    main = torch.cuda.current_stream()
    side = ctx.setdefault("side_stream", torch.cuda.Stream())
    side.wait_stream(main)  # the previous step's assemblies are done with these values
    zeroed = {}
    with torch.cuda.stream(side):  # in launch order, so the first launch waits for its own matrices only
        for _, ks, kind in launches:
            if kind == "rows":
                continue
            for k in ks:
                ctx["problems"][k]["val"].zero_()
                ev = torch.cuda.Event()
                ev.record(side)
                zeroed[k] = ev
    for j, entry in enumerate(launches):
        for k in entry[1]:
            if k in zeroed:
                main.wait_event(zeroed[k])
        if events is not None:
            events[j][0].record(main)
        launch_assembly(F, ctx, entry, ctx["cells"], ctx["verts"], precision)
        if events is not None:
            events[j][1].record(main)
    main.wait_stream(side)


def run_headline_step(F, ctx, precision, pair_degrees=(1, 2, 3), rows_degrees=(3, 4)):
    """One headline step (every matrix assembled from scratch) on the current stream."""
    if "launches" not in ctx:
        ctx["launches"] = launch_list(ctx, set(pair_degrees), set(rows_degrees) & set(ctx["plans"]))
    assemble_step(F, ctx, precision)


def launch_assembly(F, ctx, entry, cells, verts, precision):
    _, ks, kind = entry
    prs = [ctx["problems"][k] for k in ks]
    if kind == "rows":
        F.assemble_rows_pair(prs[0]["F"], prs[1]["F"], ctx["plans"][prs[0]["q"]], cells, verts, prs[0]["val"],
                             prs[1]["val"], precision=precision)
    elif kind == "pair":
        F.assemble_pair(prs[0]["F"], prs[1]["F"], cells, verts, prs[0]["slot"], prs[0]["val"], prs[1]["val"],
                        precision=precision)
    else:
        F.assemble(prs[0]["F"], cells, verts, prs[0]["slot"], prs[0]["val"], precision=precision)


def alg_bytes_assemble(ctx, prs, kind="pair"):
    """Algorithmic bytes of one assembly launch: cells + vertices + dofmap once, and the
    CSR values of each of its matrices written once, plus read once where the launch
    accumulates into them (the atomic paths; slot map and row plan not counted)."""
    m = ctx["mesh"]
    per_nnz = 8 if kind == "rows" else 16
    return m.n_elem * 16 + m.n_vert * 24 + m.n_elem * 4 * prs[0]["n_local"] + sum(per_nnz * pr["nnz"] for pr in prs)


def alg_bytes_tabulate(ctx, n_local, out_bytes):
    m = ctx["mesh"]
    return m.n_elem * 16 + m.n_vert * 24 + m.n_elem * n_local * n_local * out_bytes


# DRAM bytes (read + write) per launch, from one `ncu` capture of the kernel on a smaller
# mesh scaled by the cell count (positions, pairs, values and cells all grow with it); only
# valid for the kernels as captured, other launches report null.
# DRAM bytes per launch of the dominant kernel from an ncu capture of the current kernel
# (scaled from a smaller mesh by the cell count); none is held for the one-digit row-owner
# kernel, whose last capture (1.237 GB at 24^3 x 6, two-digit sums) predates it
CAPTURED_TRAFFIC_GB = {}

_PEAKS = {}


def compute_peaks(F):
    """Compute ceilings of this GPU, measured now by ffc_diag_peak (best of two launches
    each): FP64 and FP32 FMA (TFLOP/s), TF32 and BF16 tcgen05 MMA (TFLOP/s) and 32-bit
    shared-memory atomics (G lane-operations/s)."""
    if not _PEAKS:
        for k in F.PEAKS:
            rate = max(F.diag_peak(k)[0] for _ in range(2))
            _PEAKS[k] = rate / 1e12 if k != "smem_atomic_u32" else rate / 1e9
    return dict(_PEAKS)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ CPU oracle baseline
def _oracle_chunk(args):
    form, q, verts, dofmap, n_dof = args
    from oracle import assemble as OA
    from oracle import element as OE

    A = OE.element_tensors(form, verts, q)
    OA.assemble_csr(A, dofmap, n_dof)
    return verts.shape[0]


def cpu_oracle_step(n, frac, pool):
    """One sampled oracle step: the same fraction `frac` of the cells of each of the
    eight problems (cells spread evenly over the mesh), element tensors by quadrature
    and their Algorithm-2 insertion, split over the pool's host cores.
    Returns (cells per problem, seconds)."""
    from synthetic import mesh as M
    from synthetic import workloads as W

    cores = pool._processes
    mesh = W.tet_scalar_mesh(n)
    S = max(cores, int(round(mesh.n_elem * frac)))
    idx = np.linspace(0, mesh.n_elem - 1, S).astype(np.int64)
    verts = M.gather_cell_vertices(mesh)[idx]
    jobs = []
    for q in DEGREES:
        p = W.make_problem(mesh, W.POISSON, q)
        dm = p.dofmap[idx]
        for form in FORMS:
            jobs += [(form, q, verts[c::cores], dm[c::cores], p.n_dof) for c in range(cores)]
    t0 = time.perf_counter()
    done = sum(pool.map(_oracle_chunk, jobs, chunksize=1))
    dt = time.perf_counter() - t0
    assert done == S * len(FORMS) * len(DEGREES)
    return S, dt


def oracle_pool(cores=None):
    import multiprocessing as mp

    if cores is None:
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    pool = mp.get_context("spawn").Pool(cores)
    warm = (0, 1, np.zeros((1, 4, 3)) + np.eye(4, 3)[None], np.zeros((1, 4), np.int32), 1)
    pool.map(_oracle_chunk, [warm] * cores)
    return pool, cores


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    pool, cores = oracle_pool()
    times = []
    S = 0
    for it in range(args.warmup + args.steps):
        S, t = cpu_oracle_step(args.n, REF_FRACTION, pool)
        if it >= args.warmup:
            times.append(t)
    pool.close()
    pool.join()
    t = statistics.mean(times)
    value = len(FORMS) * len(DEGREES) * S / t
    sample = (f"{S} of the cells (1/{round(1 / REF_FRACTION)}) of each of the 8 problems per step, "
              "spread evenly over the mesh; same problem mix as the full step")
    line = {"metric": METRIC, "value": value, "unit": "elem/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "cells_per_problem_per_step": S},
            "cpu_baseline": {"value": value, "unit": "elem/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "elem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ main arm
def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "tet_scalar":
        return run_other(args)
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    device = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(device)

    # the CPU oracle pool starts before the first GPU call
    cpu = None
    pool = pool1 = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool, cores = oracle_pool()
        pool1, _ = oracle_pool(1)  # the same oracle on one host thread

    from paper_1112_0402_gb300 import build as B

    B.build()
    import paper_1112_0402_gb300 as F

    rows_degrees = _degrees(args.rows_degrees)
    fp64_rows = _degrees(args.fp64_rows_degrees)
    ctx = build_workload(F, args.n, device, rows_degrees | fp64_rows)
    ctx["launches"] = launch_list(ctx, _degrees(args.pair_degrees), rows_degrees)
    P = len(ctx["problems"])
    NL = len(ctx["launches"])
    n_elem = ctx["mesh"].n_elem
    total_nnz = sum(pr["nnz"] for pr in ctx["problems"])
    peaks = compute_peaks(F)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        assemble_step(F, ctx, args.precision)
    assert F.status_poll() == 0
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(NL * args.steps)]
    bus = None
    try:
        bus = torch.cuda.get_device_properties(device).pci_bus_id  # noqa
    except Exception:
        bus = None
    clocks = ClockSampler(bus)
    clocks.start()
    barrier()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for s in range(args.steps):
        assemble_step(F, ctx, args.precision, events[s * NL:(s + 1) * NL])
    stop.record()
    barrier()
    clk = clocks.stop()
    elapsed = max_over_ranks(start.elapsed_time(stop) / 1e3, world, device)
    assert F.status_poll() == 0
    per_launch = np.zeros(NL)
    for s in range(args.steps):
        for k in range(NL):
            ev = events[s * NL + k]
            per_launch[k] += ev[0].elapsed_time(ev[1]) / 1e3
    per_launch /= args.steps
    dom = int(np.argmax(per_launch))
    dlabel, dks, dkind = ctx["launches"][dom]
    dprs = [ctx["problems"][k] for k in dks]
    hbm_peak, peak_kind = measured_peaks()
    dbytes = alg_bytes_assemble(ctx, dprs, dkind)
    achieved = dbytes / per_launch[dom] / 1e9
    value = world * P * n_elem / elapsed * args.steps
    kernels_per_step = sum(kernels_of(e, args.precision) for e in ctx["launches"])

    # ---- the same step in FP64 arithmetic (FP64 contraction, FP64 CSR values)
    fp64 = None
    if args.precision != "fp64":
        l64 = launch_list(ctx, _degrees(args.pair_degrees), fp64_rows)
        for _ in range(2):
            assemble_step(F, ctx, "fp64", launches=l64)
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            assemble_step(F, ctx, "fp64", launches=l64)
        b.record()
        barrier()
        assert F.status_poll() == 0
        t64 = max_over_ranks(a.elapsed_time(b) / 1e3, world, device) / args.steps
        fp64 = {"value": world * P * n_elem / t64, "unit": "elem/s", "nnz_per_s": world * total_nnz / t64,
                "ms_per_step": t64 * 1e3, "dtype": "f64", "steps": args.steps,
                "launches": [lab for lab, _, _ in l64],
                "gpu_launches": sum(kernels_of(e, "fp64") for e in l64) * args.steps}

    # ---- end to end through the C ABI: pinned host inputs in, CSR values out
    e2e = None
    if not args.no_e2e:
        h_cells = torch.as_tensor(ctx["mesh"].cells).pin_memory()
        h_verts = torch.as_tensor(ctx["mesh"].vertices).pin_memory()
        h_out = [torch.empty(pr["nnz"], dtype=torch.float64).pin_memory() for pr in ctx["problems"]]
        d_cells = torch.empty_like(ctx["cells"])
        d_verts = torch.empty_like(ctx["verts"])

        # the read-back of a launch's matrices runs on its own stream while the next launch
        # assembles; a matrix is written again only after its previous read-back finished
        copy_stream = torch.cuda.Stream()
        read_done = [None] * P

        def e2e_step():
            cur = torch.cuda.current_stream()
            d_cells.copy_(h_cells, non_blocking=True)
            d_verts.copy_(h_verts, non_blocking=True)
            for entry in ctx["launches"]:
                for k in entry[1]:
                    if read_done[k] is not None:
                        cur.wait_event(read_done[k])
                    if entry[2] != "rows":
                        ctx["problems"][k]["val"].zero_()
                launch_assembly(F, ctx, entry, d_cells, d_verts, args.precision)
                copy_stream.wait_stream(cur)
                with torch.cuda.stream(copy_stream):
                    for k in entry[1]:
                        h_out[k].copy_(ctx["problems"][k]["val"], non_blocking=True)
                        read_done[k] = torch.cuda.Event()
                        read_done[k].record(copy_stream)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.current_stream().wait_stream(copy_stream)
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.current_stream().wait_stream(copy_stream)
        b.record()
        barrier()
        te = max_over_ranks(a.elapsed_time(b) / 1e3, world, device)
        e2e = {"value": world * P * n_elem * args.steps / te, "unit": "elem/s",
               "h2d_bytes_per_step": int(h_cells.numel() * 4 + h_verts.numel() * 8),
               "d2h_bytes_per_step": int(sum(pr["nnz"] for pr in ctx["problems"]) * 8),
               "ms_per_step": te / args.steps * 1e3}
        del h_out

    detail = None
    if rank == 0 and not args.no_detail:
        detail = measure_detail(F, ctx, args, device)
        detail["compute_peaks"] = {"fp64_fma_tflops": peaks["fp64_fma"], "fp32_fma_tflops": peaks["fp32_fma"],
                                   "tf32_mma_tflops": peaks["tf32_mma"], "bf16_mma_tflops": peaks["bf16_mma"],
                                   "smem_atomic_u32_g_per_s": peaks["smem_atomic_u32"],
                                   "how": "ffc_diag_peak, best of 2 launches, this run"}
    iso_ms = (detail or {}).get("launch_alone_ms", {}).get(dlabel) if args.precision == "fp32" else None
    ctx_problems = [{k: pr[k] for k in ("form", "q", "n_local")} for pr in ctx["problems"]]
    n_vert = ctx["mesh"].n_vert
    launches = ctx["launches"]
    del ctx, dprs
    torch.cuda.empty_cache()
    if detail is not None and not args.no_configs and world == 1:
        detail["configs"] = {}
        for wl in ("tri_p1", "ns_vp2", "batched", "adjoint", "source", "quad_curved"):
            detail["configs"][wl] = measure_other(F, args, device, wl)
            torch.cuda.empty_cache()

    if pool is not None:
        S, t_cpu = cpu_oracle_step(args.n, 2 * REF_FRACTION, pool)
        pool.close()
        pool.join()
        S1, t1 = cpu_oracle_step(args.n, REF_FRACTION / 8, pool1)
        pool1.close()
        pool1.join()
        cpu = {"value": P * S / t_cpu, "unit": "elem/s", "cores": cores, "kind": "oracle",
               "sample": f"{S} cells (1/8) of each of the 8 problems, spread evenly over the mesh, "
                         f"{t_cpu:.1f} s; same problem mix as the GPU step",
               "single_thread": {"value": P * S1 / t1, "unit": "elem/s", "cores": 1,
                                 "sample": f"{S1} cells (1/128) of each of the 8 problems, {t1:.1f} s"}}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "elem/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64", "data": "synthetic",
            "nnz_per_s": world * total_nnz * args.steps / elapsed,
            "insertions_per_s": world * n_elem * sum(p["n_local"] ** 2 for p in ctx_problems) * args.steps / elapsed,
            "config": {"workload": WORKLOAD, "cells": n_elem, "vertices": n_vert,
                       "problems": [f"{FORM_NAME[p['form']]}_p{p['q']}" for p in ctx_problems],
                       "contraction": args.precision, "csr_accumulation": "f64",
                       "assembly": {lab: kind for lab, _, kind in launches},
                       "nnz_total": total_nnz,
                       "l2": "inputs larger than L2: the step streams ~12 GB (CSR values, row plans) per pass",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                         "traffic": CAPTURED_TRAFFIC_GB.get((dlabel, args.precision)),
                         "traffic_unit": "GB per launch (ncu, scaled by the cell count from a smaller mesh)",
                         "algorithmic_gb": dbytes / 1e9,
                         "kernel": f"{dlabel} ({args.precision})",
                         "launch_ms": per_launch[dom] * 1e3,
                         # in the step the launch overlaps the side-stream zeroing of other
                         # matrices; the same launch timed alone (detail section):
                         "isolated_launch_ms": iso_ms,
                         "isolated_frac": dbytes / (iso_ms / 1e3) / 1e9 / hbm_peak if iso_ms else None},
            "per_launch_ms": {lab: round(per_launch[k] * 1e3, 4) for k, (lab, _, _) in enumerate(launches)},
            "fp64": fp64,
            "clocks": clk, "gpu_launches": kernels_per_step * args.steps, "e2e": e2e, "cpu_baseline": cpu,
            "detail": detail,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def measure_detail(F, ctx, args, device, reps=5):
    """ffc_tabulate alone per problem, FP64 vs the mixed path, plus FP64 assembly."""
    import torch

    out = {}
    hbm_peak, _ = measured_peaks()
    n_elem = ctx["mesh"].n_elem
    for pr in ctx["problems"]:
        key = f"{FORM_NAME[pr['form']]}_p{pr['q']}"
        n = pr["n_local"]
        rec = {}
        ref = None
        for prec in ("fp64", args.precision):
            dt = torch.float64 if prec == "fp64" else torch.float32
            A = torch.empty((n_elem, n, n), dtype=dt, device=device)
            F.tabulate(pr["F"], ctx["cells"], ctx["verts"], out=A, precision=prec)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                F.tabulate(pr["F"], ctx["cells"], ctx["verts"], out=A, precision=prec)
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3 / reps
            byts = alg_bytes_tabulate(ctx, n, 8 if prec == "fp64" else 4)
            r = {"elem_per_s": n_elem / t, "ms": t * 1e3, "hbm_frac": byts / t / 1e9 / hbm_peak}
            if prec == "fp64" and pr["form"] == 1:
                # executed FP64 FMAs: the symmetric form contracts the entries i1 <= i2 only
                nak = 3 * (3 + 1) // 2  # symmetric G of the tetrahedron: 6 columns
                fl = 2.0 * n * (n + 1) / 2 * nak * n_elem / t / 1e12
                r["fp64_tflops"] = fl
                r["fp64_frac"] = fl / compute_peaks(F)["fp64_fma"]
            if prec == "fp64":
                ref = A
            else:
                d = (A.double() - ref).reshape(n_elem, -1).norm(dim=1) / ref.reshape(n_elem, -1).norm(dim=1)
                r["max_rel_err_vs_fp64"] = float(d.max().item())
                r["mean_rel_err_vs_fp64"] = float(d.mean().item())
            rec[prec] = r
            if prec != "fp64" and pr["form"] == 1 and pr["q"] >= 3:
                # the same element tensors on the tensor cores (tcgen05, split products)
                for tc in ("tf32x3", "bf16x3"):
                    F.tabulate(pr["F"], ctx["cells"], ctx["verts"], out=A, precision=tc)
                    torch.cuda.synchronize()
                    a.record()
                    for _ in range(reps):
                        F.tabulate(pr["F"], ctx["cells"], ctx["verts"], out=A, precision=tc)
                    b.record()
                    torch.cuda.synchronize()
                    ttc = a.elapsed_time(b) / 1e3 / reps
                    d = (A.double() - ref).reshape(n_elem, -1).norm(dim=1) / ref.reshape(n_elem, -1).norm(dim=1)
                    rec[tc] = {"ms": ttc * 1e3, "hbm_frac": byts / ttc / 1e9 / hbm_peak,
                               "max_rel_err_vs_fp64": float(d.max().item())}
            del A
        ref = None
        torch.cuda.empty_cache()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            pr["val"].zero_()
            F.assemble(pr["F"], ctx["cells"], ctx["verts"], pr["slot"], pr["val"], precision="fp64")
        b.record()
        torch.cuda.synchronize()
        rec["assemble_fp64_ms"] = a.elapsed_time(b) / reps
        if pr["q"] == 4:
            # the insertion alone (Algorithm 2's add of precomputed element tensors into the
            # same slots, ffc_scatter_add, FP32 values and FP64 atomics as in the fused
            # step), zeroing included as in the fused timing: the atomic ceiling of this
            # slot pattern
            A = torch.empty((n_elem, n, n), dtype=torch.float32, device=device)
            F.tabulate(pr["F"], ctx["cells"], ctx["verts"], out=A, precision="fp32")
            pr["val"].zero_()
            F.scatter_add(A, pr["slot"], pr["val"])
            torch.cuda.synchronize()
            a.record()
            for _ in range(3):
                pr["val"].zero_()
                F.scatter_add(A, pr["slot"], pr["val"])
            b.record()
            torch.cuda.synchronize()
            rec["scatter_only_ms"] = a.elapsed_time(b) / 3
            a.record()
            for _ in range(3):
                pr["val"].zero_()
                F.assemble(pr["F"], ctx["cells"], ctx["verts"], pr["slot"], pr["val"], precision="fp32")
            b.record()
            torch.cuda.synchronize()
            rec["assemble_fp32_with_zero_ms"] = a.elapsed_time(b) / 3
            # the launch alone: no zeroing, nothing else running (the values accumulate)
            a.record()
            for _ in range(3):
                F.assemble(pr["F"], ctx["cells"], ctx["verts"], pr["slot"], pr["val"], precision="fp32")
            b.record()
            torch.cuda.synchronize()
            rec["assemble_fp32_ms"] = a.elapsed_time(b) / 3
            del A
            torch.cuda.empty_cache()
            if pr["form"] == 1:
                # the FP64 atomic ceiling of the GPU: ffc_scatter_add of as many FP32 values as
                # the P4 matrix has entries, through the identity slot map (consecutive
                # addresses, each entry once: no conflicts, fully coalesced)
                ident = torch.arange(pr["nnz"], dtype=torch.int32, device=device)
                ones = torch.ones(pr["nnz"], dtype=torch.float32, device=device)
                F.scatter_add(ones, ident, pr["val"])
                torch.cuda.synchronize()
                a.record()
                for _ in range(3):
                    F.scatter_add(ones, ident, pr["val"])
                b.record()
                torch.cuda.synchronize()
                out["fp64_atomic_ceiling_per_s"] = pr["nnz"] / (a.elapsed_time(b) / 3 / 1e3)
                del ident, ones
                torch.cuda.empty_cache()
        out[key] = rec
    # both assembly paths per degree, each launch timed alone (no zeroing, nothing else
    # running): the fused atomic pair (accumulating) and the row-owner pair (overwriting)
    out["launch_alone_ms"] = {}
    out["degrees"] = {}
    for q in DEGREES:
        pm, pp = [pr for pr in ctx["problems"] if pr["q"] == q]
        plan = ctx["plans"].get(q)
        if plan is None:
            pat = ctx["patterns"][q]
            plan = F.RowPlan(torch.as_tensor(pat["dofmap"], device=device), pat["n_dof"],
                             torch.as_tensor(pat["row_ptr"], device=device), torch.as_tensor(pat["col"], device=device))
        rec = {}

        def atomic_pair():
            F.assemble_pair(pm["F"], pp["F"], ctx["cells"], ctx["verts"], pm["slot"], pm["val"], pp["val"],
                            precision=args.precision)

        def rows_pair():
            F.assemble_rows_pair(pm["F"], pp["F"], plan, ctx["cells"], ctx["verts"], pm["val"], pp["val"],
                                 precision=args.precision)

        rec["atomic_pair_ms"] = _timed(atomic_pair, reps, 1) * 1e3
        rec["rows_pair_ms"] = _timed(rows_pair, reps, 1) * 1e3
        for pr in (pm, pp):
            rec[f"rows_{FORM_NAME[pr['form']]}_ms"] = _timed(
                lambda: F.assemble_rows(pr["F"], plan, ctx["cells"], ctx["verts"], pr["val"],
                                        precision=args.precision), reps, 1) * 1e3
        prs = [pm, pp]
        rec["rows_pair_hbm_frac"] = alg_bytes_assemble(ctx, prs, "rows") / (rec["rows_pair_ms"] / 1e3) / 1e9 / hbm_peak
        rec["atomic_pair_hbm_frac"] = alg_bytes_assemble(ctx, prs) / (rec["atomic_pair_ms"] / 1e3) / 1e9 / hbm_peak
        rec["plan_mb"] = plan.device_bytes / 1e6
        out["degrees"][f"p{q}"] = rec
        out["launch_alone_ms"][f"rows_mass+poisson_p{q}"] = rec["rows_pair_ms"]
        out["launch_alone_ms"][f"mass+poisson_p{q}"] = rec["atomic_pair_ms"]
        if q not in ctx["plans"]:
            del plan
            torch.cuda.empty_cache()
    assert F.status_poll() == 0
    return out


# ------------------------------------------------------------------ other workloads
def _timed(fn, steps, warmup):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3 / steps


def _oracle_rate(form, q, verts, coeffs, cores, seconds=4.0):
    """Oracle element tensors per second on `cores` host processes (bounded sample)."""
    import multiprocessing as mp

    pool = mp.get_context("spawn").Pool(cores)
    try:
        probe = max(cores, 64)
        t0 = time.perf_counter()
        pool.map(_oracle_tensors, [(form, q, verts[:probe:1][c::cores], None if coeffs is None else
                                    coeffs[:probe][c::cores]) for c in range(cores)])
        rate = probe / (time.perf_counter() - t0)
        S = min(verts.shape[0], max(cores, int(rate * seconds)))
        t0 = time.perf_counter()
        pool.map(_oracle_tensors, [(form, q, verts[:S][c::cores], None if coeffs is None else coeffs[:S][c::cores])
                                   for c in range(cores)])
        return S / (time.perf_counter() - t0), S
    finally:
        pool.close()
        pool.join()


def _oracle_tensors(args):
    form, q, verts, coeffs = args
    from oracle import element as OE

    OE.element_tensors(form, verts, q, coeffs=coeffs)
    return verts.shape[0]


def run_other(args):
    import torch

    from paper_1112_0402_gb300 import build as B

    B.build()
    import paper_1112_0402_gb300 as F

    print(json.dumps(measure_other(F, args, torch.device("cuda", 0), args.workload)), flush=True)
    return 0


def measure_other(F, args, device, workload):
    """One of the other workloads, as its own record (metric, roofline, clocks, CPU baseline)."""
    import torch

    from synthetic import mesh as M
    from synthetic import workloads as W

    hbm_peak, peak_kind = measured_peaks()
    cores = len(os.sched_getaffinity(0))
    clocks = ClockSampler(None)
    out = {"metric": None, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "data": "synthetic", "unit": "elem/s"}
    if workload == "tri_p1":
        # P1 Poisson on the unit square, 64 x 64 x 2 triangles, FP64: zero + fused assembly
        p = W.poisson_p1_tri()
        m = p.mesh
        cells = torch.as_tensor(m.cells, device=device)
        verts = torch.as_tensor(m.vertices, device=device)
        fm = F.Form(F.POISSON, F.TRIANGLE, 1)
        row_ptr, col, slot = F.csr_pattern(p.dofmap, p.n_dof)
        slot_d = torch.as_tensor(slot, device=device)
        val = torch.zeros(col.size, dtype=torch.float64, device=device)
        A = torch.empty((m.n_elem, 3, 3), dtype=torch.float64, device=device)
        reps = 100  # assemblies per timed step: one alone is a few microseconds

        def step():
            for _ in range(reps):
                val.zero_()
                F.assemble(fm, cells, verts, slot_d, val, precision="fp64")

        t_tab = _timed(lambda: F.tabulate(fm, cells, verts, out=A, precision="fp64"), reps * args.steps,
                       args.warmup) 
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        clocks.start()
        t = _timed(step, args.steps, 1) / reps
        # the assembly kernel alone (no zeroing), on the launching stream
        ev[0].record()
        for _ in range(reps):
            F.assemble(fm, cells, verts, slot_d, val, precision="fp64")
        ev[1].record()
        torch.cuda.synchronize()
        clk = clocks.stop()
        assert F.status_poll() == 0
        t_k = ev[0].elapsed_time(ev[1]) / 1e3 / reps
        byts = m.n_elem * (12 + 4 * 3) + m.n_vert * 16 + 16 * int(col.size)
        rate, S = (None, 0) if args.no_cpu_baseline else _oracle_rate(W.POISSON, 1, M.gather_cell_vertices(m), None,
                                                                       cores, seconds=2.0)
        out.update({"metric": "element tensors/s (P1 Poisson, 64x64x2 triangles, FP64, zero + assemble)",
                    "value": m.n_elem / t, "ms_per_step": t * 1e3, "dtype": "f64", "nnz_per_s": int(col.size) / t,
                    "config": {"workload": "tri_p1_64", "cells": m.n_elem, "vertices": m.n_vert,
                               "nnz": int(col.size), "assemblies_per_step": 1,
                               "note": "latency-bound: 8,192 cells are a fraction of one wave; the timed "
                                       f"region holds {reps} back-to-back steps",
                               "l2": "inputs and matrix (0.4 MB) stay in L2"},
                    "roofline": {"bound": "hbm", "achieved": byts / t_k / 1e9, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": byts / t_k / 1e9 / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                                 "kernel": "simt_tabulate_kernel<2,POISSON,1,double,assemble>",
                                 "kernel_us": t_k * 1e6, "latency_bound": True},
                    "clocks": clk, "gpu_launches": reps * args.steps,
                    "cpu_baseline": {"value": rate, "unit": "elem/s", "cores": cores, "kind": "oracle",
                                     "sample": f"{S} cells, element tensors"},
                    "detail": {"tabulate_fp64_us": t_tab * 1e6}})
        return out
    if workload == "ns_vp2":
        p = W.ns_vp2(40 if args.n == 48 else args.n)
        m = p.mesh
        cells = torch.as_tensor(m.cells, device=device)
        verts = torch.as_tensor(m.vertices, device=device)
        coeffs = torch.as_tensor(p.coeffs, device=device)
        fm = F.Form(F.NS_CONVECTION, F.TETRAHEDRON, 2)
        row_ptr, col, slot = F.csr_pattern(p.dofmap, p.n_dof)
        slot_d = torch.as_tensor(slot, device=device)
        del slot
        val = torch.zeros(col.size, dtype=torch.float64, device=device)
        detail = {}
        ref = None
        fm_dense = F.Form(F.NS_CONVECTION, F.TETRAHEDRON, 2, algorithm=F.ALG_DENSE)
        for prec, f_, tag in (("fp64", fm_dense, "fp64_dense"), ("fp64", fm, "fp64_block"),
                              ("fp32", fm_dense, "fp32_dense"), ("fp32", fm, "fp32_block"),
                              ("tf32", fm, "tf32"), ("tf32x3", fm, "tf32x3"), ("bf16x3", fm, "bf16x3")):
            dt = torch.float64 if prec == "fp64" else torch.float32
            A = torch.empty((m.n_elem, 30, 30), dtype=dt, device=device)
            t = _timed(lambda: F.tabulate(f_, cells, verts, coeffs=coeffs, out=A, precision=prec), args.steps,
                       args.warmup)
            byts = m.n_elem * (16 + 240 + 900 * (8 if prec == "fp64" else 4)) + m.n_vert * 24
            r = {"elem_per_s": m.n_elem / t, "ms": t * 1e3, "hbm_frac": byts / t / 1e9 / hbm_peak}
            if ref is None:
                ref = A
            else:
                d = (A.double() - ref).reshape(m.n_elem, -1).norm(dim=1) / ref.reshape(m.n_elem, -1).norm(dim=1)
                r["max_rel_err_vs_fp64"] = float(d.max())
            detail["tabulate_" + tag] = r
            if ref is not A:
                del A
        del ref
        torch.cuda.empty_cache()
        for prec, f_, tag in (("fp64", fm_dense, "fp64_dense"), ("fp64", fm, "fp64_block"),
                              ("fp32", fm, "fp32_block"), ("bf16x3", fm, "bf16x3")):
            def step():
                val.zero_()
                F.assemble(f_, cells, verts, slot_d, val, coeffs=coeffs, precision=prec)
            detail["assemble_" + tag + "_ms"] = _timed(step, max(1, args.steps // 2), 1) * 1e3
        # the reported path: the fastest one within the 1e-6 mixed-precision bound
        paths = {"fp32_block": ("fp32", "simt_block_kernel<3, convection, 2, float>"),
                 "tf32x3": ("tf32x3", "tc_ws_kernel convection P2 tf32x3"),
                 "bf16x3": ("bf16x3", "tc_ws_kernel convection P2 bf16x3")}
        ok = [k for k in paths if detail["tabulate_" + k].get("max_rel_err_vs_fp64", 1.0) <= 1e-6]
        best = min(ok, key=lambda k: detail["tabulate_" + k]["ms"])
        prec, kernel_name = paths[best]
        A32 = torch.empty((m.n_elem, 30, 30), dtype=torch.float32, device=device)
        clocks.start()
        t = _timed(lambda: F.tabulate(fm, cells, verts, coeffs=coeffs, out=A32, precision=prec), args.steps,
                   args.warmup)
        clk = clocks.stop()
        byts = m.n_elem * (16 + 240 + 3600) + m.n_vert * 24
        rate, S = (None, 0) if args.no_cpu_baseline else _oracle_rate(W.NS_CONVECTION, 2,
                                                                       M.gather_cell_vertices(m), p.coeffs, cores)
        out.update({"metric": "element tensors/s (vector-P2 convection, 40^3x6 tets, tabulate)",
                    "value": m.n_elem / t, "ms_per_step": t * 1e3, "dtype": "f32" if prec == "fp32" else prec,
                    "config": {"workload": "ns_vp2", "cells": m.n_elem, "nnz": int(col.size),
                               "contraction": best, "l2": "A_K output 1.38 GB per step > L2"},
                    "roofline": {"bound": "hbm", "achieved": byts / t / 1e9, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": byts / t / 1e9 / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                                 "kernel": kernel_name},
                    "clocks": clk, "gpu_launches": args.steps,
                    "cpu_baseline": {"value": rate, "unit": "elem/s", "cores": cores, "kind": "oracle",
                                     "sample": f"{S} cells"}, "detail": detail})
    elif workload == "batched":
        probs = W.batched(scale=args.scale)
        items = []
        total_nnz = 0
        for pb in probs:
            row_ptr, col, slot = F.csr_pattern(pb.dofmap, pb.n_dof)
            items.append({"form": F.Form(pb.form, F.TETRAHEDRON, pb.degree),
                          "cells": torch.as_tensor(pb.mesh.cells, device=device),
                          "vertices": torch.as_tensor(pb.mesh.vertices, device=device),
                          "slot": torch.as_tensor(slot, device=device),
                          "csr_val": torch.zeros(col.size, dtype=torch.float64, device=device)})
            total_nnz += int(col.size)
            del slot
        n_cells = sum(pb.n_elem for pb in probs)
        b = F.Batch(items, zero_csr=True)
        ke = b.tune()
        t_plain = _timed(lambda: b.run(graph=False), args.steps, args.warmup)
        clocks.start()
        t = _timed(lambda: b.run(graph=True), args.steps, args.warmup)
        clk = clocks.stop()
        assert F.status_poll() == 0
        # per-problem launches of the same work, for comparison
        def separate():
            for it in items:
                it["csr_val"].zero_()
                F.assemble(it["form"], it["cells"], it["vertices"], it["slot"], it["csr_val"], precision="fp32")
        t_sep = _timed(separate, args.steps, args.warmup)
        # the largest elasticity vP3 mesh of the batch, tabulated alone by each path
        big = max((pb for pb in probs if pb.form == W.ELASTICITY and pb.degree == 3), key=lambda pb: pb.n_elem)
        bc = torch.as_tensor(big.mesh.cells, device=device)
        bv = torch.as_tensor(big.mesh.vertices, device=device)
        A3 = torch.empty((big.n_elem, 60, 60), dtype=torch.float32, device=device)
        elast = {"cells": big.n_elem}
        for tag, alg, prec in (("fp32_dense", F.ALG_DENSE, "fp32"), ("fp32_block", F.ALG_BLOCK, "fp32"),
                               ("tf32x3", F.ALG_AUTO, "tf32x3"), ("bf16x3", F.ALG_AUTO, "bf16x3")):
            f3 = F.Form(F.ELASTICITY, F.TETRAHEDRON, 3, algorithm=alg)
            elast[tag + "_ms"] = _timed(lambda: F.tabulate(f3, bc, bv, out=A3, precision=prec), 3, 1) * 1e3
        del A3
        byts = sum(pb.n_elem * (16 + 4 * pb.n_local) + pb.mesh.n_vert * 24 for pb in probs) + 16 * total_nnz
        out.update({"metric": "element tensors/s (batched: 32 meshes, elasticity vP1-vP3 + Poisson P2)",
                    "value": n_cells / t, "ms_per_step": t * 1e3, "dtype": "f32", "nnz_per_s": total_nnz / t,
                    "insertions_per_s": sum(pb.n_elem * pb.n_local ** 2 for pb in probs) / t,
                    "config": {"workload": "batched", "meshes": len(probs), "cells": n_cells, "nnz": total_nnz,
                               "tile_cells_per_group": ke, "threads_per_block": b.threads_per_block,
                               "graph": True},
                    "roofline": {"bound": "hbm", "achieved": byts / t / 1e9, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": byts / t / 1e9 / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                                 "kernel": "batch_assemble_kernel"},
                    "clocks": clk, "gpu_launches": args.steps,
                    "detail": {"plain_launch_ms": t_plain * 1e3, "separate_launches_ms": t_sep * 1e3,
                               "elasticity_p3_tabulate": elast}})
        if not args.no_cpu_baseline:
            # the oracle's element-tensor rate of each (form, degree) of the batch on a sample
            # of its largest mesh, weighted by the batch's cell counts
            t_cpu, sample = 0.0, []
            for form, q in W.BATCHED_FORMS:
                grp = [pb for pb in probs if (pb.form, pb.degree) == (form, q)]
                if not grp:
                    continue
                big = max(grp, key=lambda pb: pb.n_elem)
                rate, S = _oracle_rate(form, q, M.gather_cell_vertices(big.mesh), None, cores, seconds=1.5)
                t_cpu += sum(pb.n_elem for pb in grp) / rate
                sample.append(f"{S} cells of form {form} P{q}")
            out["cpu_baseline"] = {"value": n_cells / t_cpu, "unit": "elem/s", "cores": cores, "kind": "oracle",
                                   "sample": ", ".join(sample) + " (element tensors; rates weighted by the "
                                                                 "batch's cell counts)"}
    elif workload == "source":
        # the linear form L = v f dx (P4, 48^3 x 6 tets) assembled into a global vector
        m = W.tet_scalar_mesh(args.n)
        p = W.make_problem(m, W.SOURCE, 4, seed=2)
        n = p.n_local
        cells = torch.as_tensor(m.cells, device=device)
        verts = torch.as_tensor(m.vertices, device=device)
        coeffs = torch.as_tensor(p.coeffs, device=device)
        dm = torch.as_tensor(p.dofmap, device=device)
        fm = F.Form(F.SOURCE, F.TETRAHEDRON, 4)
        b = torch.zeros(p.n_dof, dtype=torch.float64, device=device)

        def step(prec):
            b.zero_()
            F.assemble(fm, cells, verts, dm, b, coeffs=coeffs, precision=prec)

        detail = {}
        for prec in ("fp64", "fp32"):
            dt = torch.float64 if prec == "fp64" else torch.float32
            A = torch.empty((m.n_elem, n), dtype=dt, device=device)
            detail["tabulate_" + prec + "_ms"] = _timed(
                lambda: F.tabulate(fm, cells, verts, coeffs=coeffs, out=A, precision=prec), args.steps,
                args.warmup) * 1e3
            del A
        detail["assemble_fp64_ms"] = _timed(lambda: step("fp64"), args.steps, args.warmup) * 1e3
        # the assembly kernel alone, on the launching stream (the zeroing is a separate launch)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
        for _ in range(args.warmup):
            step("fp32")
        torch.cuda.synchronize()
        clocks.start()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for k in range(args.steps):
            b.zero_()
            ev[2 * k].record()
            F.assemble(fm, cells, verts, dm, b, coeffs=coeffs, precision="fp32")
            ev[2 * k + 1].record()
        t1.record()
        torch.cuda.synchronize()
        clk = clocks.stop()
        assert F.status_poll() == 0
        t = t0.elapsed_time(t1) / 1e3 / args.steps
        t_k = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps)) / 1e3 / args.steps
        # algorithmic bytes of one assembly: cells, vertices, f on each cell, dof map, and
        # the global vector read and written once
        byts = m.n_elem * (16 + 8 * n + 4 * n) + m.n_vert * 24 + 16 * p.n_dof
        detail["fp64_flops_per_s"] = 2.0 * n * n * m.n_elem / (detail["assemble_fp64_ms"] / 1e3)
        rate, S = (None, 0) if args.no_cpu_baseline else _oracle_rate(W.SOURCE, 4, M.gather_cell_vertices(m),
                                                                       p.coeffs, cores)
        out.update({"metric": "element vectors/s (source form P4, 48^3x6 tets, zero + assemble into b)",
                    "value": m.n_elem / t, "ms_per_step": t * 1e3, "dtype": "f32",
                    "config": {"workload": "source_p4", "cells": m.n_elem, "n_dof": p.n_dof,
                               "l2": "inputs 0.29 GB per step > L2"},
                    "roofline": {"bound": "hbm", "achieved": byts / t_k / 1e9, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": byts / t_k / 1e9 / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                                 "kernel": "simt_tabulate_kernel<3,SOURCE,4,float,assemble>",
                                 "kernel_ms": t_k * 1e3},
                    "clocks": clk, "gpu_launches": 2 * args.steps,
                    "cpu_baseline": {"value": rate, "unit": "elem/s", "cores": cores, "kind": "oracle",
                                     "sample": f"{S} cells"}, "detail": detail})
    elif workload == "quad_curved":
        # quadrature as a tensor contraction (Section 3.4): P2 Poisson on 40^3 x 6 curved
        # (quadratic-geometry) tets, A~0 with a point index contracted with per-point G~_K;
        # plus the same contraction on the affine cells of the headline mesh against the
        # tensor representation (the paper's T_Q / T_T comparison, here on the GPU)
        from synthetic import curved as CV

        cm = CV.curved_mesh(3, 40 if args.n == 48 else args.n, eps=0.08)
        cells = torch.as_tensor(cm.cells, device=device)
        nodes = torch.as_tensor(cm.nodes, device=device)
        qf = F.QForm(F.POISSON, F.TETRAHEDRON, 2, 2)
        n = qf.n_local
        detail = {"points": qf.n_points, "k_contract": qf.k_contract, "quad_degree": qf.quad_degree}
        A64 = torch.empty((cm.n_elem, n, n), dtype=torch.float64, device=device)
        detail["tabulate_fp64_ms"] = _timed(lambda: F.tabulate_quadrature(qf, cells, nodes, "fp64", out=A64),
                                            args.steps, args.warmup) * 1e3
        # FP64 by exact digit products on the tensor cores (Ozaki-style splitting)
        B64 = torch.empty_like(A64)
        t_oz = _timed(lambda: F.tabulate_quadrature(qf, cells, nodes, "fp64_ozaki", out=B64), args.steps, args.warmup)
        assert F.status_poll() == 0
        d_oz = (B64 - A64).reshape(cm.n_elem, -1).norm(dim=1) / A64.reshape(cm.n_elem, -1).norm(dim=1)
        oz_pieces = -(-qf.k_contract // 48) * 3
        detail["fp64_ozaki"] = {"ms": t_oz * 1e3, "max_rel_diff_vs_fp64": float(d_oz.max()),
                                "speedup_vs_fp64": detail["tabulate_fp64_ms"] / (t_oz * 1e3),
                                "bf16_digit_products_tflops": 36 * 2.0 * 128 * 64 * 16 * oz_pieces
                                * (-(-cm.n_elem // 64)) / t_oz / 1e12}
        del B64
        A32 = torch.empty((cm.n_elem, n, n), dtype=torch.float32, device=device)
        pk = compute_peaks(F)

        def max_rel(A):
            d = (A.double() - A64).reshape(cm.n_elem, -1).norm(dim=1) / A64.reshape(cm.n_elem, -1).norm(dim=1)
            return float(d.max())

        # the SIMT FP32 contraction and the tensor-core ones; the headline is 3xTF32 (FP32
        # accuracy; the worst cell's relative error against the FP64 result is recorded)
        t32 = _timed(lambda: F.tabulate_quadrature(qf, cells, nodes, "fp32", out=A32), args.steps, args.warmup)
        assert F.status_poll() == 0
        flops32 = 2.0 * n * n * qf.k_contract * cm.n_elem  # executed by the SIMT kernel (all n^2 entries)
        detail["simt_fp32"] = {"ms": t32 * 1e3, "max_rel_err_vs_fp64": max_rel(A32),
                               "tflops": flops32 / t32 / 1e12, "fp32_fma_frac": flops32 / t32 / 1e12 / pk["fp32_fma"]}
        for prec in ("tf32", "bf16x3"):
            tp = _timed(lambda: F.tabulate_quadrature(qf, cells, nodes, prec, out=A32), args.steps, args.warmup)
            assert F.status_poll() == 0
            detail[prec] = {"ms": tp * 1e3, "max_rel_err_vs_fp64": max_rel(A32)}
        clocks.start()
        t = _timed(lambda: F.tabulate_quadrature(qf, cells, nodes, "tf32x3", out=A32), args.steps, args.warmup)
        clk = clocks.stop()
        assert F.status_poll() == 0
        detail["tf32x3_max_rel_err_vs_fp64"] = max_rel(A32)
        del A64, A32
        # P3 (400 entries: four 128-entry M tiles on the tensor cores), FP32 on CUDA cores
        # against the tensor-core splits, worst cell against FP64
        q3 = F.QForm(F.POISSON, F.TETRAHEDRON, 3, 2)
        B64 = F.tabulate_quadrature(q3, cells, nodes, "fp64")
        B32 = torch.empty((cm.n_elem, 20, 20), dtype=torch.float32, device=device)
        p3 = {}
        for prec in ("fp32", "tf32x3", "bf16x3"):
            tp = _timed(lambda: F.tabulate_quadrature(q3, cells, nodes, prec, out=B32), args.steps, 1)
            assert F.status_poll() == 0
            d3 = (B32.double() - B64).reshape(cm.n_elem, -1).norm(dim=1) / B64.reshape(cm.n_elem, -1).norm(dim=1)
            p3[prec] = {"ms": tp * 1e3, "max_rel_err_vs_fp64": float(d3.max())}
        detail["poisson_p3"] = p3
        del B64, B32
        # algorithmic FLOPs of the contraction (one product, n^2 entries) and those the
        # tensor cores execute (128-entry M tiles, K padded to 48-column chunks, 3 products)
        flops_alg = 2.0 * n * n * qf.k_contract * cm.n_elem
        n_tiles = -(-cm.n_elem // 128)
        flops_exec = 3 * 2.0 * 128 * 128 * (-(-qf.k_contract // 48) * 48) * n_tiles
        flops64 = 2.0 * n * (n + 1) / 2 * qf.k_contract * cm.n_elem  # FP64 kernel: entries i1 <= i2
        detail["fp64_tflops"] = flops64 / (detail["tabulate_fp64_ms"] / 1e3) / 1e12
        detail["fp64_frac"] = detail["fp64_tflops"] / pk["fp64_fma"]
        detail["tf32x3_executed_tflops"] = flops_exec / t / 1e12
        detail["tf32x3_executed_frac"] = flops_exec / t / 1e12 / pk["tf32_mma"]
        byts = cm.n_elem * (4 * qf.n_geometry + 4 * n * n) + cm.nodes.size * 8
        # T_Q / T_T on affine cells: the headline mesh, mass and Poisson P1-P3
        m = W.tet_scalar_mesh(40)
        ca, va = torch.as_tensor(m.cells, device=device), torch.as_tensor(m.vertices, device=device)
        ratio = {}
        for form in (F.MASS, F.POISSON):
            for q in (1, 2, 3):
                f = F.Form(form, F.TETRAHEDRON, q)
                qa = F.QForm(form, F.TETRAHEDRON, q, 1, 2 * q)
                A = torch.empty((m.n_elem, f.n_local, f.n_local), dtype=torch.float32, device=device)
                tt = _timed(lambda: F.tabulate(f, ca, va, precision="fp32", out=A), args.steps, 1)
                tq = _timed(lambda: F.tabulate_quadrature(qa, ca, va, precision="fp32", out=A), args.steps, 1)
                ratio[f"{FORM_NAME[form]}_p{q}"] = {"tensor_ms": tt * 1e3, "quadrature_ms": tq * 1e3,
                                                    "TQ_over_TT": tq / tt}
                if f.n_local ** 2 <= 128:  # the quadrature contraction on the tensor cores (3xTF32)
                    tc = _timed(lambda: F.tabulate_quadrature(qa, ca, va, precision="tf32x3", out=A), args.steps, 1)
                    ratio[f"{FORM_NAME[form]}_p{q}"].update({"quadrature_tf32x3_ms": tc * 1e3,
                                                             "TQ_tf32x3_over_TT": tc / tt})
                del A
        detail["affine_fp32_T_Q_over_T_T"] = ratio
        cpu_rate, S = None, 0
        if not args.no_cpu_baseline:
            import multiprocessing as mp
            pool = mp.get_context("spawn").Pool(cores)
            S = min(cm.n_elem, 400 * cores)
            X = CV.gather_nodes(cm)[np.linspace(0, cm.n_elem - 1, S).astype(np.int64)]
            t0 = time.perf_counter()
            pool.map(_oracle_curved, [(X[c::cores], qf.quad_degree) for c in range(cores)])
            cpu_rate = S / (time.perf_counter() - t0)
            pool.close()
            pool.join()
        out.update({"metric": "element tensors/s (P2 Poisson on 40^3x6 curved tets, quadrature as contraction)",
                    "value": cm.n_elem / t, "ms_per_step": t * 1e3, "dtype": "tf32x3",
                    "config": {"workload": "quad_curved_p2_40", "cells": cm.n_elem, "geometry_degree": 2,
                               "l2": "output 154 MB per step > L2"},
                    "roofline": {"bound": "tensor", "achieved": flops_alg / t / 1e12, "peak": pk["tf32_mma"],
                                 "unit": "TFLOP/s", "frac": flops_alg / t / 1e12 / pk["tf32_mma"],
                                 "peak_kind": "measured (ffc_diag_peak TF32 tcgen05 MMA, this run)", "traffic": None,
                                 "hbm_gbs": byts / t / 1e9, "kernel": "tq_kernel<3, POISSON, 2, TF32X3>"},
                    "clocks": clk, "gpu_launches": args.steps,
                    "cpu_baseline": {"value": cpu_rate, "unit": "elem/s", "cores": cores, "kind": "oracle",
                                     "sample": f"{S} curved cells, point-by-point quadrature"},
                    "detail": detail})
    elif workload == "rows":
        # the headline's eight problems, every degree by the row-owner assembly: mass and
        # Poisson in one ffc_assemble_rows_pair launch per degree (fixed-point sums, every
        # CSR value written once, no atomics and no zeroing)
        mesh = W.tet_scalar_mesh(args.n)
        cells = torch.as_tensor(mesh.cells, device=device)
        verts = torch.as_tensor(mesh.vertices, device=device)
        probs = []
        for q in DEGREES:
            p = W.make_problem(mesh, W.POISSON, q)
            row_ptr, col, _ = F.csr_pattern(p.dofmap, p.n_dof, with_slots=False)
            plan = F.RowPlan(torch.as_tensor(p.dofmap, device=device), p.n_dof,
                             torch.as_tensor(row_ptr, device=device), torch.as_tensor(col, device=device))
            del col
            probs.append({"q": q, "plan": plan, "n_local": p.n_local, "nnz": plan.nnz,
                          "F": (F.Form(F.MASS, F.TETRAHEDRON, q), F.Form(F.POISSON, F.TETRAHEDRON, q)),
                          "val": [torch.empty(plan.nnz, dtype=torch.float64, device=device) for _ in FORMS]})
        P = len(probs)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(P * args.steps)]

        def rows_step(s=None):
            for k, pr in enumerate(probs):
                if s is not None:
                    ev[s * P + k][0].record()
                F.assemble_rows_pair(pr["F"][0], pr["F"][1], pr["plan"], cells, verts, pr["val"][0], pr["val"][1],
                                     precision=args.precision)
                if s is not None:
                    ev[s * P + k][1].record()

        for _ in range(args.warmup):
            rows_step()
        torch.cuda.synchronize()
        clocks.start()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for s_ in range(args.steps):
            rows_step(s_)
        t1.record()
        torch.cuda.synchronize()
        clk = clocks.stop()
        assert F.status_poll() == 0
        t = t0.elapsed_time(t1) / 1e3 / args.steps
        per = [sum(ev[s_ * P + k][0].elapsed_time(ev[s_ * P + k][1]) for s_ in range(args.steps)) / 1e3 / args.steps
               for k in range(P)]
        dom = int(np.argmax(per))
        dpr = probs[dom]
        # algorithmic bytes of one row-owner pair launch: cells, vertices, the dof-map
        # equivalent (4n per cell) and the two matrices' CSR values written once
        byts = mesh.n_elem * (16 + 4 * dpr["n_local"]) + mesh.n_vert * 24 + 2 * 8 * dpr["nnz"]
        cpu = None
        if not args.no_cpu_baseline:
            pool, _ = oracle_pool()
            S, t_cpu = cpu_oracle_step(args.n, REF_FRACTION, pool)
            pool.close()
            pool.join()
            cpu = {"value": 2 * P * S / t_cpu, "unit": "elem/s", "cores": cores, "kind": "oracle",
                   "sample": f"{S} cells of each of the 8 problems, element tensors and Algorithm 2, {t_cpu:.1f} s"}
        out.update({"metric": "element tensors/s (row-owner assembly, mass+Poisson P1..P4 on 48^3x6 tets)",
                    "value": 2 * P * mesh.n_elem / t, "ms_per_step": t * 1e3,
                    "dtype": "f32" if args.precision != "fp64" else "f64",
                    "config": {"workload": f"tet_scalar_{args.n}_rows", "cells": mesh.n_elem,
                               "problems": [f"mass+poisson_p{p_['q']}" for p_ in probs],
                               "csr_accumulation": "fixed point in shared memory (42-bit for FP32 contributions, "
                                                   "63-bit for FP64), rounded once to f64",
                               "l2": "inputs larger than L2: ~12 GB of positions and CSR values per step"},
                    "roofline": {"bound": "hbm", "achieved": byts / per[dom] / 1e9, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": byts / per[dom] / 1e9 / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                                 "kernel": f"rows_assemble mass+Poisson P{dpr['q']}",
                                 "launch_ms": per[dom] * 1e3},
                    "per_launch_ms": {f"mass+poisson_p{p_['q']}": round(per[k] * 1e3, 4)
                                      for k, p_ in enumerate(probs)},
                    "clocks": clk, "gpu_launches": 2 * P * args.steps, "cpu_baseline": cpu})
    else:  # adjoint
        p, u, v = W.adjoint_p2(56 if args.n == 48 else args.n)
        m = p.mesh
        cells = torch.as_tensor(m.cells, device=device)
        verts = torch.as_tensor(m.vertices, device=device)
        dm = torch.as_tensor(p.dofmap.astype(np.int64), device=device)
        uK = torch.as_tensor(u, device=device)[dm]
        vK = torch.as_tensor(v, device=device)[dm]
        dA = torch.einsum("ei,ej->eij", uK, vK).contiguous()
        fm = F.Form(F.POISSON, F.TETRAHEDRON, 2)
        fp64_peak = compute_peaks(F)["fp64_fma"]
        dv = torch.zeros_like(verts)
        A = torch.empty((m.n_elem, 10, 10), dtype=torch.float64, device=device)
        t_fwd = _timed(lambda: F.tabulate(fm, cells, verts, out=A), args.steps, args.warmup)
        clocks.start()
        t = _timed(lambda: F.tabulate_adjoint(fm, cells, verts, dA, dvertices=dv), args.steps, args.warmup)
        clk = clocks.stop()
        assert F.status_poll() == 0
        byts = m.n_elem * (16 + 800 + 12 * 8) + m.n_vert * 24 * 2
        # executed FP64 flops per cell: 6 symmetric combinations x 100 entries (FMA = 2),
        # plus about 240 for J^{-1}, det J and the chain rule
        flops = m.n_elem * (2 * 100 * 6 + 240)
        cpu_rate, S = None, 0
        if not args.no_cpu_baseline:
            import multiprocessing as mp
            pool = mp.get_context("spawn").Pool(cores)
            S = min(m.n_elem, 20000 * cores)
            sel = np.linspace(0, m.n_elem - 1, S).astype(np.int64)
            chunks = [(m.vertices, m.cells[sel[c::cores]], p.dofmap[sel[c::cores]], u, v) for c in range(cores)]
            t0 = time.perf_counter()
            pool.map(_oracle_shape, chunks)
            cpu_rate = S / (time.perf_counter() - t0)
            pool.close()
            pool.join()
        out.update({"metric": "element adjoints/s (P2 Poisson dL/dvertices, 56^3x6 tets)",
                    "value": m.n_elem / t, "ms_per_step": t * 1e3, "dtype": "f64",
                    "config": {"workload": "adjoint_p2", "cells": m.n_elem, "vertices": m.n_vert},
                    "roofline": {"bound": "alu", "achieved": flops / t / 1e12, "peak": fp64_peak,
                                 "unit": "TFLOP/s", "frac": flops / t / 1e12 / fp64_peak,
                                 "peak_kind": "measured (ffc_diag_peak FP64 FMA, this run)", "traffic": None,
                                 "hbm_gbs": byts / t / 1e9, "hbm_frac": byts / t / 1e9 / hbm_peak,
                                 "kernel": "poisson_adjoint_kernel<3,2>"},
                    "clocks": clk, "gpu_launches": args.steps,
                    "cpu_baseline": {"value": cpu_rate, "unit": "elem/s", "cores": cores, "kind": "oracle",
                                     "sample": f"{S} cells, continuous shape derivative"},
                    "detail": {"forward_tabulate_fp64_ms": t_fwd * 1e3}})
    return out


def _oracle_curved(args):
    X, p = args
    from oracle import curved as OC

    OC.element_tensors_curved(OC.POISSON, X, 2, 2, p)
    return X.shape[0]


def _oracle_shape(args):
    verts, cells, dofmap, u, v = args
    from oracle import shape as OS

    OS.poisson_shape_gradient(verts, cells, 2, dofmap, u, v)
    return cells.shape[0]


if __name__ == "__main__":
    sys.exit(main())
