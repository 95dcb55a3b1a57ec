#!/usr/bin/env python
"""Benchmark of the periodic piezoelectric cell solve on GB300.

One step = the whole hot path for one design: the design mapped into the
handle from a nodal level set on the device (ersatz rho, multigrid
hierarchies), the nine right-hand sides, SCP-GMRES (FP32 Krylov and multigrid
inside FP64 iterative refinement) to the residual tolerance, null-space
projection, the homogenised C^H, e^H, kappa^H (FP64 energy form) and the
element sensitivities of the hydrostatic coefficient d_h.

Workload (default): a 128^3 unit cell (8,388,608 dof, 9 loads), PZT-5H-class
base material, seeded level sets (sum of 8 periodic Gaussians).  The
tolerance is chosen so that C^H/e^H/kappa^H meet 1e-8 and the d_h
sensitivities 1e-5 relative error; both are measured after the timed region
against FP64 solves of the same designs to 1e-12 and reported.  The same
designs are also solved by the plain FP64 GPU path at the same tolerance and
timed.  Working set: several GB (Krylov basis, multigrid levels, FP64
vectors), far above the 129 MB L2; a 256 MB buffer is also rewritten between
timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 64]

Multi-GPU (torchrun, one rank per GPU): independent designs per rank
(replicas, no collective on the data path); value = total time / total cells.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

# The CPU oracle (reference arm and cpu_baseline) is timed on one host core:
# pin the BLAS thread pools before numpy is first imported, so that the
# reported core count is the one used.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-solve time to C^H at 1e-8 rel err; DOF·RHS/s per apply vs HBM roofline"

# Algorithmic cost per (node, load) of each timed kernel class of the library:
# (flops, bytes, bound, dtype, dof per node).  Bytes count one read of every
# input and one write of every output.
CLASS_COST = {
    "full32": (2 * (1024 + 32), 4 * 4 + 4 * 4 + 4 / 9, "alu", "f32", 4),
    "full64": (2 * (1024 + 32), 8 * 4 + 8 * 4 + 8 + 8 / 9, "alu", "f64", 4),
    "elastic0": (2 * (576 + 24), 4 * (3 + 2 * 3 + 2 * 3 + 3) + 4 * 3 / 9 + 4 / 9, "alu", "f32", 3),
    "schur0": (2 * (64 + 8), 4 * (1 + 2 + 2 + 1) + 4 / 9 + 4 / 9, "hbm", "f32", 1),
    "coupling": (2 * (192 + 8), 4 * (3 + 1 + 1) + 4 / 9, "alu", "f32", 3),
}
# The tensor-core smoothers (node-centric TF32 MMAs): each (node, load) row
# takes 15 MMAs of K = 8 against N = 32 columns, 2 x 120 x 32 flops; their
# algorithmic bytes are those of the class above, which bound them (the MMA
# work at the TF32 rate takes less time than the bytes at the HBM rate).
TC_FLOPS_PER_ROW = 2 * 120 * 32
# Algorithmic bytes per dof and load of the plain FP32 operator apply
# (read x, write y, rho amortised over 4 dof x 9 loads)
APPLY_BYTES_PER_DOF_RHS = 4 + 4 + 4 / 36
# Oracle sizes timed for the CPU baseline (a few seconds to ~10 s each on one core)
ORACLE_SIZES = (8, 12, 16)


def unit_for(n):
    return f"ms per {n}^3 cell solve (9 loads, setup+solve+C^H+d_h sensitivities)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    # residual tolerance of the solves: C^H at 1e-8 needs far less (the energy
    # form's error is quadratic in the solve error); the element sensitivities
    # are linear in it and set the tolerance (1e-5 relative at 128^3)
    ap.add_argument("--tol", type=float, default=2e-8)
    ap.add_argument("--inner-tol", type=float, default=1e-4)
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--accuracy-designs", type=int, default=2)
    # fine-grid smoothers on the tensor cores (node-centric tcgen05 TF32 kernels)
    ap.add_argument("--tensor-cores", type=int, default=1, choices=[0, 1, 2])
    # E1 benchmark of the paper's weak-scaling study instead of the headline step
    ap.add_argument("--e1", action="store_true")
    # batched uneven cells (16 each of 32^3, 48^3, 64^3) instead of the headline step
    ap.add_argument("--batch", action="store_true")
    return ap.parse_args()


def rank_seeds(rank, ndes):
    """Design seeds of one rank: disjoint across ranks (replicas solve
    independent designs, no data-path collective)."""
    return [rank * 1000 + s for s in range(ndes)]


def job_ms_per_cell(total_ms, steps, world, dist=None):
    """Whole-job figure from one rank's timed region: the slowest rank's time
    (max over ranks) for all steps x world cells."""
    if world > 1 and dist is not None:
        import torch
        t = torch.tensor([float(total_ms)], dtype=torch.float64,
                         device="cuda" if dist.get_backend() == "nccl" else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, total_ms / (steps * world)


def traffic_table():
    """DRAM bytes per (node, load) of the kernel classes from ncu captures
    (profiles/traffic.json); a class whose kernel changed since has no entry."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return {}
    with open(p) as f:
        return {k: v for k, v in json.load(f).items() if not k.startswith("_") and v}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured", d.get("sm_max_mhz", 2070.0)
    return 6800.0, "fallback", 2070.0


def peaks_tf32():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f).get("bf16_tflops", 1900.0) / 2.0
    return 1900.0 / 2.0


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        loaded = [s for s in sm if s > 500] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_step(n, seed):
    """The FP64 CPU oracle on one n^3 design: ersatz, assembly, direct solve,
    energy-form homogenisation and the d_h element sensitivities."""
    import cellgen
    from oracle import ersatz, fem, figures, sensitivity
    mat = cellgen.pzt5h_class()
    phi = cellgen.gaussian_levelset(n, seed=seed)
    rho = ersatz.rho_from_levelset(phi)
    P = fem.CellProblem(rho, *mat)
    y = P.solve()
    H, _ = P.homogenise(y)
    Ch, eh, kh = P.tensors(H)
    dC, de = figures.d_h_grad(Ch, eh)
    sensitivity.grad_rho(P, y, sensitivity.G_from_si(dC, de, 0 * kh, P.sc))
    return Ch


def oracle_fit(points, n_target):
    """Least-squares fit t = c * dof^p to measured oracle steps (n, seconds)
    and its extrapolation to an n_target^3 cell (ms).  The direct solve's fill
    grows faster than the dof count, so p > 1; with one size only p = 1."""
    xs = [math.log(4 * n ** 3) for n, _ in points]
    ys = [math.log(t) for _, t in points]
    if len(set(xs)) < 2:
        p = 1.0
        c = statistics.mean(ys) - xs[0]
    else:
        mx, my = statistics.mean(xs), statistics.mean(ys)
        p = sum((x - mx) * (y - my) for x, y in zip(xs, ys)) / sum((x - mx) ** 2 for x in xs)
        c = my - p * mx
    return math.exp(c + p * math.log(4 * n_target ** 3)) * 1e3, p


def oracle_baseline(n_target, steps=None, seed0=0):
    """Shared by cpu_baseline and the reference arm: time the oracle at the
    ORACLE_SIZES (cycled over `steps` samples), fit the growth exponent and
    extrapolate to the workload's size."""
    steps = len(ORACLE_SIZES) if steps is None else steps
    pts = []
    for k in range(steps):
        n = ORACLE_SIZES[k % len(ORACLE_SIZES)]
        t0 = time.perf_counter()
        oracle_step(n, seed0 + k)
        pts.append((n, time.perf_counter() - t0))
    ms, p = oracle_fit(pts, n_target)
    timed = sum(t for _, t in pts)
    per_size = {f"{n}^3": round(min(t for m, t in pts if m == n), 3) for n in sorted({n for n, _ in pts})}
    sample = (f"FP64 oracle (sparse assembly + SuperLU direct solve + energy form + d_h sensitivities, "
              f"one thread) timed on {steps} seeded cells of sizes {sorted({n for n, _ in pts})} "
              f"(s per cell: {per_size}; {timed:.1f} s in total); time = c * dof^p fitted "
              f"(p = {p:.2f}) and extrapolated to {n_target}^3")
    return ms, p, pts, timed, sample


def workload_config(args, world):
    """The workload keys both arms report (the GPU arm adds its timing notes)."""
    n = args.n
    return {"workload": f"{n}^3 periodic piezoelectric cell ({4 * n ** 3} dof), 9 loads, "
                        "seeded Gaussian level sets, PZT-5H-class",
            "tol": args.tol, "inner_tol": args.inner_tol, "tensor_cores": args.tensor_cores,
            "precision": args.precision, "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for w in range(args.warmup):
        oracle_step(ORACLE_SIZES[0], 100 + w)
    ms, p, pts, timed, sample = oracle_baseline(args.n, steps=args.steps)
    unit = unit_for(args.n)
    line = {
        "impl": "reference", "metric": METRIC, "value": ms, "unit": unit, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {**workload_config(args, int(os.environ.get("WORLD_SIZE", "1"))),
                   "l2": "host cores: FP64 direct solves, no GPU"},
        "cpu_baseline": {"value": ms, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample,
                         "extrapolated": True, "fit_exponent": p, "timed_region_s": timed,
                         "points_s": [[n, t] for n, t in pts]},
        "e2e": {"value": ms, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_e1(args):
    """E1 benchmark (§2.5.4, Table 1): level set -prod cos(2 pi x_i) - 0.2, the
    single load eps_bar^(11), outer tolerance 1e-8; SCP and DBP, FP64 and mixed,
    1 and 2 V-cycles per block.  Prints one JSON line per configuration with
    the GMRES iterations and the solve time (CUDA events around cell_solve)."""
    import torch
    import cellgen
    from paper_2410_03148_gb300 import Cell, load
    load()
    dev = torch.device("cuda", 0)
    mat = cellgen.pzt5h_class()
    n = args.n
    phi = torch.as_tensor(cellgen.e1_levelset(n), device=dev)
    stream = torch.cuda.current_stream(dev)
    for prec in (1, 0):
        for pc in (0, 1):
            for vc in (1, 2):
                cell = Cell(phi, mat, kind="phi", precision=prec, precond=pc, load_mask=1, tol=1e-8,
                            vcycles_u=vc, vcycles_phi=vc, tensor_cores=args.tensor_cores, max_iter=4000)
                cell.solve()                   # warm-up (graph capture, first-touch)
                ms = []
                for _ in range(2):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    st = cell.solve()
                    e1.record(stream)
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
                print(json.dumps({"workload": f"E1 {n}^3 ({4 * n ** 3} dof), load eps11, tol 1e-8",
                                  "precision": "mixed" if prec else "fp64",
                                  "precond": "SCP" if pc == 0 else "DBP", "vcycles": vc,
                                  "gmres_iters": st["iters"][0], "refinements": st["refinements"],
                                  "rel_residual": st["rel_residual"][0], "solve_ms": min(ms)}), flush=True)
                cell.close()
                torch.cuda.empty_cache()


def run_batch(args):
    """Batched uneven cells: 48 seeded designs (16 each of 32^3, 48^3, 64^3), 9
    loads each, mixed precision at the bench tolerance, solved by one
    cell_solve_batch call: all 48 solves as branches of one CUDA graph (one
    launch); against the same designs with one graph launch per handle on its
    own stream, the same handles solved one after another, and one-by-one FP64
    solves.  Prints one JSON line with the wall times (synchronised, host
    clock, best of three for the batched forms)."""
    import numpy as np
    import torch
    import cellgen
    from paper_2410_03148_gb300 import Cell, load, solve_batch
    load()
    dev = torch.device("cuda", 0)
    mat = cellgen.pzt5h_class()
    sizes = [32] * 16 + [48] * 16 + [64] * 16
    phis = [torch.as_tensor(cellgen.gaussian_levelset(n, seed=s), device=dev) for s, n in enumerate(sizes)]
    opt = dict(tol=args.tol, inner_tol=args.inner_tol, tensor_cores=args.tensor_cores)

    def timed_batches(graphs):
        cells = []
        for phi in phis:
            with torch.cuda.stream(torch.cuda.Stream(dev)):
                cells.append(Cell(phi, mat, kind="phi", precision=1, graphs=graphs, **opt))
        torch.cuda.synchronize()
        solve_batch(cells)             # warm-up: graph capture
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(3):
            t0 = time.perf_counter()
            sts = solve_batch(cells)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        return cells, sts, best

    cells3, _, t_streams = timed_batches(3)
    H3 = [c.homogenise() for c in cells3]
    for c in cells3:
        c.close()
    del cells3
    cells, sts, t_batch = timed_batches(2)
    t0 = time.perf_counter()
    for c in cells:
        c.solve()
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    H = [c.homogenise() for c in cells]
    same = all(all(np.array_equal(a, b) for a, b in zip(h, h3)) for h, h3 in zip(H, H3))
    for c in cells:
        c.close()
    del cells
    torch.cuda.empty_cache()
    t64 = 0.0
    err = 0.0
    for phi, h in zip(phis, H):
        c = Cell(phi, mat, kind="phi", precision=0, tol=args.tol, max_iter=4000)
        c.solve()                      # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c.solve()
        torch.cuda.synchronize()
        t64 += time.perf_counter() - t0
        for a, b in zip(h, c.homogenise()):
            err = max(err, float(np.abs(a - b).max() / np.abs(b).max()))
        c.close()
    print(json.dumps({"workload": "48 designs: 16 each of 32^3, 48^3, 64^3 (seeds 0-47), 9 loads, mixed",
                      "tol": args.tol, "batch_one_graph_s": t_batch, "designs_per_s": len(sizes) / t_batch,
                      "batch_graph_per_handle_s": t_streams, "sequential_s": t_seq, "fp64_one_by_one_s": t64,
                      "batch_speedup_vs_sequential": t_seq / t_batch, "batch_speedup_vs_fp64": t64 / t_batch,
                      "one_graph_equals_per_handle_bitwise": same,
                      "max_iters": max(max(st["iters"]) for st in sts),
                      "CH_eH_kH_block_rel_vs_fp64": err}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.e1:
        run_e1(args)
        return
    if args.batch:
        run_batch(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import cellgen
    from paper_2410_03148_gb300 import Cell, dh, load
    from paper_2410_03148_gb300 import _binding as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    load()
    mat = cellgen.pzt5h_class()
    n = args.n
    prec = 1 if args.precision == "mixed" else 0
    ndes = 8
    designs = [torch.as_tensor(cellgen.gaussian_levelset(n, seed=sd), device=dev)
               for sd in rank_seeds(rank, ndes)]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    # One handle per process (all device memory allocated here, once); every
    # step maps a new design into it (cell_update: rho_e and the multigrid
    # hierarchy, S1) and runs S2-S9 on it, as an optimisation loop does.
    # Handle 1 times every kernel class (class shares, untimed pass); handle 2
    # times only the dominant class inside the timed region (its roofline).
    sopt = dict(tol=args.tol, inner_tol=args.inner_tol, tensor_cores=args.tensor_cores)
    cells = {0: Cell(designs[0], mat, kind="phi", precision=prec, **sopt),
             1: Cell(designs[0], mat, kind="phi", precision=prec, profile=1, **sopt)}

    def step(phi, profile=0):
        cell = cells[profile]
        cell.update(phi)
        st = cell.solve()
        Ch, eh, kh = cell.homogenise()
        d, dC, de = dh(Ch, eh)
        g = cell.sensitivity(dC, de, None, dtype=torch.float32)
        return st, (Ch, eh, kh), g

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for w in range(args.warmup):
        step(designs[w % ndes])
    # class shares from a fully profiled pass over the timed designs (untimed)
    shares = [step(designs[k % ndes], profile=1)[0] for k in range(min(args.steps, 2))]
    share_ms = {c: sum(s_["class_ms"][c] for s_ in shares) / len(shares) for c in B.PROF_CLASSES}
    dom = max((c for c in CLASS_COST), key=lambda c: share_ms[c])
    cells[2] = Cell(designs[0], mat, kind="phi", precision=prec, profile=1,
                    profile_mask=1 << B.PROF_CLASSES.index(dom), **sopt)
    step(designs[0], profile=2)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    stats = []
    step_ms = []
    outputs = {}
    launches0 = B.cell_launch_count()
    stream = torch.cuda.current_stream(dev)
    t_start = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, tens, g = step(designs[k % ndes], profile=2)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        stats.append(st)
        outputs[k % ndes] = (tens, g)
    barrier()
    wall = time.perf_counter() - t_start
    launches = B.cell_launch_count() - launches0
    clocks = sampler.stop()
    total_ms, ms_per_cell = job_ms_per_cell(sum(step_ms), args.steps, world, dist if world > 1 else None)
    unit = unit_for(n)

    # roofline of the dominant kernel class, from the live CUDA events
    hbm, hbm_kind, sm_max = peaks()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    tot = {c: sum(s["class_ms"][c] for s in stats) for c in B.PROF_CLASSES}
    cnt = {c: sum(s["class_count"][c] for s in stats) for c in B.PROF_CLASSES}
    units = {c: sum(s["class_units"][c] for s in stats) for c in B.PROF_CLASSES}
    flops_u, bytes_u, bound, kdt, ndof = CLASS_COST[dom]
    tc_class = args.tensor_cores >= 1 and prec == 1 and dom in ("elastic0", "schur0")
    if tc_class:
        bound = "hbm"
    nn = n ** 3
    avg_ms = tot[dom] / max(cnt[dom], 1)
    per_launch_units = units[dom] / max(cnt[dom], 1)
    fp32_peak = nsm * 128 * 2 * sm_max * 1e6 / 1e12           # TFLOP/s, FP32 FMA lanes
    fp64_peak = 1.25 * sm_max / 2070.0                        # TFLOP/s, nominal FP64 rate
    alg_bytes = bytes_u * nn * per_launch_units
    if bound == "hbm":
        achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": None}
    else:
        achieved = flops_u * nn * per_launch_units / (avg_ms * 1e-3) / 1e12
        peak = fp32_peak if kdt == "f32" else fp64_peak
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None}
    tt = traffic_table().get(dom)
    if tt and tt.get("bytes_per_node_load"):
        roof["traffic"] = tt["bytes_per_node_load"] * nn * per_launch_units
        roof["traffic_source"] = (f"ncu dram__bytes_read+write of one {tt.get('n')}^3 launch "
                                  f"({tt.get('profile')}), per node and load, scaled to this launch")
    if tc_class:
        # tensor-pipe view: MMA flops per launch (the Schur kernel packs four loads per row)
        rows = nn * per_launch_units / (4 if dom == "schur0" else 1)
        tf32_peak = peaks_tf32()
        roof["tensor_view"] = {"mma_tflops": TC_FLOPS_PER_ROW * rows / (avg_ms * 1e-3) / 1e12,
                               "tf32_peak_tflops": tf32_peak,
                               "frac": TC_FLOPS_PER_ROW * rows / (avg_ms * 1e-3) / 1e12 / tf32_peak,
                               "peak_source": "measured bf16 burst (MEASURED_PEAKS.json) / 2, the nominal TF32 ratio"}
    dof_rate = ndof * nn * per_launch_units / (avg_ms * 1e-3)
    roof.update({"kernel": dom,
                 "peak_source": (f"hbm {hbm_kind} (MEASURED_PEAKS.json)" if bound == "hbm" else
                                 f"{nsm} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz"),
                 "launches": cnt[dom], "avg_launch_ms": avg_ms, "loads_per_launch": per_launch_units,
                 "algorithmic_bytes_per_launch": alg_bytes,
                 "hbm_frac_of_algorithmic_bytes": alg_bytes / (avg_ms * 1e-3) / 1e9 / hbm,
                 "dof_per_node": ndof,
                 "dof_rhs_per_s": dof_rate,
                 "dof_rhs_per_s_apply_roofline": hbm * 1e9 / APPLY_BYTES_PER_DOF_RHS,
                 "dof_rhs_per_s_frac_of_apply_roofline": dof_rate / (hbm * 1e9 / APPLY_BYTES_PER_DOF_RHS)})
    step_avg = total_ms / args.steps
    class_share = {c: round(share_ms[c] / max(step_avg, 1e-9), 4) for c in B.PROF_CLASSES}

    # accuracy of the timed results (untimed): against FP64 solves to 1e-12 of
    # the same designs (the FP64 path is pinned to the oracle at small sizes and
    # to the laminate closed form at any size)
    def errors(tens, g, R, gr):
        blk = ent = 0.0
        for a, b in zip(tens, R):
            blk = max(blk, float(np.abs(a - b).max() / np.abs(b).max()))
            m = np.abs(b) > 1e-6 * np.abs(b).max()
            ent = max(ent, float((np.abs(a - b)[m] / np.abs(b)[m]).max()))
        grad = float(np.abs(g.double().cpu().numpy() - gr).max() / np.abs(gr).max())
        return blk, ent, grad

    # the plain FP64 GPU solve of the same designs at the same tolerance (timed
    # like the mixed step, outside the headline's timed region)
    fp64 = None
    fp64_out = {}
    if not args.no_fp64 and prec == 1:
        c64 = Cell(designs[0], mat, kind="phi", precision=0, tol=args.tol, max_iter=4000)
        cells[3] = c64
        step(designs[0], profile=3)
        t64 = []
        for k in range(min(args.steps, 2)):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st64, tens64, g64 = step(designs[k % ndes], profile=3)
            e1.record(stream)
            e1.synchronize()
            t64.append(e0.elapsed_time(e1))
            fp64_out[k % ndes] = (tens64, g64)
        c64.close()
        del cells[3]
        fp64 = {"ms_per_step": statistics.mean(t64), "steps": len(t64),
                "mixed_speedup": statistics.mean(t64) / statistics.mean(step_ms[:len(t64)]),
                "what": "same step (update + solve + C^H + d_h sensitivities) with every operator, "
                        "smoother and Krylov vector in FP64, same designs and tolerance"}

    accuracy = None
    if not args.no_accuracy:
        ref = Cell(designs[0], mat, kind="phi", precision=0, tol=1e-12, max_iter=4000)
        blk = ent = grad = 0.0
        b64 = e64 = g64e = 0.0
        keys = sorted(outputs)[:max(1, args.accuracy_designs)]
        for k in keys:
            tens, g = outputs[k]
            ref.update(designs[k])
            ref.solve()
            R = ref.homogenise()
            _, rdC, rde = dh(*R[:2])
            gr = ref.sensitivity(rdC, rde, None).cpu().numpy()
            a, b_, c = errors(tens, g, R, gr)
            blk, ent, grad = max(blk, a), max(ent, b_), max(grad, c)
            if k in fp64_out:
                a, b_, c = errors(*fp64_out[k], R, gr)
                b64, e64, g64e = max(b64, a), max(e64, b_), max(g64e, c)
        ref.close()
        accuracy = {"designs": len(keys), "target_CH": 1e-8, "target_sensitivity": 1e-5,
                    "CH_eH_kH_block_rel_max": blk, "entry_rel_max": ent,
                    "dh_sensitivity_rel_max": grad,
                    "reference": "FP64 GPU solves of the same designs to residual 1e-12",
                    "block_rel": "max |dH| / max |H| per block (C^H, e^H, kappa^H)",
                    "entry_rel": "max |dH_ij| / |H_ij| over entries with |H_ij| > 1e-6 max |H|"}
        if fp64_out:
            accuracy["fp64_path"] = {"CH_eH_kH_block_rel_max": b64, "entry_rel_max": e64,
                                     "dh_sensitivity_rel_max": g64e}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        host = [torch.as_tensor(cellgen.gaussian_levelset(n, seed=rank * 1000 + 500 + s)).pin_memory()
                for s in range(2)]
        e2e_ms = []
        for k in range(max(2, min(args.steps, 4))):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            phi = host[k % 2].to(dev, non_blocking=True)
            _, tens, g = step(phi)
            g_host = g.cpu()
            _ = [np.asarray(t) for t in tens]
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e = {"value": statistics.mean(e2e_ms), "unit": unit,
               "h2d_bytes_per_step": nn * 8, "d2h_bytes_per_step": nn * 4 + (36 + 18 + 9) * 8}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ms, p, pts, timed, sample = oracle_baseline(n)
        cpu = {"value": ms, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample,
               "extrapolated": True, "fit_exponent": p, "points_s": [[m, t] for m, t in pts]}

    if rank == 0:
        iters = [max(s["iters"]) for s in stats]
        line = {
            "metric": METRIC, "value": ms_per_cell, "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == 1 else "f64", "data": "synthetic",
            "config": {**workload_config(args, world),
                       "handle": "allocated once per process outside the timed region; each step = "
                                 "cell_update (rho, multigrid hierarchy) + solve + homogenise + "
                                 "d_h sensitivities",
                       "l2": "working set of several GB > L2, plus a 256 MB flush between steps"},
            "roofline": roof,
            "accuracy": accuracy,
            "fp64_gpu_same_accuracy": fp64,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "detail": {"wall_s": wall, "step_ms": step_ms, "gmres_iters_max": iters,
                       "refinements": [s["refinements"] for s in stats],
                       "tc_tiles_autotuned": {"elastic": stats[0]["tc_tiles"][0], "schur": stats[0]["tc_tiles"][1]},
                       "class_ms_per_step": share_ms, "class_share": class_share,
                       "class_source": "separate fully profiled pass over the same designs "
                                       "(untimed); the timed region times only the roofline kernel"},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
