#!/usr/bin/env python
"""BP5 Jacobi-PCG throughput on one GB300: DOFs/s per CG iteration, n_0.8, roofline fraction.

The metric is the paper's rate of work (Eq. (3)): DOFs x CG iterations / seconds
with DOFs = E N^3 (Sec. 2), on a synthetic deformed-box mesh (Sec. 3), BP5
(Table 1) at order N = 7.  A "step" is one PCG iteration over the whole
problem: the element kernel (BK5 with the fused p^T A p), the gather-scatter
plus vector update, and the direction update.  Setup (mesh, geometric factors,
Jacobi diagonal) is outside the timed region, as in the paper (Sec. 3).

    python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

The headline arm runs native FP64 arithmetic; the line also carries the
FP64-accurate FP32-pair arm and the recomputed-factor arm as `variants`, an n
sweep of both arithmetics (r_max, n_0.8, t_0.8), the roofline of the element
kernel, the end-to-end rate with host copies and the CPU oracle's rate.

Under torchrun (N > 1) every rank solves its own independent problem (replicas,
weak scaling); rank 0 prints one JSON line.  ``--impl reference`` times the
CPU FP64 oracle on the host cores instead (a bounded sample of the workload).

Other workloads (``--workload``): ``bp-sweep`` (BP1/BP3/BP5 at N = 3..15 over
n = 1e4..1e8), ``bk-sweep`` (unassembled BK5, FP64 and pairs), ``mixed`` (BP6
defect correction against plain PCG), ``batched`` (256 uneven BP5 problems),
``adjoint`` (dJ/dkappa with finite-difference checks), ``bp-point`` (one BP, order and size).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BP5 DOFs/sec per CG iter vs n on 1 GB300; n_0.8; % of HBM roofline"
UNIT = "DOFs/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100, help="timed PCG iterations")
    ap.add_argument("--warmup", type=int, default=5, help="untimed PCG iterations before the timed ones")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--order", type=int, default=7)
    ap.add_argument("--arith", choices=["fp64", "df64"], default="fp64",
                    help="headline arithmetic: fp64 native FP64 instructions; df64 FP64-accurate FP32 pairs")
    ap.add_argument("--headline-only", action="store_true", help="skip the other arithmetic variant")
    ap.add_argument("--k", type=int, default=18, help="E = 2^k elements (N=7: k=18 is n = 8.99e7)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the n sweep (r_max, n_0.8, t_0.8)")
    ap.add_argument("--sweep-iters", type=int, default=100)
    ap.add_argument("--mixed-e", type=int, default=48, help="elements per direction of the mixed workload")
    ap.add_argument("--mixed-bp", type=int, default=6, choices=[5, 6], help="bake-off problem of the mixed workload")
    ap.add_argument("--bp", type=int, default=3, help="bake-off problem of the bp-point workload")
    ap.add_argument("--bps", default="1,3,5", help="bake-off problems of the bp-sweep workload")
    ap.add_argument("--bk-bps", default="", help="element operators of the bk-sweep workload (default: 5)")
    ap.add_argument("--bk-orders", default="1,2,3,5,7,9,11,15", help="orders N of the bk-sweep workload")
    ap.add_argument("--df-tile", default=None,
                    help="pin the pair kernel's shape 'eb,schedule,seq' instead of the autotuner's choice")
    ap.add_argument("--geom", choices=["stored", "recompute"], default="stored",
                    help="geometric factors of the headline arm: stored, or recomputed in the element kernel")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the compact runs of the other configurations (BP1/BP3 points, BP6 defect "
                         "correction, batched solves, adjoint gradient)")
    ap.add_argument("--cpu-sample-k", type=int, default=9, help="E = 2^k elements for the oracle sample")
    ap.add_argument("--cpu-max-k", type=int, default=13, help="largest E = 2^k of the cpu-sweep workload")
    ap.add_argument("--workload", choices=["sweep", "batched", "mixed", "adjoint", "bp-sweep", "bk-sweep", "bp-point",
                                           "cpu-sweep"], default="sweep",
                    help="sweep: BP5 n-sweep headline; batched: 256 BP5 problems batched vs one at a time; "
                         "mixed: BP6 defect correction vs FP64 PCG; adjoint: dJ/dkappa pipeline")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------------
def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def fp64_peak_tflops(peaks):
    """FP64 FMA peak of the GB300 derived from its unit count and clock: the nominal
    1.25 TFLOP/s over 152 SMs at 2070 MHz is 4 flops (2 DFMA) per clock per SM.  Used only
    when the measured peak (measured_fma_peaks) is not available."""
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return 4.0 * 152 * mhz * 1e6 / 1e12, "derived: 2 DFMA/clk/SM x 152 SMs x sm_max_mhz"


_FMA_PEAKS = None


def measured_fma_peaks(pkg):
    """FP64 and FP32 FMA throughput of this GPU measured by the library's FMA-chain kernel
    (ceedbp_fma_peak; the SM count comes from the device), measured once per process."""
    global _FMA_PEAKS
    if _FMA_PEAKS is None:
        f64, sms = pkg.fma_peak(True)
        f32, _ = pkg.fma_peak(False)
        _FMA_PEAKS = {"fp64_tflops": f64, "fp32_tflops": f32, "sm_count": sms,
                      "how": "ceedbp_fma_peak: 8 independent FMA chains per thread, 8 blocks of 256 threads "
                             "per SM, best of 3 launches after a warm-up, CUDA events"}
    return _FMA_PEAKS


def ncu_value(name: str, key: str):
    """A number recorded as '<key>: value' in a committed ncu summary (profiles/<name>), else None."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        for line in open(path):
            if line.startswith(key + ":"):
                return float(line.split(":")[1])
    except (OSError, ValueError):
        pass
    return None


def ncu_traffic(name: str):
    """dram bytes per launch of a kernel from a committed ncu summary (profiles/<name>.md), else None."""
    return ncu_value(name, "dram_bytes_per_launch")


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: str):
        self.index = index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.index, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        self.proc.wait(timeout=5)
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        smax = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------------
def bp5_units(N: int):
    """Algorithmic bytes and flops per DOF (n = E N^3) of the BK5 element kernel and of one PCG
    iteration (FP64 words): p read once, w written once, six G words per quadrature point,
    one int32 l2g entry per local node; apply flops 12 p1^4 + 15 p1^3 per element."""
    p1 = N + 1
    ratio = (p1 / N) ** 3
    elem_bytes = 8 * 2 + (6 * 8 + 4) * ratio
    iter_bytes = 8 * 13 + (6 * 8 + 4) * ratio
    elem_flops = (12 * p1 ** 4 + 15 * p1 ** 3) / N ** 3
    return elem_bytes, iter_bytes, elem_flops


def bp5_units_recompute(N: int):
    """As bp5_units with the factors recomputed in the element kernel: three coordinate words per
    local node replace the six factor words; flops add the Jacobian (9 contractions, 18 p1 per node)
    and adj(J), |J| and the six factors (71 per node)."""
    p1 = N + 1
    ratio = (p1 / N) ** 3
    elem_bytes = 8 * 2 + (3 * 8 + 4) * ratio
    iter_bytes = 8 * 13 + (3 * 8 + 4) * ratio
    elem_flops = (30 * p1 ** 4 + 86 * p1 ** 3) / N ** 3
    return elem_bytes, iter_bytes, elem_flops


def n_08(ns, rates):
    """Smallest n with rate >= 0.8 r_max, log-linearly interpolated between samples."""
    rmax = max(rates)
    target = 0.8 * rmax
    for i, (n, r) in enumerate(zip(ns, rates)):
        if r >= target:
            if i == 0:
                return float(n)
            n0, r0 = ns[i - 1], rates[i - 1]
            t = (target - r0) / (r - r0)
            return float(math.exp(math.log(n0) + t * (math.log(n) - math.log(n0))))
    return float(ns[-1])


def max_over_ranks(ms: float, world: int, dist, device) -> float:
    """The slowest rank's time (the whole-job time of independent replicas)."""
    if world <= 1:
        return float(ms)
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_mesh(pkg, N, k):
    from synth import box_dims
    dims = box_dims(k)
    coords, l2g, dirichlet = pkg.mesh_box(*dims, N, 0.05)
    return dims, coords, l2g, dirichlet


def make_problem(pkg, N, mesh, seed, device, arith=0, geom=0):
    import numpy as np
    import torch

    from synth import uniform_pm1
    dims, coords, l2g, dirichlet = mesh
    op = pkg.Operator(5, N, coords, l2g, dirichlet, device=device, arith=arith, geom=geom)
    r = torch.from_numpy(uniform_pm1(seed, np.arange(op.nglobal))).to(device)
    mask = torch.from_numpy(1.0 - dirichlet.astype(np.float64)).to(device)
    b = op.mass(r) * mask
    E = dims[0] * dims[1] * dims[2]
    return op, b, E * N ** 3


def measure(pkg, args, mesh, arith, device, rank, world, dist, geom=0):
    """One arithmetic variant at the headline size: timed graph, per-kernel profile, end-to-end."""
    import torch
    N, K, W = args.order, args.steps, max(3, args.warmup)
    op, b, n_dofs = make_problem(pkg, N, mesh, seed=rank, device=device, arith=arith, geom=geom)
    if arith == pkg.ARITH_DF64 and args.df_tile:
        op.set_tile(*[int(v) for v in args.df_tile.split(",")])
    dims = mesh[0]
    x = op.empty()
    op.solve(b, x, fixed_iters=K, chunk=K)  # graph capture for the timed chunk length
    op.solve(b, x, fixed_iters=W, chunk=W)
    torch.cuda.synchronize()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = Clocks(vis.split(",")[device.index] if vis else str(device.index))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    _, info = op.solve(b, x, fixed_iters=K, chunk=K)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(info["device_ms"], world, dist, device)
    value = world * n_dofs * K / (ms * 1e-3)
    # per-kernel durations: the same K-iteration graph with event-record nodes around each kernel
    _, pinfo = op.solve(b, x, fixed_iters=K, chunk=K, profile=True)
    elem_ms = pinfo["kernel_ms"][0]
    # end to end through the public API: pinned host RHS in, solution back to pinned host memory
    b_h = b.cpu().pin_memory()
    x_h = torch.empty_like(b_h).pin_memory()
    b_d = torch.empty_like(b)
    s = torch.cuda.current_stream(device)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(s)
    b_d.copy_(b_h, non_blocking=True)
    xe, _ = op.solve(b_d, x, fixed_iters=K, chunk=K)
    x_h.copy_(xe, non_blocking=True)
    ev1.record(s)
    torch.cuda.synchronize()
    e2e_ms = ev0.elapsed_time(ev1)

    peaks, peak_src = load_peaks()
    rc = geom == pkg.GEOM_RECOMPUTE
    elem_bytes_dof, iter_bytes_dof, elem_flops_dof = bp5_units_recompute(N) if rc else bp5_units(N)
    fma = measured_fma_peaks(pkg)
    fp64_tf, fp64_src = fma["fp64_tflops"], "measured: " + fma["how"]
    elem_flops = elem_flops_dof * n_dofs
    elem_bytes = elem_bytes_dof * n_dofs
    name = ("fp64rc" if rc else "fp64") if arith == pkg.ARITH_FP64 else "df64"
    pair_eo = arith != pkg.ARITH_FP64 and op.tile_info()[1] == 3  # even-odd pair kernel chosen
    if pair_eo:
        name = "df64eo"
    traffic = ncu_traffic(f"bk5_{name}_n{N}.md")
    if arith == pkg.ARITH_FP64:
        ach = elem_flops / (elem_ms * 1e-3) / 1e12
        kname = "elem_rc_kernel (BK5, FP64, factors recomputed)" if rc else "elem_eo_kernel (BK5, FP64, even-odd)"
        roof = {"bound": "alu", "achieved": ach, "peak": fp64_tf, "unit": "TFLOP/s", "frac": ach / fp64_tf,
                "traffic": traffic, "kernel": kname, "peak_source": fp64_src,
                "peak_derived_tflops": fp64_peak_tflops(peaks)[0],
                "hbm_frac": (elem_bytes / (elem_ms * 1e-3) / 1e9) / peaks["hbm_gbs"]}
        # the FP64 work the kernel actually executes (ncu thread-instruction counts per element of
        # the same kernel): DFMA counts 2 flops, DADD and DMUL 1
        name_i = f"bk5_{'fp64rc' if rc else 'fp64'}_n{N}.md"
        inst = [ncu_value(name_i, k) for k in ("dfma_per_element", "dadd_per_element", "dmul_per_element")]
        if all(v is not None for v in inst):
            E = n_dofs // N ** 3
            exec_flops = (2 * inst[0] + inst[1] + inst[2]) * E
            roof["executed_tflops"] = exec_flops / (elem_ms * 1e-3) / 1e12
            roof["frac_executed"] = roof["executed_tflops"] / fp64_tf
            roof["executed_flops_per_dof"] = exec_flops / n_dofs
            # FP64 pipe: one DFMA, DADD or DMUL per slot, 2 slots per clock per SM (the peak's rate)
            roof["fp64_pipe_frac"] = sum(inst) * E / (elem_ms * 1e-3) / (fp64_tf * 1e12 / 2)
    else:
        ach = elem_bytes / (elem_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": ("elem_dfeo_kernel (BK5, FP64-accurate FP32 pairs, even-odd)" if pair_eo
                           else "elem_dfp_kernel (BK5, FP64-accurate FP32 pairs)"),
                "peak_source": f"{peak_src} hbm_gbs",
                "fp64_equiv_tflops": elem_flops / (elem_ms * 1e-3) / 1e12,
                "fp32_peak_measured_tflops": fma["fp32_tflops"]}
    roof.update({"elem_ms": elem_ms, "update_ms": pinfo["kernel_ms"][1], "dir_ms": pinfo["kernel_ms"][2],
                 "algorithmic_bytes_per_dof": elem_bytes_dof, "flops_per_dof": elem_flops_dof})
    out = {
        "value": value, "ms_per_step": ms / K,
        "dtype": "f64" if arith == pkg.ARITH_FP64 else "df64 (FP32 pairs, FP64-accurate)",
        "hbm_roofline": {"bytes_per_dof_iter": iter_bytes_dof,
                         "roofline_dofs_per_s": peaks["hbm_gbs"] * 1e9 / iter_bytes_dof,
                         "frac": value / world / (peaks["hbm_gbs"] * 1e9 / iter_bytes_dof)},
        "roofline": roof,
        "e2e": {"value": world * n_dofs * K / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": b.numel() * 8 / K, "d2h_bytes_per_step": b.numel() * 8 / K,
                "note": "per solve call of K iterations: H2D of b, solve, D2H of x"},
        "gpu_launches": 3 * K,
        "clocks": clk,
        "wall_s_timed": wall,
        "solver": {"rel_res_after_K": info["rel_res"][0], "status": info["status"]},
        "n": n_dofs, "nglobal": op.nglobal, "elements": list(dims),
    }
    if arith != pkg.ARITH_FP64:
        eb, sched, seq = op.tile_info()
        out["roofline"]["tile"] = {"elements_per_block": eb,
                                   "schedule": ["G ring (cp.async)", "G staged (bulk copy)", "pipelined sequences", "even-odd octets"][sched],
                                   "elements_per_sequence": seq}
    op.close()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2004_06722_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    N, K, W = args.order, args.steps, max(3, args.warmup)
    mesh = make_mesh(pkg, N, args.k)
    head_arith = pkg.ARITH_DF64 if args.arith == "df64" else pkg.ARITH_FP64
    head_geom = pkg.GEOM_RECOMPUTE if args.geom == "recompute" else pkg.GEOM_STORED
    head = measure(pkg, args, mesh, head_arith, device, rank, world, dist, geom=head_geom)
    variants = {}
    if not args.headline_only:
        other = pkg.ARITH_FP64 if head_arith == pkg.ARITH_DF64 else pkg.ARITH_DF64
        variants["df64" if other == pkg.ARITH_DF64 else "fp64"] = measure(pkg, args, mesh, other, device, rank,
                                                                           world, dist)
        variants["fp64_recompute"] = measure(pkg, args, mesh, pkg.ARITH_FP64, device, rank, world, dist,
                                             geom=pkg.GEOM_RECOMPUTE)
    dims, n_dofs = head["elements"], head["n"]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": head["dtype"], "data": "synthetic",
        "config": {"workload": f"BP5 Jacobi-PCG, N={N}, E={dims[0]}x{dims[1]}x{dims[2]}={dims[0]*dims[1]*dims[2]} "
                               f"deformed box (amp 0.05), n=E*N^3={n_dofs}, RHS B*r with r seeded U[-1,1]",
                   "n": n_dofs, "order": N, "elements": dims, "nglobal": head["nglobal"],
                   "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 "
                   f"(geometric factors {6 * 8 * (N + 1) ** 3 * dims[0] * dims[1] * dims[2] / 1e9:.1f} GB per iteration)",
                   "timing": "CUDA events around one captured graph of K iterations on the solver stream"},
        "hbm_roofline": head["hbm_roofline"], "roofline": head["roofline"], "e2e": head["e2e"],
        "gpu_launches": head["gpu_launches"], "clocks": head["clocks"], "wall_s_timed": head["wall_s_timed"],
        "solver": head["solver"], "variants": variants,
    }
    # the HBM-roofline fraction of the iteration in each arithmetic, side by side: native FP64 is
    # bound by the FP64 pipe; the pair arithmetic carries 47-bit (not 53-bit) significands
    line["hbm_roofline_by_arith"] = {
        head["dtype"]: head["hbm_roofline"]["frac"],
        **{v["dtype"] + (" recomputed factors" if k == "fp64_recompute" else ""): v["hbm_roofline"]["frac"]
           for k, v in variants.items()}}
    del mesh
    if not args.no_sweep and rank == 0:
        line["sweep"] = run_sweep(pkg, N, args.sweep_iters, device, [head_arith] + (
            [] if args.headline_only else [pkg.ARITH_DF64 if head_arith == pkg.ARITH_FP64 else pkg.ARITH_FP64]))
    if not args.no_extras and rank == 0 and world == 1:
        line["configs"] = config_summaries()
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline(N, args.cpu_sample_k)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_sweep(pkg, N, iters, device, ariths):
    import torch

    from synth import sweep_ks
    res = {a: {"n": [], "dofs_per_s": [], "ms_per_iter": []} for a in ariths}
    for k in sweep_ks(N):
        mesh = make_mesh(pkg, N, k)
        for a in ariths:
            op, b, n_dofs = make_problem(pkg, N, mesh, seed=0, device=device, arith=a)
            x = op.empty()
            op.solve(b, x, fixed_iters=iters, chunk=iters)
            best = None
            for _ in range(3):
                _, info = op.solve(b, x, fixed_iters=iters, chunk=iters)
                best = info["device_ms"] if best is None else min(best, info["device_ms"])
            res[a]["n"].append(n_dofs)
            res[a]["dofs_per_s"].append(n_dofs * iters / (best * 1e-3))
            res[a]["ms_per_iter"].append(best / iters)
            op.close()
            del b, x
        del mesh
        torch.cuda.empty_cache()
    out = {}
    for a, r in res.items():
        rmax = max(r["dofs_per_s"])
        n80 = n_08(r["n"], r["dofs_per_s"])
        out["fp64" if a == pkg.ARITH_FP64 else "df64"] = dict(
            r, order=N, iters=iters, r_max=rmax, **{"n_0.8": n80, "t_0.8_s": 1.25 * n80 / rmax})
    return out


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:  # Arm hosts name the core in lscpu only
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample(N, k):
    """The oracle's assembled BP5 problem on E = 2^k elements (assembly is not timed)."""
    import numpy as np

    from oracle.problems import BakeoffProblem
    from synth import box_dims, uniform_pm1
    dims = box_dims(k)
    t0 = time.perf_counter()
    prob = BakeoffProblem(5, *dims, N, amp=0.05)
    t_setup = time.perf_counter() - t0
    b = prob.rhs(uniform_pm1(0, np.arange(prob.n_global)))[prob.free]
    return dims, prob, b, t_setup


def timed_cpu_pcg(pcg_threads, A, b, diag, threads, min_warm_s=0.5, min_timed_s=1.0):
    """(iterations, seconds) of the oracle's threaded PCG after a warm-up of at least min_warm_s (the
    host cores reach their clock under sustained load), timing at least min_timed_s."""
    t0 = time.perf_counter()
    pcg_threads(A, b, diag, 5, threads)
    per_it = (time.perf_counter() - t0) / 5
    pcg_threads(A, b, diag, max(5, int(math.ceil(min_warm_s / per_it))), threads)
    iters = max(10, int(math.ceil(min_timed_s / per_it)))
    t0 = time.perf_counter()
    pcg_threads(A, b, diag, iters, threads)
    return iters, time.perf_counter() - t0


def cpu_baseline(N, k):
    """The oracle as it stands (assembled CSR, textbook Jacobi PCG) on a bounded sample: BP5 at the
    same order on E = 2^k elements, the PCG on every host core (the oracle's C PCG on POSIX threads,
    same arithmetic as oracle/pcg.py) for at least a second after a warm-up; rate = E N^3 x
    iterations / PCG seconds (assembly excluded)."""
    from oracle.cpu_pcg import host_threads, pcg_threads
    dims, prob, b, t_setup = oracle_sample(N, k)
    threads = host_threads()
    iters, t = timed_cpu_pcg(pcg_threads, prob.A_free, b, prob.diag_free, threads)
    n = dims[0] * dims[1] * dims[2] * N ** 3
    return {"value": n * iters / t, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"BP5 N={N}, E={dims[0]}x{dims[1]}x{dims[2]} (n={n}, CSR nnz={prob.A_free.nnz}), {iters} PCG "
                      f"iterations of the oracle on the assembled CSR matrix, rows split over {threads} POSIX "
                      f"threads; assembly by naive full quadrature {t_setup:.1f} s excluded",
            "host_cpus": os.cpu_count(), "cpu_model": cpu_model()}


def _assemble_chunk(task):
    """Element matrices of one range of elements by the oracle (naive full quadrature) and their
    assembled sum over that range (the oracle's own assembly); a worker of cpu_sweep's pool."""
    import numpy as np

    from oracle.assemble import assemble
    from oracle.element import element_matrices
    from oracle.mesh import box_mesh, global_count
    from oracle.quadrature import bp_rule
    dims, N, e0, e1 = task
    coords, l2g = box_mesh(*dims, N, 0.05, elements=np.arange(e0, e1))
    rule = bp_rule(5, N)
    mats = [element_matrices(coords[e], N, rule, want=("A",))["A"] for e in range(e1 - e0)]
    A = assemble(l2g, mats, global_count(*dims, N)).tocoo()
    return A.row.astype(np.int32), A.col.astype(np.int32), A.data


def run_cpu_sweep(args):
    """The oracle's PCG rate on all host cores against the problem size: BP5 at order --order on
    E = 2^k for k = 9 .. --cpu-max-k, assembled by the oracle's element matrices on a process pool
    (spawn; assembly not timed), 20 PCG iterations of the oracle's C PCG on POSIX threads."""
    import multiprocessing as mp

    import numpy as np
    import scipy.sparse as sp

    from oracle.assemble import restrict
    from oracle.cpu_pcg import host_threads, pcg_threads
    from oracle.mesh import boundary_nodes, global_count
    from synth import box_dims, uniform_pm1
    N = args.order
    threads = host_threads()
    out = []

    def make_pool():
        # one BLAS thread per worker process (the pool already uses every core)
        saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for v in saved:
            os.environ[v] = "1"
        pool = mp.get_context("spawn").Pool(threads)
        for v, old in saved.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old
        return pool

    for k in range(9, args.cpu_max_k + 1):
        dims = box_dims(k)
        E = dims[0] * dims[1] * dims[2]
        ng = global_count(*dims, N)
        t0 = time.perf_counter()
        step = 32
        # a pool per size, ended before the timed PCG so that no worker shares the cores
        with make_pool() as pool:
            parts = pool.map(_assemble_chunk, [(dims, N, e, min(E, e + step)) for e in range(0, E, step)])
        rows = np.concatenate([p[0] for p in parts])
        cols = np.concatenate([p[1] for p in parts])
        vals = np.concatenate([p[2] for p in parts])
        del parts
        A = sp.csr_matrix((vals, (rows, cols)), shape=(ng, ng))
        del rows, cols, vals
        A.sum_duplicates()
        free = ~boundary_nodes(*dims, N)
        A_free = restrict(A, free)
        del A
        t_asm = time.perf_counter() - t0
        b = uniform_pm1(0, np.arange(ng))[free]
        diag = A_free.diagonal()
        iters, t = timed_cpu_pcg(pcg_threads, A_free, b, diag, threads)
        n = E * N ** 3
        row = {"k": k, "elements": list(dims), "n": n, "nnz": int(A_free.nnz),
               "csr_gb": (A_free.nnz * 12 + A_free.shape[0] * 8) / 1e9, "assembly_s": t_asm,
               "dofs_per_s": n * iters / t, "ms_per_iter": t / iters * 1e3, "iters": iters}
        out.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
        del A_free
    print(json.dumps({"metric": "oracle PCG DOFs/s per iteration on all host cores vs n (BP5)", "unit": "DOFs/s",
                      "order": N, "threads": threads, "cpu_model": cpu_model(), "host_cpus": os.cpu_count(),
                      "results": out}), flush=True)


def run_reference(args):
    """The oracle timed on all host cores, one PCG iteration per step, on a bounded sample."""
    from oracle.cpu_pcg import host_threads, pcg_threads
    from synth import box_dims
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    N, K, W = args.order, args.steps, max(3, args.warmup)
    dims, prob, b, t_setup = oracle_sample(N, args.cpu_sample_k)
    threads = host_threads()
    # W warm-up steps, and at least half a second of them: the host cores reach their clock only
    # under sustained load
    t0 = time.perf_counter()
    pcg_threads(prob.A_free, b, prob.diag_free, W, threads)
    per_it = (time.perf_counter() - t0) / W
    if per_it * W < 0.5:
        pcg_threads(prob.A_free, b, prob.diag_free, int(math.ceil(0.5 / per_it)), threads)
    t0 = time.perf_counter()
    pcg_threads(prob.A_free, b, prob.diag_free, K, threads)
    t = time.perf_counter() - t0
    n = dims[0] * dims[1] * dims[2] * N ** 3
    big = box_dims(args.k)
    value = n * K / t
    sample = (f"BP5 N={N}, E={dims[0]}x{dims[1]}x{dims[2]} (n={n}) instead of E=2^{args.k}; {K} PCG iterations "
              f"of the oracle (assembled CSR, rows split over {threads} POSIX threads; assembly {t_setup:.1f} s "
              f"excluded)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": K, "warmup": W, "ms_per_step": t / K * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"BP5 FP64 Jacobi-PCG, N={N}, E={big[0]}x{big[1]}x{big[2]} deformed box",
                   "order": N},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model(), "host_cpus": os.cpu_count()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def batched_summary(n_problems=256, arith_names=("fp64", "df64")):
    """n_problems BP5 problems (E = k^3, k log-uniform in [2, 16], N in {3, 5, 7}, amplitude U[0, 0.1],
    seed 0) solved to 1e-8 by one batched solve, against solving them one at a time with the
    single-problem path, in each arithmetic."""
    import numpy as np
    import torch

    import paper_2004_06722_gb300 as pkg
    from synth import batched_problems, uniform_pm1
    draws = batched_problems(n_problems, seed=0)
    meshes = [pkg.mesh_box(q["k"], q["k"], q["k"], q["N"], q["amp"]) for q in draws]
    out = {"problems": n_problems, "total_dofs": sum(q["k"] ** 3 * q["N"] ** 3 for q in draws),
           "orders": {str(N): sum(1 for q in draws if q["N"] == N) for N in (3, 5, 7)}, "tol": 1e-8}
    for name in arith_names:
        arith = pkg.ARITH_FP64 if name == "fp64" else pkg.ARITH_DF64
        probs, rhs, ops = [], [], []
        for q, (coords, l2g, dirichlet) in zip(draws, meshes):
            probs.append((q["N"], coords, l2g, dirichlet))
            op = pkg.Operator(5, q["N"], coords, l2g, dirichlet, arith=arith)
            r = torch.from_numpy(uniform_pm1(q["rhs_seed"], np.arange(op.nglobal))).cuda()
            rhs.append(op.mass(r) * torch.from_numpy(1.0 - dirichlet.astype(np.float64)).cuda())
            ops.append(op)
        batch = pkg.Batch(probs, arith=arith)
        for _ in range(2):
            xs, infos = batch.solve(rhs, tol=1e-8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xs, infos = batch.solve(rhs, tol=1e-8)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        for op, b in zip(ops, rhs):
            op.solve(b, tol=1e-8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        single = [op.solve(b, tol=1e-8) for op, b in zip(ops, rhs)]
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        dofs_iters = sum(q["k"] ** 3 * q["N"] ** 3 * inf["iters"][0] for q, inf in zip(draws, infos))
        diff_its = max(abs(a["iters"][0] - b[1]["iters"][0]) for a, b in zip(infos, single))
        diff_x = max((torch.linalg.norm(x - b[0]) / torch.linalg.norm(b[0])).item() for x, b in zip(xs, single))
        out[name] = {"batched_s": t_batch, "sequential_s": t_seq, "speedup": t_seq / t_batch,
                     "dofs_iters_per_s": dofs_iters / t_batch, "max_iteration_difference": diff_its,
                     "max_rel_diff_vs_single": diff_x, "all_converged": all(i["status"] == "OK" for i in infos),
                     "dtype": "f64" if arith == pkg.ARITH_FP64 else "df64 (FP32 pairs, FP64-accurate)"}
        batch.close()
        for op in ops:
            op.close()
        del rhs, xs, single
        torch.cuda.empty_cache()
    return out


def run_batched(args):
    """256 BP5 problems batched against one at a time, FP64 and FP32-pair arithmetic."""
    res = batched_summary(256)
    print(json.dumps({"metric": "batched BP5 solve time (256 problems to 1e-8)", "value": res["fp64"]["batched_s"],
                      "unit": "s", "higher_is_better": False, "dtype": "f64", "results": res}), flush=True)


def mixed_summary(E1, chunk=64, bp=6):
    """BP6 (three components; or BP5), N = 7, E = E1^3, seeded RHS: plain PCG (native FP64 and FP32 pairs) against
    FP64 defect correction with FP32 and BF16-storage inner solves, all to 1e-10 relative residual; the
    difference of every solution from the native FP64 one."""
    import numpy as np
    import torch

    import paper_2004_06722_gb300 as pkg
    from synth import uniform_pm1
    N = 7
    coords, l2g, dirichlet = pkg.mesh_box(E1, E1, E1, N, 0.05)
    res = {}
    x_ref = None
    for name, arith, mixed in [("fp64_pcg", pkg.ARITH_FP64, 0), ("df64_pcg", pkg.ARITH_DF64, 0),
                               ("fp32_defect_correction", pkg.ARITH_DF64, pkg.MIXED_FP32),
                               ("bf16_defect_correction", pkg.ARITH_DF64, pkg.MIXED_BF16),
                               ("fp32_tc_defect_correction", pkg.ARITH_DF64, pkg.MIXED_FP32_TC)]:
        op = pkg.Operator(bp, N, coords, l2g, dirichlet, arith=arith)
        if mixed:
            op.prepare_mixed(mixed)
        r = np.stack([uniform_pm1(c, np.arange(op.nglobal)) for c in range(op.ncomp)], axis=1)
        mask = torch.from_numpy(1.0 - dirichlet.astype(np.float64)).cuda()[:, None]
        b = op.mass(torch.from_numpy(np.ascontiguousarray(r if op.ncomp == 3 else r[:, 0])).cuda())
        b = b * (mask if op.ncomp == 3 else mask[:, 0])
        op.solve(b, tol=1e-3, mixed=mixed)  # warm-up (graphs, autotuned shapes)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, info = op.solve(b, tol=1e-10, mixed=mixed, chunk=chunk)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if x_ref is None:
            x_ref = x.clone()
        err = (torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)).item()
        res[name] = {"wall_s": wall, "device_ms": info["device_ms"], "iters": info["iters"],
                     "outer_iters": info["outer_iters"], "rel_res": info["rel_res"],
                     "rel_diff_vs_fp64_pcg": err}
        op.close()
        del b, x
        torch.cuda.empty_cache()
    return {"n_per_component": E1 ** 3 * N ** 3, "elements": [E1] * 3, "results": res,
            "speedup_fp32_dc_vs_fp64": res["fp64_pcg"]["wall_s"] / res["fp32_defect_correction"]["wall_s"],
            "speedup_fp32_dc_vs_df64": res["df64_pcg"]["wall_s"] / res["fp32_defect_correction"]["wall_s"]}


def run_mixed(args):
    """BP6 N = 7, E = 48^3 (--mixed-e): FP64 PCG against FP32 / BF16 defect correction to 1e-10."""
    E1 = args.mixed_e
    out = mixed_summary(E1, bp=args.mixed_bp)
    print(json.dumps(dict({"metric": f"BP{args.mixed_bp} N=7 E={E1}^3 solve time to 1e-10 relative residual", "unit": "s",
                           "higher_is_better": False}, **out)), flush=True)


def adjoint_summary(E1=32, n_dirs=20, arith_name="fp64", n_smooth=5):
    """-div(kappa grad u) = f, BP5 N = 7, E = E1^3, kappa = exp(g) with 16 random Fourier modes; target u*
    from a second kappa; J = 1/2 ||u - u*||_B^2; dJ/dkappa by one adjoint solve and the fused gradient
    kernel, checked by central differences (h = 1e-6) along n_dirs seeded directions, in both measures:
    the plain relative error |fd - <g,d>| / |<g,d>| and the error in the scale of the direction,
    |fd - <g,d>| / sum |g_i d_i|.  Forcing f = 1."""
    import numpy as np
    import torch

    import paper_2004_06722_gb300 as pkg
    from synth import fourier_field, fourier_modes
    N = 7
    coords, l2g, dirichlet = pkg.mesh_box(E1, E1, E1, N, 0.05)
    kappa = torch.from_numpy(np.exp(fourier_field(fourier_modes(0), coords))).cuda()
    kappa_star = torch.from_numpy(np.exp(fourier_field(fourier_modes(1), coords))).cuda()
    op = pkg.Operator(5, N, coords, l2g, dirichlet, arith=pkg.ARITH_DF64 if arith_name == "df64" else pkg.ARITH_FP64)
    mask = torch.from_numpy(1.0 - dirichlet.astype(np.float64)).cuda()
    # smooth forcing f = 1 (b = M B 1): u and u - u* are O(1e-2), so J is well conditioned for differences
    b = op.mass(torch.ones(op.nglobal, dtype=torch.float64, device="cuda")) * mask
    op.set_kappa(kappa_star)
    u_star, _ = op.solve(b, tol=1e-13, chunk=64)
    u_star = u_star.clone()
    k = kappa.clone().requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = pkg.kappa_misfit(k, op, b, u_star, tol=1e-10)
    (g,) = torch.autograd.grad(J, k)
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t0

    def Jof(kap):
        op.set_kappa(kap)
        u, _ = op.solve(b, tol=1e-13, chunk=64)
        return op.misfit(u, u_star)[1]

    # the same gradient with forward and adjoint solved to 1e-13: separates the error of the 1e-10 solves
    # from that of the adjoint formula and the gradient kernel
    k13 = kappa.clone().requires_grad_(True)
    (g13,) = torch.autograd.grad(pkg.kappa_misfit(k13, op, b, u_star, tol=1e-13), k13)

    rng = np.random.default_rng(20)
    h, errs, errs13, cancel, scaled = 1e-6, [], [], [], []
    for _ in range(n_dirs):
        d = torch.from_numpy(rng.uniform(-1, 1, size=tuple(kappa.shape))).cuda()
        d /= d.abs().max()
        fd = (Jof(kappa + h * d) - Jof(kappa - h * d)) / (2 * h)
        ad, ad13 = float((g * d).sum()), float((g13 * d).sum())
        mag = float((g13 * d).abs().sum())
        errs.append(abs(fd - ad) / abs(ad))
        errs13.append(abs(fd - ad13) / abs(ad13))
        cancel.append(mag / abs(ad13))
        scaled.append(abs(fd - ad) / mag)
    # smooth directions: log-kappa perturbations of the same Fourier form as g (seeds 100..104)
    smooth = []
    for sd in range(100, 100 + n_smooth):
        d = torch.from_numpy(fourier_field(fourier_modes(sd), coords)).cuda()
        d /= d.abs().max()
        fd = (Jof(kappa + h * d * kappa) - Jof(kappa - h * d * kappa)) / (2 * h)
        ad = float((g * d * kappa).sum())
        smooth.append(abs(fd - ad) / abs(ad))
    op.close()
    return {"value": t_grad, "unit": "s", "J": float(J.detach()),
            "kappa_values": int(kappa.numel()), "n": E1 ** 3 * N ** 3, "elements": [E1] * 3,
            "fd_rel_err_max": max(errs), "fd_rel_err_median": float(np.median(errs)),
            "fd_rel_err_max_tol13": max(errs13), "fd_rel_err_median_tol13": float(np.median(errs13)),
            "cancellation_max": max(cancel), "fd_err_over_abs_sum_max": max(scaled),
            "fd_rel_err_smooth_max": max(smooth), "fd_directions": n_dirs, "smooth_directions": n_smooth,
            "h": h, "dtype": "f64" if arith_name == "fp64" else "df64 (FP32 pairs, FP64-accurate)"}


def run_adjoint(args):
    """The adjoint workload at E = 32^3 with 20 finite-difference directions."""
    out = adjoint_summary(32, 20, args.arith)
    print(json.dumps(dict({"metric": "adjoint gradient dJ/dkappa (forward + adjoint solve to 1e-10 + gradient)",
                           "higher_is_better": False}, **out)), flush=True)


def run_bp_sweep(args):
    """BP1, BP3 and BP5 (FP64) at N in {3, 5, 7, 9, 11, 15} on E = 2^k deformed boxes with n = E N^3 stepping
    by 2x from 1e4 to 1e8; fixed 100 PCG iterations; r_max, n_0.8 and t_0.8 = 1.25 n_0.8 / r_max per (BP, N)."""
    import numpy as np
    import torch

    import paper_2004_06722_gb300 as pkg
    from synth import box_dims, sweep_ks, uniform_pm1
    iters = args.sweep_iters
    out = {}
    for bp in [int(v) for v in args.bps.split(",")]:
        for N in (3, 5, 7, 9, 11, 15):
            ns, rates = [], []
            for k in sweep_ks(N):
                dims = box_dims(k)
                coords, l2g, dirichlet = pkg.mesh_box(*dims, N, 0.05)
                op = pkg.Operator(bp, N, coords, l2g, dirichlet)
                del coords, l2g
                r = torch.from_numpy(uniform_pm1(0, np.arange(op.nglobal))).cuda()
                mask = torch.from_numpy(1.0 - dirichlet.astype(np.float64)).cuda() if bp != 1 else 1.0
                b = op.mass(r) * mask
                x = op.empty()
                op.solve(b, x, fixed_iters=iters, chunk=iters)
                best = min(op.solve(b, x, fixed_iters=iters, chunk=iters)[1]["device_ms"] for _ in range(2))
                n = dims[0] * dims[1] * dims[2] * N ** 3
                ns.append(n)
                rates.append(n * iters / (best * 1e-3))
                op.close()
                del b, x, r
                torch.cuda.empty_cache()
            rmax = max(rates)
            n80 = n_08(ns, rates)
            out[f"BP{bp}_N{N}"] = {"n": ns, "dofs_per_s": rates, "r_max": rmax, "n_0.8": n80,
                                   "t_0.8_s": 1.25 * n80 / rmax}
            print(json.dumps({f"BP{bp}_N{N}": {"r_max": rmax, "n_0.8": n80, "t_0.8_s": 1.25 * n80 / rmax}}),
                  file=sys.stderr, flush=True)
    print(json.dumps({"metric": "DOFs/s per CG iteration vs n (FP64), r_max, n_0.8, t_0.8 per BP and order",
                      "unit": "DOFs/s", "iters": iters, "results": out}), flush=True)


def bk_flops(bp: int, N: int) -> int:
    """Algorithmic flops of one element of BK`bp` (per component): BK5/BK6 12 p1^4 + 15 p1^3 (Eq. (22)
    with J = I); BK3/BK4 the interpolate-then-differentiate count 4 p1^4 (3 g^4 + g^3 + g^2 + g) +
    15 g^3 p1^3 with g = q / p1 (Eqs. (31)-(33)); BK1/BK2 the mass J^T B J, 4 p1^4 (g + g^2 + g^3) + g^3 p1^3
    (Eq. (34))."""
    p1 = N + 1
    if bp in (5, 6):
        return 12 * p1 ** 4 + 15 * p1 ** 3
    g = (N + 2) / p1
    if bp in (3, 4):
        return int(round(4 * p1 ** 4 * (3 * g ** 4 + g ** 3 + g ** 2 + g) + 15 * g ** 3 * p1 ** 3))
    return int(round(4 * p1 ** 4 * (g + g ** 2 + g ** 3) + g ** 3 * p1 ** 3))


def run_bk_sweep(args):
    """Unassembled BK kernels (the element operators of the BPs in --bps, no Q, Q^T or mask;
    ceedbp_bk_apply) at N in --bk-orders (default {1, 2, 3, 5, 7, 9, 11, 15}), FP64 and FP32 pairs (where built), on E = 2^k boxes
    (k <= 21) with n = E N^3 from ~1e3 to ~1e8 (k in steps of 2): time per apply (CUDA events over
    `--sweep-iters` applies after 3 warm-ups), algorithmic GFLOP/s (bk_flops per element), DOFs/s and r_max,
    n_0.8 per (BK, arith, N).  The default runs BK5; --bk-bps 1,3,5 adds BK1 and BK3."""
    import numpy as np
    import torch

    import paper_2004_06722_gb300 as pkg
    from synth import box_dims, uniform_pm1
    reps = args.sweep_iters
    bps = [int(v) for v in (args.bk_bps or "5").split(",")]
    orders = [int(v) for v in args.bk_orders.split(",")]
    out = {}
    for bp in bps:
        for name, arith in (("fp64", pkg.ARITH_FP64), ("df64", pkg.ARITH_DF64)):
            for N in orders:
                p1 = N + 1
                ns, rates, gflops, tpp = [], [], [], []
                k = 0
                while 2 ** k * N ** 3 < 1e3:
                    k += 1
                while 2 ** k * N ** 3 <= 1.2e8 and k <= 21:
                    dims = box_dims(k)
                    E = dims[0] * dims[1] * dims[2]
                    coords, l2g, dirichlet = pkg.mesh_box(*dims, N, 0.05)
                    op = pkg.Operator(bp, N, coords, l2g, dirichlet, arith=arith)
                    del coords, l2g
                    uL = torch.from_numpy(uniform_pm1(0, np.arange(E * p1 ** 3)).reshape(E, p1 ** 3)).cuda()
                    wL = torch.empty_like(uL)
                    for _ in range(3):
                        op.bk_apply(uL, wL)
                    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    with torch.cuda.stream(op.stream):
                        torch.cuda.synchronize()
                        ev0.record(op.stream)
                        for _ in range(reps):
                            op.bk_apply(uL, wL)
                        ev1.record(op.stream)
                    torch.cuda.synchronize()
                    t = ev0.elapsed_time(ev1) * 1e-3 / reps
                    n = E * N ** 3
                    ns.append(n)
                    rates.append(n / t)
                    gflops.append(E * bk_flops(bp, N) / t / 1e9)
                    tpp.append(t / n)
                    op.close()
                    del uL, wL
                    torch.cuda.empty_cache()
                    k += 2
                rmax = max(rates)
                n80 = n_08(ns, rates)
                key = f"BK{bp}_{name}_N{N}"
                out[key] = {"n": ns, "dofs_per_s": rates, "gflops": gflops, "s_per_dof": tpp,
                            "r_max": rmax, "n_0.8": n80, "gflops_max": max(gflops)}
                print(json.dumps({key: {"r_max": rmax, "n_0.8": n80, "gflops_max": max(gflops)}}),
                      file=sys.stderr, flush=True)
    print(json.dumps({"metric": "unassembled BK apply: DOFs/s and GFLOP/s vs n (FP64 and FP32 pairs)",
                      "unit": "DOFs/s", "reps": reps, "bks": bps, "results": out}), flush=True)


def bp_point_summary(bp, N, k, K, warmup=3, arith_name="fp64"):
    """One point of the BP sweep: BP `bp` at order N on E = 2^k, FP64 (or FP32 pairs), K fixed PCG
    iterations in one graph; DOFs/s and the per-kernel split (element / update / direction)."""
    import numpy as np
    import torch

    import paper_2004_06722_gb300 as pkg
    from synth import box_dims, uniform_pm1
    dims = box_dims(k)
    coords, l2g, dirichlet = pkg.mesh_box(*dims, N, 0.05)
    op = pkg.Operator(bp, N, coords, l2g, dirichlet,
                      arith=pkg.ARITH_DF64 if arith_name == "df64" else pkg.ARITH_FP64)
    del coords, l2g
    ncomp = op.ncomp
    r = np.stack([uniform_pm1(c, np.arange(op.nglobal)) for c in range(ncomp)], axis=1)
    rt = torch.from_numpy(np.ascontiguousarray(r if ncomp == 3 else r[:, 0])).cuda()
    mask = torch.from_numpy(1.0 - dirichlet.astype(np.float64)).cuda() if bp not in (1, 2) else None
    b = op.mass(rt) if bp in (1, 3, 5) else rt.clone()
    if mask is not None:
        b = b * (mask if ncomp == 1 else mask[:, None])
    x = op.empty()
    op.solve(b, x, fixed_iters=K, chunk=K)
    for _ in range(max(3, warmup) // K + 1):
        op.solve(b, x, fixed_iters=K, chunk=K)
    ms = min(op.solve(b, x, fixed_iters=K, chunk=K)[1]["device_ms"] for _ in range(2))
    _, pinfo = op.solve(b, x, fixed_iters=K, chunk=K, profile=True)
    op.close()
    n = dims[0] * dims[1] * dims[2] * N ** 3
    return {"bp": bp, "value": n * ncomp * K / (ms * 1e-3), "unit": "DOFs/s", "n": n, "ncomp": ncomp,
            "elements": list(dims), "order": N, "steps": K, "ms_per_iter": ms / K, "kernel_ms": pinfo["kernel_ms"],
            "dtype": "f64" if arith_name == "fp64" else "df64 (FP32 pairs, FP64-accurate)"}


def run_bp_point(args):
    """One point of the BP sweep (--bp, --order, --k, --steps)."""
    out = bp_point_summary(args.bp, args.order, args.k, args.steps, args.warmup, args.arith)
    print(json.dumps(dict({"metric": f"BP{args.bp} DOFs/s per CG iteration ({args.arith})"}, **out)), flush=True)


def config_summaries():
    """Compact, bounded runs of the other configurations for the default bench line (about three
    minutes): BP1 and BP3 at N = 7 on E = 2^18 (100 fixed iterations, FP64 and FP32 pairs), BP6
    defect correction at E = 16^3, 64 batched BP5 problems (FP64 and pairs) and the adjoint gradient
    at the configuration's E = 32^3 with 4 random and 1 smooth finite-difference directions (both
    error measures)."""
    import torch
    out = {}
    t_all = time.perf_counter()
    for bp in (1, 3):
        for arith in ("fp64", "df64"):
            key = f"bp{bp}_n7" + ("" if arith == "fp64" else "_df64")
            t0 = time.perf_counter()
            out[key] = bp_point_summary(bp, 7, 18, 100, arith_name=arith)
            out[key]["wall_s"] = time.perf_counter() - t0
            torch.cuda.empty_cache()
    t0 = time.perf_counter()
    out["bp6_defect_correction"] = mixed_summary(16)
    out["bp6_defect_correction"]["wall_s"] = time.perf_counter() - t0
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    out["batched"] = batched_summary(64)
    out["batched"]["wall_s"] = time.perf_counter() - t0
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    # the configuration's size with 4 + 1 directions (each costs two solves to 1e-13 of 1.1e7
    # DOFs); --workload adjoint runs the 20 + 5 of the configuration
    out["adjoint"] = adjoint_summary(32, 4, "fp64", n_smooth=1)
    out["adjoint"]["wall_s"] = time.perf_counter() - t0
    torch.cuda.empty_cache()
    out["wall_s"] = time.perf_counter() - t_all
    return out


def main():
    args = parse_args()
    if args.workload == "bp-point":
        return run_bp_point(args)
    if args.workload == "bp-sweep":
        return run_bp_sweep(args)
    if args.workload == "bk-sweep":
        return run_bk_sweep(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "mixed":
        return run_mixed(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload == "cpu-sweep":
        return run_cpu_sweep(args)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
