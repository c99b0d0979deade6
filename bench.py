#!/usr/bin/env python3
"""Throughput of the SDC hydro + reaction hot path on GB300.

Metric: zone-node-iterations/s = zones x (M-1) x K per SDC step / time, one
unit being one zone's node m -> m+1 update in one SDC iteration (advective term,
right-hand side and implicit reaction solve).  A step is one sdc_step (CUDA
graph) over the whole box from the same seeded initial state.

Default workload: 64^3 periodic box, 7-species alpha chain, 3 Gauss-Lobatto
nodes, 3 SDC iterations, FP64.  Inputs are resident in HBM when the timed
region starts; L2 is flushed (256 MB write) before every timed step.

Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64|fp32jac]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores
Under torchrun each rank runs its own box (independent problems, weak scaling).
"""
from __future__ import annotations

import argparse
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

from paper_1910_12578_gb300 import workloads as W  # noqa: E402

METRIC = "zone-node-iterations/s on 1 GB300 at stated FP64-oracle error; % of roofline"
UNIT = "zone-node-iterations/s"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per zone of one Newton launch, from one ncu
# capture per kernel variant on the 64^3 workload (262,144 zones), keyed by (nspec, Newton variant, prec).
# The traffic of these kernels grows in proportion to the zones (no re-reads), so a launch over N zones
# moves N times this.  A variant or precision without a capture reports null.
NEWTON_TRAFFIC_PER_ZONE = {
    (7, 1, "fp64"): (44.363264e6 + 4.091392e6) / 262144,    # newton_queue_kernel<7, chain, double>; its writes
                                                              # stay in the 129 MB L2 at the 64^3 size
    (13, 3, "fp64"): (70.107904e6 + 71.510016e6) / 262144,  # newton_queue_kernel<13, chain, double> on a 64^3
                                                              # box of the 256^3 workload's network; its writes
                                                              # already reach DRAM there, so 256^3 scales by zones
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--config", choices=["box64", "box256", "batch200"], default="box64")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--prec", choices=["fp64", "fp32jac"], default="fp64")
    p.add_argument("--space-order", type=int, choices=[2, 4], default=2,
                   help="2: PLM/MC/HLLC; 4: the fourth-order finite-volume operators")
    p.add_argument("--limiter", type=int, choices=[0, 1], default=1,
                   help="1: MC slopes (order 2) or limited face states with HLLC (order 4); 0: unlimited centred "
                        "slopes (order 2) or the smooth-flow form (order 4)")
    p.add_argument("--nodes", choices=["lobatto", "radau", "radau4"], default="lobatto",
                   help="temporal node set: Gauss-Lobatto (trapezoid/Simpson), node 0 + the Radau IIA points "
                        "1/3, 1, or (radau4) node 0 + the three Radau IIA points of s = 3")
    p.add_argument("--seed", type=int, default=None,
                   help="network / box seed (default: 1 for the single boxes, 3 for the batch)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--strang", action=argparse.BooleanOptionalAction, default=True,
                   help="also time the Strang-split baseline step and compare its error with the SDC step's")
    p.add_argument("--adjoint", action=argparse.BooleanOptionalAction, default=True,
                   help="also time one backward step (sdc_step_backward) of the workload")
    return p.parse_args()


def space_desc(args):
    if args.space_order == 4:
        return ("; fourth-order finite-volume operators, " +
                ("limited face states and HLLC" if args.limiter else "smooth-flow form (no limiter)"))
    return "" if args.limiter else "; unlimited centred slopes"


def workload(name, seed, nodes="lobatto"):
    """(problems, initial state, description): a Problem and its U, or for the
    batched workload a list of Problems and the concatenated U."""
    if name == "batch200":
        import numpy as np
        net, boxes = W.batched_boxes(nbox=200, nspec=7, seed=seed)
        Ps = [b[0] for b in boxes]
        U = np.concatenate([b[1].reshape(b[0].nvar, -1) for b in boxes], axis=1)
        desc = ("200 ragged periodic boxes (edges from {16,24,32,48,64} per axis, dx=1/64), 7-species alpha chain "
                "(seeded), hot spots 1.2-3x over T0=0.5, 3 Gauss-Lobatto nodes, 3 SDC iterations, CFL 0.5")
        for p in Ps:
            _set_nodes(p, nodes)
        return Ps, U, _nodes_desc(desc, nodes)
    if name == "box64":
        P, U = W.config_box(n=64, nspec=7, n_nodes=3, n_iters=3, seed=seed, T0=0.5)
        desc = ("64^3 periodic box, 7-species alpha chain (seeded), hot spot 2x over T0=0.5, "
                "3 Gauss-Lobatto nodes, 3 SDC iterations, CFL 0.5")
    else:
        P, U = W.config_box(n=256, nspec=13, n_nodes=3, n_iters=4, seed=seed, T0=0.5)
        desc = ("256^3 periodic box, 13-species alpha chain (seeded), hot spot 2x over T0=0.5, "
                "3 Gauss-Lobatto nodes, 4 SDC iterations, CFL 0.5")
    _set_nodes(P, nodes)
    return P, U, _nodes_desc(desc, nodes)


def _set_nodes(P, nodes):
    P.nodes = "lobatto" if nodes == "lobatto" else "radau"
    if nodes == "radau4":
        P.n_nodes = 4


def _nodes_desc(desc, nodes):
    if nodes == "lobatto":
        return desc
    if nodes == "radau4":
        return desc.replace("3 Gauss-Lobatto nodes", "4 nodes (0 and the Radau IIA points (4 -/+ sqrt 6)/10, 1; the "
                            "integral through the Radau points)")
    return desc.replace("3 Gauss-Lobatto nodes", "3 nodes (0 and the Radau IIA points 1/3, 1; the integral through the "
                        "Radau points)")


def units_per_step(P):
    if isinstance(P, (list, tuple)):
        return sum(units_per_step(p) for p in P)
    return P.nzones * (P.n_nodes - 1) * P.n_iters


def as_list(P):
    return list(P) if isinstance(P, (list, tuple)) else [P]


def nzones(P):
    return sum(p.nzones for p in as_list(P))


def newton_flops_per_iter(nspec):
    """Algorithmic flops of one Newton / pseudo-time iteration of one zone
    (alpha chain, n = nspec + 1 unknowns, nspec - 1 reactions):
      state evaluation  9 (n_r) + 3 nspec + 5 n   (rate constants and their T
                                                  derivative, sources, residual, norm)
      Jacobian / matrix 14 n_r + n
      LU, partial pivot 2n^3/3 - n^2/2 - n/6 + n  (multiply-add = 2, n reciprocals)
      two triangular solves 2 n^2 - n
      update and tests  3 n
    The transcendental calls (1 log, n_r exp per evaluation) are not counted."""
    n, nr = nspec + 1, nspec - 1
    ev = 9 * nr + 3 * nspec + 5 * n
    jac = 14 * nr + n
    lu = 2 * n ** 3 / 3 - n ** 2 / 2 - n / 6 + n
    sol = 2 * n ** 2 - n
    return ev, jac + lu + sol, 3 * n


def stencil_bytes_per_zone(P, rhs_mode):
    nv, n, M = P.nvar, P.net.nspec + 1, P.n_nodes
    if not rhs_mode:
        return 8 * 2 * nv                               # read U, write A
    return 8 * ((1 + 1 + 1 + M + 1) * nv + (M + 1) * n)  # U, A new, A old m, A old l, rhs; R old l, R next


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
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
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_seed(seed, rank):
    """Each rank runs its own box: the ranks' problems are independent (weak scaling)."""
    return seed + rank


def job_value(local_ms, units_per_rank, steps, world_size, reduce_max=None):
    """Whole-job throughput: the slowest rank's time (max over ranks) and the
    units of all ranks.  reduce_max(x) returns the maximum of x over the ranks."""
    t = reduce_max(local_ms) if (reduce_max and world_size > 1) else local_ms
    return units_per_rank * steps * world_size / (t * 1e-3), t


def torch_reduce_max(device):
    def f(x):
        import torch
        import torch.distributed as tdist
        v = torch.tensor([x], dtype=torch.float64, device=device)
        tdist.all_reduce(v, op=tdist.ReduceOp.MAX)
        return float(v.item())
    return f


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """The FP64 CPU oracle, as it stands, on the host cores: each step is one
    full SDC step of the same workload."""
    ws, rank, _ = dist()
    if rank != 0:
        return 0
    import oracle as O
    P, U, desc = workload(args.config, args.seed, args.nodes)
    for p_ in (P if isinstance(P, list) else [P]):
        p_.space_order, p_.limiter = args.space_order, args.limiter
    desc += space_desc(args)
    if args.config == "box256":
        # bounded sample: a 64^3 box with the same network and parameters
        P, U = W.config_box(n=64, nspec=13, n_nodes=3, n_iters=4, seed=args.seed, T0=0.5)
        _set_nodes(P, args.nodes)
        P.space_order, P.limiter = args.space_order, args.limiter
        desc += " (sample: 64^3 box, same network)"
    if isinstance(P, list):
        # bounded sample: the first 8 boxes of the batch, each its own oracle step
        Ps = P[:8]
        Us = []
        off = 0
        for p in P:
            if len(Us) == len(Ps):
                break
            Us.append(U[:, off:off + p.nzones].reshape((p.nvar,) + tuple(reversed(p.n))).copy())
            off += p.nzones
        orcs = [O.Oracle(p) for p in Ps]
        dt = min(o.cfl_dt(u) for o, u in zip(orcs, Us))
        run = lambda: [o.step(u, dt) for o, u in zip(orcs, Us)]
        P = Ps
        desc += " (sample: the first 8 boxes)"
    else:
        o = O.Oracle(P)
        dt = o.cfl_dt(U)
        run = lambda: o.step(U, dt)
    for _ in range(args.warmup):
        run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    el = time.perf_counter() - t0
    v = units_per_step(P) * args.steps / el
    P0 = as_list(P)[0]
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "zones": nzones(P), "nspec": P0.net.nspec, "nodes": P0.n_nodes,
                       "iters": P0.n_iters, "seed": args.seed},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d full SDC steps of the workload (or of its sample), OpenMP over zones"
                                       % args.steps},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sampled(P, U, dt, gpu_out, seed, target_s=10.0, max_steps=3):
    """Large boxes: the oracle as it stands on a bounded sample (whole SDC steps
    of a 64^3 box with the same network and parameters), and the GPU step's
    error per field on a contiguous 64^3 block at the hot spot: one step moves
    information at most 2 zones per advective evaluation, 2 (1 + K (M-1)) zones
    in all (fourth order: 5 (1 + K (M-1))), so the oracle run on the block's
    periodic surrounding with that much padding gives the exact result in the
    block."""
    import numpy as np
    import oracle as O
    Pc, Uc = W.config_box(n=64, nspec=P.net.nspec, n_nodes=P.n_nodes, n_iters=P.n_iters, seed=seed, T0=0.5)
    Pc.nodes = P.nodes
    Pc.space_order, Pc.limiter = P.space_order, P.limiter
    oc = O.Oracle(Pc)
    dtc = oc.cfl_dt(Uc)
    t0 = time.perf_counter()
    steps = 0
    while steps < 1 or (time.perf_counter() - t0 < target_s and steps < max_steps):
        oc.step(Uc, dtc)
        steps += 1
    el = time.perf_counter() - t0
    h = 64
    # per advective evaluation 2 zones (PLM/HLLC), 3 (fourth order, smooth form) or 4
    # (limited: the zone limiter reads two zones out); the fourth-order implicit
    # update reaches 2 more through its average <-> centre maps
    reach = 2 if P.space_order == 2 else (6 if P.limiter else 5)
    pad = reach * (1 + P.n_iters * (P.n_nodes - 1))
    c0 = P.n[0] // 2 - h // 2
    blk = np.arange(c0 - pad, c0 + h + pad) % P.n[0]
    Ub = U.reshape(P.nvar, P.n[2], P.n[1], P.n[0])[:, blk][:, :, blk][:, :, :, blk].copy()
    Pb = W.Problem(dim=3, n=(h + 2 * pad,) * 3, dx=P.dx, gamma=P.gamma, net=P.net, n_nodes=P.n_nodes,
                   n_iters=P.n_iters, nodes=P.nodes, space_order=P.space_order, limiter=P.limiter)
    Vb, _ = O.Oracle(Pb).step(Ub, dt)
    Vb = Vb.reshape(P.nvar, h + 2 * pad, h + 2 * pad, h + 2 * pad)[:, pad:pad + h, pad:pad + h, pad:pad + h]
    g = gpu_out.reshape(P.nvar, P.n[2], P.n[1], P.n[0])[:, c0:c0 + h, c0:c0 + h, c0:c0 + h]
    scale = np.abs(gpu_out).reshape(P.nvar, -1).max(1)
    scale[2 + P.dim:] = np.maximum(scale[2 + P.dim:], 1e-6 * scale[0])
    names = ["rho"] + ["mom%d" % d for d in range(P.dim)] + ["rhoE"] + ["X%d" % i for i in range(P.net.nspec)]
    errs = {n: float(e) for n, e in zip(names, np.abs(g - Vb).reshape(P.nvar, -1).max(1) / scale)}
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return ({"value": units_per_step(Pc) * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": "%d full SDC step(s) of a 64^3 box with the same network and parameters, OpenMP over zones"
                       % steps},
            {"max_rel": max(errs.values()), "per_field": errs,
             "sample": "every zone of the 64^3 block at the hot spot, from the oracle on its %d^3 periodic "
                       "surrounding (%d zones of padding: the step's domain of dependence)" % (h + 2 * pad, pad)})


def cpu_baseline_batched(Ps, U, dt, gpu_out, target_s=10.0):
    """Batched boxes: the oracle as it stands on a bounded sample (boxes taken in
    order until ~10 s of CPU work), and the GPU step's error on the smallest
    boxes of the batch, each compared zone by zone with the oracle run on it."""
    import numpy as np
    import oracle as O
    offs = np.cumsum([0] + [p.nzones for p in Ps])
    box = lambda i, A: A[:, offs[i]:offs[i + 1]].reshape((Ps[i].nvar,) + tuple(reversed(Ps[i].n)))
    t0 = time.perf_counter()
    units = 0
    i = 0
    while i < len(Ps) and (i == 0 or time.perf_counter() - t0 < target_s):
        O.Oracle(Ps[i]).step(box(i, U).copy(), dt)
        units += units_per_step(Ps[i])
        i += 1
    el = time.perf_counter() - t0
    worst = 0.0
    smallest = sorted(range(len(Ps)), key=lambda j: Ps[j].nzones)[:3]
    for j in smallest:
        Uo, _ = O.Oracle(Ps[j]).step(box(j, U).copy(), dt)
        g = box(j, gpu_out).reshape(Ps[j].nvar, -1)
        r = Uo.reshape(Ps[j].nvar, -1)
        scale = np.abs(r).max(1)
        scale[2 + Ps[j].dim:] = np.maximum(scale[2 + Ps[j].dim:], 1e-6 * scale[0])
        worst = max(worst, float((np.abs(g - r) / scale[:, None]).max()))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return ({"value": units / el, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": "one SDC step of each of the first %d boxes, OpenMP over zones" % i},
            {"max_rel": worst, "per_field": None,
             "sample": "every zone of the %d smallest boxes, each box run alone in the oracle" % len(smallest)})


def cpu_baseline_and_error(P, U, dt, gpu_out, target_s=10.0, max_steps=4):
    """The oracle as it stands on the host cores (bounded sample: whole SDC steps
    of the workload until ~10 s of CPU work), plus the error of the GPU step
    against it (this leg is the only one that runs the oracle)."""
    import numpy as np
    import oracle as O
    o = O.Oracle(P)
    t0 = time.perf_counter()
    Uo, _ = o.step(U, dt)
    steps = 1
    while time.perf_counter() - t0 < target_s and steps < max_steps:
        o.step(U, dt)
        steps += 1
    el = time.perf_counter() - t0
    g = gpu_out.reshape(P.nvar, -1)
    r = Uo.reshape(P.nvar, -1)
    rho_max = np.abs(r[0]).max()
    errs = {}
    names = ["rho"] + ["mom%d" % d for d in range(P.dim)] + ["rhoE"] + ["X%d" % i for i in range(P.net.nspec)]
    for f in range(P.nvar):
        den = np.abs(r[f]).max()
        if f >= 2 + P.dim:
            den = max(den, 1e-6 * rho_max)
        errs[names[f]] = float(np.abs(g[f] - r[f]).max() / max(den, 1e-300))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return ({"value": units_per_step(P) * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": "%d full SDC step(s) of the workload from the initial state, OpenMP over zones" % steps},
            {"max_rel": max(errs.values()), "per_field": errs})


def run_ours(args):
    import numpy as np
    import torch

    from paper_1910_12578_gb300 import build as B
    from paper_1910_12578_gb300 import sdc

    ws, rank, local = dist()
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if not os.path.exists(sdc.LIB_PATH):
        B.build()
    P, U, desc = workload(args.config, rank_seed(args.seed, rank), args.nodes)
    for p_ in as_list(P):
        p_.space_order, p_.limiter = args.space_order, args.limiter
    desc += space_desc(args)
    P0 = as_list(P)[0]
    prec = sdc.PREC_FP64 if args.prec == "fp64" else sdc.PREC_FP32_JAC
    ctx = sdc.Context(P, prec=prec)
    U0 = torch.from_numpy(U).cuda()
    Ud = torch.empty_like(U0)
    dt = ctx.cfl_dt(U0, P0.cfl)
    tuning = None
    if not args.no_autotune:
        tuning = ctx.autotune(U0, dt).as_dict()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    units = units_per_step(P)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # warm-up (also captures the graph)
    for _ in range(max(args.warmup, 1)):
        Ud.copy_(U0)
        ctx.step(Ud, dt, stats=False)
    torch.cuda.synchronize()

    # ---- timed region: K steps, each from the same initial state, L2 flushed before each
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    for i, (a, b) in enumerate(evs):
        Ud.copy_(U0)
        flush.fill_(i & 0xFF)
        a.record()
        ctx.step(Ud, dt, stats=False)
        b.record()
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    value, total_ms = job_value(sum(step_ms), units, args.steps, ws, torch_reduce_max("cuda"))

    # ---- end to end through the public API with host buffers (pinned), copies timed
    Uh = U0.cpu().pin_memory()
    Uout = torch.empty_like(Uh).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    Ud.copy_(U0)
    ctx.step(Ud, dt, stats=False)
    torch.cuda.synchronize()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ea.record()
    for _ in range(e2e_steps):
        Ud.copy_(Uh, non_blocking=True)
        ctx.step(Ud, dt, stats=False)
        Uout.copy_(Ud, non_blocking=True)
    eb.record()
    torch.cuda.synchronize()
    e2e_value, _ = job_value(ea.elapsed_time(eb) / e2e_steps, units, 1, ws, torch_reduce_max("cuda"))
    nbytes = U0.numel() * 8

    # ---- per-kernel-class times of the same step (eager launches, CUDA events on the context stream)
    Ud.copy_(U0)
    st, pr = ctx.step_profile(Ud, dt)
    Ud.copy_(U0)
    st2 = ctx.step(Ud, dt, stats=True)
    torch.cuda.synchronize()
    gpu_out = Ud.cpu().numpy()
    ev_f, lin_f, upd_f = newton_flops_per_iter(P0.net.nspec)
    iters = st.newton_iters_total
    newton_ms_launch = pr.ms_newton / max(pr.launches_newton, 1)
    if prec == sdc.PREC_FP64:
        fp64_flops = iters * (ev_f + lin_f + upd_f)
        fp32_flops = 0
    else:
        fp64_flops = iters * (ev_f + upd_f)
        fp32_flops = iters * lin_f
    achieved = fp64_flops / max(pr.launches_newton, 1) / (newton_ms_launch * 1e-3) / 1e12
    newton_choice = tuning["newton_choice"] if tuning else 0
    per_zone = NEWTON_TRAFFIC_PER_ZONE.get((P0.net.nspec, newton_choice, args.prec))
    roof = {"kernel": "newton_kernel (implicit reaction update)", "bound": "alu",
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": per_zone * nzones(P) if per_zone is not None else None,
            "traffic_unit": "bytes per launch (ncu DRAM read + write)",
            "peak_source": "FP64: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (recipe unit counts and clock; "
                           "an FMA-chain probe measured 1.256 TFLOP/s)",
            "flops_per_launch": fp64_flops / max(pr.launches_newton, 1), "ms_per_launch": newton_ms_launch,
            "newton_iters_per_solve": iters / max(st.newton_solves, 1),
            "note": "algorithmic flops count a dense pivoted LU per Newton iteration; the alpha chain's kernels "
                    "solve the same system by an O(n) elimination of its bordered bidiagonal form, so frac is "
                    "the algorithmic rate over the FP64 peak, not the FP64 pipe's occupancy (ncu: 84-85 %)"}
    if fp32_flops:
        roof["fp32_achieved"] = fp32_flops / max(pr.launches_newton, 1) / (newton_ms_launch * 1e-3) / 1e12
        roof["fp32_peak"] = FP32_PEAK_TFLOPS
    n_st = pr.launches_stencil
    st_bytes = nzones(P) * (stencil_bytes_per_zone(P0, False) * P0.n_iters +
                            stencil_bytes_per_zone(P0, True) * (P0.n_nodes - 2) * P0.n_iters) / max(n_st, 1)
    stencil_ms = pr.ms_stencil / max(n_st, 1)
    hbm_peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm_peak = json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        pass
    hbm_peak = hbm_peak or 6800.0
    st_gbs = st_bytes / (stencil_ms * 1e-3) / 1e9
    roof_st = {"kernel": "stencil_kernel (advective term + fused rhs)", "bound": "hbm", "achieved": st_gbs,
               "peak": hbm_peak, "unit": "GB/s", "frac": st_gbs / hbm_peak, "traffic": None,
               "bytes_per_launch": st_bytes, "ms_per_launch": stencil_ms}

    # ---- one backward (adjoint) step of the same workload, where the network has one
    adjoint = None
    if args.adjoint:
        gU = torch.ones_like(U0)
        gUn = torch.empty_like(U0)
        ga = torch.zeros(P0.net.nreac, dtype=torch.float64, device="cuda")
        try:
            ctx.step_backward(U0, dt, gU, gUn, ga)          # allocates the adjoint workspace
            torch.cuda.synchronize()
            ab = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ab[0].record()
            for _ in range(2):
                ctx.step_backward(U0, dt, gU, gUn, ga)
            ab[1].record()
            torch.cuda.synchronize()
            bms = ab[0].elapsed_time(ab[1]) / 2
            adjoint = {"ms_per_backward_step": bms, "ms_per_forward_step": total_ms / args.steps,
                       "ratio": bms / (total_ms / args.steps),
                       "note": "recomputes the forward step from its checkpoint, then the reverse sweep; "
                               "gradient of sum(U^{n+1}) with respect to U^n and the rate prefactors"}
        except sdc.SdcError as e:
            adjoint = {"unavailable": str(e)}

    # ---- the Strang-split baseline on the same kernels: its cost, and the coupling
    # error the SDC step removes (both against the coupled step in 8 steps of dt/8)
    strang = None
    if args.strang:
        Us = torch.empty_like(U0)
        Us.copy_(U0)
        ctx.step_strang(Us, dt, stats=False)
        torch.cuda.synchronize()
        sa = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        reps = 3
        sa[0].record()
        for _ in range(reps):
            Us.copy_(U0)
            ctx.step_strang(Us, dt, stats=False)
        sa[1].record()
        torch.cuda.synchronize()
        ca = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ca[0].record()
        for _ in range(reps):
            Us.copy_(U0)
        ca[1].record()
        torch.cuda.synchronize()
        copy_ms = ca[0].elapsed_time(ca[1]) / reps
        s_ms = sa[0].elapsed_time(sa[1]) / reps - copy_ms
        Uref = U0.clone()
        for _ in range(8):
            ctx.step(Uref, dt / 8, stats=False)
        Uc = U0.clone()
        ctx.step(Uc, dt, stats=False)
        Us.copy_(U0)
        sst = ctx.step_strang(Us, dt)
        torch.cuda.synchronize()
        ref = Uref.cpu().numpy().reshape(P0.nvar, -1)

        names = ["rho"] + ["mom%d" % d for d in range(P0.dim)] + ["rhoE"] + \
            ["rhoX%d" % i for i in range(P0.net.nspec)]
        den = np.abs(ref).max(1)
        den[2 + P0.dim:] = np.maximum(den[2 + P0.dim:], 1e-6 * den[0])
        l1den = np.abs(ref).sum(1)

        def field_err(a):
            a = a.cpu().numpy().reshape(P0.nvar, -1)
            inf = np.abs(a - ref).max(1) / den
            l1 = np.abs(a - ref).sum(1) / np.maximum(l1den, 1e-300)
            return float(inf.max()), {n: [float(x), float(y)] for n, x, y in zip(names, inf, l1)}

        es, fs = field_err(Us)
        ec, fc = field_err(Uc)
        strang = {"ms_per_step": s_ms, "sdc_ms_per_step": total_ms / args.steps,
                  "error_vs_fine_sdc": es, "sdc_error_vs_fine_sdc": ec,
                  "per_field_inf_l1": {"strang": fs, "sdc": fc},
                  "newton_fails": sst.n_fail,
                  "reference": "the coupled SDC step in 8 steps of dt/8 on the GPU (same kernels); errors are "
                               "|U - U_ref|_inf / |U_ref|_inf per field (max over fields) and |U - U_ref|_1 / "
                               "|U_ref|_1 at the benchmark dt"}

    line = None
    if rank == 0:
        cpu, err = (None, None)
        if ws == 1 and not args.no_cpu_baseline:
            if isinstance(P, list):
                cpu, err = cpu_baseline_batched(P, U, dt, gpu_out)
            elif P.nzones > 64 ** 3:
                cpu, err = cpu_baseline_sampled(P, U, dt, gpu_out, args.seed)
            else:
                cpu, err = cpu_baseline_and_error(P, U, dt, gpu_out)
        per_step = ctx.launches_per_step()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == sdc.PREC_FP64 else "f64 residual/update, f32 Jacobian/LU",
            "data": "synthetic",
            "config": {"workload": desc, "zones": nzones(P), "nspec": P0.net.nspec, "n_nodes": P0.n_nodes,
                       "iters": P0.n_iters, "nodes": args.nodes, "space_order": args.space_order,
                       "limiter": args.limiter, "prec": args.prec, "seed": args.seed,
                       "kernel_variants": tuning,
                       "l2": "flushed before every timed step (256 MB write)",
                       "parallelism": "independent box per GPU" if ws > 1 else "1 GPU"},
            "clocks": ck,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes},
            "gpu_launches": per_step * args.steps,
            "roofline": roof,
            "roofline_stencil": roof_st,
            "profile_ms": {"stencil": pr.ms_stencil, "newton": pr.ms_newton, "other": pr.ms_other,
                           "launches": [pr.launches_stencil, pr.launches_newton, pr.launches_other]},
            "newton": {"iters_total": st2.newton_iters_total, "solves": st2.newton_solves,
                       "fails": st2.n_fail},
            "cpu_baseline": cpu,
            "oracle_error": err,
            "adjoint": adjoint,
            "strang": strang,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.seed is None:
        # the batch uses seed 3: with seeds 0-2 some strongly igniting boxes of the
        # batch make the SDC iteration diverge in the oracle and on the GPU alike
        args.seed = 3 if args.config == "batch200" else 1
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
