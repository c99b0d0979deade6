#!/usr/bin/env python3
"""Throughput of the SDC hydro + reaction hot path on GB300.

Metric: zone-node-iterations/s = zones x (M-1) x K per SDC step / time, one
unit being one zone's node m -> m+1 update in one SDC iteration (advective term,
right-hand side and implicit reaction solve).  A step is one sdc_step (CUDA
graph) over the whole box from the same seeded initial state.

Default workload: 256^3 periodic box (16.8M zones), 13-species alpha chain
(14 x 14 Newton system), 3 Gauss-Lobatto nodes, 4 SDC iterations: the FP64
path is the headline; the FP32-Jacobian / FP64-residual path and the
float-pair Jacobian path of the same workload are measured in the same run (the
"fp32jac" and "fp32x2jac" objects), each with its error against the FP64
oracle.  Inputs are resident in HBM when the timed
region starts; the state (2.4 GB) is larger than L2, and L2 is also flushed
(256 MB write) before every timed step.

Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--config box256|box64|batch200]
                  [--prec all|both|fp64|fp32jac|fp32x2jac]
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
# capture per kernel variant and precision, keyed by (nspec, Newton variant, prec).  The captures ran on a 128^3
# box of the 256^3 workload's network (2.1M zones: every array of the launch exceeds L2, so its writes reach
# DRAM and the traffic grows in proportion to the zones; algorithmic 624 B per zone: the rhs, R^{m+1,(k)} and
# the step's rate anchors read, the new state and R written), mean over the 8 launches of a step, so a launch
# over N zones moves N times this.  A variant or precision without a capture of the current kernels reports null.
NEWTON_TRAFFIC_PER_ZONE = {
    (13, 2, "fp64"): (771.9e6 + 818.0e6) / 2097152,       # newton_kernel<13, chain, double>, static grid: its
                                                          # spills (168 registers) reach DRAM
    (13, 2, "fp32jac"): (791.9e6 + 771.1e6) / 2097152,    # newton_kernel<13, chain, float>: the same
    (13, 2, "fp32x2jac"): (767.9e6 + 577.6e6) / 2097152,  # newton_kernel<13, chain, f2>: the same
}
# The same for one advective term of the direction-split passes (x, y, z; A only), 128^3 box, 13 species.
PREC_NAMES = {0: "fp64", 1: "fp32jac", 2: "fp32x2jac"}   # sdc_precision values
STENCIL_TRAFFIC_PER_ZONE = {13: (302.3e6 + 546.5e6 + 604.3e6 + 259.6e6 + 654.7e6 + 261.8e6) / 2097152}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--config", choices=["box64", "box256", "batch200"], default="box256")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--prec", choices=["all", "both", "fp64", "fp32jac", "fp32x2jac"], default="all",
                   help="all: the FP64 path is the headline, the FP32-Jacobian and the float-pair Jacobian paths "
                        "of the same workload are measured in the same run; both: FP64 and FP32 Jacobian; "
                        "otherwise that path alone")
    p.add_argument("--space-order", type=int, choices=[2, 4], default=2,
                   help="2: PLM/MC/HLLC; 4: the fourth-order finite-volume operators")
    p.add_argument("--limiter", type=int, choices=[0, 1], default=1,
                   help="1: MC slopes (order 2) or limited face states with HLLC (order 4); 0: unlimited centred "
                        "slopes (order 2) or the smooth-flow form (order 4)")
    p.add_argument("--nodes", choices=["lobatto", "radau", "radau4"], default="lobatto",
                   help="temporal node set: Gauss-Lobatto (trapezoid/Simpson), node 0 + the Radau IIA points "
                        "1/3, 1, or (radau4) node 0 + the three Radau IIA points of s = 3")
    p.add_argument("--batch-T0", type=float, default=1.0,
                   help="background temperature of the batched boxes (1.15: a stiffer batch, 2-21 Newton "
                        "iterations per zone in its first step)")
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


def workload(name, seed, nodes="lobatto", batch_T0=1.0):
    """(problems, initial state, description): a Problem and its U, or for the
    batched workload a list of Problems and the concatenated U."""
    if name == "batch200":
        import numpy as np
        net, boxes = W.batched_boxes(nbox=200, nspec=7, seed=seed, T0=batch_T0)
        Ps = [b[0] for b in boxes]
        U = np.concatenate([b[1].reshape(b[0].nvar, -1) for b in boxes], axis=1)
        desc = ("200 ragged periodic boxes (edges from {16,24,32,48,64} per axis, dx=1/64), 7-species alpha chain "
                "(seeded), hot spots 1.2-3x over T0=%g, 3 Gauss-Lobatto nodes, 3 SDC iterations, CFL 0.5" % batch_T0)
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


def newton_flops(nspec):
    """Algorithmic flops of one zone's implicit reaction update on the alpha
    chain as the kernels compute it (nspec species, n_r = nspec - 1 reactions,
    n_c = nspec - 1 chain columns; a reciprocal counts as one flop, a fused
    multiply-add as two; the transcendental calls, 1 log2 T and n_r exp2 per
    evaluation, are counted apart):
      evaluation   11 + 9 n_r + 7 nspec   T, 1/T and the rate constants k_j
                                          (2 per reaction), Y, the rates and
                                          their species and energy sums, the
                                          residual G = w - dt_m R - rhs, its
                                          scaled norm
      matrix       2 + 18 + 30 (n_r - 1)  entries of c I - dt_m dR/dw in its
                                          bordered bidiagonal form
      elimination  28 (n_c - 1) + 15 + 11 + 7 n_c
                                          the chain columns with the border
                                          rows, the 2 x 2 border block,
                                          back substitution
      update       nspec + 3              trial state and stop-test scales
      setup        6 + nspec + 2 n_r      per solve: 1/rho, kinetic energy,
                                          1/(rho mass_i), a_j rho^(o_j-1), the
                                          energy scale
    One iteration is one linear solve: matrix + elimination + update + the
    evaluation at the trial (whose residual decides the step and whose R is
    the source at the solution); one solve adds the setup and the evaluation at
    the start.  Returns (per_solve, per_iter_fp64_part, per_iter_linear_part)."""
    nr = nspec - 1
    nc = nspec - 1
    evaluation = 11 + 9 * nr + 7 * nspec
    matrix = 2 + 18 + 30 * (nr - 1)
    elimination = 28 * (nc - 1) + 15 + 11 + 7 * nc
    update = nspec + 3
    setup = 6 + nspec + 2 * nr
    return {"per_solve": setup + evaluation, "per_iter_eval_update": evaluation + update,
            "per_iter_linear": matrix + elimination, "evaluation": evaluation, "matrix": matrix,
            "elimination": elimination, "update": update, "setup": setup,
            "transcendentals_per_evaluation": 1 + nr}


def stencil_flops_per_zone(P, rhs_mode):
    """Algorithmic FP64 flops of one advective term per zone (PLM / MC / HLLC,
    3D, nspec species, nvar = 5 + nspec fields; a fused multiply-add counts 2,
    a refined reciprocal or reciprocal square root 1):
      primitives            13 + nspec      (once per zone)
      per direction, per zone:
        differences         nvar            (one per face and field)
        half slopes         nvar            (dl + dr; the MC limiting on bit patterns)
        face flux           87 + 3 nspec    (both face states of the hydro fields,
                                             the Davis speeds, S*, the upwind flux,
                                             the star-region correction; the upwind
                                             mass fractions, their sum, renormalised
                                             species fluxes)
        flux difference     3 nvar
    so 349 + 25 nspec per zone (7 species 524, 13 species 674).  The fused
    right-hand side of Eq. sdc:general adds per field the A difference (3),
    the integral's terms (2 per term and a reactive source add per term) and
    the reactive R term (2)."""
    ns = P.net.nspec
    nv = P.nvar
    f = 13 + ns + 3 * (2 * nv + 87 + 3 * ns + 3 * nv)
    if rhs_mode:
        terms = P.n_nodes
        nw = ns + 1
        f += nv * (3 + 2 * terms) + nw * (2 + terms)
    return f


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


def field_names(P):
    return ["rho"] + ["mom%d" % d for d in range(P.dim)] + ["rhoE"] + ["X%d" % i for i in range(P.net.nspec)]


def field_errors(P, g, r):
    """Error of the GPU state g against the oracle's r (both [nvar][zones]),
    per field, in the two forms the results are stated in:
      per_field   |g - r|_inf / |r|_inf for every field, species included
                  (relative to each species' own largest value, floor 1e-30);
      per_field_floored
                  the same with the species measured against
                  max(|rho X_i|_inf, 1e-6 |rho|_inf), i.e. in units of the mass
                  below 1e-6 of it."""
    import numpy as np
    g = g.reshape(P.nvar, -1)
    r = r.reshape(P.nvar, -1)
    d = np.abs(g - r).max(1)
    own = np.maximum(np.abs(r).max(1), 1e-30)
    floored = own.copy()
    floored[2 + P.dim:] = np.maximum(floored[2 + P.dim:], 1e-6 * np.abs(r[0]).max())
    names = field_names(P)
    pf = {n: float(x) for n, x in zip(names, d / own)}
    pff = {n: float(x) for n, x in zip(names, d / floored)}
    hydro = names[:2 + P.dim]
    return {"max_rel": max(pf.values()), "max_rel_hydro": max(pf[n] for n in hydro),
            "max_rel_floored": max(pff.values()), "per_field": pf, "per_field_floored": pff,
            "norm": "per field |gpu - oracle|_inf / |oracle|_inf (species: relative to their own largest value, "
                    "floor 1e-30; per_field_floored: relative to max(|rho X_i|_inf, 1e-6 |rho|_inf))"}


def bench_config(args, desc, P):
    """The workload description shared by both arms of the benchmark."""
    P0 = as_list(P)[0]
    return {"workload": desc, "zones": nzones(P), "nspec": P0.net.nspec, "n_nodes": P0.n_nodes,
            "iters": P0.n_iters, "nodes": args.nodes, "space_order": args.space_order, "limiter": args.limiter,
            "seed": args.seed, "prec": args.prec if args.prec in ("fp32jac", "fp32x2jac") else "fp64",
            "l2": "inputs larger than L2 at 256^3; L2 also flushed before every timed step (256 MB write)",
            "parallelism": "independent box per GPU" if args.gpus > 1 else "1 GPU"}


def oracle_sample(args, P, U):
    """The bounded sample of the workload that the oracle runs as a CPU
    baseline: the whole problem when it is small, a 64^3 box with the same
    network and parameters for the 256^3 box, the first 8 boxes of the batch.
    Returns (list of (Problem, U) pairs, description)."""
    if isinstance(P, list):
        out, off = [], 0
        for p in P[:8]:
            out.append((p, U[:, off:off + p.nzones].reshape((p.nvar,) + tuple(reversed(p.n))).copy()))
            off += p.nzones
        return out, "one SDC step of each of the first 8 boxes of the batch"
    if P.nzones > 64 ** 3:
        Pc, Uc = W.config_box(n=64, nspec=P.net.nspec, n_nodes=P.n_nodes, n_iters=P.n_iters, seed=args.seed, T0=0.5)
        Pc.nodes, Pc.n_nodes = P.nodes, P.n_nodes
        Pc.space_order, Pc.limiter = P.space_order, P.limiter
        return [(Pc, Uc)], "one full SDC step of a 64^3 box with the same network and parameters"
    return [(P, U)], "one full SDC step of the workload"


def run_reference(args):
    """The FP64 CPU oracle, as it stands, on the host cores: each step is one
    SDC step of a bounded sample of the workload (oracle_sample)."""
    ws, rank, _ = dist()
    if rank != 0:
        return 0
    import oracle as O
    P, U, desc = workload(args.config, args.seed, args.nodes, args.batch_T0)
    for p_ in as_list(P):
        p_.space_order, p_.limiter = args.space_order, args.limiter
    desc += space_desc(args)
    sample, sdesc = oracle_sample(args, P, U)
    orcs = [O.Oracle(p) for p, _ in sample]
    dt = min(o.cfl_dt(u) for o, (_, u) in zip(orcs, sample))
    run = lambda: [o.step(u, dt) for o, (_, u) in zip(orcs, sample)]
    for _ in range(args.warmup):
        run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    el = time.perf_counter() - t0
    v = units_per_step([p for p, _ in sample]) * args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, desc, P),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "per step: %s (%d zones), OpenMP over zones"
                                       % (sdesc, sum(p.nzones for p, _ in sample))},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(args, P, U, dt, target_s=10.0, max_steps=3):
    """The oracle as it stands on the host cores, on the bounded sample of
    oracle_sample, repeated until about target_s seconds of CPU work."""
    import oracle as O
    sample, sdesc = oracle_sample(args, P, U)
    orcs = [O.Oracle(p) for p, _ in sample]
    t0 = time.perf_counter()
    steps = 0
    while steps < 1 or (time.perf_counter() - t0 < target_s and steps < max_steps):
        for o, (_, u) in zip(orcs, sample):
            o.step(u, dt)
        steps += 1
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": units_per_step([p for p, _ in sample]) * steps / el, "unit": UNIT, "cores": cores,
            "kind": "oracle", "sample": "%d x %s, OpenMP over zones" % (steps, sdesc)}


def oracle_reference(P, U, dt):
    """The oracle's result on the part of the workload it can run, and a
    function that cuts the same part out of a GPU result:
      a box of at most 64^3 zones: the whole box;
      a larger box: the contiguous 64^3 block at the hot spot, from the oracle
        run on the block's periodic surrounding padded by the step's domain of
        dependence (2 zones per advective evaluation for PLM/HLLC, 1 + K (M-1)
        evaluations; fourth order 5 or 6);
      the batch: its 3 smallest boxes, each run alone.
    Returns (Problem, oracle state [nvar][zones], cut(gpu_out) -> [nvar][zones], description)."""
    import numpy as np
    import oracle as O
    if isinstance(P, list):
        offs = np.cumsum([0] + [p.nzones for p in P])
        small = sorted(range(len(P)), key=lambda j: P[j].nzones)[:3]
        refs = []
        for j in small:
            Uj = U[:, offs[j]:offs[j + 1]].reshape((P[j].nvar,) + tuple(reversed(P[j].n))).copy()
            refs.append(O.Oracle(P[j]).step(Uj, dt)[0].reshape(P[j].nvar, -1))
        cut = lambda G: np.concatenate([G[:, offs[j]:offs[j + 1]] for j in small], axis=1)
        return P[0], np.concatenate(refs, axis=1), cut, \
            "every zone of the %d smallest boxes of the batch, each box run alone in the oracle" % len(small)
    if P.nzones <= 64 ** 3:
        Uo, _ = O.Oracle(P).step(U, dt)
        return P, Uo.reshape(P.nvar, -1), (lambda G: G.reshape(P.nvar, -1)), "every zone of the workload"
    h = 64
    reach = 2 if P.space_order == 2 else (6 if P.limiter else 5)
    pad = reach * (1 + P.n_iters * (P.n_nodes - 1))
    c0 = P.n[0] // 2 - h // 2
    blk = np.arange(c0 - pad, c0 + h + pad) % P.n[0]
    Ub = U.reshape(P.nvar, P.n[2], P.n[1], P.n[0])[:, blk][:, :, blk][:, :, :, blk].copy()
    Pb = W.Problem(dim=3, n=(h + 2 * pad,) * 3, dx=P.dx, gamma=P.gamma, net=P.net, n_nodes=P.n_nodes,
                   n_iters=P.n_iters, nodes=P.nodes, space_order=P.space_order, limiter=P.limiter)
    Vb, _ = O.Oracle(Pb).step(Ub, dt)
    Vb = Vb.reshape(P.nvar, h + 2 * pad, h + 2 * pad, h + 2 * pad)[:, pad:pad + h, pad:pad + h, pad:pad + h]
    cut = lambda G: G.reshape(P.nvar, P.n[2], P.n[1], P.n[0])[:, c0:c0 + h, c0:c0 + h, c0:c0 + h].reshape(
        P.nvar, -1)
    return P, Vb.reshape(P.nvar, -1), cut, \
        ("every zone and field of the 64^3 block at the hot spot, from the oracle on its %d^3 periodic "
         "surrounding (%d zones of padding: the step's domain of dependence)" % (h + 2 * pad, pad))


def hist_summary(hist):
    """Newton iterations per zone solve: the histogram (index = iterations,
    the last bin counts 63 and more) and its range."""
    h = [int(x) for x in hist]
    nz = [i for i, x in enumerate(h) if x]
    top = max(nz) if nz else 0
    return {"hist": h[:top + 1], "min_iters": min(nz) if nz else 0, "max_iters": top,
            "solves": sum(h), "mean_iters": (sum(i * x for i, x in enumerate(h)) / max(sum(h), 1))}


def measure(args, P, U, prec, ws, barrier, flush, with_e2e=True):
    """One context at one precision: autotune, warm-up, K timed steps (device
    time, inputs resident), end to end with host buffers, the per-class
    profile, the Newton roofline; returns (record, final state of one step
    from U (numpy), context)."""
    import numpy as np
    import torch

    from paper_1910_12578_gb300 import sdc

    P0 = as_list(P)[0]
    ctx = sdc.Context(P, prec=prec)
    U0 = torch.from_numpy(U).cuda()
    Ud = torch.empty_like(U0)
    dt = ctx.cfl_dt(U0, P0.cfl)
    tuning = None
    if not args.no_autotune:
        tuning = ctx.autotune(U0, dt).as_dict()
    units = units_per_step(P)

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

    # ---- end to end through the public API with host buffers (pinned), copies timed.  Every step
    # copies its input state from pinned host memory into one of two device buffers, steps that
    # buffer in place and copies the result back; the copies of step i+1's input and of step i-1's
    # result run on a second stream while step i computes, as a caller streaming states through the
    # library would (the context keeps the step's graph for both buffers).
    e2e = None
    if with_e2e:
        Uh = U0.cpu().pin_memory()
        Uout = [torch.empty_like(Uh).pin_memory() for _ in range(2)]
        Din = [torch.empty_like(U0) for _ in range(2)]
        e2e_steps = max(3, args.steps)
        comp = torch.cuda.current_stream()
        copy = torch.cuda.Stream()
        for b in range(2):   # capture the graph of each buffer outside the timed region
            Din[b].copy_(U0)
            ctx.step(Din[b], dt, stats=False)
        torch.cuda.synchronize()
        ev = lambda: torch.cuda.Event()
        in_ready, out_ready = ([ev() for _ in range(2)] for _ in range(2))

        def h2d(i):
            # on the copy stream after the previous result read from this buffer (stream order)
            b = i % 2
            with torch.cuda.stream(copy):
                Din[b].copy_(Uh, non_blocking=True)
                in_ready[b].record(copy)

        def pipeline(n):
            """n steps, each with its input copied in and its result copied out; the device time"""
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(comp)
            copy.wait_event(ea)
            h2d(0)
            for i in range(n):
                b = i % 2
                if i + 1 < n:
                    h2d(i + 1)
                comp.wait_event(in_ready[b])
                ctx.step(Din[b], dt, stats=False)
                out_ready[b].record(comp)
                with torch.cuda.stream(copy):
                    copy.wait_event(out_ready[b])
                    Uout[b].copy_(Din[b], non_blocking=True)
            comp.wait_stream(copy)
            eb.record(comp)
            torch.cuda.synchronize()
            return ea.elapsed_time(eb)

        # warm-up: the first copies from and into freshly pinned host buffers take several times
        # as long as the later ones (about 110 against 12 ms for 2.4 GB at 256^3)
        pipeline(3)
        # the copies alone (for the record: the first input and the last result of the timed region
        # are the copies that no compute hides)
        h2d_ms = d2h_ms = float("inf")
        for _ in range(3):   # the fastest of three (single copies vary several-fold on the host side)
            cev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            with torch.cuda.stream(copy):
                cev[0].record(copy)
                Din[0].copy_(Uh, non_blocking=True)
                cev[1].record(copy)
                Uout[0].copy_(Din[0], non_blocking=True)
                cev[2].record(copy)
            torch.cuda.synchronize()
            h2d_ms = min(h2d_ms, cev[0].elapsed_time(cev[1]))
            d2h_ms = min(d2h_ms, cev[1].elapsed_time(cev[2]))
        barrier()
        e2e_ms = pipeline(e2e_steps)
        e2e_value, _ = job_value(e2e_ms / e2e_steps, units, 1, ws, torch_reduce_max("cuda"))
        nbytes = U0.numel() * 8
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "steps": e2e_steps, "h2d_ms": round(h2d_ms, 3), "d2h_ms": round(d2h_ms, 3),
               "note": "per step: host->device copy of the input state (pinned) into one of two device buffers, "
                       "the step in place on it, device->host copy of the result (pinned); copies overlap the "
                       "neighbouring steps' compute on a second stream; after 3 untimed steps of the same loop "
                       "(h2d_ms, d2h_ms: one copy alone, the fastest of three)"}
        del Uh, Uout, Din

    # ---- per-kernel-class times of the same step (eager launches, CUDA events on the context stream)
    Ud.copy_(U0)
    st, pr = ctx.step_profile(Ud, dt)
    Ud.copy_(U0)
    st2 = ctx.step(Ud, dt, stats=True)
    torch.cuda.synchronize()
    gpu_out = Ud.cpu().numpy()

    fl = newton_flops(P0.net.nspec)
    iters, solves = st.newton_iters_total, st.newton_solves
    nl = max(pr.launches_newton, 1)
    newton_ms_launch = pr.ms_newton / nl
    fp64_total = solves * fl["per_solve"] + iters * fl["per_iter_eval_update"]
    lin_total = iters * fl["per_iter_linear"]
    if prec == sdc.PREC_FP64:
        fp64_total += lin_total
        fp32_total = 0
    else:
        fp32_total = lin_total   # in FP32, or in float pairs on the FP32 pipe
    achieved = fp64_total / nl / (newton_ms_launch * 1e-3) / 1e12
    newton_choice = tuning["newton_choice"] if tuning else 0
    pkey = PREC_NAMES[prec]
    per_zone = NEWTON_TRAFFIC_PER_ZONE.get((P0.net.nspec, newton_choice, pkey))
    roof = {"kernel": "newton_*_kernel<%d> (implicit reaction update, variant %d)" % (P0.net.nspec, newton_choice),
            "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": per_zone * nzones(P) if per_zone is not None else None,
            "traffic_unit": "bytes per launch (ncu DRAM read + write)",
            "peak_source": "FP64: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (recipe unit counts and clock; "
                           "an FMA-chain probe measured 1.256 TFLOP/s)",
            "fp64_flops_per_launch": fp64_total / nl, "ms_per_launch": newton_ms_launch,
            "launches_per_step": pr.launches_newton,
            "newton_iters_per_solve": iters / max(solves, 1),
            "flops_per_zone": fl,
            "note": "algorithmic flops of the bordered bidiagonal elimination the kernel runs (not a dense LU): "
                    "per solve setup + evaluation, per iteration matrix + elimination + update + evaluation"}
    if fp32_total:
        roof["fp32_flops_per_launch"] = fp32_total / nl
        roof["fp32_achieved"] = fp32_total / nl / (newton_ms_launch * 1e-3) / 1e12
        roof["fp32_peak"] = FP32_PEAK_TFLOPS
        if prec == sdc.PREC_FP32_JAC:
            roof["note"] += "; FP32 Jacobian: matrix and elimination in FP32 (fp32_*), the rest in FP64"
        else:
            roof["note"] += ("; float-pair Jacobian: matrix and elimination in double-float arithmetic on the FP32 "
                             "pipe (fp32_* counts their algorithmic flops, each about 10-15 FP32 instructions), "
                             "the rest in FP64")
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
    st_flops = nzones(P) * (stencil_flops_per_zone(P0, False) * P0.n_iters +
                            stencil_flops_per_zone(P0, True) * (P0.n_nodes - 2) * P0.n_iters) / max(n_st, 1)
    st_tf = st_flops / (stencil_ms * 1e-3) / 1e12
    split = (tuning is not None and tuning["stencil_choice"] == tuning["stencil_variants"] - 1 and P0.dim == 3
             and P0.space_order == 2)
    if P0.space_order == 4:
        st_tf = None
    roof_st = {"kernel": ("stencil_split_kernel x, y, z passes" if split else "stencil_kernel") +
                         " (advective term, fused rhs at the inner nodes)",
               "bound": "alu", "achieved": st_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
               "frac": st_tf / FP64_PEAK_TFLOPS if st_tf is not None else None, "traffic": None,
               "flops_per_launch": st_flops if st_tf is not None else None,
               "ms_per_launch": stencil_ms,
               "hbm": {"achieved": st_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": st_gbs / hbm_peak,
                       "bytes_per_launch": st_bytes, "peak_source": "measured copy bandwidth (hbm_gbs)",
                       "traffic_A_only": (STENCIL_TRAFFIC_PER_ZONE[P0.net.nspec] * nzones(P)
                                          if split and P0.net.nspec in STENCIL_TRAFFIC_PER_ZONE else None),
                       "traffic_note": "ncu DRAM read + write of the three passes of one advective term without "
                                       "the rhs, 128^3 capture scaled by zones"},
               "note": "one launch = one advective term (the direction-split variant's three passes); algorithmic "
                       "FP64 flops per zone from stencil_flops_per_zone; the term is bound by the FP64 pipe, not by "
                       "HBM (its algorithmic bytes are the hbm object)"}
    rec = {"value": value, "ms_per_step": total_ms / args.steps, "step_ms": step_ms, "clocks": ck, "e2e": e2e,
           "kernel_variants": tuning, "roofline": roof, "roofline_stencil": roof_st,
           "profile_ms": {"stencil": pr.ms_stencil, "newton": pr.ms_newton, "other": pr.ms_other,
                          "launches": [pr.launches_stencil, pr.launches_newton, pr.launches_other]},
           "newton": {"iters_total": st2.newton_iters_total, "solves": st2.newton_solves, "fails": st2.n_fail,
                      "iterations_per_solve": hist_summary(st2.hist)},
           "gpu_launches": ctx.launches_per_step() * args.steps, "dt": dt}
    return rec, gpu_out, ctx, U0


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
    P, U, desc = workload(args.config, rank_seed(args.seed, rank), args.nodes, args.batch_T0)
    for p_ in as_list(P):
        p_.space_order, p_.limiter = args.space_order, args.limiter
    desc += space_desc(args)
    P0 = as_list(P)[0]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    precs = {"all": [sdc.PREC_FP64, sdc.PREC_FP32_JAC, sdc.PREC_FP32X2_JAC],
             "both": [sdc.PREC_FP64, sdc.PREC_FP32_JAC], "fp64": [sdc.PREC_FP64],
             "fp32jac": [sdc.PREC_FP32_JAC], "fp32x2jac": [sdc.PREC_FP32X2_JAC]}[args.prec]
    head, head_out, ctx, U0 = measure(args, P, U, precs[0], ws, barrier, flush)
    dt = head["dt"]

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
            adjoint = {"ms_per_backward_step": bms, "ms_per_forward_step": head["ms_per_step"],
                       "ratio": bms / head["ms_per_step"],
                       "note": "recomputes the forward step from its checkpoint, then the reverse sweep; "
                               "gradient of sum(U^{n+1}) with respect to U^n and the rate prefactors"}
        except sdc.SdcError as e:
            adjoint = {"unavailable": str(e)}
        del gU, gUn

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
        ref = Uref.cpu().numpy().reshape(P0.nvar, -1)
        del Uref
        Uc = U0.clone()
        ctx.step(Uc, dt, stats=False)
        Us.copy_(U0)
        sst = ctx.step_strang(Us, dt)
        torch.cuda.synchronize()

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
        strang = {"ms_per_step": s_ms, "sdc_ms_per_step": head["ms_per_step"],
                  "error_vs_fine_sdc": es, "sdc_error_vs_fine_sdc": ec,
                  "per_field_inf_l1": {"strang": fs, "sdc": fc},
                  "newton_fails": sst.n_fail,
                  "reference": "the coupled SDC step in 8 steps of dt/8 on the GPU (same kernels); errors are "
                               "|U - U_ref|_inf / max(|U_ref|_inf, 1e-6 |rho|_inf) per field (max over fields) "
                               "and |U - U_ref|_1 / |U_ref|_1 at the benchmark dt"}
        del Us, Uc
    ctx.close()
    del ctx, U0
    torch.cuda.empty_cache()

    # ---- the FP32-Jacobian and float-pair Jacobian paths of the same workload
    others = []
    for pr_ in precs[1:]:
        rec2, out2, ctx2, U02 = measure(args, P, U, pr_, ws, barrier, flush)
        others.append((pr_, rec2, out2))
        ctx2.close()
        del ctx2, U02
        torch.cuda.empty_cache()

    line = None
    if rank == 0:
        cpu, err = None, None
        errs = [None] * len(others)
        if ws == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(args, P, U, dt)
            Pr, ref, cut, rdesc = oracle_reference(P, U, dt)
            err = field_errors(Pr, cut(head_out.reshape(P0.nvar, -1)), ref)
            err["sample"] = rdesc
            for i, (_, _, out2) in enumerate(others):
                errs[i] = field_errors(Pr, cut(out2.reshape(P0.nvar, -1)), ref)
                errs[i]["sample"] = rdesc
        dtype = lambda p: {sdc.PREC_FP64: "f64", sdc.PREC_FP32_JAC: "f64 residual/update, f32 Jacobian/LU",
                           sdc.PREC_FP32X2_JAC: "f64 residual/update, float-pair (2 x f32) Jacobian/LU"}[p]
        cfg = bench_config(args, desc, P)
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype(precs[0]), "data": "synthetic",
            "config": cfg, "clocks": head["clocks"], "e2e": head["e2e"],
            "gpu_launches": head["gpu_launches"] + sum(r["gpu_launches"] for _, r, _ in others),
            "roofline": head["roofline"], "roofline_stencil": head["roofline_stencil"],
            "kernel_variants": head["kernel_variants"], "profile_ms": head["profile_ms"],
            "newton": head["newton"], "cpu_baseline": cpu, "oracle_error": err,
        }
        for (pr_, rec2, _), err2 in zip(others, errs):
            line[PREC_NAMES[pr_]] = {
                "prec": PREC_NAMES[pr_], "dtype": dtype(pr_), "value": rec2["value"],
                "ms_per_step": rec2["ms_per_step"], "speedup_vs_fp64": head["ms_per_step"] / rec2["ms_per_step"],
                # the implicit reaction update alone (eager per-class profile): the part the precision changes
                "newton_speedup_vs_fp64": (head["profile_ms"]["newton"] / rec2["profile_ms"]["newton"]
                                           if head.get("profile_ms") and rec2.get("profile_ms") else None),
                "e2e": rec2["e2e"], "clocks": rec2["clocks"], "roofline": rec2["roofline"],
                "kernel_variants": rec2["kernel_variants"], "profile_ms": rec2["profile_ms"],
                "newton": rec2["newton"], "oracle_error": err2,
                "note": "same workload, steps and warm-up as the headline; gpu_launches counts every run"}
        line["adjoint"] = adjoint
        line["strang"] = strang
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
