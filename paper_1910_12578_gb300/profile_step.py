"""Run SDC steps of a named workload for a profiler (ncu) or a quick timing.

    python -m paper_1910_12578_gb300.profile_step --config box64 --stencil-variant 1 --newton-variant 1 \\
        --warmup 1 --steps 2 [--eager] [--prec fp32jac|fp32x2jac] [--space-order 4] [--limiter 0] [--nodes radau] \\
        [--backward]

Every step starts from the same seeded initial state.  With --eager the kernels
are launched one by one (sdc_step_profile, CUDA events per kernel class);
otherwise each step replays the captured CUDA graph (sdc_step), as bench.py
times it.  Kernel variants are set explicitly (no autotuning launches in the
profile); --autotune picks them first instead.  Prints one JSON line with the
per-step times and the variants used."""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1910_12578_gb300 import workloads as W  # noqa: E402


def workload(name, seed, batch_T0=1.0):
    import numpy as np
    if name == "batch200":
        net, boxes = W.batched_boxes(nbox=200, nspec=7, seed=seed, T0=batch_T0)
        Ps = [b[0] for b in boxes]
        U = np.concatenate([b[1].reshape(b[0].nvar, -1) for b in boxes], axis=1)
        return Ps, U
    n, nspec, K = {"box32": (32, 7, 3), "box64": (64, 7, 3), "box128": (128, 7, 3), "box64_13": (64, 13, 4),
                   "box128_13": (128, 13, 4), "box256": (256, 13, 4)}[name]
    return W.config_box(n=n, nspec=nspec, n_nodes=3, n_iters=K, seed=seed, T0=0.5)


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--config", default="box64", choices=["box32", "box64", "box128", "box64_13", "box128_13", "box256",
                                                         "batch200"])
    p.add_argument("--seed", type=int, default=None)
    p.add_argument("--prec", choices=["fp64", "fp32jac", "fp32x2jac"], default="fp64")
    p.add_argument("--stencil-variant", type=int, default=0)
    p.add_argument("--newton-variant", type=int, default=0)
    p.add_argument("--autotune", action="store_true")
    p.add_argument("--eager", action="store_true")
    p.add_argument("--warmup", type=int, default=1)
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--space-order", type=int, choices=[2, 4], default=2)
    p.add_argument("--limiter", type=int, choices=[0, 1], default=1)
    p.add_argument("--nodes", choices=["lobatto", "radau"], default="lobatto")
    p.add_argument("--backward", action="store_true", help="then one adjoint step (sdc_step_backward)")
    p.add_argument("--batch-T0", type=float, default=1.0, help="background temperature of the batched boxes")
    a = p.parse_args(argv)
    seed = a.seed if a.seed is not None else (3 if a.config == "batch200" else 1)

    import torch

    from paper_1910_12578_gb300 import sdc
    P, U = workload(a.config, seed, a.batch_T0)
    for q in (P if isinstance(P, list) else [P]):
        q.space_order, q.nodes, q.limiter = a.space_order, a.nodes, a.limiter
    P0 = P[0] if isinstance(P, list) else P
    ctx = sdc.Context(P, prec={"fp64": sdc.PREC_FP64, "fp32jac": sdc.PREC_FP32_JAC,
                               "fp32x2jac": sdc.PREC_FP32X2_JAC}[a.prec])
    U0 = torch.from_numpy(U).cuda()
    Ud = torch.empty_like(U0)
    dt = ctx.cfl_dt(U0, P0.cfl)
    if a.autotune:
        t = ctx.autotune(U0, dt)
        variants = (t.stencil_choice, t.newton_choice)
    else:
        variants = (a.stencil_variant, a.newton_variant)
        ctx.set_variants(*variants)
    out = []
    for i in range(a.warmup + a.steps):
        Ud.copy_(U0)
        if a.eager:
            st, pr = ctx.step_profile(Ud, dt)
            rec = {"stencil_ms": pr.ms_stencil, "newton_ms": pr.ms_newton, "other_ms": pr.ms_other,
                   "fails": st.n_fail}
        else:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            ctx.step(Ud, dt, stats=False)
            ev[1].record()
            torch.cuda.synchronize()
            rec = {"ms": ev[0].elapsed_time(ev[1])}
        if i >= a.warmup:
            out.append(rec)
    torch.cuda.synchronize()
    back = None
    if a.backward:
        gU, gUn = torch.ones_like(U0), torch.empty_like(U0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        ctx.step_backward(U0, dt, gU, gUn)
        ev[1].record()
        torch.cuda.synchronize()
        back = ev[0].elapsed_time(ev[1])
    print(json.dumps({"config": a.config, "seed": seed, "prec": a.prec, "variants": variants,
                      "space_order": a.space_order, "limiter": a.limiter, "nodes": a.nodes, "eager": a.eager, "steps": out,
                      "backward_ms": back}), flush=True)
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
