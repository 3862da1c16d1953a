"""Time one level operator of a hierarchy (a profiling target).

  python -m paper_2405_05047_gb300.opbench --workload td_adaptive --op smooth --prec fp32 --reps 3
  python -m paper_2405_05047_gb300.opbench --workload ns_cavity --steps 3     (driven-cavity steps)
  python -m paper_2405_05047_gb300.opbench --workload batch_small            (one batched launch)
  python -m paper_2405_05047_gb300.opbench --workload td_adaptive --op vcycle --nu 5 --tail-rows 1024
                                                                (whole FP32 V-cycles, small-level kernel)

Sets up the hierarchy of the named workload, runs the operator `reps` times
back to back on the finest level (or --level) through mg_time_op and prints
one JSON line with the mean device time per launch and the algorithmic bytes
of that launch.  Under a profiler, `-k regex:<kernel> -s <warm-up launches>
-c <n>` selects the launches to capture.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

from . import binding as B  # noqa: E402
from . import build as BLD  # noqa: E402

OPS = {"smooth": B.MG_OP_SMOOTH, "matvec": B.MG_OP_MATVEC, "restrict": B.MG_OP_RESTRICT,
       "prolong": B.MG_OP_PROLONG_ADD}


def make(workload):
    if workload == "td_adaptive":
        return (W.td_adaptive(rounds=8, gamma=0.18),
                B.make_problem(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5)), {})
    if workload.startswith("poisson"):
        n = int(workload[len("poisson"):])
        return W.uniform_leaves(2, (1, 1), n.bit_length() - 1), B.make_problem(kind=B.MG_POISSON), {}
    if workload.startswith("elasticity"):
        n = int(workload[len("elasticity"):])
        return (W.elasticity3d(n), B.make_problem(kind=B.MG_ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,)),
                {"omega": 0.5})
    if workload.startswith("oseen"):
        vanka = workload.startswith("oseen_vanka")      # oseen_vanka[rounds]: cell-patch Vanka levels
        rounds = int(workload[len("oseen_vanka" if vanka else "oseen"):] or 12)
        lm = W.oseen_channel(1, rounds)
        beta = W.oseen_beta(B.mg_mesh_nodes(lm))
        okw = {"krylov": B.MG_GMRES}
        if vanka:
            okw["smoother"] = B.MG_SMOOTHER_VANKA
        return (lm, B.make_problem(kind=B.MG_OSEEN, dirichlet=(0xD, 0xD, 0x0), nu=1e-3, dt=0.01, conv=beta), okw)
    raise SystemExit(f"unknown workload {workload}")


def alg_bytes(info, level, nc, op, vbytes):
    """Bytes the operator must move once: stored values + column indices of
    the level matrix (for "vanka": of the level's Vanka matrix) (2 bytes where the level stores 16-bit column offsets,
    else 4; 6 values per 3x3 block where the level stores the
    velocity-pressure pattern, else nc*nc), plus its vectors (x, b, S^-1 and
    the output for a sweep)."""
    nnz = info.level_rows_nnzb[level] * info.level_block_values[level]
    rows = info.level_nodes[level] * nc
    ib = 2 if info.level_col16[level] else 4
    if op == "smooth":
        return nnz * vbytes + info.level_rows_nnzb[level] * ib + rows * vbytes * 3 + info.level_nodes[level] * nc * nc * vbytes
    if op == "matvec":
        return nnz * vbytes + info.level_rows_nnzb[level] * ib + rows * vbytes * 2
    if op == "vanka":       # x_out = x_in + w S r: S (dense nc x nc blocks), r, x_in, x_out
        return info.level_vanka_nnzb[level] * (nc * nc * vbytes + ib) + rows * vbytes * 3
    return None


def run_ns(steps):
    """Three-phase steps of the driven cavity (32x32x64, FP32 multigrid + CG)."""
    import paper_2405_05047_gb300 as G
    ctx = G.Context(0)
    sim = B.NavierStokes(ctx, nx=32, ny=32, nz=64, prec=B.MG_MIXED_FP32, krylov=B.MG_CG, rtol=1e-8, max_it=400)
    st = sim.steps(steps)
    print(json.dumps({"workload": "ns_cavity", "steps": st.steps, "status": st.status, "iters": st.iters,
                      "ms_momentum_per_step": st.ms_momentum / max(st.steps, 1)}))
    sim.free()
    ctx.close()


def run_batch():
    """One batched launch of 304 small Poisson problems (2D 24..72, 3D 12, 20)."""
    import torch
    import paper_2405_05047_gb300 as G
    ctx = G.Context(0)
    hs = [G.Hierarchy(ctx, W.uniform_leaves(2, (m, m), 3), B.make_problem(kind=B.MG_POISSON),
                      B.make_opts(autotune=0)) for m in (3, 5, 7, 9)]
    hs += [G.Hierarchy(ctx, W.uniform_leaves(3, (m, m, m), 2), B.make_problem(kind=B.MG_POISSON),
                       B.make_opts(autotune=0)) for m in (3, 5)]
    probs = [hs[k % len(hs)] for k in range(304)]
    bs, xs = [], []
    for h in probs:
        b = torch.empty(h.n_dofs, device="cuda", dtype=torch.float64)
        h.assemble_rhs(torch.ones(h.n_dofs, device="cuda", dtype=torch.float64), b)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    rc, st = ctx.solve_batch(probs, bs, xs, rtol=1e-8, max_it=200)
    print(json.dumps({"workload": "batch_small", "problems": len(probs), "status": rc, "device_ms": st[0].solve_ms}))
    for h in hs:
        h.free()
    ctx.close()


def run_vcycle(G, ctx, lm, pb, okw, prec, args):
    """`reps` V-cycles of the finest level from a seeded residual; wall time
    per cycle (mg_vcycle synchronises after each one)."""
    import time

    import numpy as np
    import torch
    if args.nu > 0:
        okw.update(nu1=args.nu, nu2=args.nu)
    h = G.Hierarchy(ctx, lm, pb, B.make_opts(**okw))
    if args.tail_rows >= 0:
        h.tune(prec, tail_rows=args.tail_rows, cluster=0)
    dt = torch.float64 if prec == B.MG_FP64 else torch.float32
    r = torch.from_numpy(np.random.default_rng(7).standard_normal(h.n_dofs)).to(device="cuda", dtype=dt)
    z = torch.empty_like(r)
    h.vcycle(r, z, prec)
    t0 = time.perf_counter()
    for _ in range(args.reps):
        h.vcycle(r, z, prec)
    ms = (time.perf_counter() - t0) * 1e3 / args.reps
    print(json.dumps({"workload": args.workload, "op": "vcycle", "prec": args.prec, "levels": h.levels,
                      "tail_levels": h.info.tail_levels, "tail_cluster": h.info.tail_cluster,
                      "nu": args.nu, "ms_per_cycle_wall": ms}))
    h.free()
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="td_adaptive",
                    help="a hierarchy workload (level operator timing), or ns_cavity / batch_small")
    ap.add_argument("--steps", type=int, default=3, help="ns_cavity: time steps")
    ap.add_argument("--op", default="smooth", choices=sorted(OPS) + ["vcycle"])
    ap.add_argument("--nu", type=int, default=0, help="vcycle: pre- and post-smoothing sweeps (0: default)")
    ap.add_argument("--tail-rows", type=int, default=-1,
                    help="vcycle: small-level kernel over the levels of at most this many rows, one CTA in "
                         "shared memory (-1: the setup default)")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--level", type=int, default=-1)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    BLD.build()
    if args.workload == "ns_cavity":
        return run_ns(args.steps)
    if args.workload == "batch_small":
        return run_batch()
    import paper_2405_05047_gb300 as G
    lm, pb, okw = make(args.workload)
    prec = B.MG_MIXED_FP32 if args.prec == "fp32" else B.MG_FP64
    # no setup autotuner: its V-cycles would put many more launches of the
    # same kernels ahead of the timed ones in a profiler's launch list
    okw.update(store_fp64=int(prec == B.MG_FP64), store_fp32=int(prec != B.MG_FP64), autotune=0)
    ctx = G.Context(0)
    if args.op == "vcycle":
        return run_vcycle(G, ctx, lm, pb, okw, prec, args)
    h = G.Hierarchy(ctx, lm, pb, B.make_opts(**okw))
    level = args.level if args.level >= 0 else h.levels - 1
    ms = h.time_op(level, OPS[args.op], prec, reps=args.reps)
    op = "vanka" if args.op == "smooth" and h.info.level_smoother[level] == B.MG_SMOOTHER_VANKA else args.op
    nb = alg_bytes(h.info, level, h.nc, op, 4 if prec != B.MG_FP64 else 8)   # Vanka: the k_vanka update
    print(json.dumps({"workload": args.workload, "op": args.op, "prec": args.prec, "level": level,
                      "rows": int(h.info.level_nodes[level] * h.nc), "ms_per_launch": ms, "alg_bytes": nb,
                      "achieved_gbs": (nb / (ms * 1e-3) / 1e9) if nb else None}))
    h.free()
    ctx.close()


if __name__ == "__main__":
    main()
