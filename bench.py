#!/usr/bin/env python3
"""Benchmark of the GMG-preconditioned Krylov solve on GB300.

Metric: DoF/s to 1e-8 relative residual = free DoFs / device time of one
mg_solve from x0 = 0 until the true FP64 residual satisfies
||b - A x|| <= 1e-8 ||b||, for the FP32-multigrid + FP64-Krylov path (value)
and the plain FP64 path (reported beside it).  One "step" is one such solve.

Default workload: the adaptive 2D transport-diffusion problem (eps = 1e-3,
beta = (1, 0.5), SUPG) on a 1-irregular mesh refined around 16 seeded points
(about 1.2 M nodes), BiCGStab preconditioned by a V(5,5) cycle with damped
Jacobi (NU_TD).  Inputs are synthetic and seeded; L2 is flushed between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload td_adaptive|poisson64|elasticity128|oseen|serving]

Other workloads (same JSON line): poisson64 (64x64 Poisson, CG), elasticityN
(N^3 elasticity, CG), oseen (Oseen/LPS channel, 658 k nodes, GMRES(30)),
serving (a Poisson(200/s) stream of mixed requests through mg_submit/mg_poll:
p50/p99 latency and aggregate DoF/s, plus a rate sweep).

Under torchrun each rank solves its own copy of the workload on its own GPU
(replicas: the solve does not shard); value = all ranks' DoFs / max time.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
if "--impl" in sys.argv and "reference" in sys.argv:      # the oracle arm runs on one host thread
    for _k, _v in {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}.items():
        os.environ[_k] = _v

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "DoF/s to 1e-8 rel. residual (FP32-MG + FP64 Krylov)"
GAMMA_TD = 0.18          # radius decay chosen so that the mesh has ~1.2 M nodes
# Jacobi sweeps before and after the coarse correction on the transport-diffusion
# workload: the paper fixes no number; the one with the shortest time to the
# tolerance on GB300 (V(nu,nu) sweep, nu = 1..8).  The oracle's CPU baseline
# runs the same cycle.
NU_TD = 5


OSEEN_ROUNDS = 12       # refinement rounds towards the circle: ~658 k nodes, ~1.97 M DoFs


def workload(name):
    """(leaf mesh, problem kwargs, opts kwargs, rhs function, description,
    Dirichlet data function or None)."""
    from paper_2405_05047_gb300 import binding as B
    if name in ("oseen", "oseen_small"):
        rounds = OSEEN_ROUNDS if name == "oseen" else 7
        lm = W.oseen_channel(1, rounds)
        xy = B.mg_mesh_nodes(lm)
        pk = dict(kind=B.MG_OSEEN, dirichlet=(0xD, 0xD, 0x0), nu=1e-3, dt=0.01, conv=W.oseen_beta(xy))
        return lm, pk, dict(krylov=B.MG_GMRES, restart=30, smoother=B.MG_SMOOTHER_VANKA), (
            lambda c: np.zeros(c.shape[0] * 3)), (
            "2D Oseen (one backward-Euler step, nu=1e-3, dt=0.01) equal-order Q1 (u,v,p) + LPS on the channel "
            f"[0,2.2]x[0,0.41], 22x4 macro cells refined once, then {rounds} rounds towards the circle "
            "|x-(0.2,0.2)|=0.05 by sibling families, 2:1; seeded divergence-free convection field, parabolic "
            "inflow (lifted), no-slip walls, do-nothing outflow; GMRES(30) + V(2,2) with the additive "
            "cell-patch Vanka smoother (12x12 local problems, w = 1) on every level"), W.oseen_inflow
    if name == "td_adaptive":
        lm = W.td_adaptive(rounds=8, gamma=GAMMA_TD)
        pk = dict(kind=B.MG_TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
        return lm, pk, dict(krylov=B.MG_BICGSTAB, nu1=NU_TD, nu2=NU_TD), (
            lambda xy: W.f_transport(xy, 1e-3, (1.0, 0.5))), (
            "2D transport-diffusion eps=1e-3 beta=(1,0.5) Q1+SUPG, 32x32 start + 8 rounds refined within "
            f"r_k=0.05*2^(-{GAMMA_TD}k) of 16 seeded points, 2:1, hanging nodes; BiCGStab + V({NU_TD},{NU_TD}) "
            "Jacobi w=0.8"), None
    if name == "poisson64":
        lm = W.poisson64(64)
        return lm, dict(kind=B.MG_POISSON), dict(krylov=B.MG_CG), W.f_poisson, (
            "2D Poisson 64x64 Q1, CG + V(2,2) Jacobi w=0.8, 5 levels"), None
    if name.startswith("elasticity"):
        n = int(name[len("elasticity"):] or 128)
        lm = W.elasticity3d(n)
        pk = dict(kind=B.MG_ELASTICITY, mu=1.0, lam=10.0, dirichlet=(0x1,))
        return lm, pk, dict(krylov=B.MG_CG), (
            lambda xyz: np.tile([0.0, 0.0, -1.0], (xyz.shape[0], 1)).ravel()), (
            f"3D linear elasticity {n}^3 Q1 hexes, mu=1 lambda=10, clamped x=0, f=(0,0,-1); "
            "CG + V(2,2) point-block Jacobi, w_l = 1.2/lambda_max(S_l A_l) per level"), None
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------- helpers
def whole_job_rate(dofs_local, steps, t_local_ms, world, device="cpu"):
    """Whole-job DoF/s over replicas: every rank's DoFs x steps divided by the
    slowest rank's time (max over ranks, the bench contract's clock)."""
    import torch
    t = torch.tensor([float(t_local_ms)], dtype=torch.float64, device=device)
    d = torch.tensor([float(dofs_local)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(d, op=dist.ReduceOp.SUM)
    return float(d.item()) * steps / (float(t.item()) * 1e-3), float(t.item())


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: $BENCH_CLOCKS_DIR (default: the system's temporary directory)
        out = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


ONE_THREAD = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def start_oracle_child(outdir, steps=2, rtol=1e-8, procs=8):
    """The oracle on the headline workload itself, in a child process started
    before this process touches the GPU (it runs on the host cores while the
    GPU is measured).  It writes oracle.json (CPU baseline: one thread, then
    `procs` concurrent single-thread solves) and the FP64 reference solution
    to rtol 1e-12 with the lumped-mass weights (xref.npy, w.npy) to outdir."""
    env = dict(os.environ, **ONE_THREAD)
    code = f"import bench; bench._oracle_child({outdir!r}, {steps}, {rtol}, {procs})"
    log = open(os.path.join(outdir, "oracle.log"), "w")
    return subprocess.Popen([sys.executable, "-c", code], cwd=ROOT, env=env, stdout=log, stderr=subprocess.STDOUT)


def _oracle_system(rounds=8):
    """Oracle hierarchy, finest system and right-hand side of the adaptive TD
    workload (setup, not timed)."""
    from oracle import fem, mg
    from oracle import problems as PB
    lm = W.td_adaptive(rounds=rounds, gamma=GAMMA_TD)
    prob = PB.Problem(PB.TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
    Hh = mg.Hierarchy(lm, prob, nu1=NU_TD, nu2=NU_TD)
    S = Hh.fine.sys
    S.F = fem.assemble(Hh.fine.mesh, PB.load_element(prob, 2), 1)
    b = S.rhs(W.f_transport(Hh.fine.mesh.coords, 1e-3, (1.0, 0.5)))
    return Hh, S, b


def _oracle_child(outdir, steps, rtol, procs):
    import multiprocessing as mp
    from oracle import krylov
    t0 = time.perf_counter()
    Hh, S, b = _oracle_system()
    t_setup = time.perf_counter() - t0
    n_free = int((~S.fixed).sum())
    times, iters = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        _, info = krylov.bicgstab(Hh.fine.A, b, Hh.precondition, rtol=rtol, maxit=500)
        times.append(time.perf_counter() - t0)
        iters.append(info["iters"])
    t1 = statistics.mean(times)
    out = {"value": n_free / t1, "unit": "DoF/s", "cores": 1, "kind": "oracle",
           "sample": f"oracle (numpy/scipy FP64) BiCGStab+V({NU_TD},{NU_TD}) solve to {rtol:g} of the headline TD "
                     f"workload itself ({n_free} free DoFs, {len(Hh.levels)} levels), mean of {steps} solves, one "
                     f"host thread, setup {t_setup:.0f} s untimed",
           "iters": iters, "sec_per_solve": t1}

    # `procs` concurrent single-thread solves (forked after setup; no GPU in this process)
    def one(q):
        t = time.perf_counter()
        krylov.bicgstab(Hh.fine.A, b, Hh.precondition, rtol=rtol, maxit=500)
        q.put(time.perf_counter() - t)
    try:
        ctx = mp.get_context("fork")
        q = ctx.Queue()
        t0 = time.perf_counter()
        ps = [ctx.Process(target=one, args=(q,)) for _ in range(procs)]
        for p in ps:
            p.start()
        walls = [q.get(timeout=900) for _ in ps]
        for p in ps:
            p.join()
        span = time.perf_counter() - t0
        out["concurrent"] = {"cores": procs, "value": procs * n_free / span, "unit": "DoF/s",
                             "sample": f"{procs} single-thread oracle solves of the same system at once "
                                       f"(forked processes, {os.cpu_count()} host cores); value = {procs} x free "
                                       f"DoFs / wall time of all",
                             "sec_per_solve_max": max(walls)}
    except Exception as e:          # reported, never required
        out["concurrent"] = {"error": str(e)}
    t0 = time.perf_counter()
    xref, info = krylov.bicgstab(Hh.fine.A, b, Hh.precondition, rtol=1e-12, maxit=500)
    xall = S.H @ xref
    np.save(os.path.join(outdir, "xref.npy"), xall)
    np.save(os.path.join(outdir, "w.npy"), np.asarray(S.F.sum(axis=1)).ravel())
    out["reference_solve"] = {"rtol": 1e-12, "true_rel": info["true_rel"], "sec": time.perf_counter() - t0}
    with open(os.path.join(outdir, "oracle.json"), "w") as f:
        json.dump(out, f)


def rel_err(x, xref, w):
    """Relative lumped-mass-weighted L2 error ||x - xref||_M / ||xref||_M."""
    e = np.asarray(x, dtype=np.float64) - xref
    return float(np.sqrt(np.sum(w * e * e) / np.sum(w * xref * xref)))


def cpu_baseline(steps=4, rounds=7, rtol=1e-8, threads=1):
    """The oracle (numpy/scipy FP64, as it stands) on a bounded sample of the
    same workload (the adaptive TD mesh with `rounds` refinement rounds), run
    in a child process with `threads` BLAS/OpenMP threads."""
    env = dict(os.environ, **{k: str(threads) for k in ONE_THREAD})
    code = (f"import json, bench; print(json.dumps(bench._cpu_baseline_inproc({steps}, {rounds}, {rtol}, {threads})))")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr[-500:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def _cpu_baseline_inproc(steps, rounds, rtol, threads=1):
    from oracle import krylov, mg
    from oracle import problems as PB
    lm = W.td_adaptive(rounds=rounds, gamma=GAMMA_TD)
    prob = PB.Problem(PB.TRANSPORT, eps=1e-3, beta=(1.0, 0.5))
    t0 = time.perf_counter()
    Hh = mg.Hierarchy(lm, prob, nu1=NU_TD, nu2=NU_TD)
    s = PB.build_system(Hh.fine.mesh, prob)
    b = s.rhs(W.f_transport(Hh.fine.mesh.coords, 1e-3, (1.0, 0.5)))
    t_setup = time.perf_counter() - t0
    n_free = int((~s.fixed).sum())
    times, iters = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        x, info = krylov.bicgstab(Hh.fine.A, b, Hh.precondition, rtol=rtol, maxit=500)
        times.append(time.perf_counter() - t0)
        iters.append(info["iters"])
    t = statistics.mean(times)
    return {"value": n_free / t, "unit": "DoF/s", "cores": threads, "kind": "oracle",
            "sample": f"oracle BiCGStab+V({NU_TD},{NU_TD}) FP64 solve to {rtol:g} of the same TD workload with {rounds} "
                      f"refinement rounds ({n_free} free DoFs, {len(Hh.levels)} levels), mean of {steps} solves, "
                      f"{threads} thread(s) (setup {t_setup:.1f}s untimed)",
            "iters": iters, "sec_per_solve": t}


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle as it stands (numpy/scipy FP64, one host thread) on the
    headline workload itself: setup untimed, then --warmup and --steps solves
    of the same system to 1e-8."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    from oracle import krylov
    t0 = time.perf_counter()
    Hh, S, b = _oracle_system()
    t_setup = time.perf_counter() - t0
    n_free = int((~S.fixed).sum())
    for _ in range(warm):
        krylov.bicgstab(Hh.fine.A, b, Hh.precondition, rtol=args.rtol)
    t0 = time.perf_counter()
    for _ in range(steps):
        krylov.bicgstab(Hh.fine.A, b, Hh.precondition, rtol=args.rtol)
    dt = (time.perf_counter() - t0) / max(steps, 1)
    value = n_free / dt
    sample = (f"oracle BiCGStab+V({NU_TD},{NU_TD}) FP64 solve to {args.rtol:g} of the headline TD workload itself "
              f"({n_free} free DoFs), one host thread, setup {t_setup:.0f} s untimed")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "td_adaptive", "n_free_dofs": n_free, "same_config": True},
        "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------- serving workload
SERVE_EPS = (1e-3, 1e-2, 1e-1, 1.0)


def serve_sizes(lo, hi, mult, odd_max):
    """Mesh sizes n = m 2^L (m odd <= odd_max) in [lo, hi] that are multiples
    of `mult`: the macro grid is m^dim cells, so the coarsest level (and its
    dense direct solve) stays small."""
    out = set()
    for m in range(1, odd_max + 1, 2):
        n = m
        while n <= hi:
            if n >= lo and n % mult == 0:
                out.add(n)
            n *= 2
    return tuple(sorted(out))


SERVE_2D = serve_sizes(16, 1024, 8, 15)
SERVE_3D = serve_sizes(8, 96, 4, 7)


def _serve_mesh(dim, n):
    m = n
    while m % 2 == 0:
        m //= 2
    return W.uniform_leaves(dim, (m,) * dim, int(round(np.log2(n // m))))


def serving_stream(n_req, rate, seed=W.MASTER_SEED):
    """Seeded request stream: arrival times (Poisson process), kind, size,
    eps and RHS seed.  Sizes log-uniform in 16..1024 (2D) / 8..96 (3D),
    rounded to the nearest multiple of 8 (2D) / 4 (3D) whose odd factor is
    small (SERVE_2D, SERVE_3D); eps log-uniform in [1e-3, 1], rounded to the
    nearest power of ten so that operators are shared by requests."""
    rng = np.random.Generator(np.random.PCG64([seed, 4]))
    t = np.cumsum(rng.exponential(1.0 / rate, n_req))
    out = []
    for k in range(n_req):
        kind = int(rng.integers(4))             # 0: 2D Poisson, 1: 2D TD, 2: 3D Poisson, 3: 3D TD
        dim = 2 if kind < 2 else 3
        if dim == 2:
            n = 2.0 ** rng.uniform(4, 10)
            cat = SERVE_2D
        else:
            n = 2.0 ** rng.uniform(3, np.log2(96))
            cat = SERVE_3D
        n = min(cat, key=lambda c: abs(np.log(c) - np.log(n)))
        eps = 10.0 ** rng.uniform(-3, 0)
        eps = min(SERVE_EPS, key=lambda e: abs(np.log(e) - np.log(eps))) if kind in (1, 3) else 1.0
        out.append((float(t[k]), kind, dim, n, eps, int(rng.integers(1 << 30))))
    return out


def run_serving(args):
    import torch
    import paper_2405_05047_gb300 as G
    from paper_2405_05047_gb300 import binding as B
    from paper_2405_05047_gb300 import build as BLD
    BLD.build()
    stream = serving_stream(args.requests, args.rate)
    ctx = G.Context(0)
    ctx.serve_config(args.slots)
    hiers = {}
    t0 = time.perf_counter()
    for (_, kind, dim, n, eps, _) in stream:
        key = (kind, n, eps)
        if key in hiers:
            continue
        beta = (1.0, 0.5) if dim == 2 else (1.0, 0.5, 0.25)
        pk = dict(kind=B.MG_POISSON) if kind in (0, 2) else dict(kind=B.MG_TRANSPORT, eps=eps, beta=beta)
        # transport: the cell-patch Vanka smoother (damped Jacobi does not
        # converge on the convection-dominated 3D requests, eps = 1e-3)
        ok = dict(krylov=B.MG_CG, store_fp64=0) if kind in (0, 2) else dict(
            krylov=B.MG_BICGSTAB, store_fp64=0, smoother=B.MG_SMOOTHER_VANKA)
        hiers[key] = G.Hierarchy(ctx, _serve_mesh(dim, n), B.make_problem(**pk), B.make_opts(**ok))
    setup_s = time.perf_counter() - t0
    # solve slots reserved up front (workspaces and their graphs): the
    # scheduler never allocates on the serving path
    t0 = time.perf_counter()
    for h in hiers.values():
        ctx.serve_reserve(h, args.reserve, B.MG_MIXED_FP32)
    reserve_s = time.perf_counter() - t0
    # right-hand sides: f = a0 + seeded low-frequency modes, assembled by the library
    reqs = []
    for (ta, kind, dim, n, eps, seed) in stream:
        h = hiers[(kind, n, eps)]
        rng = np.random.Generator(np.random.PCG64(seed))
        xy = h.coords()
        a = rng.standard_normal(5)
        f = a[0] + sum(a[m] * np.prod(np.sin(m * np.pi * xy), axis=1) for m in range(1, 5))
        b = torch.empty(h.n_dofs, device="cuda", dtype=torch.float64)
        h.assemble_rhs(torch.from_numpy(np.ascontiguousarray(f)).cuda(), b)
        reqs.append((ta, h, b, torch.zeros_like(b)))
    torch.cuda.synchronize()

    def play(rate_scale):
        for (_, _, _, x) in reqs:
            x.zero_()
        torch.cuda.synchronize()
        gc.collect()
        gc.disable()           # no collector pauses inside the client's polling loop
        try:
            return _play(rate_scale)
        finally:
            gc.enable()

    def _play(rate_scale):
        pending = {}
        done_t = {}
        stats = {}
        start = time.perf_counter()
        limit = 60.0 + 2.0 * reqs[-1][0] / rate_scale
        next_log = 10.0
        i = 0
        while i < len(reqs) or pending:
            now = time.perf_counter() - start
            if now > next_log:
                print(f"[serving] replay x{rate_scale:g}: {i}/{len(reqs)} submitted, {len(pending)} pending, "
                      f"{len(done_t)} done at {now:.1f} s", file=sys.stderr, flush=True)
                next_log += 10.0
            if now > limit:
                raise RuntimeError(f"serving replay x{rate_scale:g}: {len(pending)} requests still pending after "
                                   f"{now:.0f} s ({i} of {len(reqs)} submitted)")
            while i < len(reqs) and reqs[i][0] / rate_scale <= now:
                ta, h, b, x = reqs[i]
                pending[ctx.submit(h, b, x, rtol=1e-8, max_it=500)] = i
                i += 1
            for t in list(pending):
                rc, st = ctx.poll(t)
                if rc != B.MG_PENDING:
                    k = pending.pop(t)
                    done_t[k] = time.perf_counter() - start
                    stats[k] = (rc, st.iters, st.rel_res, st.setup_ms + st.solve_ms, st.launches)
            if not pending and i < len(reqs):
                time.sleep(max(0.0, reqs[i][0] / rate_scale - (time.perf_counter() - start)))
        lat = np.array([done_t[k] - reqs[k][0] / rate_scale for k in range(len(reqs))]) * 1e3
        span = max(done_t.values()) - reqs[0][0] / rate_scale
        dofs = sum(reqs[k][1].info.n_free for k in range(len(reqs)))
        ok = all(stats[k][0] == 0 and stats[k][2] <= 1e-8 for k in stats)
        iterated = all(stats[k][1] > 0 for k in stats)
        # the library's own submit-to-finish time (queue + device), without the client's polling
        lib = np.array([stats[k][3] for k in range(len(reqs))])
        return {"rate_req_s": args.rate * rate_scale, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                "lib_p50_ms": float(np.percentile(lib, 50)), "lib_p99_ms": float(np.percentile(lib, 99)),
                "dof_per_s": dofs / span, "span_s": span, "all_converged": ok, "all_iterated": iterated,
                "batched_requests": sum(int(stats[k][4] <= 2) for k in stats)}

    def log(msg):
        print(f"[serving {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)

    log(f"{len(hiers)} operators set up in {setup_s:.1f} s, slots reserved in {reserve_s:.1f} s")
    play(1.0)                                   # warm-up: graphs, pooled workspaces
    base = play(1.0)
    log(f"base stream: p50 {base['p50_ms']:.2f} ms, p99 {base['p99_ms']:.2f} ms")
    mixed = [r[3].clone() for r in reqs]        # every result of the measured stream
    sweep = [play(s) for s in args.sweep]
    sizes = [r[1].info.n_free for r in reqs]
    # verification: each result solved (iterations > 0, residual reached) and,
    # on a seeded subset, bitwise equal to the same solve run alone
    rng = np.random.Generator(np.random.PCG64([W.MASTER_SEED, 5]))
    subset = sorted(rng.choice(len(reqs), size=min(64, len(reqs)), replace=False).tolist())
    same = 0
    for k in subset:
        _, h, b, x = reqs[k]
        x.zero_()
        st = h.solve(b, x, rtol=1e-8, max_it=500, prec=B.MG_MIXED_FP32)
        same += int(st.status == 0 and torch.equal(x, mixed[k]))
    verified = {"all_converged": base["all_converged"], "all_iterated": base["all_iterated"],
                "alone_equals_mix": f"{same}/{len(subset)}"}
    # the same stream with batched launches on: whenever two or more queued
    # requests fit the batched kernel they go out as one launch
    log("sweep and verification done; batched launches on")
    ctx.serve_batching(256, 2)
    play(1.0)
    bbase = play(1.0)
    log(f"batched base stream: p50 {bbase['p50_ms']:.2f} ms, {bbase['batched_requests']} batched")
    bmixed = [r[3].clone() for r in reqs]
    bsweep = [play(s) for s in args.sweep]
    log("batched sweep done")
    ctx.serve_batching(0, 2)
    same_b = 0
    for k in subset:
        _, h, b, x = reqs[k]
        x.zero_()
        if h.batch_fits(B.MG_MIXED_FP32):
            rc, (st,) = ctx.solve_batch([h], [b], [x], rtol=1e-8, max_it=500, prec=B.MG_MIXED_FP32)
            eq = torch.equal(x, bmixed[k]) or torch.equal(mixed[k], bmixed[k])
        else:
            st = h.solve(b, x, rtol=1e-8, max_it=500, prec=B.MG_MIXED_FP32)
            eq = torch.equal(x, bmixed[k])
        same_b += int(st.status == 0 and eq)
    batched = {"p50_ms": bbase["p50_ms"], "p99_ms": bbase["p99_ms"], "dof_per_s": bbase["dof_per_s"],
               "batched_requests": bbase["batched_requests"], "sweep": bsweep,
               "verified": {"all_converged": bbase["all_converged"], "all_iterated": bbase["all_iterated"],
                            "result_equals_its_path_alone": f"{same_b}/{len(subset)}"},
               "note": "mg_serve_batching(256, 2): two or more queued requests that fit the batched kernel "
                       "(Poisson at 2D n <= 80 / 3D n <= 20 here; transport requests smooth with Vanka and "
                       "take the graph path) go out as one launch; a batched result equals mg_solve_batch of "
                       "that request alone, a graph one mg_solve"}
    print(json.dumps({
        "metric": "serving p50/p99 latency and aggregate DoF/s (FP32-MG + FP64 Krylov, rtol 1e-8)",
        "value": base["dof_per_s"], "unit": "DoF/s", "n_gpus": 1, "steps": len(reqs), "warmup": len(reqs),
        "ms_per_step": base["mean_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-mg+f64", "data": "synthetic",
        "config": {"workload": "serving", "requests": len(reqs), "rate_req_s": args.rate, "slots": args.slots,
                   "catalogue": {"2d": SERVE_2D, "3d": SERVE_3D, "eps": SERVE_EPS},
                   "operators_resident": len(hiers), "mean_dofs": float(np.mean(sizes)),
                   "setup_s": setup_s, "reserved_slots_per_operator": args.reserve, "reserve_s": reserve_s,
                   "smoothers": "Poisson: damped Jacobi, CG; transport: cell-patch Vanka, BiCGStab; V(2,2)"},
        "p50_ms": base["p50_ms"], "p99_ms": base["p99_ms"], "verified": verified,
        "lib_p50_ms": base["lib_p50_ms"], "lib_p99_ms": base["lib_p99_ms"],
        "sweep": sweep, "batched": batched,
    }))
    for h in hiers.values():
        h.free()
    ctx.close()


EL_RUNS = (("face", 5), ("edge", 6), ("vertex", 6))
EL_PAPER_H100_S = {("face", 5): 122.57, ("edge", 6): 14.7, ("vertex", 6): 7.9}   # Tables tab:elasticity:times:*


def measure_elastodyn(G, B, ctx, kind, levels, rtol=1e-8, steps=None, oracle_check=False):
    """The paper's elastodynamics run (Sec. 5.2) on one adaptive hex mesh:
    100 backward-Euler steps (dt = 0.025) of the first-order system in
    (u, v) through mg_time_steps2 (v eliminated: CG + V(2,2) point-block
    Jacobi on M/dt^2 + K per step, warm-started), f = (0, -1, 0), clamped
    boundary, zero initial data."""
    import torch
    steps = steps or W.EL_STEPS
    dt = W.EL_DT
    lm = W.elasticity_adaptive(kind, levels)
    pk = dict(kind=B.MG_ELASTICITY, mu=W.EL_MU, lam=W.EL_LAMBDA, dirichlet=(0x3F,), mass=1.0 / dt ** 2)
    t0 = time.perf_counter()
    h = G.Hierarchy(ctx, lm, B.make_problem(**pk), B.make_opts(krylov=B.MG_CG))
    setup_s = time.perf_counter() - t0
    nd = h.n_dofs
    f = torch.from_numpy(np.tile(W.EL_F, h.n_nodes)).cuda()
    fs = f.unsqueeze(0).expand(steps, nd).contiguous()
    out = {"mesh": f"{kind} refinement, level {levels}", "nodes": int(h.n_nodes),
           "hanging_nodes": int(h.info.n_hanging), "paper_dofs": int(6 * h.n_nodes), "levels": int(h.levels),
           "steps": steps, "setup_s": setup_s}
    for key, prec in (("mixed", B.MG_MIXED_FP32), ("fp64", B.MG_FP64)):
        u = torch.zeros(nd, device="cuda", dtype=torch.float64)
        v = torch.zeros_like(u)
        h.time_steps2(u, v, fs, None, 3, dt, rtol=rtol, max_it=300, prec=prec)        # warm-up
        u.zero_()
        v.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        rc, sts = h.time_steps2(u, v, fs, None, steps, dt, rtol=rtol, max_it=300, prec=prec)
        e1.record(ctx.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out[key] = {"s": ms * 1e-3, "dof_steps_per_s": 6 * h.n_nodes * steps / (ms * 1e-3), "status": rc,
                    "iters_total": int(sum(s_.iters for s_ in sts)), "iters_max": int(max(s_.iters for s_ in sts)),
                    "rel_res_max": float(max(s_.rel_res for s_ in sts)),
                    "launches": int(sum(s_.launches for s_ in sts))}
        out[key + "_u"] = u.cpu().numpy()
    if oracle_check:
        from oracle import mesh as M
        from oracle import problems as PB
        from oracle import timestep as TS
        m = M.Q1Mesh(3, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor)
        prob = PB.Problem(PB.ELASTICITY, mu=W.EL_MU, lam=W.EL_LAMBDA, dirichlet=(0x3F,))
        fn = np.tile(W.EL_F, m.n_nodes)
        S, ref = TS.run_first_order(m, prob, dt, np.zeros(nd), np.zeros(nd), lambda t: fn, lambda t: None, steps)
        w = np.repeat(np.asarray(S.F.sum(axis=1)).ravel(), 3)
        for key in ("mixed", "fp64"):
            out[key]["err_vs_oracle_u"] = rel_err(out[key + "_u"], ref[-1][0], w)
    for key in ("mixed", "fp64"):
        out.pop(key + "_u")
    out["paper_h100_solve_s"] = EL_PAPER_H100_S.get((kind, levels))
    h.free()
    return out


# ---------------------------------------------------------------- our arm
def flush_l2(buf):
    buf.add_(1.0)


class Solver:
    """One resident hierarchy of a workload with its right-hand side, timed
    through mg_solve (CUDA events on the library's stream, L2 flushed before
    every timed solve)."""

    def __init__(self, G, B, ctx, name, flush, launch="graph", tail=None):
        import torch
        self.B, self.ctx, self.flush, self.name = B, ctx, flush, name
        lm, pk, ok, ffun, desc, gfun = workload(name)
        self.lm, self.pk, self.ok, self.desc = lm, pk, dict(ok), desc
        ok["launch_mode"] = 1 if launch == "direct" else 0
        ok["store_bf16"] = 1
        if tail:
            ok["autotune"] = 0
        t0 = time.perf_counter()
        self.h = G.Hierarchy(ctx, lm, B.make_problem(**pk), B.make_opts(**ok))
        if tail:
            rows, cl = (int(v) for v in tail.split(","))
            for p in (B.MG_MIXED_FP32, B.MG_FP64, B.MG_MIXED_BF16):
                self.h.tune(p, rows, cl)
        self.setup_s = time.perf_counter() - t0
        self.info = self.h.info
        self.coords = self.h.coords()
        self.f_host = np.ascontiguousarray(ffun(self.coords), dtype=np.float64)
        self.g_host = None if gfun is None else np.ascontiguousarray(gfun(self.coords), dtype=np.float64).ravel()
        f = torch.from_numpy(self.f_host).cuda()
        self.b = torch.empty(self.h.n_dofs, device="cuda", dtype=torch.float64)
        g = None if self.g_host is None else torch.from_numpy(self.g_host).cuda()
        self.h.assemble_rhs(f, self.b, g)
        self.x = torch.zeros_like(self.b)

    def timed(self, prec, k, warm, rtol, hh=None):
        import torch
        hh = hh or self.h
        stats, ms = [], []
        for _ in range(warm):
            self.x.zero_()
            hh.solve(self.b, self.x, rtol=rtol, max_it=500, prec=prec)
        for _ in range(k):
            self.x.zero_()
            flush_l2(self.flush)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.ctx.stream)
            st = hh.solve(self.b, self.x, rtol=rtol, max_it=500, prec=prec)
            e1.record(self.ctx.stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            stats.append(st)
        return ms, stats, self.x.cpu().numpy()

    def profile(self, prec, k, rtol, iters_expected=None):
        """Per-kernel device time inside k solves (mg_solve_profiled), summed
        per (kernel, level); returns (table, floor_ms per interval)."""
        import torch
        prof = {}
        for _ in range(k):
            self.x.zero_()
            flush_l2(self.flush)
            torch.cuda.synchronize()
            st_p, ents = self.h.solve_profiled(self.b, self.x, rtol=rtol, max_it=500, prec=prec)
            assert st_p.status == 0, st_p.as_dict()
            if iters_expected is not None:
                assert st_p.iters == iters_expected, (st_p.iters, iters_expected)
            for e in ents:
                a = prof.setdefault((e["kernel"], e["level"]), [0, 0.0])
                a[0] += e["launches"]
                a[1] += e["ms"]
        floor_n, floor_ms = prof.pop(("k_prof_empty", -2), [1, 0.0])
        return prof, floor_ms / floor_n

    def smoother_roofline(self, prof, floor_ms, peak):
        """Roofline of the finest-level fused FP32 smoother sweep (a2 / a3):
        algorithmic bytes per launch / its mean interval inside the solve."""
        from paper_2405_05047_gb300 import opbench
        fine = self.h.levels - 1
        total = sum(v[1] for v in prof.values())
        vanka = self.info.level_smoother[fine] == self.B.MG_SMOOTHER_VANKA
        key = "k_vanka<float" if vanka else "k_smooth<float"
        cand = [kv for kv in prof.items() if kv[0][0].startswith(key) and kv[0][1] == fine
                and (vanka or ", false," in kv[0][0])]
        (name, _), (n, ms) = max(cand, key=lambda kv: kv[1][1])
        alg = opbench.alg_bytes(self.info, fine, self.h.nc, "vanka" if vanka else "smooth", 4)
        ach = alg / (ms / n * 1e-3) / 1e9
        what = "Vanka update x + w S r" if vanka else "fused residual + (block-)Jacobi sweep"
        return {"bound": "hbm", "kernel": f"{name} on the finest level ({what})", "achieved": ach, "peak": peak,
                "unit": "GB/s", "frac": ach / peak, "alg_bytes_per_launch": int(alg), "ms_per_launch": ms / n,
                "launches_timed": int(n), "share_of_solve": ms / total, "interval_floor_ms": floor_ms}

    def free(self):
        self.h.free()


def top_table(prof, k=12):
    total = sum(v[1] for v in prof.values())
    ranked = sorted(prof.items(), key=lambda kv: -kv[1][1])
    return [{"kernel": kk, "level": l, "launches": n, "ms": round(t, 4), "share": round(t / total, 4)}
            for (kk, l), (n, t) in ranked[:k]]


def oracle_reference(name, coords_check=None):
    """The oracle's FP64 solution of a (small) workload by sparse LU (3D
    elasticity: the oracle's MG-CG to 1e-12), with the lumped-mass weights:
    (x_all, w)."""
    import scipy.sparse.linalg as spl
    from oracle import mesh as M
    from oracle import problems as PB
    lm, pk, _, ffun, _, gfun = workload(name)
    from paper_2405_05047_gb300 import binding as B
    kind = {B.MG_POISSON: PB.POISSON, B.MG_TRANSPORT: PB.TRANSPORT, B.MG_ELASTICITY: PB.ELASTICITY,
            B.MG_OSEEN: PB.OSEEN}[pk["kind"]]
    kw = {k: v for k, v in pk.items() if k in ("eps", "beta", "mu", "nu", "dt", "conv")}
    if "lam" in pk:
        kw["lam"] = pk["lam"]
    if "dirichlet" in pk:
        kw["dirichlet"] = pk["dirichlet"]
    prob = PB.Problem(kind, **kw)
    m = M.Q1Mesh(lm.dim, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor)
    if coords_check is not None:
        assert np.array_equal(m.coords, coords_check)
    S = PB.build_system(m, prob, beta=prob.conv)
    g = None if gfun is None else gfun(m.coords).ravel()
    b = S.rhs(ffun(m.coords), g)
    if kind == PB.ELASTICITY:     # 3D: sparse LU fills in; the oracle's own MG-CG to 1e-12 instead
        from oracle import krylov, mg
        Hh = mg.Hierarchy(lm, prob)
        x, _ = krylov.pcg(Hh.fine.A, b, Hh.precondition, rtol=1e-12, maxit=500)
    else:
        x = spl.spsolve(S.A.tocsc(), b)
    w = np.repeat(np.asarray(S.F.sum(axis=1)).ravel(), prob.nc)
    return S.H @ x, w


def err_on_sample(G, B, ctx, name, flush, rtol=1e-10):
    """Error of both GPU paths against the oracle's solve on a smaller
    instance of the same workload (the full-size system does not fit the
    oracle): relative lumped-mass L2 at rtol 1e-10."""
    sv = Solver(G, B, ctx, name, flush)
    xref, w = oracle_reference(name, sv.coords)
    out = {"workload": name, "n_free_dofs": int(sv.info.n_free), "rtol": rtol}
    for key, prec in (("mixed", B.MG_MIXED_FP32), ("fp64", B.MG_FP64)):
        _, st, x = sv.timed(prec, 1, 0, rtol)
        out[key] = {"err": rel_err(x, xref, w), "rel_res": st[0].rel_res, "iters": st[0].iters}
    sv.free()
    return out


def measure_config(G, B, ctx, name, flush, peak, steps=3, rtol=1e-8, err_sample=None):
    """Compact record of one more configuration: both precisions, the BF16
    ablation, the in-solve roofline of the finest smoother sweep and the error
    against the oracle (on the full size where the oracle's direct solve fits,
    else on `err_sample`, a smaller instance of the same workload)."""
    sv = Solver(G, B, ctx, name, flush)
    n_free = int(sv.info.n_free)
    ms32, st32, x32 = sv.timed(B.MG_MIXED_FP32, steps, 1, rtol)
    ms64, st64, x64 = sv.timed(B.MG_FP64, max(2, steps - 1), 1, rtol)
    ms16, st16, _ = sv.timed(B.MG_MIXED_BF16, 2, 1, rtol)
    prof, floor = sv.profile(B.MG_MIXED_FP32, 1, rtol, st32[0].iters)
    rec = {"description": sv.desc, "n_nodes": int(sv.info.n_nodes), "n_free_dofs": n_free,
           "levels": int(sv.info.levels), "setup_s": sv.setup_s,
           "value": n_free / (statistics.mean(ms32) * 1e-3), "unit": "DoF/s", "ms_per_step": statistics.mean(ms32),
           "iters": [s.iters for s in st32], "rel_res": max(s.rel_res for s in st32),
           "converged": all(s.status == 0 for s in st32 + st64),
           "fp64": {"value": n_free / (statistics.mean(ms64) * 1e-3), "ms_per_step": statistics.mean(ms64),
                    "iters": [s.iters for s in st64], "rel_res": max(s.rel_res for s in st64)},
           "speedup_mixed_vs_fp64": statistics.mean(ms64) / statistics.mean(ms32),
           "bf16_values_ablation": {"value": n_free / (statistics.mean(ms16) * 1e-3),
                                    "ms_per_step": statistics.mean(ms16), "iters": [s.iters for s in st16],
                                    "converged": all(s.status == 0 for s in st16)},
           "roofline": sv.smoother_roofline(prof, floor, peak),
           "top_kernels_in_solve": top_table(prof, 5)}
    if sv.ok.get("smoother") == B.MG_SMOOTHER_VANKA:
        # the same solve with the point-block Jacobi smoother, for comparison
        hj = G.Hierarchy(ctx, sv.lm, B.make_problem(**sv.pk), B.make_opts(**dict(sv.ok, smoother=0)))
        msj, stj, _ = sv.timed(B.MG_MIXED_FP32, 2, 1, rtol, hj)
        rec["point_block_jacobi"] = {"value": n_free / (statistics.mean(msj) * 1e-3),
                                     "ms_per_step": statistics.mean(msj), "iters": [s_.iters for s_ in stj]}
        hj.free()
    if err_sample is None:
        xref, w = oracle_reference(name, sv.coords)
        rec["err_vs_oracle"] = rel_err(x32, xref, w)
        rec["fp64_err_vs_oracle"] = rel_err(x64, xref, w)
        rec["err_note"] = f"relative lumped-mass L2 against the oracle's sparse LU solve, at rtol {rtol:g}"
    if name.startswith("elasticity"):
        okd = dict(sv.ok, store_bf16=0, inner_rtol=1e-4)
        hd = G.Hierarchy(ctx, sv.lm, B.make_problem(**sv.pk), B.make_opts(**okd))
        msd, std, _ = sv.timed(B.MG_MIXED_FP32, 2, 1, rtol, hd)
        rec["defect_correction"] = {"value": n_free / (statistics.mean(msd) * 1e-3),
                                    "ms_per_step": statistics.mean(msd), "inner_rtol": 1e-4,
                                    "iters": [s.iters for s in std], "rel_res": max(s.rel_res for s in std),
                                    "converged": all(s.status == 0 for s in std)}
        hd.free()
    sv.free()
    if err_sample is not None:
        rec["err_vs_oracle_sample"] = err_on_sample(G, B, ctx, err_sample, flush)
    return rec


BATCH_2D = tuple(n for n in SERVE_2D if n <= 80)
BATCH_3D = tuple(n for n in SERVE_3D if n <= 20)


def measure_batch(G, B, ctx, n_req=1000, rtol=1e-8, reps=3):
    """Many small uneven problems in one launch (mg_solve_batch) against the
    same problems through the serving path (every request submitted at once,
    one graph per request on concurrent streams).  Problems: the serving
    stream's kinds (2D / 3D Poisson and transport-diffusion, eps as there),
    sizes log-uniform over the catalogue sizes whose V-cycle fits the
    batched kernel (2D n <= 80, 3D n <= 20), seeded right-hand sides; the
    transport problems smooth with damped Jacobi here (the batched kernel's
    smoother) at eps >= 1e-2.  Hierarchies and right-hand sides are set up
    before the timed region."""
    import torch
    rng = np.random.Generator(np.random.PCG64([W.MASTER_SEED, 6]))
    hiers, probs = {}, []
    for _ in range(n_req):
        kind = int(rng.integers(4))
        dim = 2 if kind < 2 else 3
        cat = BATCH_2D if dim == 2 else BATCH_3D
        n = int(cat[int(rng.integers(len(cat)))])
        eps = float(10.0 ** rng.integers(-2, 1)) if kind in (1, 3) else 1.0
        key = (kind, n, eps)
        if key not in hiers:
            beta = (1.0, 0.5) if dim == 2 else (1.0, 0.5, 0.25)
            pk = dict(kind=B.MG_POISSON) if kind in (0, 2) else dict(kind=B.MG_TRANSPORT, eps=eps, beta=beta)
            hiers[key] = G.Hierarchy(ctx, _serve_mesh(dim, n), B.make_problem(**pk),
                                     B.make_opts(store_fp64=0, autotune=0))
        probs.append((hiers[key], int(rng.integers(1 << 30))))
    hs, bs = [], []
    for h, seed in probs:
        r = np.random.Generator(np.random.PCG64(seed))
        xy = h.coords()
        a = r.standard_normal(5)
        f = a[0] + sum(a[m] * np.prod(np.sin(m * np.pi * xy), axis=1) for m in range(1, 5))
        b = torch.empty(h.n_dofs, device="cuda", dtype=torch.float64)
        h.assemble_rhs(torch.from_numpy(np.ascontiguousarray(f)).cuda(), b)
        hs.append(h)
        bs.append(b)
    xs = [torch.zeros_like(b) for b in bs]
    dofs = sum(int(h.info.n_free) for h in hs)
    assert all(h.batch_fits(B.MG_MIXED_FP32) for h in hs)
    dev_ms, wall_ms = [], []
    for _ in range(reps + 1):
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = ctx.solve_batch(hs, bs, xs, rtol=rtol, max_it=500, prec=B.MG_MIXED_FP32)
        wall_ms.append((time.perf_counter() - t0) * 1e3)
        dev_ms.append(st[0].solve_ms)
    dev_ms, wall_ms = dev_ms[1:], wall_ms[1:]
    ok = rc == 0 and all(s.status == 0 and s.iters > 0 and s.rel_res <= rtol for s in st)
    xb = [x.clone() for x in xs]
    # the same problems through the serving path (graphs warmed first)
    for h in hiers.values():
        ctx.serve_reserve(h, 4, B.MG_MIXED_FP32)
    serve_ms = []
    for _ in range(2):
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pend = {ctx.submit(h, b, x, rtol=rtol, max_it=500): k for k, (h, b, x) in enumerate(zip(hs, bs, xs))}
        sst = {}
        while pend:
            for t in list(pend):
                rc2, s2 = ctx.poll(t)
                if rc2 != B.MG_PENDING:
                    sst[pend.pop(t)] = (rc2, s2.iters)
        serve_ms.append((time.perf_counter() - t0) * 1e3)
    ok_serve = all(v[0] == 0 for v in sst.values())
    diff = max(float((a - c).norm() / c.norm()) for a, c in zip(xb, xs))
    iters_equal = sum(int(st[k].iters == sst[k][1]) for k in range(len(hs)))
    rec = {"description": f"{n_req} seeded small problems (2D/3D Poisson and transport-diffusion, 2D n in "
                          f"{list(BATCH_2D)}, 3D n in {list(BATCH_3D)}, {len(hiers)} hierarchies) solved to "
                          f"rel. residual {rtol:g} by one batched launch: a thread block per problem runs CG "
                          "(Poisson) or BiCGStab (transport) with the V(2,2) cycle of every level in shared "
                          "memory, FP32 V-cycle + FP64 Krylov",
           "metric": "DoF/s (sum of free DoFs / device time of the batched launch)",
           "value": dofs / (statistics.median(dev_ms) * 1e-3), "unit": "DoF/s", "problems": n_req,
           "free_dofs": dofs, "device_ms": dev_ms, "wall_ms": wall_ms, "launches": st[0].launches,
           "iters_max": max(s.iters for s in st), "all_converged": ok,
           "streams": {"value": dofs / (min(serve_ms) * 1e-3), "unit": "DoF/s", "wall_ms": serve_ms,
                       "all_converged": ok_serve,
                       "note": "mg_submit of every problem at once, mg_poll until all finished (16 slots, "
                               "4 reserved workspaces per hierarchy); wall clock"},
           "batched_over_streams_wall": min(serve_ms) / statistics.median(wall_ms),
           "max_rel_diff_vs_graph_solve": diff, "iters_equal_graph_solve": f"{iters_equal}/{len(hs)}"}
    for h in hiers.values():
        h.free()
    return rec


NS_PAPER_H100 = {"steps": 40000, "sum_s": 1660.0, "momentum_s": 231.1, "pres_s": 1356.7, "pres_solve_s": 1303.4,
                 "pres_up_s": 72.2}   # Table "tab:ns", GPU column


def measure_ns(G, B, ctx, shape=(32, 32, 64), steps=100, warm=10):
    """The explicit Navier-Stokes pressure correction of Sec. 5.3 (3D driven
    cavity, Re 1000, dt 1e-4, cosine-graded 32 x 32 x 64 pressure mesh,
    velocity on its refinement): warm-up steps from rest, then `steps` timed
    steps, per phase; both pressure-solve precisions; an oracle check of a
    smaller cavity."""
    from oracle import ns as ONS
    nx, ny, nz = shape
    rec = {"description": "3D driven cavity (Sec. 5.3): explicit lumped-mass momentum step with the interpolated "
                          "nonlinearity (matrix-free 27-point stencils of the tensor-product Q1 operators, FP64), "
                          "pressure-increment Poisson problem (pure Neumann, mean-zero solution) by GMRES (as in "
                          "the paper; CG in mixed_cg) + V(4,4) geometric multigrid on the graded pressure mesh "
                          "(warm start), explicit pressure update; "
                          f"Re 1000, dt 1e-4, {nx}x{ny}x{nz} pressure cells, velocity on the refined mesh",
           "paper_context": "Table tab:ns, GPU column on an H100 PCIe (40,000 steps): 1660 s in total, i.e. "
                            f"{NS_PAPER_H100['sum_s'] / NS_PAPER_H100['steps'] * 1e3:.1f} ms per step "
                            f"(momentum {NS_PAPER_H100['momentum_s'] / NS_PAPER_H100['steps'] * 1e3:.2f}, pressure "
                            f"{NS_PAPER_H100['pres_s'] / NS_PAPER_H100['steps'] * 1e3:.2f}, update "
                            f"{NS_PAPER_H100['pres_up_s'] / NS_PAPER_H100['steps'] * 1e3:.2f} ms)"}
    for name, prec, kr in (("mixed", B.MG_MIXED_FP32, B.MG_GMRES), ("fp64", B.MG_FP64, B.MG_GMRES),
                           ("mixed_cg", B.MG_MIXED_FP32, B.MG_CG)):
        t0 = time.perf_counter()
        sim = B.NavierStokes(ctx, nx=nx, ny=ny, nz=nz, prec=prec, krylov=kr, rtol=1e-8, max_it=400)
        setup_s = time.perf_counter() - t0
        sim.steps(warm)
        st = sim.steps(steps)
        n_dof = 3 * sim.nv + sim.np
        ms = st.ms_total / st.steps
        r = {"steps": st.steps, "status": st.status, "ms_per_step": ms,
             "ms_per_step_phases": {"momentum": st.ms_momentum / st.steps, "pres_rhs": st.ms_pres_rhs / st.steps,
                                    "pres_solve": st.ms_pres_solve / st.steps, "pres_up": st.ms_pres_up / st.steps},
             "iters_per_step": st.iters / st.steps, "iters_max": st.iters_max, "rel_res_max": st.rel_res_max,
             "dofs": n_dof, "velocity_nodes": sim.nv, "pressure_nodes": sim.np, "setup_s": setup_s,
             "dof_steps_per_s": n_dof * st.steps / (st.ms_total * 1e-3)}
        rec[name] = r
        sim.free()
    rec["value"] = rec["mixed"]["dof_steps_per_s"]
    rec["unit"] = "DoF*steps/s"
    rec["metric"] = "DoF*steps/s (velocity 3 x nodes + pressure nodes)"
    # oracle check on a smaller graded cavity, 10 steps from rest
    S = ONS.cavity(8, 8, 16)
    sim = B.NavierStokes(ctx, nx=8, ny=8, nz=16, prec=B.MG_MIXED_FP32, rtol=1e-10, max_it=400)
    sim.steps(10)
    ug, pg, _ = (t.cpu().numpy() for t in sim.get_state())
    sim.free()
    u, p, _ = ONS.run(S, 10)
    rec["oracle_check"] = {"mesh": "8x8x16 graded", "steps": 10,
                           "u_max_rel_err": float(np.abs(ug - u).max() / np.abs(u).max()),
                           "p_max_rel_err": float(np.abs(pg - p).max() / np.abs(p).max()),
                           "note": "mixed-precision pressure solve at rtol 1e-10 against the oracle's sparse LU"}
    return rec


TD_SIZES = (128, 256, 512, 1024)
TD_PAPER_H100_S = {128: 2.05, 256: 2.85, 512: 4.47, 1024: 9.0}   # Table "tab:td", GPU solve column


def measure_timedep(G, B, ctx, n, krylov, rtol=1e-8, steps=None, oracle_check=False):
    """The paper's time-dependent transport-diffusion run (Sec. 5.1) on the
    uniform n x n mesh: 100 backward-Euler steps (dt = 0.02) through
    mg_time_steps, right-hand side and warm-started solve per step on the
    device, hierarchy resident.  Source and boundary data of every step are
    inputs, resident before the timed region."""
    import torch
    steps = steps or W.TD_STEPS
    dt = W.TD_DT
    lm = W.td_uniform(n)
    pk = dict(kind=B.MG_TRANSPORT, eps=W.TD_LAMBDA, beta=W.TD_B, supg_delta0=0.0, mass=1.0 / dt)
    t0 = time.perf_counter()
    h = G.Hierarchy(ctx, lm, B.make_problem(**pk), B.make_opts(krylov=krylov))
    setup_s = time.perf_counter() - t0
    xy = h.coords()
    f = torch.from_numpy(np.stack([W.td_source((k + 1) * dt, xy) for k in range(steps)])).cuda()
    g = torch.from_numpy(np.stack([W.td_theta((k + 1) * dt, xy) for k in range(steps)])).cuda()
    th0 = torch.from_numpy(W.td_theta(0.0, xy)).cuda()
    out = {"n": n, "dofs": int(h.n_dofs), "steps": steps, "setup_s": setup_s}
    for key, prec in (("mixed", B.MG_MIXED_FP32), ("fp64", B.MG_FP64)):
        th = th0.clone()
        h.time_steps(th, f, g, 3, rtol=rtol, max_it=200, prec=prec)        # warm-up
        th = th0.clone()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        rc, sts = h.time_steps(th, f, g, steps, rtol=rtol, max_it=200, prec=prec)
        e1.record(ctx.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        thn = th.cpu().numpy()
        r = {"s": ms * 1e-3, "dof_solves_per_s": h.n_dofs * steps / (ms * 1e-3), "status": rc,
             "iters_total": int(sum(s.iters for s in sts)), "iters_max": int(max(s.iters for s in sts)),
             "rel_res_max": float(max(s.rel_res for s in sts)),
             "launches": int(sum(s.launches for s in sts)),
             "err_vs_exact_max": float(np.abs(thn - W.td_theta(steps * dt, xy)).max())}
        out[key] = (r, thn)
    if oracle_check:
        from oracle import mesh as M
        from oracle import problems as PB
        from oracle import timestep as TS
        m = M.Q1Mesh(2, lm.origin, lm.extent, lm.macro, lm.level, lm.anchor)
        prob = PB.Problem(PB.TRANSPORT, eps=W.TD_LAMBDA, beta=W.TD_B, supg_delta0=0.0)
        S, ref = TS.run(m, prob, dt, W.td_theta(0.0, xy), lambda t: W.td_source(t, xy),
                        lambda t: W.td_theta(t, xy), steps)
        w = np.asarray(S.F.sum(axis=1)).ravel()
        for key in ("mixed", "fp64"):
            out[key][0]["err_vs_oracle"] = rel_err(out[key][1], ref[-1], w)
    for key in ("mixed", "fp64"):
        out[key] = out[key][0]
    out["paper_h100_solve_s"] = TD_PAPER_H100_S.get(n)
    h.free()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="td_adaptive")
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="headline workload only (no records of the other configurations)")
    ap.add_argument("--requests", type=int, default=1000, help="serving: requests per stream")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean arrivals per second")
    ap.add_argument("--slots", type=int, default=16, help="serving: solves in flight")
    ap.add_argument("--reserve", type=int, default=4, help="serving: solve slots reserved per operator")
    ap.add_argument("--sweep", type=float, nargs="*", default=[10.0, 100.0], help="serving: rate multipliers")
    ap.add_argument("--launch", default="graph", choices=["graph", "direct"],
                    help="direct: per-kernel launches (for profilers that cannot see inside graphs)")
    ap.add_argument("--tail", default=None,
                    help="ROWS,CLUSTER: fixed tail shape instead of the setup autotuner (profiling runs, "
                         "where the autotuner's timings would be distorted)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    headline = args.workload == "td_adaptive"
    # the oracle on the host cores, started before this process touches the GPU
    tmp = tempfile.mkdtemp(prefix="mg_bench_")
    orc = None
    if rank == 0 and world == 1 and headline and not args.no_cpu_baseline:
        orc = start_oracle_child(tmp)

    import torch
    import torch.distributed as dist
    import paper_2405_05047_gb300 as G
    from paper_2405_05047_gb300 import binding as B
    from paper_2405_05047_gb300 import build as BLD

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    BLD.build()
    torch.cuda.set_device(local)
    ctx = G.Context(local)
    stream = ctx.stream
    flush = torch.empty(64 * 1024 * 1024, device="cuda", dtype=torch.float32)   # 256 MB > L2
    sv = Solver(G, B, ctx, args.workload, flush, args.launch, args.tail)
    h, info = sv.h, sv.info
    # kernels launched by setup (autotuner V-cycles): a profiler skips these to reach the solves
    print(f"launches after setup: {h.launch_count()}", file=sys.stderr, flush=True)
    n_free = info.n_free

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    with ClockSampler(local) as clk:
        barrier()
        ms_mixed, st_mixed, x_mixed = sv.timed(B.MG_MIXED_FP32, args.steps, args.warmup, args.rtol)
        barrier()
    # FP64 path of the same fused kernels (reported beside the value)
    ms64, st64, x_fp64 = sv.timed(B.MG_FP64, max(2, args.steps // 2), 1, args.rtol)
    barrier()
    # ablation: BF16-stored matrix values in the FP32 V-cycle
    ms16, st16, _ = sv.timed(B.MG_MIXED_BF16, max(2, args.steps // 2), 1, args.rtol)
    barrier()
    value, t_max = whole_job_rate(n_free, args.steps, sum(ms_mixed), world, "cuda")
    assert all(s.status == 0 for s in st_mixed + st64), [s.as_dict() for s in st_mixed + st64]

    # end to end through the public host-buffer entry point (pinned host memory)
    bh = torch.empty(h.n_dofs, dtype=torch.float64, pin_memory=True)
    bh.copy_(sv.b.cpu())
    xh = torch.zeros(h.n_dofs, dtype=torch.float64, pin_memory=True)
    bhn, xhn = bh.numpy(), xh.numpy()
    h.solve_host(bhn, xhn, rtol=args.rtol, max_it=500, prec=B.MG_MIXED_FP32)
    e2e_ms = []
    for _ in range(args.steps):
        xhn[:] = 0.0
        flush_l2(flush)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.solve_host(bhn, xhn, rtol=args.rtol, max_it=500, prec=B.MG_MIXED_FP32)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_value = world * n_free * args.steps / (sum(e2e_ms) * 1e-3)

    # roofline of the dominant kernel, timed inside the solve: the same K
    # solves (L2 flushed before each) with every kernel between two CUDA
    # events on the library's stream, summed per (kernel, level)
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs", 6800.0)
    prof, floor_ms = sv.profile(B.MG_MIXED_FP32, args.steps, args.rtol, st_mixed[0].iters)
    prof_total = sum(v[1] for v in prof.values())
    for (k, l), (n, t) in sorted(prof.items(), key=lambda kv: -kv[1][1]):   # whole table, for the profiles
        print(f"prof {k:48s} level {l:3d} launches {n:6d} ms {t:9.4f} us/launch {1e3 * t / n:8.2f} "
              f"share {t / prof_total:.4f}", file=sys.stderr)
    roof = sv.smoother_roofline(prof, floor_ms, peak)
    fine = h.levels - 1
    # the same sweep alone: cold (L2 flushed before each single launch) and warm
    cold = []
    for _ in range(10):
        flush_l2(flush)
        torch.cuda.synchronize()
        cold.append(h.time_op(fine, B.MG_OP_SMOOTH, B.MG_MIXED_FP32, reps=1))
    hot_ms = h.time_op(fine, B.MG_OP_SMOOTH, B.MG_MIXED_FP32, reps=50)
    per_level = []
    for lvl in range(h.levels):
        row = {"level": lvl, "nodes": int(info.level_nodes[lvl])}
        for opn, op in (("smooth", B.MG_OP_SMOOTH), ("restrict", B.MG_OP_RESTRICT),
                        ("prolong", B.MG_OP_PROLONG_ADD)):
            if lvl == 0 and op != B.MG_OP_SMOOTH:
                continue
            row[opn + "_us"] = 1e3 * h.time_op(lvl, op, B.MG_MIXED_FP32, reps=20)
        per_level.append(row)
    traffic = None       # DRAM bytes per launch from the ncu capture, while it matches the current kernel
    tr_path = os.path.join(ROOT, "profiles", f"traffic_{args.workload}.txt")
    if os.path.exists(tr_path):
        for line in open(tr_path):
            if line.startswith("bytes_per_launch:"):
                v = line.split(":", 1)[1].strip()
                traffic = None if v == "null" else int(v)
    roof.update({"traffic": traffic,
                 "timing": "CUDA events between consecutive kernels inside the solve (one graph per Krylov "
                           "iteration, L2 flushed before each solve); an empty kernel timed the same way takes "
                           f"{floor_ms * 1e3:.2f} us",
                 "ms_per_launch_alone_cold": statistics.mean(cold), "ms_per_launch_alone_l2_warm": hot_ms,
                 "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs, copy)" if peaks else "fallback"})
    sv.free()

    # the other configurations (one GPU, rank 0 only)
    configs = None
    if rank == 0 and world == 1 and headline and not args.no_configs:
        configs = {}
        for name, sample in (("poisson64", None), ("elasticity128", "elasticity32"), ("oseen", "oseen_small")):
            try:
                configs[name] = measure_config(G, B, ctx, name, flush, peak, rtol=args.rtol, err_sample=sample)
            except Exception as e:        # a failing record is reported, never hides the headline
                configs[name] = {"error": repr(e)}
        try:
            configs["batch_small"] = measure_batch(G, B, ctx, rtol=args.rtol)
        except Exception as e:
            configs["batch_small"] = {"error": repr(e)}
        try:
            configs["ns_cavity"] = measure_ns(G, B, ctx)
        except Exception as e:
            configs["ns_cavity"] = {"error": repr(e)}
        try:
            runs = [measure_timedep(G, B, ctx, n, B.MG_BICGSTAB, args.rtol, oracle_check=(n == 128))
                    for n in TD_SIZES]
            big = runs[-1]
            configs["td_timedep"] = {
                "description": "the paper's time-dependent transport-diffusion problem (lambda=0.01, b=(0,-1), "
                               "exact solution theta_ex, backward Euler dt=0.02, 100 steps, uniform meshes "
                               "h=2^-7..2^-10): per step the right-hand side and a warm-started BiCGStab + "
                               "V(2,2) solve to 1e-8 on the device, hierarchy resident",
                "metric": "DoF*solves/s (FP32-MG + FP64 Krylov)", "value": big["mixed"]["dof_solves_per_s"],
                "unit": "DoF*solves/s", "sizes": runs,
                "paper_context": "Table tab:td, GPU solve column on an H100 PCIe (FP64, GMRES+MG; rhs on the CPU "
                                 "and not included there): 2.05 / 2.85 / 4.47 / 9.0 s for 100 steps"}
        except Exception as e:
            configs["td_timedep"] = {"error": repr(e)}
        try:
            runs = [measure_elastodyn(G, B, ctx, kind, lv, args.rtol) for kind, lv in EL_RUNS]
            chk = measure_elastodyn(G, B, ctx, "edge", 3, args.rtol, steps=10, oracle_check=True)
            configs["elasticity_timedep"] = {
                "description": "the paper's elastodynamics problem (lambda=8e4, mu=2e4, f=(0,-1,0), clamped "
                               "boundary, zero initial data, backward Euler dt=0.025, 100 steps) on its adaptive "
                               "face / edge / vertex meshes (Table table:ndofs); per step the right-hand side and a "
                               "warm-started CG + V(2,2) point-block solve of M/dt^2 + K to 1e-8 on the device "
                               "(v eliminated), hierarchy resident",
                "metric": "DoF*steps/s, DoF = 6 x nodes as in the paper (FP32-MG + FP64 Krylov)",
                "value": runs[0]["mixed"]["dof_steps_per_s"], "unit": "DoF*steps/s", "meshes": runs,
                "oracle_check": {k: chk[k] for k in ("mesh", "nodes", "steps")} | {
                    "mixed_err_u": chk["mixed"]["err_vs_oracle_u"], "fp64_err_u": chk["fp64"]["err_vs_oracle_u"],
                    "note": "relative lumped-mass L2 of u after the steps against the oracle's coupled "
                            "first-order block solve (sparse LU)"},
                "paper_context": "Tables tab:elasticity:times:face/edge/vertex, GPU solve column on an H100 PCIe "
                                 "(FP64, GMRES+MG on the 6-component system): 122.57 s (face 5), 14.7 s (edge 6), "
                                 "7.9 s (vertex 6) for 100 steps"}
        except Exception as e:
            configs["elasticity_timedep"] = {"error": repr(e)}

    # error against the oracle and the CPU baseline on the headline mesh
    cpu, err = None, None
    if orc is not None:
        try:
            orc.wait(timeout=1200)
            oj = json.load(open(os.path.join(tmp, "oracle.json")))
            xref, w = np.load(os.path.join(tmp, "xref.npy")), np.load(os.path.join(tmp, "w.npy"))
            err = {"err_vs_oracle": rel_err(x_mixed, xref, w), "fp64_err_vs_oracle": rel_err(x_fp64, xref, w),
                   "note": f"relative lumped-mass L2 of the bench's solutions (rtol {args.rtol:g}) against the "
                           f"oracle's FP64 solve to {oj['reference_solve']['rtol']:g}"}
            cpu = {k: oj[k] for k in ("value", "unit", "cores", "kind", "sample", "iters", "sec_per_solve")}
            cpu["concurrent"] = oj.get("concurrent")
        except Exception as e:       # the baseline is reported, never required
            cpu = {"error": repr(e)}

    out = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(ms_mixed), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-mg+f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": sv.desc, "n_nodes": int(info.n_nodes),
                   "n_free_dofs": int(n_free), "levels": int(info.levels), "hanging_nodes": int(info.n_hanging),
                   "rtol": args.rtol, "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"replicas x{world}", "tail_levels": int(info.tail_levels),
                   "tail_cluster": int(info.tail_cluster), "tuned_vcycle_ms": info.vcycle_ms,
                   "col16_slices": int(info.col16_slices), "col32_slices": int(info.col32_slices)},
        "iters": [s.iters for s in st_mixed], "rel_res": max(s.rel_res for s in st_mixed),
        "fp64": {"value": world * n_free / (statistics.mean(ms64) * 1e-3), "ms_per_step": statistics.mean(ms64),
                 "iters": [s.iters for s in st64], "rel_res": max(s.rel_res for s in st64)},
        "speedup_mixed_vs_fp64": statistics.mean(ms64) / statistics.mean(ms_mixed),
        "bf16_values_ablation": {"value": world * n_free / (statistics.mean(ms16) * 1e-3),
                                 "ms_per_step": statistics.mean(ms16), "iters": [s.iters for s in st16],
                                 "rel_res": max(s.rel_res for s in st16),
                                 "converged": all(s.status == 0 for s in st16)},
        "err_vs_oracle": err["err_vs_oracle"] if err else None,
        "fp64_err_vs_oracle": err["fp64_err_vs_oracle"] if err else None,
        "err_note": err["note"] if err else None,
        "setup_s": sv.setup_s,
        "gpu_launches": int(sum(s.launches for s in st_mixed)),
        "e2e": {"value": e2e_value, "unit": "DoF/s", "h2d_bytes_per_step": int(2 * 8 * h.n_dofs),
                "d2h_bytes_per_step": int(8 * h.n_dofs), "ms_per_step": statistics.mean(e2e_ms)},
        "roofline": roof,
        "clocks": clk.summary(),
        "per_level_fp32_us": per_level,
        "top_kernels_in_solve": top_table(prof),
        "cpu_baseline": cpu,
        "configs": configs,
    }
    if rank == 0:
        print(json.dumps(out))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
