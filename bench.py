#!/usr/bin/env python3
"""IBDL solve benchmark on one GB300 (or N independent replicas).

Workload: the 2D star problem, periodic box [0,1)^2 with N=1024^2 nodes, star
r(theta) = 0.3 (1 + 0.2 cos 5 theta), M = 3525 arclength-equispaced points,
Peskin 4-point delta, kappa = 1e-3, seeded 10-mode Fourier boundary data.
One step = one Dirichlet solve (seed 0) + one Neumann solve (seed 1) to a
relative residual of 1e-8, solved together in one batched persistent launch
(``--mode solo``: one launch each) (the whole hot path: spread-divergence, FFT
Helmholtz solve, interpolation + jump, GMRES Arnoldi/Givens, the Neumann
right-hand side).

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import configs, geometry  # noqa: E402

METRIC = "IBDL solves/s at 1e-8 relative residual (2D star N=1024^2, M=3525, Dirichlet+Neumann)"
WORKLOAD = "c2-star-n1024-m3525-kappa1e-3-dirichlet+neumann"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ibdl", choices=["ibdl", "reference"])
    ap.add_argument("--precision", default="fp32-refined", choices=["fp32-refined", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="batched", choices=["batched", "solo"],
                    help="batched: each step solves the Dirichlet + Neumann pair in one "
                         "persistent launch; solo: one launch per solve")
    ap.add_argument("--engine", type=int, default=0, choices=[0, 1],
                    help="0: persistent single-launch solver, 1: host-driven loop")
    ap.add_argument("--no-matvec", action="store_true",
                    help="skip the matvec HBM-roofline measurement")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 256-instance batched measurement")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the mixed serving stream per offered rate (0: skip it)")
    ap.add_argument("--no-c1", action="store_true", help="skip the C1 latency row")
    ap.add_argument("--profile-case", default=None,
                    choices=["matvec-c2-f32", "matvec-c2-f64", "matvec-c2-dd",
                             "matvec-c3-f32", "matvec-c3-f64", "matvec-c3-dd",
                             "solve-c2", "pair-c2"],
                    help="run one small fixed workload for a profiler (ncu) and exit: "
                         "matvecs of the 2D star (c2) or the 3D sphere (c3) in float32, "
                         "float64 or with double-float transforms, float32-refined c2 "
                         "solves, or the benchmark's batched c2 pair")
    ap.add_argument("--reps", type=int, default=None,
                    help="--profile-case: repetitions (matvec 5, solve/pair 2)")
    ap.add_argument("--trace", action="store_true",
                    help="--profile-case pair-c2: after the repetitions, trace one more "
                         "launch's work items and print a summary (phase hand-offs, "
                         "starts, busy share) as one JSON line")
    ap.add_argument("--rows", type=int, default=None,
                    help="--profile-case: pin the x-pass tiling (rows per tile); the "
                         "autotuner's timings are distorted under a profiler")
    ap.add_argument("--pencils", default=None,
                    help="--profile-case: pin the pencils per item of the solve pass and "
                         "of the 3D y passes, as 'c_solve,c_y' (c_y 0 in 2D)")
    ap.add_argument("--plan", type=int, default=None,
                    help="--profile-case: pin the float32 FFT plan variant of 2D "
                         "float32-refined kinds (0 or 1)")
    return ap.parse_args()


def combine_ranks(local_ms, local_solves, dist=None, device=None):
    """Whole-job aggregate over ranks: the slowest rank's timed duration and
    the sum of all ranks' solves (independent replicas, no data exchange)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_ms, local_solves
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    s = torch.tensor([float(local_solves)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t.item()), int(s.item())


def run_serving(pkg, reqs, rate, precision, base_rate=2000.0, budget=120 << 30):
    """Replay the seeded mixed serving stream (Poisson arrivals generated at
    `base_rate`, their times scaled to the offered `rate`) in real time
    through the continuous-batching server; latency = arrival -> result."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    budget = int(min(budget, 0.8 * free))
    srv = pkg.Server(memory_budget=budget, max_active=64, rounds_per_step=4, reserve_sms=8,
                     tol=1e-8)
    scale = base_rate / rate
    t0 = srv.clock() + 0.02
    nxt = 0
    outstanding = {}
    recs = []
    while nxt < len(reqs) or outstanding:
        now = srv.clock()
        while nxt < len(reqs) and t0 + reqs[nxt].t * scale <= now:
            r = reqs[nxt]
            rid = srv.submit(r.problem.geom, r.problem.bdata, bc=r.problem.bc,
                             precision=precision, t_arrival=t0 + r.t * scale)
            outstanding[rid] = r
            nxt += 1
        st = srv.stats()
        if st["active"] == 0 and st["queued"] == 0 and nxt < len(reqs):
            time.sleep(max(0.0, t0 + reqs[nxt].t * scale - srv.clock()))
            continue
        for rid in srv.step():
            r = outstanding.pop(rid)
            _, rec = srv.take(rid, r.problem.geom.m)
            rec["kind"] = r.kind
            recs.append(rec)
    stats = srv.stats()
    srv.close()
    lat = np.array([(x["t_done"] - x["t_arrival"]) * 1e3 for x in recs])
    qwait = np.array([(x["t_admit"] - x["t_arrival"]) * 1e3 for x in recs])
    insvc = np.array([(x["t_done"] - x["t_admit"]) * 1e3 for x in recs])
    span = max(x["t_done"] for x in recs) - t0
    ok = [x for x in recs if x["status"] == 0]
    kinds = {}
    for x in recs:
        k = x["kind"].rsplit("-", 1)[0]
        kinds.setdefault(k, []).append((x["t_done"] - x["t_arrival"]) * 1e3)
    pct = (lambda a: {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99))})
    return {
        "offered_rate_per_s": rate, "requests": len(reqs), "completed_ok": len(ok),
        "solves_per_s": len(ok) / span,
        "latency_ms": {**pct(lat), "max": float(lat.max())},
        "queue_wait_ms": pct(qwait), "in_service_ms": pct(insvc),
        "latency_p50_ms_by_kind": {k: float(np.median(v)) for k, v in sorted(kinds.items())},
        "max_rel_residual": float(max(x["rel_residual"] for x in ok)) if ok else None,
        "memory_budget_bytes": budget, "peak_device_bytes": int(stats["peak_bytes"]),
        "slices": int(stats["launches"]),
        "host_admit_s": float(stats["admit_seconds"]),
        "host_wait_for_gpu_s": float(stats["wait_seconds"]),
        "offered_span_s": float(reqs[-1].t * scale), "makespan_s": float(span),
    }


def run_serving_sweep(pkg, nreq, seed=3, base_rate=2000.0):
    """The C5 stream (`nreq` requests, seed 3) offered at the specified
    2000/s (above one GPU's capacity: a saturated queue, which measures the
    capacity), then at 80% and 50% of the capacity that run measured (the
    steady states), float32-refined; and the same stream offered at 2000/s
    to plain float64 solves (the same tolerance), for the refined-vs-float64
    serving comparison."""
    from paper_2203_12126_gb300 import ibdl
    t = time.perf_counter()
    reqs = configs.c5_requests(nreq, seed=seed, rate=base_rate)
    gen_s = time.perf_counter() - t
    sat = run_serving(pkg, reqs, base_rate, ibdl.FP32_REFINED, base_rate)
    cap = sat["solves_per_s"]
    rows = {"saturated_2000_per_s": sat}
    for frac in (0.8, 0.5):
        rows[f"steady_{int(frac * 100)}pct_of_capacity"] = run_serving(
            pkg, reqs, frac * cap, ibdl.FP32_REFINED, base_rate)
    f64 = run_serving(pkg, reqs, base_rate, ibdl.FP64, base_rate)
    return {
        "workload": f"mixed stream, {nreq} requests, Poisson arrivals (seed {seed}): 80% 2D "
                    "stars N in {256,512,1024}^2, 20% 3D spheres/ellipsoids N in "
                    "{64,128,256}^3, kappa log-U[1e-4,1e-1], Dirichlet/Neumann 50/50, "
                    "tol 1e-8; the same requests at every offered rate",
        "capacity_solves_per_s": cap,
        "float32_refined": rows,
        "float64_saturated_2000_per_s": f64,
        "refined_over_float64_capacity": cap / f64["solves_per_s"],
        "request_generation_s": gen_s,
    }


def run_c3_solve(pkg, reps=3):
    """C3: the 3D sphere (N=256^3, M=38039) Neumann solve, float32-refined to
    1e-8 through the persistent solver; event-timed; error against a float64
    GPU solve at 1e-12."""
    import torch
    from paper_2203_12126_gb300 import ibdl
    dev = torch.device("cuda", torch.cuda.current_device())
    p = configs.c3()
    b = torch.tensor(p.bdata, dtype=torch.float64, device=dev)
    g = pkg.Geometry.from_workload(p.geom, bc=p.bc, precision=ibdl.FP32_REFINED)
    q = torch.zeros_like(b)
    info = g.solve(b, q, tol=1e-8)
    rows = g.info()["rows_per_tile"]
    ms = []
    for _ in range(reps):
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        info = g.solve(b, q, tol=1e-8)
        c.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(c))
    g.close()
    g64 = pkg.Geometry.from_workload(p.geom, bc=p.bc, precision=ibdl.FP64)
    q64 = torch.zeros_like(b)
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    i64 = g64.solve(b, q64, tol=1e-8)
    c.record()
    torch.cuda.synchronize()
    fp64_ms = a.elapsed_time(c)
    g64.solve(b, q64, tol=1e-12)
    g64.close()
    return {"workload": "3D sphere r=0.3, N=256^3, M=38039, kappa=1e-3, Neumann, "
                        "float32-refined to 1e-8",
            "solve_ms": float(np.median(ms)), "solves_per_s": 1e3 / float(np.median(ms)),
            "iters": info["iters"], "matvecs": info["matvecs"],
            "refine_steps": info["refine_steps"], "rel_residual": info["rel_residual"],
            "rel_err_vs_fp64_1e-12": float(torch.linalg.norm(q - q64) / torch.linalg.norm(q64)),
            "fp64_solve_ms": fp64_ms, "fp64_iters": i64["iters"], "rows_per_tile": rows}


def run_c1(pkg, solos=200, count=64, reps=5):
    """C1: the plain float64 Dirichlet solve of the Sec. 6.1 circle shape
    (N=128^2, r=0.3, M=242, cosine delta, kappa=1e-2, modified-Bessel data)
    at tol 1e-10: single-solve latency over `solos` event-timed solves
    (one persistent launch each, L2 flushed between), and throughput of
    `count` copies solved in one batched launch; error against the dense-LU
    density of the oracle."""
    import torch
    from oracle import ibdl_oracle as O
    from paper_2203_12126_gb300 import ibdl
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    p = configs.c1()
    g = pkg.Geometry.from_workload(p.geom, bc=p.bc, precision=ibdl.FP64)
    b = torch.tensor(p.bdata, dtype=torch.float64, device=dev)
    q = torch.zeros_like(b)
    info = {}

    def one():
        info.update(g.solve(b, q, tol=1e-10))
    for _ in range(5):
        one()
    lat = []
    for _ in range(solos):
        flush.fill_(5.0)
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        one()
        c.record()
        torch.cuda.synchronize()
        lat.append(a.elapsed_time(c))
    qstar = O.solve_dense(p.geom, p.bc, p.bdata)
    err = float(np.linalg.norm(q.cpu().numpy() - qstar) / np.linalg.norm(qstar))
    gs = [pkg.Geometry.from_workload(p.geom, bc=p.bc, precision=ibdl.FP64) for _ in range(count)]
    bs = [b] * count
    qs = [torch.zeros_like(b) for _ in range(count)]
    batch = ibdl.Batch(count)
    batch.solve(gs, bs, qs, tol=1e-10)
    ms = []
    for _ in range(reps):
        flush.fill_(6.0)
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        infos = batch.solve(gs, bs, qs, tol=1e-10)
        c.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(c))
    berr = max(float(np.linalg.norm(x.cpu().numpy() - qstar) / np.linalg.norm(qstar)) for x in qs)
    batch.close()
    for gg in gs:
        gg.close()
    g.close()
    med = float(np.median(ms))
    return {"workload": "circle r=0.3, N=128^2, M=242, cos4 delta, kappa=1e-2, Dirichlet "
                        "I_2 data, float64, tol 1e-10",
            "solo": {"solves": solos, "solves_per_s": solos / (sum(lat) / 1e3),
                     "latency_ms": {"p50": float(np.percentile(lat, 50)),
                                    "p99": float(np.percentile(lat, 99))},
                     "iters": info["iters"], "rel_err_vs_dense_lu": err},
            "batched": {"instances": count, "launch_ms": med,
                        "solves_per_s": count / (med / 1e3),
                        "all_ok": all(f["status"] == 0 for f in infos),
                        "max_rel_err_vs_dense_lu": berr}}


def run_batched_c4(pkg, count=256, reps=5):
    """C4: `count` uneven 2D star instances (N in {128,256,512}^2, kappa
    log-uniform [1e-4,1e-1], seed 2) solved in ONE persistent launch,
    float32-refined to 1e-8; event-timed, L2 flushed between launches."""
    import torch
    from paper_2203_12126_gb300 import ibdl
    dev = torch.device("cuda", torch.cuda.current_device())
    insts = configs.c4_instances(count)
    geoms = [pkg.Geometry.from_workload(p.geom, bc=p.bc, precision=ibdl.FP32_REFINED)
             for p in insts]
    # the autotuner's tiling per grid size (the batch's time depends on it)
    picks = {}
    for p, g in zip(insts, geoms):
        picks.setdefault(str(p.geom.n), g.info()["rows_per_tile"])
    bs = [torch.tensor(p.bdata, dtype=torch.float64, device=dev) for p in insts]
    qs = [torch.zeros(p.geom.m, dtype=torch.float64, device=dev) for p in insts]
    batch = ibdl.Batch(count)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    batch.solve(geoms, bs, qs, tol=1e-8)
    ms, infos = [], None
    for _ in range(reps):
        flush.fill_(4.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        infos = batch.solve(geoms, bs, qs, tol=1e-8)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    batch.close()
    for g in geoms:
        g.close()
    med = float(np.median(ms))
    return {"workload": f"{count} 2D star instances, N in {{128,256,512}}^2 (seed 2), "
                        "float32-refined, tol 1e-8, one persistent launch",
            "rows_per_tile": picks,
            "solves_per_s": count / (med / 1e3), "launch_ms": med,
            "max_rel_residual": float(max(f["rel_residual"] for f in infos)),
            "all_ok": all(f["status"] == 0 for f in infos),
            "iters": {"min": min(f["iters"] for f in infos),
                      "max": max(f["iters"] for f in infos)}}


def _event_ms(fn, reps, flush):
    import torch
    fn()
    ms = []
    for _ in range(reps):
        flush.fill_(3.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return float(np.median(ms))


def run_method_rows(pkg, peaks, reps=10):
    """The method rows beyond the Helmholtz hot path, event-timed with L2
    flushed between calls.  Poisson limit:
    the interior indicator (App. D) and the near-boundary values (App. A,
    m1 = 6, m2 = 8) on the C2 star (N = 1024^2, M = 3525); a Dirichlet
    Poisson solve on the same star (kappa = inf, float32-refined, tol 1e-8);
    the completed solve of Sec. 6.3 (exterior of r = 0.25 in [-4, 4)^2,
    N = 1024^2, eta = 10, u = exp(sin 2 pi x)), with its error against the
    closed form away from Gamma."""
    import dataclasses
    import torch
    from paper_2203_12126_gb300 import ibdl
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    p = configs.c2()
    g = p.geom
    nn = g.n * g.n
    out = {}
    G = pkg.Geometry.from_workload(g)
    chi = torch.empty(nn, dtype=torch.uint8, device=dev)
    ind_ms = _event_ms(lambda: G.indicator(None, chi), reps, flush)
    P = configs.grid_nodes(g)
    uin = torch.tensor(np.sin(3 * P[:, 0]) * np.cos(2 * P[:, 1]), dtype=torch.float64,
                       device=dev)
    ub = torch.tensor(p.bdata, dtype=torch.float64, device=dev)
    uout = torch.empty_like(uin)
    near_ms = _event_ms(lambda: G.near_boundary(uin, ub, chi, 6, 8.0, uout), reps, flush)
    fixed = int((uout != uin).sum().item())
    out["indicator_c2"] = {"us": ind_ms * 1e3, "inside_nodes": int(chi.sum().item()),
                           "note": "spread-divergence of Q = 1, float64 Poisson solve, "
                                   "threshold; n = 1024^2"}
    out["near_boundary_c2"] = {"us": near_ms * 1e3, "replaced_nodes": fixed,
                               "ns_per_replaced_node": near_ms * 1e6 / max(fixed, 1),
                               "note": "m1 = 6, m2 = 8; the three nearest boundary points "
                                       "of each node from a cell list (3 x 3 cells of 8 h)"}
    G.close()
    # the same two steps on the C3 sphere (N = 256^3, M = 38039)
    c3 = configs.c3()
    G3n = pkg.Geometry.from_workload(c3.geom)
    n3 = c3.geom.n ** 3
    chi3 = torch.empty(n3, dtype=torch.uint8, device=dev)
    ind3_ms = _event_ms(lambda: G3n.indicator(None, chi3), 3, flush)
    P3 = configs.grid_nodes(c3.geom)
    u3in = torch.tensor(np.sin(3 * P3[:, 0]) * np.cos(2 * P3[:, 1]) * np.cos(P3[:, 2]),
                        dtype=torch.float64, device=dev)
    ub3n = torch.tensor(c3.bdata, dtype=torch.float64, device=dev)
    u3out = torch.empty_like(u3in)
    near3_ms = _event_ms(lambda: G3n.near_boundary(u3in, ub3n, chi3, 6, 8.0, u3out), 3, flush)
    fixed3 = int((u3out != u3in).sum().item())
    out["indicator_c3"] = {"us": ind3_ms * 1e3, "inside_nodes": int(chi3.sum().item())}
    out["near_boundary_c3"] = {"us": near3_ms * 1e3, "replaced_nodes": fixed3,
                               "ns_per_replaced_node": near3_ms * 1e6 / max(fixed3, 1),
                               "note": "3D generalisation (Sec. 6.7), m1 = 6, m2 = 8"}
    G3n.close()
    del u3in, u3out, chi3
    gp = dataclasses.replace(g, kappa=float("inf"))
    Gp = pkg.Geometry.from_workload(gp, bc=configs.DIRICHLET, precision=ibdl.FP32_REFINED)
    q = torch.zeros(g.m, dtype=torch.float64, device=dev)
    info = {}

    def psolve():
        info.update(Gp.solve(ub, q, tol=1e-8))
    ps_ms = _event_ms(psolve, 3, flush)
    out["poisson_solve_c2"] = {"ms": ps_ms, "iters": info["iters"],
                               "rel_residual": info["rel_residual"],
                               "note": "Dirichlet, kappa = inf, float32-refined, tol 1e-8, "
                                       "persistent launch"}
    Gp.close()
    ge, gt, ube, uex = configs.poisson_exterior(1024, 8.0)
    Gc = pkg.Geometry.from_workload(ge, bc=configs.DIRICHLET, precision=ibdl.FP32_REFINED,
                                    eta=10.0)
    z = torch.zeros(ge.m + 1, dtype=torch.float64, device=dev)
    ubt = torch.tensor(ube, dtype=torch.float64, device=dev)
    gtt = torch.tensor(gt.reshape(-1), dtype=torch.float64, device=dev)
    cinfo = {}

    def csolve():
        cinfo.update(Gc.solve(ubt, z, g_grid=gtt, tol=1e-8))
    cs_ms = _event_ms(csolve, 3, flush)
    u = torch.empty(ge.n * ge.n, dtype=torch.float64, device=dev)
    Gc.evaluate(z, u, g_grid=gtt)
    Pe = configs.grid_nodes(ge)
    far = np.linalg.norm(Pe, axis=1) > 0.25 + 6 * ge.h
    err = float(np.max(np.abs(u.cpu().numpy()[far] - uex[far])))
    out["completed_solve_sec6_3"] = {"ms": cs_ms, "iters": cinfo["iters"], "m": ge.m,
                                     "max_err_away_from_gamma": err,
                                     "note": "L = 8, N = 1024^2, eta = 10, float32-refined, "
                                             "tol 1e-8, launch-based engine"}
    Gc.close()
    # Fourier-spectral discretisation (Sec. 6.2.1): matvecs on C2 and C3
    for name, prob in (("c2", configs.c2()), ("c3", configs.c3())):
        Gs = pkg.Geometry.from_workload(prob.geom, bc=prob.bc, precision=ibdl.FP32_REFINED,
                                        disc="spectral")
        qv = torch.tensor(np.random.default_rng(0).standard_normal(prob.geom.m),
                          dtype=torch.float64, device=dev)
        yv = torch.empty_like(qv)
        for prec, tag in ((1, "f32"), (0, "f64")):
            us = _event_ms(lambda: Gs.apply(qv, yv, precision=prec), reps, flush) * 1e3
            out[f"spectral_matvec_{name}_{tag}"] = {"us": us}
        Gs.close()
    # Sec. 6.7: the 3D Dirichlet problem (spectral), dx = 2^-8, 14400 points
    g3 = geometry.sphere(256, 0.25, m=14400, center=(0, 0, 0), origin=(-0.5,) * 3, kappa=1.0)
    x, y, z = (g3.X - np.array(g3.center)).T
    ub3 = torch.tensor(0.25 * z * 2 * x * y / np.maximum(x * x + y * y, 1e-300),
                       dtype=torch.float64, device=dev)
    G3 = pkg.Geometry.from_workload(g3, precision=ibdl.FP32_REFINED, disc="spectral")
    q3 = torch.zeros(g3.m, dtype=torch.float64, device=dev)
    i3 = {}

    def s3():
        i3.update(G3.solve(ub3, q3, tol=1e-8))
    s3_ms = _event_ms(s3, 3, flush)
    out["spectral_solve_sec6_7"] = {"ms": s3_ms, "iters": i3["iters"],
                                    "note": "sphere r = 0.25, N = 256^3, M = 14400 (Fibonacci), "
                                            "k = 1, Dirichlet, float32-refined, tol 1e-8 "
                                            "(Table 3 lists 5 iterations at dx = 2^-8)"}
    G3.close()
    return out


def problems():
    return [configs.c2(bc=configs.DIRICHLET), configs.c2(bc=configs.NEUMANN)]


def run_profile_case(args):
    """One small fixed workload for a profiler, then exit (no timing, no JSON
    line): ``matvec-<c2|c3>-<f32|f64|dd>`` applies the boundary operator of
    the 2D star (N=1024^2, M=3525) or the 3D sphere (N=256^3, M=38039)
    ``--reps`` times (default 5); ``solve-c2`` runs float32-refined Dirichlet
    solves of the star at tol 1e-8 (default 2); ``pair-c2`` runs the
    benchmark's step, the Dirichlet + Neumann pair in one batched launch
    (default 2).  ``--rows`` pins the x-pass tiling."""
    import torch
    import paper_2203_12126_gb300 as pkg
    from paper_2203_12126_gb300 import ibdl
    pkg.load()
    dev = torch.device("cuda:0")
    what = args.profile_case
    if what.startswith("matvec"):
        _, case, tag = what.split("-")
        prob = configs.c3() if case == "c3" else configs.c2()
        prec = {"f32": ibdl.FP32_REFINED, "f64": ibdl.FP64, "dd": 2}[tag]
        reps = args.reps or 5
        if args.rows:
            ibdl.tuning_set(prob.geom.dim, prob.geom.n, min(prec, 1), args.rows)
        if args.pencils:
            cs, cy = (int(v) for v in args.pencils.split(","))
            ibdl.tuning_set_pencils(prob.geom.dim, prob.geom.n, min(prec, 1), cs, cy)
        if args.plan is not None and prob.geom.dim == 2:
            ibdl.tuning_set_plan(2, prob.geom.n, ibdl.FP32_REFINED, args.plan)
        g = pkg.Geometry.from_workload(prob.geom, bc=prob.bc, precision=min(prec, 1))
        q = torch.tensor(np.random.default_rng(0).standard_normal(prob.geom.m), device=dev)
        y = torch.empty_like(q)
        for _ in range(reps):
            g.apply(q, y, precision=prec)
        torch.cuda.synchronize()
        print(f"{what} x{reps}: |y| = {float(y.norm()):.6e}")
        g.close()
        return 0
    reps = args.reps or 2
    probs = [configs.c2(bc=configs.DIRICHLET)] if what == "solve-c2" else problems()
    if args.rows:
        ibdl.tuning_set(2, probs[0].geom.n, ibdl.FP32_REFINED, args.rows)
    if args.pencils:
        cs, cy = (int(v) for v in args.pencils.split(","))
        ibdl.tuning_set_pencils(2, probs[0].geom.n, ibdl.FP32_REFINED, cs, cy)
    if args.plan is not None:
        ibdl.tuning_set_plan(2, probs[0].geom.n, ibdl.FP32_REFINED, args.plan)
    gs = [pkg.Geometry.from_workload(p.geom, bc=p.bc, precision=ibdl.FP32_REFINED)
          for p in probs]
    bs = [torch.tensor(p.bdata, device=dev) for p in probs]
    qs = [torch.empty_like(b) for b in bs]
    if what == "solve-c2":
        for _ in range(reps):
            info = gs[0].solve(bs[0], qs[0], tol=1e-8)
        print(f"{what} x{reps}: iters {info['iters']} rel_res {info['rel_residual']:.2e}")
    else:
        batch = ibdl.Batch(len(gs))
        for _ in range(reps):
            infos = batch.solve(gs, bs, qs, tol=1e-8)
        print(f"{what} x{reps}: iters {[f['iters'] for f in infos]}")
        if args.trace:
            ibdl.profile_enable(True)
            ibdl.profile_trace(True)
            batch.solve(gs, bs, qs, tol=1e-8)
            rec, _ = ibdl.profile_trace_read()
            ibdl.profile_trace(False)
            ibdl.profile_enable(False)
            print(json.dumps(trace_summary(rec)))
        batch.close()
    torch.cuda.synchronize()
    for g in gs:
        g.close()
    return 0


TRACE_PHASES = {0: "x_fwd", 1: "y_fwd", 2: "solve", 3: "y_inv", 4: "x_inv", 5: "D", 6: "E",
                7: "F", 9: "single"}


def trace_summary(rec):
    """Per instance: phases, the phase hand-offs (last item done -> next phase
    published) and the start gaps (publication -> first item of the phase);
    per phase kind and precision: count, median span and median item; the
    busy share of blocks x launch."""
    r = rec.astype(np.int64)
    t0 = int(r[:, 0].min())
    s, e, meta = r[:, 0] - t0, r[:, 1] - t0, r[:, 2]
    blk, inst = meta >> 40, (meta >> 24) & 0xFFFF
    ph, prec = (meta >> 20) & 15, (meta >> 18) & 3
    span = int(e.max())
    nblk = int(blk.max()) + 1
    out = {"span_us": span / 1e3, "blocks": nblk,
           "busy_share": float((e - s)[ph != 15].sum() / (span * nblk)), "instances": {}}
    for k in np.unique(inst):
        m = inst == k
        ho = np.sort(e[m & (ph == 15)])
        hod = (e - s)[m & (ph == 15)]
        items = m & (ph != 15)
        grp = np.searchsorted(ho, s[items])
        kinds = {}
        gaps = []
        for g in np.unique(grp):
            sel = grp == g
            ss, ee = s[items][sel], e[items][sel]
            kind = f"{TRACE_PHASES.get(int(ph[items][sel][0]), '?')}_{'f32' if prec[items][sel][0] else 'f64'}"
            kinds.setdefault(kind, []).append(((ee.max() - ss.min()) / 1e3,
                                               float(np.median(ee - ss)) / 1e3))
            if g > 0:
                gaps.append((ss.min() - ho[g - 1]) / 1e3)
        out["instances"][int(k)] = {
            "phases": int(len(np.unique(grp))),
            "handoff_us_median": float(np.median(hod)) / 1e3 if len(hod) else None,
            "start_gap_us_median": float(np.median(gaps)) if gaps else None,
            "by_kind": {kk: {"phases": len(v), "span_us_median": float(np.median([a for a, _ in v])),
                             "item_us_median": float(np.median([b for _, b in v]))}
                        for kk, v in sorted(kinds.items())}}
    return out


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping: algorithmic bytes / flops per launch of each kernel
# family on this workload (2D, n^2 grid, M points)
# ---------------------------------------------------------------------------

def kernel_model(name, n, m):
    """Algorithmic bytes and flops per launch of a kernel family or solver
    phase on a 2D n^2 grid with M points (the same passes whether launched
    alone or as a phase of the persistent solver)."""
    name = name.replace("phase:", "")
    p = 8 if name.endswith("f64") else 4
    spec = (n // 2 + 1) * n * 2 * p            # half spectrum, complex
    grid = n * n * p
    fft = 5.0 * n * math.log2(n)               # flops of one complex length-n FFT
    pts = m * (8 * 4 + 4 * 2 + 8 * 8)          # q, w, normals, base, W per point
    if name.startswith("rows_fwd"):
        return {"bytes": spec + pts, "flops": (n // 2) * fft}
    if name.startswith("pencils_solve") or name.startswith("solve"):
        return {"bytes": 2 * spec, "flops": (n // 2 + 1) * (2 * fft + 6 * n)}
    if name.startswith("rows_inv"):
        return {"bytes": spec + grid, "flops": (n // 2) * fft}
    if name.startswith("interp"):
        return {"bytes": m * (16 * p + 8 * 3 + 4 * 2 + 8 * p), "flops": m * 40.0}
    return None


def model_matvec_bytes(dim, n, m, p):
    """Algorithmic bytes of one matvec, the fixed model
    B = 9 p N^d + p M (4^d + 2d + 4): one grid write by the spread, two
    read+write passes per transform, the taps and point I/O."""
    return 9 * p * n ** dim + p * m * (4 ** dim + 2 * dim + 4)


def launch_field_solves(infos, per_launch, refined, neumann, n, m, dim=2):
    """Field solves of one persistent launch by precision, and its
    algorithmic bytes by the matvec model: (float64-grade, float32, bytes).
    infos: the solve infos of the launches timed (per_launch solves each,
    in the order of `neumann`, a flag per problem).  A refined solve's
    matvecs are its inner iterations and residual updates (float32) and its
    float64-grade residuals; a Neumann solve adds one field solve for its
    right-hand side (float32 when refined: its residuals carry the S V_b
    term; float64 else)."""
    mv = float(np.mean([f["matvecs"] for f in infos])) * per_launch
    it = float(np.mean([f["iters"] for f in infos])) * per_launch
    up = float(np.mean([f.get("residual_updates", 0) for f in infos])) * per_launch
    mv64 = (mv - it - up) if refined else mv
    mv32 = (it + up) if refined else 0.0
    nneu = per_launch * sum(bool(x) for x in neumann) / len(neumann)
    if refined:
        mv32 += nneu
    else:
        mv64 += nneu
    B = mv64 * model_matvec_bytes(dim, n, m, 8) + mv32 * model_matvec_bytes(dim, n, m, 4)
    return mv64, mv32, B


def run_matvec_roofline(pkg, peaks, reps=30):
    """Event-timed matvecs (float32, float64, and float64 with double-float
    transforms) on the 3D 256^3 sphere (the HBM-bound case) and the 2D
    1024^2 star, L2 flushed between launches; then one profiled pass that
    splits each matvec into its kernels (library event pairs)."""
    import torch
    from paper_2203_12126_gb300 import ibdl
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = {}
    for name, prob in (("c3-sphere-n256-m38039", configs.c3()),
                       ("c2-star-n1024-m3525", configs.c2())):
        g = pkg.Geometry.from_workload(prob.geom, bc=prob.bc, precision=1)
        q = torch.tensor(np.random.default_rng(0).standard_normal(prob.geom.m),
                         dtype=torch.float64, device=dev)
        y = torch.empty_like(q)
        for prec, tag, p in ((1, "f32", 4), (0, "f64", 8), (2, "dd", 8)):
            for _ in range(3):
                g.apply(q, y, precision=prec)
            ev = []
            for _ in range(reps):
                flush.fill_(2.0)
                a = torch.cuda.Event(enable_timing=True)
                c = torch.cuda.Event(enable_timing=True)
                a.record()
                g.apply(q, y, precision=prec)
                c.record()
                ev.append((a, c))
            torch.cuda.synchronize()
            us = float(np.median([a.elapsed_time(c) for a, c in ev])) * 1e3
            B = model_matvec_bytes(prob.geom.dim, prob.geom.n, prob.geom.m, p)
            gbs = B / (us * 1e-6) / 1e9
            # per-kernel split of the same matvec (event pairs around each
            # launch; a few microseconds of event overhead per launch)
            ibdl.profile_enable(True)
            ibdl.profile_read(reset=True)
            for _ in range(5):
                flush.fill_(2.0)
                g.apply(q, y, precision=prec)
            st = ibdl.profile_read(reset=True)
            ibdl.profile_enable(False)
            split = {k: v[1] / v[0] * 1e3 for k, v in sorted(st.items())
                     if not k.startswith("phase:")}
            out[f"{name}-{tag}"] = {"us_median": us, "algorithmic_bytes": B,
                                    "achieved_gbs": gbs, "peak_gbs": peaks["hbm_gbs"],
                                    "frac_of_hbm": gbs / peaks["hbm_gbs"],
                                    "peak_src": peaks["src"],
                                    "kernel_us": split,
                                    "rows_per_tile": g.info()["rows_per_tile"],
                                    "pencils_per_item": g.info()["pencils_per_item"],
                                    "fft_plan": g.info()["fft_plan"]}
        g.close()
    return out


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "src": "fallback"}


# DRAM bytes (read + write) of one batched-pair launch of the persistent
# solver, from one ncu capture of that launch (53.5 MB read + 119.5 MB
# write); None whenever the solver kernel changes, until it is captured again
PAIR_LAUNCH_DRAM_BYTES = (53.455872 + 119.521536) * 1e6
PAIR_LAUNCH_DRAM_SRC = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one pair launch "
                        "(profiles/c2_persistent_solve.md)")


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# ---------------------------------------------------------------------------

def oracle_sample(probs, tol, budget_s):
    """Run oracle solves (alternating Dirichlet / Neumann) for ~budget_s."""
    from oracle import ibdl_oracle as O
    t0 = time.perf_counter()
    done, iters = 0, []
    sols = {}
    while True:
        p = probs[done % len(probs)]
        r = O.solve(p.geom, p.bc, p.bdata, tol=tol)
        iters.append(r.iters)
        sols.setdefault(p.name, r.x)
        done += 1
        if time.perf_counter() - t0 >= budget_s and done % len(probs) == 0:
            break
    el = time.perf_counter() - t0
    return done, el, iters, sols


def _oracle_worker(args):
    """One spawned worker of the all-cores baseline: `rounds` rounds of one
    Dirichlet + one Neumann oracle solve; returns the seconds of each round."""
    tol, rounds = args
    probs = problems()
    from oracle import ibdl_oracle as O
    out = []
    for _ in range(rounds):
        t = time.perf_counter()
        for p in probs:
            O.solve(p.geom, p.bc, p.bdata, tol=tol)
        out.append(time.perf_counter() - t)
    return out


def cpu_baseline(probs, tol, samples=5):
    """The oracle as it stands on this host's cores: single thread (median
    of `samples` rounds of one Dirichlet + one Neumann solve, plus the
    per-matvec time) and all cores (one spawned process per core, each
    solving pairs; throughput = solves of a round / its slowest worker,
    median of `samples` rounds after a warm-up round)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    from oracle import ibdl_oracle as O
    t_all = time.perf_counter()
    pair_s, x0 = [], None
    for _ in range(samples):
        t = time.perf_counter()
        for k, p in enumerate(probs):
            r = O.solve(p.geom, p.bc, p.bdata, tol=tol)
            if k == 0:
                x0 = r.x
        pair_s.append(time.perf_counter() - t)
    op = O.Operator(probs[0].geom, probs[0].bc)
    qv = np.random.default_rng(0).standard_normal(probs[0].geom.m)
    mv_s = []
    for _ in range(samples):
        t = time.perf_counter()
        op.apply(qv)
        mv_s.append(time.perf_counter() - t)
    one = {"solves_per_s": len(probs) / statistics.median(pair_s),
           "matvecs_per_s": 1.0 / statistics.median(mv_s),
           "matvec_ms": statistics.median(mv_s) * 1e3, "cores": 1}
    cores = os.cpu_count() or 1
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                               "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"      # one thread per worker process
    try:
        with ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
            res = list(ex.map(_oracle_worker, [(tol, samples + 1)] * cores))
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    rounds = [max(r[i] for r in res) for i in range(1, samples + 1)]  # skip the warm-up
    allc = {"solves_per_s": cores * len(probs) / statistics.median(rounds), "cores": cores}
    return {"value": allc["solves_per_s"], "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"all {cores} host cores: one spawned process per core, each solving "
                      f"{samples} + 1 Dirichlet+Neumann pairs (tol {tol:g}); value = median "
                      f"round throughput; single thread: median of {samples} pairs",
            "single_thread": one, "all_cores": allc, "nproc": cores,
            "wall_s": time.perf_counter() - t_all, "_x0": x0}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    probs = problems()
    # each step is one bounded sample: a Dirichlet + Neumann oracle solve pair
    for _ in range(args.warmup):
        oracle_sample(probs, args.tol, 0.0)
    t0 = time.perf_counter()
    solves = 0
    lat = []
    for _ in range(args.steps):
        s0 = time.perf_counter()
        n, _, _, _ = oracle_sample(probs, args.tol, 0.0)
        solves += n
        lat.append((time.perf_counter() - s0) / n * 1e3)
    el = time.perf_counter() - t0
    value = solves / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64 (numpy oracle)",
                   "tol": args.tol},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} steps x (1 Dirichlet + 1 Neumann oracle "
                                   f"solve at tol {args.tol:g})"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.profile_case:
        return run_profile_case(args)

    import torch
    import paper_2203_12126_gb300 as pkg
    from paper_2203_12126_gb300 import ibdl

    assert torch.cuda.is_available(), "bench.py needs a GPU"
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    pkg.load()
    stream = torch.cuda.current_stream()

    prec = ibdl.FP32_REFINED if args.precision == "fp32-refined" else ibdl.FP64
    probs = problems()
    geoms, bs, qs = [], [], []
    for p in probs:
        geoms.append(pkg.Geometry.from_workload(p.geom, bc=p.bc, precision=prec))
        bs.append(torch.tensor(p.bdata, dtype=torch.float64, device=dev))
        qs.append(torch.zeros(p.geom.m, dtype=torch.float64, device=dev))
    m, n = probs[0].geom.m, probs[0].geom.n
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def solve(i, b=None, q=None):
        return geoms[i].solve(bs[i] if b is None else b, qs[i] if q is None else q,
                              tol=args.tol, engine=args.engine)

    batch = ibdl.Batch(len(probs))

    def step_batched(gs=None, qq=None):
        # the Dirichlet + Neumann pair advances together in one persistent launch
        return batch.solve(gs or geoms, bs, qq or qs, tol=args.tol)

    def step_solo():
        return [solve(i) for i in range(len(probs))]

    run_step = step_batched if args.mode == "batched" else step_solo

    for _ in range(args.warmup):
        run_step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, per-step CUDA events, L2 flushed between
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    infos = []
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = pkg.kernel_launch_count()
    w0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        infos.extend(run_step())
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    launches = pkg.kernel_launch_count() - l0
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    lat = [a.elapsed_time(b) for a, b in ev]
    total_ms, solves = combine_ranks(float(sum(lat)), args.steps * len(probs), dist, dev)
    value = solves / (total_ms / 1e3)

    # ---- the same pair solved one at a time (single-solve latency) and the
    # plain float64 path at the same tolerance (batched), for comparison
    def timed(fn, reps):
        evs = []
        for _ in range(reps):
            flush.fill_(3.0)
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            c.record(stream)
            evs.append((a, c))
        torch.cuda.synchronize()
        return [a.elapsed_time(c) for a, c in evs]

    solo_lat = []
    for _ in range(max(5, args.steps // 2)):
        for i in range(len(probs)):
            solo_lat.extend(timed(lambda: solve(i), 1))
    solo = {"solves_per_s": len(solo_lat) / (sum(solo_lat) / 1e3),
            "latency_ms": {"p50": float(np.percentile(solo_lat, 50)),
                           "p99": float(np.percentile(solo_lat, 99))},
            "note": "each solve alone through ibdl_solve (one persistent launch)"}
    g64s = [pkg.Geometry.from_workload(p.geom, bc=p.bc, precision=ibdl.FP64) for p in probs]
    q64s = [torch.zeros_like(q) for q in qs]
    step_batched(g64s, q64s)
    f64_lat = timed(lambda: step_batched(g64s, q64s), max(5, args.steps // 2))
    fp64 = {"solves_per_s": len(probs) * len(f64_lat) / (sum(f64_lat) / 1e3),
            "latency_ms_per_pair": {"p50": float(np.percentile(f64_lat, 50))},
            "note": "plain float64 GMRES, same pair, same tolerance, batched launch"}

    # ---- accuracy of the timed path against a float64 GPU solve at 1e-12
    errs = []
    for i, p in enumerate(probs):
        g64 = pkg.Geometry.from_workload(p.geom, bc=p.bc, precision=ibdl.FP64)
        q64 = torch.zeros_like(qs[i])
        g64.solve(bs[i], q64, tol=1e-12)
        errs.append(float(torch.linalg.norm(qs[i] - q64) / torch.linalg.norm(q64)))
        fp64.setdefault("rel_err_vs_fp64_1e-12", 0.0)
        fp64["rel_err_vs_fp64_1e-12"] = max(fp64["rel_err_vs_fp64_1e-12"], float(
            torch.linalg.norm(q64s[i] - q64) / torch.linalg.norm(q64)))
        g64.close()
    for g in g64s:
        g.close()

    # ---- profiled pass: per-kernel CUDA-event durations (library event pairs
    # on the launching stream) and, inside the persistent solver, per-phase
    # wall times from the device's global timer -> dominant kernel roofline
    pkg.ibdl.profile_enable(True)
    pkg.ibdl.profile_read(reset=True)
    pinfos = []
    for _ in range(max(3, args.steps // 4)):
        flush.fill_(1.0)
        pinfos.extend(run_step())
    per_launch = len(probs) if args.mode == "batched" else 1
    stats = pkg.ibdl.profile_read(reset=True)
    pkg.ibdl.profile_enable(False)
    peaks = load_peaks()
    kstats = {k: v for k, v in stats.items() if not k.startswith("phase:")}
    pstats = {k: v for k, v in stats.items() if k.startswith("phase:")}
    dom = max(kstats.items(), key=lambda kv: kv[1][1]) if kstats else None
    roofline = None
    kernels = {}
    tot_prof = sum(v[1] for v in kstats.values()) or 1.0
    for name, (cnt, ms) in kstats.items():
        kernels[name] = {"launches": cnt, "avg_us": ms / cnt * 1e3, "share": ms / tot_prof}
    # solver items: per phase, the summed duration of its work items (blocks
    # run items of different phases and instances at the same time)
    phases = {}
    tot_phase = sum(v[1] for k, v in pstats.items() if "idle" not in k) or 1.0
    for name, (cnt, ms) in pstats.items():
        phases[name] = {"items": cnt, "avg_item_us": ms / cnt * 1e3, "item_ms": ms,
                        "share_of_busy_item_time": (ms / tot_phase) if "idle" not in name
                        else None}
    if dom:
        name, (cnt, ms) = dom
        avg_s = ms / cnt / 1e3
        if name == "persistent_solve":
            # one launch = whole solves (per_launch of them).  The matvec
            # byte model B = 9 p N^d + p M (4^d + 2d + 4) per field solve:
            # p = 4 for the float32 Arnoldi matvecs (and a refined launch's
            # Neumann right-hand side and residual updates), p = 8 for the
            # float64-grade ones (the residuals, transformed in double-float)
            mv64, mv32, B = launch_field_solves(
                pinfos, per_launch, prec == ibdl.FP32_REFINED,
                [p.bc == configs.NEUMANN for p in probs], n, m)
            ach = B / avg_s / 1e9
            roofline = {"kernel": name, "bound": "hbm", "achieved": ach,
                        "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": ach / peaks["hbm_gbs"],
                        "peak_src": peaks["src"] + " (STREAM-style copy, MEASURED_PEAKS.json)",
                        "traffic": PAIR_LAUNCH_DRAM_BYTES if args.mode == "batched" else None,
                        "traffic_src": PAIR_LAUNCH_DRAM_SRC,
                        "algorithmic_bytes_per_launch": B,
                        "byte_model": "9 p N^d + p M (4^d + 2d + 4) per field solve, "
                                      "p = 4 (float32 matvec) or 8 (float64-grade)",
                        "float64_grade_field_solves_per_launch": mv64,
                        "float32_matvecs_per_launch": mv32,
                        "avg_launch_us": avg_s * 1e6,
                        "l2_resident": "the working set of the pair (about 40 MB) fits the "
                                       "129 MB L2; L2 is flushed between launches, so the "
                                       "first touch of each buffer per launch comes from HBM"}
        else:
            model = kernel_model(name, n, m)
            if model is not None:
                ach = model["bytes"] / avg_s / 1e9
                roofline = {"kernel": name, "bound": "hbm", "achieved": ach,
                            "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": ach / peaks["hbm_gbs"], "traffic": None,
                            "peak_src": peaks["src"], "algorithmic_bytes": model["bytes"],
                            "avg_launch_us": avg_s * 1e6}

    # ---- end to end through the C ABI with pinned host buffers
    hb = [torch.tensor(p.bdata, dtype=torch.float64).pin_memory() for p in probs]
    hq = [torch.zeros(p.geom.m, dtype=torch.float64).pin_memory() for p in probs]
    e2e_steps = max(3, args.steps // 2)
    e2e_s = 0.0
    for _ in range(e2e_steps):
        # the same L2 state as the device-timed steps: flushed before each
        # step, outside the host timer
        flush.fill_(7.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if args.mode == "batched":
            batch.solve(geoms, hb, hq, tol=args.tol)
        else:
            for i in range(len(probs)):
                solve(i, hb[i], hq[i])
        e2e_s += time.perf_counter() - t0
    e2e = {"value": e2e_steps * len(probs) * world / e2e_s, "unit": "solves/s",
           "h2d_bytes_per_step": int(sum(8 * p.geom.m for p in probs)),
           "d2h_bytes_per_step": int(sum(8 * p.geom.m for p in probs)),
           "note": ("ibdl_solve_batched" if args.mode == "batched" else "ibdl_solve") +
                   " with pinned host U_b/V_b in and host Q/U out; copies inside the "
                   "call; host wall clock per step, L2 flushed before each step outside "
                   "the clock"}

    matvec = run_matvec_roofline(pkg, peaks) if not args.no_matvec else None
    if matvec and roofline:
        # the single-matvec fractions of the same byte model, per precision
        roofline["matvec_frac_of_hbm"] = {k: v["frac_of_hbm"] for k, v in matvec.items()}

    batched_c4 = run_batched_c4(pkg) if not args.no_batched else None
    c1 = run_c1(pkg) if not args.no_c1 else None
    c3_solve = run_c3_solve(pkg) if not args.no_matvec else None
    method_rows = run_method_rows(pkg, peaks) if not args.no_matvec else None

    serving = None
    if args.serve_requests > 0:
        serving = run_serving_sweep(pkg, args.serve_requests)

    out = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(probs, args.tol)
            qd = qs[0].cpu().numpy()
            ref = cpu.pop("_x0")
            cpu["gpu_vs_oracle_rel_diff"] = float(np.linalg.norm(qd - ref) / np.linalg.norm(ref))
        iters = [f["iters"] for f in infos]
        mv = [f["matvecs"] for f in infos]
        out = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            # float32 inner operator; float64 spread, interpolation and Krylov
            # work; double-float transforms for the residuals of the pair
            "dtype": "f32+f64+dd" if prec == ibdl.FP32_REFINED else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "m": m, "kappa": 1e-3,
                       "tol": args.tol, "precision": args.precision,
                       "l2": "flushed between steps (512 MiB write, outside the events)",
                       "engine": "persistent" if args.engine == 0 else "host-loop",
                       "mode": args.mode,
                       "parallelism": f"replicas x{world}"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)),
                           "p99": float(np.percentile(lat, 99)),
                           "mean": float(np.mean(lat)),
                           "per": "step (the Dirichlet + Neumann pair)" if args.mode == "batched"
                                  else "step (two solves in sequence)"},
            "solo": solo,
            "fp64": fp64,
            # the autotuner's picks for the benchmark's geometry kind
            "tuner_picks": {k: geoms[0].info()[k]
                            for k in ("rows_per_tile", "pencils_per_item", "fft_plan")},
            "iters_per_solve": {"min": min(iters), "max": max(iters)},
            # per solve: float64-grade residuals and float32 residual updates
            "residuals_per_solve": {
                "float64_grade": float(np.mean([f["matvecs"] - f["iters"]
                                                - f.get("residual_updates", 0)
                                                for f in infos])),
                "float32_updates": float(np.mean([f.get("residual_updates", 0)
                                                  for f in infos]))},
            "matvecs_per_s": float(sum(mv)) * world / (total_ms / 1e3),
            "rel_err_vs_fp64_1e-12": max(errs),
            "roofline": roofline,
            "kernels": kernels,
            "phases": phases,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "matvec": matvec,
            "batched_c4": batched_c4,
            "c1": c1,
            "c3_solve": c3_solve,
            "method_rows": method_rows,
            "serving": serving,
            "gpu_launches": int(launches),
            "wall_s_timed": wall,
            "clocks": clocks,
        }
        print(json.dumps(out), flush=True)
    for g in geoms:
        g.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
