"""Small fixed workloads for profilers (ncu) and quick timing.

    python -m paper_2203_12126_gb300.probe matvec c3 f32 [reps] [rows_per_tile]
    python -m paper_2203_12126_gb300.probe solve c2 [reps] [rows_per_tile]
    python -m paper_2203_12126_gb300.probe pair c2 [reps] [rows_per_tile]

``matvec`` applies the boundary operator of the 3D sphere (c3: N=256^3,
M=38039) or the 2D star (c2: N=1024^2, M=3525) ``reps`` times (default 5)
in float32 (f32), float64 (f64) or with double-float transforms (dd); ``solve`` runs ``reps`` (default 2)
float32-refined Dirichlet solves of c2 at tolerance 1e-8 through the
persistent solver; ``pair`` runs ``reps`` (default 2) batched launches of the
benchmark's step, the c2 Dirichlet + Neumann pair in one persistent launch.
``rows_per_tile`` pins the x-pass tiling (the autotuner's timings are not
trustworthy under a profiler).  Everything runs in the CUDA library; the
script only builds the inputs.
"""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv):
    import numpy as np
    import torch

    import paper_2203_12126_gb300 as pkg
    from workloads import configs

    pkg.load()
    what, case = argv[0], argv[1]
    prob = configs.c3() if case == "c3" else configs.c2()
    dev = torch.device("cuda:0")
    if what == "matvec":
        tag = argv[2] if len(argv) > 2 else "f32"
        prec = {"f32": 1, "f64": 0, "dd": 2}[tag]
        reps = int(argv[3]) if len(argv) > 3 else 5
        if len(argv) > 4:
            # a fixed x-pass tiling: under a profiler the tuner's timings mislead
            from paper_2203_12126_gb300 import ibdl
            ibdl.tuning_set(prob.geom.dim, prob.geom.n, min(prec, 1), int(argv[4]))
        g = pkg.Geometry.from_workload(prob.geom, bc=prob.bc, precision=min(prec, 1))
        q = torch.tensor(np.random.default_rng(0).standard_normal(prob.geom.m), device=dev)
        y = torch.empty_like(q)
        for _ in range(reps):
            g.apply(q, y, precision=prec)
        torch.cuda.synchronize()
        print(f"matvec {case} {tag} x{reps}: |y| = {float(y.norm()):.6e}")
    elif what == "solve":
        reps = int(argv[2]) if len(argv) > 2 else 2
        if len(argv) > 3:
            from paper_2203_12126_gb300 import ibdl
            ibdl.tuning_set(prob.geom.dim, prob.geom.n, pkg.FP32_REFINED, int(argv[3]))
        g = pkg.Geometry.from_workload(prob.geom, bc=prob.bc, precision=pkg.FP32_REFINED)
        b = torch.tensor(prob.bdata, device=dev)
        q = torch.empty_like(b)
        for _ in range(reps):
            info = g.solve(b, q, tol=1e-8)
        torch.cuda.synchronize()
        print(f"solve {case} x{reps}: iters {info['iters']} rel_res {info['rel_residual']:.2e}")
    elif what == "pair":
        reps = int(argv[2]) if len(argv) > 2 else 2
        from paper_2203_12126_gb300 import ibdl
        probs = [configs.c2(bc=configs.DIRICHLET), configs.c2(bc=configs.NEUMANN)]
        if len(argv) > 3:
            ibdl.tuning_set(2, probs[0].geom.n, pkg.FP32_REFINED, int(argv[3]))
        gs = [pkg.Geometry.from_workload(p.geom, bc=p.bc, precision=pkg.FP32_REFINED)
              for p in probs]
        bs = [torch.tensor(p.bdata, device=dev) for p in probs]
        qs = [torch.empty_like(b) for b in bs]
        batch = ibdl.Batch(2)
        for _ in range(reps):
            infos = batch.solve(gs, bs, qs, tol=1e-8)
        torch.cuda.synchronize()
        print(f"pair {case} x{reps}: iters {[f['iters'] for f in infos]}")
        batch.close()
        for gg in gs:
            gg.close()
        return 0
    else:
        raise SystemExit(__doc__)
    g.close()
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
