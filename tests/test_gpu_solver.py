"""The persistent single-launch solver (default engine) and the batched
solver against the host-driven loop, individual solves and the oracle."""
import numpy as np
import pytest
from parity_util import assert_parity

torch = pytest.importorskip("torch")

from oracle import ibdl_oracle as O  # noqa: E402
from workloads import configs, geometry  # noqa: E402

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2203_12126_gb300 as pkg
    from paper_2203_12126_gb300 import ibdl
    DEV = torch.device("cuda:0")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def gpu(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def mixed_instances():
    """Uneven 2D/3D instances: sizes, kappa, bc and precision all differ."""
    out = []
    rng = np.random.default_rng(40)
    specs = [
        (geometry.star(64, 0.3, 0.15, 4, kappa=1e-2), configs.DIRICHLET, 0),
        (geometry.star(128, 0.25, 0.2, 6, kappa=3e-3), configs.NEUMANN, 0),
        (geometry.star(256, 0.3, 0.1, 3, kappa=1e-3), configs.DIRICHLET, 1),
        (geometry.circle(64, 0.35, center=(-0.25, 1.95), box_len=2.0, origin=(-0.3, 0.1),
                         kappa=5e-2), configs.NEUMANN, 1),
        (geometry.sphere(32, 0.3, kappa=1e-2), configs.DIRICHLET, 0),
        (geometry.ellipsoid(32, (0.3, 0.22, 0.26), kappa=3e-2), configs.NEUMANN, 1),
        (geometry.circle(16, 0.3, m=7, kappa=1e-1), configs.DIRICHLET, 0),
        (geometry.star(512, 0.28, 0.2, 7, kappa=2e-4), configs.DIRICHLET, 0),
        # m > 4096: this one keeps the multi-block vector phases while the
        # others (batch >= 8, m <= 4096) each run on one block
        (geometry.sphere(64, 0.3, spacing=1.0, kappa=1e-2), configs.NEUMANN, 0),
    ]
    for g, bc, prec in specs:
        out.append((g, bc, prec, rng.standard_normal(g.m)))
    return out


@pytest.mark.parametrize("bc", [configs.DIRICHLET, configs.NEUMANN])
@pytest.mark.parametrize("prec", [0, 1])
def test_persistent_engine_matches_host_loop(bc, prec):
    g = geometry.star(256, 0.3, 0.2, 5, kappa=1e-3)
    b = np.random.default_rng(1).standard_normal(g.m)
    G = pkg.Geometry.from_workload(g, bc=bc, precision=prec)
    q0 = torch.empty(g.m, dtype=torch.float64, device=DEV)
    q1 = torch.empty_like(q0)
    i0 = G.solve(gpu(b), q0, tol=1e-10, engine=0)
    i1 = G.solve(gpu(b), q1, tol=1e-10, engine=1)
    assert abs(i0["iters"] - i1["iters"]) <= 1
    assert_parity(q0.cpu(), q1.cpu(), 1e-8)
    assert i0["rel_residual"] <= 1e-10
    ref = O.solve(g, bc, b, tol=1e-13).x
    assert_parity(q0.cpu(), ref, 1e-8)
    G.close()


def test_persistent_solve_c1_tight():
    p = configs.c1()
    q_star = O.solve_dense(p.geom, p.bc, p.bdata)
    G = pkg.Geometry.from_workload(p.geom, bc=p.bc)
    q = torch.empty(p.geom.m, dtype=torch.float64, device=DEV)
    info = G.solve(gpu(p.bdata), q, tol=1e-12)
    assert_parity(q.cpu(), q_star, 1e-10)
    assert 4 <= info["iters"] <= 8 and info["matvecs"] >= info["iters"]
    assert len(info["history"]) == info["iters"]
    G.close()


def test_persistent_restarts_and_max_iters():
    g = geometry.star(128, 0.3, 0.2, 5, kappa=1e-3)
    b = np.random.default_rng(2).standard_normal(g.m)
    G = pkg.Geometry.from_workload(g)
    q = torch.empty(g.m, dtype=torch.float64, device=DEV)
    info = G.solve(gpu(b), q, tol=1e-12, restart=2)       # many short cycles
    ref = O.solve(g, configs.DIRICHLET, b, tol=1e-13).x
    assert_parity(q.cpu(), ref, 1e-10)
    info = G.solve(gpu(b), q, tol=1e-14, max_iters=3, raise_on_error=False)
    assert info["status"] == ibdl.ERR_NOT_CONVERGED and info["iters"] == 3
    G.close()


def test_persistent_with_initial_guess():
    g = geometry.star(128, 0.3, 0.2, 5, kappa=1e-3)
    b = np.random.default_rng(3).standard_normal(g.m)
    G = pkg.Geometry.from_workload(g)
    q = torch.empty(g.m, dtype=torch.float64, device=DEV)
    G.solve(gpu(b), q, tol=1e-12)
    q2 = torch.empty_like(q)
    info = G.solve(gpu(b), q2, tol=1e-10, x0=q.clone())
    assert info["iters"] == 0 and rel(q2.cpu(), q.cpu()) <= 1e-14
    G.close()


def test_batched_matches_individual_and_oracle():
    inst = mixed_instances()
    geoms = [pkg.Geometry.from_workload(g, bc=bc, precision=prec) for g, bc, prec, _ in inst]
    bs = [gpu(b) for *_, b in inst]
    qs = [torch.empty(g.m, dtype=torch.float64, device=DEV) for g, *_ in inst]
    batch = ibdl.Batch(16)
    infos = batch.solve(geoms, bs, qs, tol=1e-10)
    for k, (g, bc, prec, b) in enumerate(inst):
        alone = torch.empty_like(qs[k])
        ia = geoms[k].solve(bs[k], alone, tol=1e-10)
        assert infos[k]["status"] == 0
        # the spread's shared-memory atomics make rounding order vary between
        # launches, so the two runs agree to the solve tolerance, not bitwise
        assert abs(infos[k]["iters"] - ia["iters"]) <= 1
        assert_parity(qs[k].cpu(), alone.cpu(), (1e-8 if prec else 1e-10))
        ref = O.solve(g, bc, b, tol=1e-13).x
        assert_parity(qs[k].cpu(), ref, (1e-8 if prec else 1e-9), str((k, infos[k])))
    batch.close()
    for G in geoms:
        G.close()


def test_batched_rejects_duplicates_and_overflow():
    g = geometry.circle(32, 0.3, kappa=1e-2)
    G = pkg.Geometry.from_workload(g)
    b = gpu(np.ones(g.m))
    q = torch.empty_like(b)
    batch = ibdl.Batch(2)
    with pytest.raises(ibdl.IbdlError):
        batch.solve([G, G], [b, b], [q, q])
    with pytest.raises(ibdl.IbdlError):
        batch.solve([G, G, G], [b, b, b], [q, q, q])
    batch.close()
    G.close()


def test_c4_style_batch_of_64():
    """64 instances from the C4 generator (N in {128, 256}), FP32-refined to
    1e-8, in one launch: each matches its own solve."""
    probs = configs.c4_instances(64, seed=2, sizes=(128, 256))
    geoms = [pkg.Geometry.from_workload(p.geom, precision=1) for p in probs]
    bs = [gpu(p.bdata) for p in probs]
    qs = [torch.empty(p.geom.m, dtype=torch.float64, device=DEV) for p in probs]
    batch = ibdl.Batch(64)
    infos = batch.solve(geoms, bs, qs, tol=1e-8)
    for k in (0, 17, 42, 63):
        ref = torch.empty_like(qs[k])
        geoms[k].solve(bs[k], ref, tol=1e-12)
        assert infos[k]["rel_residual"] <= 1e-8
        assert_parity(qs[k].cpu(), ref.cpu(), 1e-7)
    batch.close()
    for G in geoms:
        G.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_multiblock_vector_path_3d_large_m(prec):
    """M > 4096 takes the multi-block vector phases (partials + grid barriers)."""
    g = geometry.sphere(64, 0.3, spacing=1.0, kappa=1e-2)
    assert g.m > 4096
    b = np.random.default_rng(5).standard_normal(g.m)
    G = pkg.Geometry.from_workload(g, bc=configs.NEUMANN, precision=prec)
    q = torch.empty(g.m, dtype=torch.float64, device=DEV)
    info = G.solve(gpu(b), q, tol=1e-10)
    ref = O.solve(g, configs.NEUMANN, b, tol=1e-13).x
    assert_parity(q.cpu(), ref, (1e-8 if prec else 1e-9), str(info))
    G.close()


def test_forced_multiblock_path_matches_single_block():
    """The same small solves with the multi-block vector phases forced on
    (environment switch read at library load, so in a child process)."""
    import json
    import os
    import subprocess
    import sys
    code = r'''
import json, sys, numpy as np, torch
sys.path.insert(0, ".")
import paper_2203_12126_gb300 as pkg
from workloads import geometry, configs
out = []
for prec in (0, 1):
    g = geometry.star(256, 0.3, 0.2, 5, kappa=1e-3)
    b = np.random.default_rng(6).standard_normal(g.m)
    G = pkg.Geometry.from_workload(g, bc=configs.NEUMANN, precision=prec)
    q = torch.empty(g.m, dtype=torch.float64, device="cuda:0")
    info = G.solve(torch.tensor(b, device="cuda:0"), q, tol=1e-10)
    out.append([q.cpu().numpy().tolist(), info["iters"]])
print(json.dumps(out))
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, IBDL_SOLVER_MULTIBLOCK="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    forced = json.loads(r.stdout.strip().splitlines()[-1])
    g = geometry.star(256, 0.3, 0.2, 5, kappa=1e-3)
    b = np.random.default_rng(6).standard_normal(g.m)
    ref = O.solve(g, configs.NEUMANN, b, tol=1e-13).x
    for prec, (q, iters) in zip((0, 1), forced):
        assert_parity(q, ref, (1e-8 if prec else 1e-9))


def test_scheduler_stress_many_tiny_instances():
    """128 tiny instances (phases of one to a few items, so the dynamic
    scheduler publishes new phases constantly and idle blocks race for
    them), solved five times: every run converges and equals the solo
    solves."""
    rng = np.random.default_rng(77)
    specs = []
    for k in range(128):
        n = 16 if k % 2 else 32
        g = geometry.circle(n, 0.25 + 0.05 * (k % 3), m=12 + k % 17,
                            kappa=float(10.0 ** rng.uniform(-2, -1)))
        specs.append((g, configs.DIRICHLET if k % 3 else configs.NEUMANN, k % 2))
    geoms = [pkg.Geometry.from_workload(g, bc=bc, precision=prec) for g, bc, prec in specs]
    bs = [gpu(rng.standard_normal(g.m)) for g, _, _ in specs]
    solo = []
    for G, b in zip(geoms, bs):
        q = torch.empty_like(b)
        G.solve(b, q, tol=1e-10)
        solo.append(q.cpu().numpy())
    batch = ibdl.Batch(len(specs))
    for _ in range(5):
        qs = [torch.full_like(b, float("nan")) for b in bs]
        infos = batch.solve(geoms, bs, qs, tol=1e-10)
        for k, info in enumerate(infos):
            assert info["status"] == 0 and info["rel_residual"] <= 1e-10, (k, info)
            assert_parity(qs[k].cpu(), solo[k], 1e-8, str(k))
    batch.close()
    for G in geoms:
        G.close()


def test_double_float_and_float64_residuals_agree():
    """Float32-refined launches of at most 16 instances take double-float
    residuals and right-hand sides, larger ones float64: the same refined
    problems solved both ways meet the dense-LU solution to 1e-8 (tol 1e-10)."""
    probs = [configs.table1(64, 1.0), configs.c1()]
    geoms, bs, refs = [], [], []
    for p in probs:
        for bc in (configs.DIRICHLET, configs.NEUMANN):
            g = p.geom
            b = np.cos(2 * np.arange(g.m) * 2 * np.pi / g.m) + 0.3
            refs.append(O.solve_dense(g, bc, b))
            geoms.append(pkg.Geometry.from_workload(g, bc=bc, precision=ibdl.FP32_REFINED))
            bs.append(gpu(b))
    small = ibdl.Batch(4)
    q_small = [torch.zeros(g.m, dtype=torch.float64, device=DEV) for g in geoms]
    infos = small.solve(geoms, bs, q_small, tol=1e-10)
    assert all(f["status"] == 0 for f in infos)
    # 20 entries: the same four problems on fresh handles, five times over
    many = [pkg.Geometry.from_workload(probs[k // 2 % 2].geom,
                                      bc=(configs.DIRICHLET, configs.NEUMANN)[k % 2],
                                      precision=ibdl.FP32_REFINED) for k in range(20)]
    big = ibdl.Batch(20)
    q_big = [torch.zeros(g.m, dtype=torch.float64, device=DEV) for g in many]
    infos = big.solve(many, [bs[k % 4] for k in range(20)], q_big, tol=1e-10)
    assert all(f["status"] == 0 for f in infos)
    for k in range(4):
        assert_parity(q_small[k].cpu().numpy(), refs[k], 1e-8)
    for k in range(20):
        assert_parity(q_big[k].cpu().numpy(), refs[k % 4], 1e-8)
    small.close()
    big.close()
    for g in geoms + many:
        g.close()


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """The solver's inter-block waits are bounded: a two-party barrier that
    only one block joins gives up after its poll limit and reports
    IBDL_ERR_TIMEOUT (no fault, no hang); a solve right after succeeds."""
    import time
    t0 = time.time()
    assert ibdl.selftest_bounded_wait(1 << 14) == ibdl.ERR_TIMEOUT
    assert time.time() - t0 < 30
    p = configs.c1()
    G = pkg.Geometry.from_workload(p.geom, bc=p.bc)
    q = torch.zeros(p.geom.m, dtype=torch.float64, device=DEV)
    assert G.solve(gpu(p.bdata), q, tol=1e-10)["status"] == 0
    G.close()
