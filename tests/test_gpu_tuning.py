"""The autotuner of the x-pass tiling and of the pencil items: whatever it
picks, the operator is the fixed rule's to rounding (float64 1e-12, float32
1e-6 relative), and every admissible pencils-per-item choice matches the
float64 oracle element-wise at the matvec tolerances (float64 1e-12, float32
1e-5)."""
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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
@pytest.mark.parametrize("which", ["star256", "ellipsoid32"])
def test_tuned_tiling_matches_fixed_rule(which, prec, tol):
    if which == "star256":
        g = geometry.star(256, 0.3, 0.2, 5, kappa=1e-3)
        rule, admissible = 4, {2, 4, 8, 16, 32}
    else:
        g = geometry.ellipsoid(32, (0.3, 0.22, 0.26), kappa=1e-2)
        rule, admissible = 8, {2, 4, 8}
    q = torch.tensor(np.random.default_rng(5).standard_normal(g.m), device=DEV)
    out = {}
    try:
        for on in (False, True):
            ibdl.tuning_enable(on)
            G = pkg.Geometry.from_workload(g, bc=configs.NEUMANN, precision=prec)
            rows = G.info()["rows_per_tile"]
            assert rows == rule if not on else rows in admissible
            y = torch.empty_like(q)
            G.apply(q, y, precision=prec)
            out[on] = y.cpu().numpy()
            G.close()
    finally:
        ibdl.tuning_enable(True)
    assert_parity(out[True], out[False], tol)


def test_pinned_tiling_is_used_and_checked():
    """ibdl_tuning_set pins the tiling of a kind; the operator stays the
    fixed rule's to rounding, and inadmissible pins are refused."""
    g2 = geometry.circle(64, 0.3, kappa=1e-2)
    g3 = geometry.sphere(32, 0.25, m=400, center=(0, 0, 0), origin=(-0.5,) * 3, kappa=1.0)
    try:
        for g, dim, pin in ((g2, 2, 8), (g3, 3, 4)):
            q = torch.tensor(np.random.default_rng(9).standard_normal(g.m), device=DEV)
            out = {}
            for pinned in (False, True):
                ibdl.tuning_enable(pinned)
                if pinned:
                    ibdl.tuning_set(dim, g.n, ibdl.FP64, pin)
                G = pkg.Geometry.from_workload(g, bc=configs.DIRICHLET, precision=ibdl.FP64)
                if pinned:
                    assert G.info()["rows_per_tile"] == pin
                y = torch.empty_like(q)
                G.apply(q, y)
                out[pinned] = y.cpu().numpy()
                G.close()
            assert_parity(out[True], out[False], 1e-12)
        bad = [(4, 64, 0, 8), (2, 100, 0, 8), (2, 64, 2, 8), (2, 64, 0, 6), (2, 64, 0, 32),
               (2, 64, 0, -2), (3, 32, 0, 16)]
        for args in bad:
            with pytest.raises(ibdl.IbdlError) as e:
                ibdl.tuning_set(*args)
            assert e.value.status == 1, args
    finally:
        ibdl.tuning_set(2, 64, ibdl.FP64, 0)
        ibdl.tuning_set(3, 32, ibdl.FP64, 0)
        ibdl.tuning_enable(True)


PENCIL_CASES = [
    # (geometry, pinned precision, matvec precisions and tolerances, c_solve, c_y)
    ("star256", 0, ((0, 1e-12), (2, 1e-12)),
     (1, 2, 4), (0,)),
    ("star256", 1, ((1, 1e-5),), (1, 2, 4, 8), (0,)),
    ("sphere64", 1, ((1, 1e-5),), (2, 4, 8, 16), (1, 4, 16)),
    ("sphere64", 0, ((0, 1e-12),), (2, 4, 8), (2, 8)),
]


@pytest.mark.parametrize("name,prec,checks,csolve,cy", PENCIL_CASES)
def test_every_pencil_choice_matches_oracle(name, prec, checks, csolve, cy):
    if name == "star256":
        g = geometry.star(256, 0.3, 0.2, 5, kappa=1e-3)
    else:
        g = geometry.sphere(64, 0.3, kappa=1e-2)
    q = np.random.default_rng(17).standard_normal(g.m)
    ref = O.Operator(g, configs.DIRICHLET).apply(q)
    try:
        for c in csolve:
            for y in cy:
                ibdl.tuning_set_pencils(g.dim, g.n, prec, c, y)
                G = pkg.Geometry.from_workload(g, bc=configs.DIRICHLET, precision=prec)
                info = G.info()
                assert info["pencils_per_item"][0] == c, info
                if g.dim == 3 and y:
                    assert info["pencils_per_item"][1] == y, info
                for mp, tol in checks:
                    out = torch.empty(g.m, dtype=torch.float64, device=DEV)
                    G.apply(torch.tensor(q, device=DEV), out, precision=mp)
                    assert_parity(out.cpu().numpy(), ref, tol, f"{name} c={c} y={y} prec={mp}")
                G.close()
        with pytest.raises(ibdl.IbdlError):
            ibdl.tuning_set_pencils(g.dim, g.n, prec, 3, 0)
    finally:
        ibdl.tuning_set_pencils(g.dim, g.n, prec, 0, 0)


@pytest.mark.parametrize("n", [512, 1024])
@pytest.mark.parametrize("plan", [0, 1])
def test_every_fft_plan_matches_the_oracle(n, plan):
    """Both FFT plan variants of the float32 transforms (radices as even as
    possible after a first radix-16 pass, or radix-16 passes first: 1024 =
    16*8*8 or 16*16*4, 512 = 16*8*4 or 16*16*2), pinned for a 2D
    float32-refined kind, give the float64 oracle's operator element-wise at
    the float32 matvec tolerance, through the launch-based passes; the
    geometry reports the plan it uses."""
    g = geometry.star(n, 0.3, 0.2, 5, kappa=1e-3)
    q = np.random.default_rng(40 + n + plan).standard_normal(g.m)
    try:
        ibdl.tuning_set_plan(2, n, ibdl.FP32_REFINED, plan)
        G = pkg.Geometry.from_workload(g, bc=configs.DIRICHLET, precision=ibdl.FP32_REFINED)
        assert G.info()["fft_plan"] == plan
        y = torch.empty(g.m, dtype=torch.float64, device=DEV)
        G.apply(torch.tensor(q, device=DEV), y, precision=ibdl.FP32_REFINED)
        torch.cuda.synchronize()
        G.close()
    finally:
        ibdl.tuning_set_plan(2, n, ibdl.FP32_REFINED, -1)
    ref = O.Operator(g, configs.DIRICHLET).apply(q)
    assert_parity(y.cpu().numpy(), ref, 1e-5, f"plan {plan} n={n}")


def test_radix16_first_plan_in_the_persistent_solver():
    """With the radix-16-first plan pinned for the C2 kind, the persistent
    solver's float32 items transform in that plan too: the benchmark's
    Dirichlet + Neumann pair, solved in one batched launch at tol 1e-8,
    matches the oracle's solves (Sec. 5.3) to 1e-8."""
    probs = [configs.c2(bc=configs.DIRICHLET), configs.c2(bc=configs.NEUMANN)]
    try:
        ibdl.tuning_set_plan(2, 1024, ibdl.FP32_REFINED, 1)
        gs = [pkg.Geometry.from_workload(p.geom, bc=p.bc, precision=ibdl.FP32_REFINED)
              for p in probs]
    finally:
        ibdl.tuning_set_plan(2, 1024, ibdl.FP32_REFINED, -1)
    qs = [torch.zeros(p.geom.m, dtype=torch.float64, device=DEV) for p in probs]
    batch = ibdl.Batch(2)
    try:
        assert all(G.info()["fft_plan"] == 1 for G in gs)
        infos = batch.solve(gs, [torch.tensor(p.bdata, device=DEV) for p in probs], qs,
                            tol=1e-8)
    finally:
        batch.close()
        for G in gs:
            G.close()
    for p, q, info in zip(probs, qs, infos):
        assert info["status"] == ibdl.OK and info["rel_residual"] <= 1e-8, info
        ref = O.solve(p.geom, p.bc, p.bdata, tol=1e-13).x
        assert_parity(q.cpu().numpy(), ref, 1e-8, f"{p.name} plan 1")
