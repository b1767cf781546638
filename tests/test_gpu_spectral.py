"""Parity of the Fourier-spectral discretisation (Sec. 5.1, Sec. 6.2.1,
Sec. 6.7) on the GPU with the float64 oracle.  Tolerances as for the
finite-difference operators: float64 1e-12 relative, float32 1e-5, solves
at tol 1e-12 against dense LU 1e-10."""
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def gpu(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def host(t):
    return t.detach().cpu().numpy()


def case(name):
    if name == "star256":
        return geometry.star(256, 0.3, 0.2, 5, kappa=1e-3)
    if name == "wrap":
        return geometry.circle(64, 0.35, center=(-0.25, 1.95), box_len=2.0, origin=(-0.3, 0.1),
                               kappa=5e-2)
    if name == "poisson128":
        return geometry.circle(128, 0.3, spacing=0.75, kappa=np.inf)
    if name == "sphere32":
        return geometry.sphere(32, 0.25, m=400, center=(0, 0, 0), origin=(-0.5,) * 3, kappa=1.0)
    return geometry.ellipsoid(64, (0.3, 0.22, 0.26), kappa=1e-2)


@pytest.mark.parametrize("name", ["star256", "wrap", "poisson128", "sphere32", "ellipsoid64"])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_spectral_matvec_parity(name, prec, tol):
    g = case(name)
    bcs = [configs.DIRICHLET] if np.isinf(g.kappa) else [configs.DIRICHLET, configs.NEUMANN]
    q = np.random.default_rng(4).standard_normal(g.m)
    for bc in bcs:
        ref = O.Operator(g, bc, disc="spectral").apply(q)
        G = pkg.Geometry.from_workload(g, bc=bc, precision=prec, disc="spectral")
        y = torch.empty(g.m, dtype=torch.float64, device=DEV)
        G.apply(gpu(q), y, precision=prec)
        assert_parity(host(y), ref, tol, str(bc))
        G.close()


@pytest.mark.parametrize("bc", [0, 1])
def test_spectral_solve_matches_dense_lu(bc):
    p = configs.table1(64, 1.0)
    g = p.geom
    ub = np.random.default_rng(6).standard_normal(g.m)
    qstar = O.solve_dense(g, bc, ub, disc="spectral")
    G = pkg.Geometry.from_workload(g, bc=bc, disc="spectral")
    q = torch.zeros(g.m, dtype=torch.float64, device=DEV)
    info = G.solve(gpu(ub), q, tol=1e-12)
    assert info["status"] == 0
    assert_parity(host(q), qstar, 1e-10)
    G.close()


def test_spectral_refined_solve_and_table3_count():
    """Sec. 6.7's 3D problem at dx = 2^-5 with 900 points: the paper's 6
    iterations (the oracle's count) and the float64 solution to 1e-8."""
    g = geometry.sphere(32, 0.25, m=900, center=(0, 0, 0), origin=(-0.5,) * 3, kappa=1.0)
    x, y, z = (g.X - np.array(g.center)).T
    ub = 0.25 * z * 2 * x * y / np.maximum(x * x + y * y, 1e-300)
    ref = O.solve(g, configs.DIRICHLET, ub, tol=1e-8, disc="spectral")
    qstar = O.solve_dense(g, configs.DIRICHLET, ub, disc="spectral")
    G = pkg.Geometry.from_workload(g, precision=ibdl.FP32_REFINED, disc="spectral")
    q = torch.zeros(g.m, dtype=torch.float64, device=DEV)
    info = G.solve(gpu(ub), q, tol=1e-10)
    assert info["status"] == 0
    assert_parity(host(q), qstar, 1e-8)
    G.close()
    G = pkg.Geometry.from_workload(g, disc="spectral")
    info = G.solve(gpu(ub), q, tol=1e-8)
    assert abs(info["iters"] - ref.iters) <= 1
    G.close()


def test_spectral_evaluate_with_forcing_and_neumann_vb():
    g = geometry.star(128, 0.3, 0.2, 5, kappa=1e-2)
    r = np.random.default_rng(8)
    q, vb, gt = r.standard_normal(g.m), r.standard_normal(g.m), r.standard_normal((128, 128))
    for bc, v in ((configs.DIRICHLET, None), (configs.NEUMANN, vb)):
        op = O.Operator(g, bc, disc="spectral")
        ref = op.evaluate(q, vb=v, g_grid=gt).reshape(-1)
        G = pkg.Geometry.from_workload(g, bc=bc, disc="spectral")
        u = torch.empty(128 * 128, dtype=torch.float64, device=DEV)
        G.evaluate(gpu(q), u, vb=None if v is None else gpu(v), g_grid=gpu(gt))
        assert_parity(host(u), ref, 1e-12)
        # the right-hand side with forcing goes through the same spectral path
        qs = torch.zeros(g.m, dtype=torch.float64, device=DEV)
        G.solve(gpu(q), qs, g_grid=gpu(gt), tol=1e-12)
        qd = O.solve_dense(g, bc, q, g_grid=gt, disc="spectral")
        assert_parity(host(qs), qd, 1e-10)
        G.close()


def test_spectral_unsupported_paths():
    g = geometry.circle(64, 0.3, kappa=1e-2)
    G = pkg.Geometry.from_workload(g, disc="spectral")
    q = gpu(np.ones(g.m))
    f = torch.empty(64 * 64, dtype=torch.float64, device=DEV)
    for call in (lambda: G.spread_div(q, f), lambda: G.helmholtz(f, f)):
        with pytest.raises(ibdl.IbdlError) as e:
            call()
        assert e.value.status == 8
    G.spread(q, f)  # the plain spread has no derivative: allowed
    b = ibdl.Batch(2)
    with pytest.raises(ibdl.IbdlError) as e:
        b.solve([G], [q], [torch.zeros_like(q)])
    assert e.value.status == 8
    b.close()
    G.close()
    with pytest.raises(ibdl.IbdlError) as e:
        pkg.Geometry.from_workload(geometry.circle(64, 0.3, kappa=np.inf), eta=1.0,
                                   disc="spectral")
    assert e.value.status == 8
