"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative, 2-norm unless stated):
* float64 operators: 1e-12.  Each output is a sum of at most a few hundred
  terms (36 spread taps per point and tile, an FFT of depth log2 n <= 12,
  16/64 interpolation taps); the rounding of either side is ~1e-15 relative,
  so 1e-12 leaves three orders of margin while any indexing or sign error
  shows up at O(1).
* float32 operators: 1e-5 (the raw float32 matvec bound).
* double-float transforms (IBDL_FP64_DF, the refined solver's residual
  operator): 1e-12 as for float64 (about 2^-48 per operation on either side
  of the transforms, float64 spread and interpolation).
* float64 solves at tol 1e-12 vs the dense-LU density: 1e-10.
* float32-refined solves at tol 1e-10 vs the dense-LU density: 1e-8.
"""
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
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def host(t):
    return t.detach().cpu().numpy()


# ---- geometries ---------------------------------------------------------------

def geo_c1():
    return configs.c1().geom


def geo_star256():
    return geometry.star(256, 0.3, 0.2, 5, kappa=1e-3)


def geo_wrap():
    # circle straddling the periodic boundary; non-unit box, shifted origin
    return geometry.circle(64, 0.35, center=(-0.25, 1.95), box_len=2.0,
                           origin=(-0.3, 0.1), kappa=5e-2)


def geo_tiny():
    return geometry.circle(16, 0.3, m=7, kappa=1e-1)


def geo_single():
    g = geometry.circle(32, 0.2, m=1, kappa=1e-2)
    return g


def geo_cos4():
    return geometry.star(128, 0.25, 0.15, 3, kappa=1e-2, delta="cos4")


def geo_sphere32():
    return geometry.sphere(32, 0.3, kappa=1e-2)


def geo_ellipsoid32():
    return geometry.ellipsoid(32, (0.3, 0.22, 0.26), kappa=3e-2, delta="cos4")


def geo_sphere_wrap():
    return geometry.sphere(16, 0.3, center=(0.1, 0.95, 0.5), kappa=1e-1)


GEOS2 = {"c1": geo_c1, "star256": geo_star256, "wrap": geo_wrap, "tiny": geo_tiny,
         "single": geo_single, "cos4": geo_cos4}
GEOS3 = {"sphere32": geo_sphere32, "ellipsoid32": geo_ellipsoid32,
         "sphere_wrap16": geo_sphere_wrap}
ALL = {**GEOS2, **GEOS3}


def make(g, bc=configs.DIRICHLET, precision=0):
    return pkg.Geometry.from_workload(g, bc=bc, precision=precision)


def density(g, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(g.m)


# ---- component operators --------------------------------------------------------

@pytest.mark.parametrize("name", list(ALL))
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_spread_div_parity(name, prec, tol):
    g = ALL[name]()
    G = make(g)
    q = density(g)
    f = torch.empty((g.n,) * g.dim, dtype=torch.float64, device=DEV)
    G.spread_div(gpu(q), f, precision=prec)
    ref = O.spread_div(O.Box.of(g), g.X, g.normals, g.weights, q, g.delta)
    assert_parity(host(f), ref, tol)
    G.close()


@pytest.mark.parametrize("name", list(ALL))
def test_spread_parity(name):
    g = ALL[name]()
    G = make(g)
    v = density(g, 1)
    f = torch.empty((g.n,) * g.dim, dtype=torch.float64, device=DEV)
    G.spread(gpu(v), f)
    ref = O.spread(O.Box.of(g), g.X, v, g.weights, g.delta)
    assert_parity(host(f), ref, 1e-12)
    G.close()


@pytest.mark.parametrize("name", ["c1", "wrap", "tiny", "sphere32", "sphere_wrap16"])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_helmholtz_parity(name, prec, tol):
    g = ALL[name]()
    G = make(g)
    rng = np.random.default_rng(7)
    f = rng.standard_normal((g.n,) * g.dim)
    v = torch.empty_like(gpu(f))
    G.helmholtz(gpu(f), v, precision=prec)
    box = O.Box.of(g)
    ref = g.kappa * O.helmholtz_solve(box, g.kappa, f)
    assert_parity(host(v), ref, tol)
    G.close()


@pytest.mark.parametrize("name", list(ALL))
@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 1e-6)])
def test_interp_parity(name, prec, tol):
    g = ALL[name]()
    G = make(g)
    rng = np.random.default_rng(8)
    u = rng.standard_normal((g.n,) * g.dim)
    y = torch.empty(g.m, dtype=torch.float64, device=DEV)
    G.interp(gpu(u), y, precision=prec)
    ref = O.interp(O.Box.of(g), g.X, u, g.delta)
    assert_parity(host(y), ref, tol)
    G.close()


# ---- the matvec ------------------------------------------------------------------

@pytest.mark.parametrize("name", list(ALL))
@pytest.mark.parametrize("bc", [configs.DIRICHLET, configs.NEUMANN])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5), (2, 1e-12)])
def test_matvec_parity(name, bc, prec, tol):
    g = ALL[name]()
    G = make(g, bc=bc)
    q = density(g, 3)
    y = torch.empty(g.m, dtype=torch.float64, device=DEV)
    G.apply(gpu(q), y, precision=prec)
    ref = O.Operator(g, bc).apply(q)
    assert_parity(host(y), ref, tol)
    G.close()


def test_matvec_host_pointers_match_device_pointers():
    g = geo_star256()
    G = make(g)
    q = density(g, 4)
    y_host = np.zeros(g.m)
    G.apply(q, y_host)                      # numpy in, numpy out
    y_dev = torch.empty(g.m, dtype=torch.float64, device=DEV)
    G.apply(gpu(q), y_dev)
    torch.cuda.synchronize()
    # the spread accumulates with shared-memory atomics, so two applications
    # agree to rounding, not bit for bit
    assert_parity(y_host, host(y_dev), 1e-14)
    pinned = torch.tensor(q).pin_memory()
    y_pin = torch.zeros(g.m, dtype=torch.float64).pin_memory()
    G.apply(pinned, y_pin)
    assert_parity(y_pin.numpy(), y_host, 1e-14)
    G.close()


def test_matvec_in_place_alias():
    g = geo_c1()
    G = make(g)
    q = density(g, 5)
    t = gpu(q)
    G.apply(t, t)
    assert_parity(host(t), O.Operator(g, configs.DIRICHLET).apply(q), 1e-12)
    G.close()


@pytest.mark.parametrize("bc", [configs.DIRICHLET, configs.NEUMANN])
def test_matvec_parity_full_c2(bc):
    """Config C2 geometry at full size (N=1024^2, M=3525), both precisions."""
    p = configs.c2(bc=bc)
    g = p.geom
    q = density(g, 6)
    ref = O.Operator(g, bc).apply(q)
    for prec, tol in ((0, 1e-12), (1, 1e-5), (2, 1e-12)):
        G = make(g, bc=bc, precision=min(prec, 1))
        y = torch.empty(g.m, dtype=torch.float64, device=DEV)
        G.apply(gpu(q), y, precision=prec)
        assert_parity(host(y), ref, tol)
        G.close()


def test_matvec_parity_full_c3_sampled():
    """Config C3 (N=256^3, M=38038) float32 and float64 matvecs against the
    oracle on all points (the oracle runs the full 256^3 FFT once)."""
    p = configs.c3()
    g = p.geom
    q = density(g, 9)
    ref = O.Operator(g, configs.NEUMANN).apply(q)
    for prec, tol in ((0, 1e-12), (1, 1e-5), (2, 1e-12)):
        G = make(g, bc=configs.NEUMANN, precision=min(prec, 1))
        y = torch.empty(g.m, dtype=torch.float64, device=DEV)
        G.apply(gpu(q), y, precision=prec)
        assert_parity(host(y), ref, tol)
        G.close()


def test_matvec_parity_512_cube():
    """3D at N=512^3 (M=3000): the smallest 3D grid whose pencil transforms
    take three radix passes, so the strided z solve and the y passes run
    their global-memory first and last passes in the three-pass plan.  The
    oracle runs the full 512^3 FFTs once (about half a minute)."""
    g = geometry.sphere(512, 0.3, m=3000, center=(0.0, 0.0, 0.0), origin=(-0.5,) * 3,
                        kappa=1e-3)
    q = density(g, 10)
    ref = O.Operator(g, configs.NEUMANN).apply(q)
    for prec, tol in ((0, 1e-12), (1, 1e-5), (2, 1e-12)):
        G = make(g, bc=configs.NEUMANN, precision=min(prec, 1))
        y = torch.empty(g.m, dtype=torch.float64, device=DEV)
        G.apply(gpu(q), y, precision=prec)
        assert_parity(host(y), ref, tol, str(prec))
        G.close()


# ---- solves ----------------------------------------------------------------------

@pytest.mark.parametrize("name", ["c1", "wrap", "tiny", "cos4", "sphere_wrap16"])
@pytest.mark.parametrize("bc", [configs.DIRICHLET, configs.NEUMANN])
def test_fp64_solve_matches_dense_lu(name, bc):
    g = ALL[name]()
    b = np.cos(3 * np.arange(g.m) * 2 * np.pi / g.m) + 0.2
    q_star = O.solve_dense(g, bc, b)
    G = make(g, bc=bc)
    q = torch.empty(g.m, dtype=torch.float64, device=DEV)
    info = G.solve(gpu(b), q, tol=1e-12)
    assert_parity(host(q), q_star, 1e-10, str(info))
    assert info["rel_residual"] <= 1e-12
    G.close()


@pytest.mark.parametrize("name", ["c1", "star256", "sphere32"])
@pytest.mark.parametrize("bc", [configs.DIRICHLET, configs.NEUMANN])
def test_fp32_refined_solve_reaches_1e8(name, bc):
    g = ALL[name]()
    b = density(g, 11)
    ref = O.solve(g, bc, b, tol=1e-13)
    G = make(g, bc=bc, precision=1)
    q = torch.empty(g.m, dtype=torch.float64, device=DEV)
    info = G.solve(gpu(b), q, tol=1e-10)
    assert info["refine_steps"] >= 1
    assert_parity(host(q), ref.x, 1e-8, str(info))
    G.close()


def test_iteration_counts_match_oracle_table1_cases():
    """GPU GMRES counts equal the oracle's within +-1 (threshold crossing)
    on the Table 1 problem, and are flat in N and point spacing."""
    counts = []
    for n in (64, 128, 256, 512):
        for c in (2.0, 0.75):
            p = configs.table1(n, c)
            ro = O.solve(p.geom, p.bc, p.bdata, tol=1e-8)
            G = make(p.geom)
            q = torch.empty(p.geom.m, dtype=torch.float64, device=DEV)
            info = G.solve(gpu(p.bdata), q, tol=1e-8)
            assert abs(info["iters"] - ro.iters) <= 1, (n, c, info["iters"], ro.iters)
            counts.append(info["iters"])
            G.close()
    assert max(counts) - min(counts) <= 2


def test_solve_with_forcing_and_evaluate():
    """Dirichlet with forcing g~ (rhs U_b + kappa S* L'^{-1} g~) and the
    grid evaluation u = kappa L'^{-1}(S~Q - g~)."""
    g = geo_star256()
    rng = np.random.default_rng(12)
    gg = rng.standard_normal((g.n,) * g.dim)
    b = density(g, 13)
    op = O.Operator(g, configs.DIRICHLET)
    rhs = op.rhs(b, gg)
    q_ref = O.gmres(op, rhs, tol=1e-13).x
    G = make(g)
    q = torch.empty(g.m, dtype=torch.float64, device=DEV)
    G.solve(gpu(b), q, g_grid=gpu(gg), tol=1e-12)
    assert_parity(host(q), q_ref, 1e-10)
    u = torch.empty((g.n,) * 2, dtype=torch.float64, device=DEV)
    G.evaluate(q, u, g_grid=gpu(gg))
    assert_parity(host(u), op.evaluate(host(q), g_grid=gg), 1e-12)
    G.close()


def test_neumann_evaluate_with_vb():
    g = geo_sphere32()
    vb = density(g, 14)
    G = make(g, bc=configs.NEUMANN)
    U = torch.empty(g.m, dtype=torch.float64, device=DEV)
    G.solve(gpu(vb), U, tol=1e-12)
    op = O.Operator(g, configs.NEUMANN)
    ref = O.gmres(op, op.rhs(vb), tol=1e-13).x
    assert_parity(host(U), ref, 1e-10)
    u = torch.empty((g.n,) * 3, dtype=torch.float64, device=DEV)
    G.evaluate(U, u, vb=gpu(vb))
    assert_parity(host(u), op.evaluate(host(U), vb=vb), 1e-12)
    G.close()


def test_c1_solve_against_closed_form():
    p = configs.c1()
    G = make(p.geom)
    q = torch.empty(p.geom.m, dtype=torch.float64, device=DEV)
    info = G.solve(gpu(p.bdata), q, tol=1e-10)
    assert info["iters"] <= 8
    u = torch.empty((p.geom.n,) * 2, dtype=torch.float64, device=DEV)
    G.evaluate(q, u)
    P = configs.grid_nodes(p.geom)
    # L1 error over the nodes of Omega farther than 6h from Gamma
    mask = configs.interior_mask_circle(p.geom, 0.3, 6 * p.geom.h)
    err = np.mean(np.abs(host(u).reshape(-1)[mask] - p.exact(P)[mask]))
    assert err < 5e-3
    G.close()


# ---- status / error behaviour on the GPU ---------------------------------------

def test_nonfinite_boundary_data_is_reported():
    g = geo_c1()
    G = make(g)
    b = density(g)
    b[3] = np.nan
    q = torch.zeros(g.m, dtype=torch.float64, device=DEV)
    info = G.solve(gpu(b), q, raise_on_error=False)
    assert info["status"] == ibdl.ERR_NONFINITE
    G.close()


def test_not_converged_returns_best_iterate():
    g = geo_star256()
    G = make(g)
    b = density(g)
    q = torch.zeros(g.m, dtype=torch.float64, device=DEV)
    info = G.solve(gpu(b), q, tol=1e-14, max_iters=2, raise_on_error=False)
    assert info["status"] == ibdl.ERR_NOT_CONVERGED
    assert info["iters"] == 2 and np.isfinite(host(q)).all()
    G.close()


def test_zero_rhs_gives_zero_density():
    g = geo_c1()
    G = make(g)
    q = torch.ones(g.m, dtype=torch.float64, device=DEV)
    info = G.solve(gpu(np.zeros(g.m)), q)
    assert info["iters"] == 0 and float(q.abs().max()) == 0.0
    G.close()


def test_launch_counter_counts_library_kernels():
    g = geo_c1()
    G = make(g)
    q = gpu(density(g))
    y = torch.empty_like(q)
    n0 = pkg.kernel_launch_count()
    G.apply(q, y)
    assert pkg.kernel_launch_count() - n0 == 4   # rows_fwd, pencils, rows_inv, interp
    G.close()


def test_c3_refined_solve_matches_fp64_solve():
    """C3 at full size (3D sphere N=256^3, M=38039, Neumann): the
    float32-refined solve to 1e-10 equals the float64 solve to 1e-12 within
    the refined path's 1e-8."""
    p = configs.c3()
    b = gpu(p.bdata)
    out = {}
    for prec, tol in ((1, 1e-10), (0, 1e-12)):
        G = make(p.geom, bc=p.bc, precision=prec)
        q = torch.empty(p.geom.m, dtype=torch.float64, device=DEV)
        info = G.solve(b, q, tol=tol)
        assert info["rel_residual"] <= tol, info
        out[prec] = host(q)
        G.close()
    assert_parity(out[1], out[0], 1e-8)
