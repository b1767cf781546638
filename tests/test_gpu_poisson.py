"""Parity of the Poisson limit (kappa = inf, Sec. 5.4), the completed system
(App. C), the interior indicator (App. D) and the near-boundary values
(App. A) on the GPU with the float64 oracle.

Tolerances:
* float64 operators: 1e-12 relative (as for the Helmholtz operators: a few
  hundred rounded terms per output on either side).
* solves at tol 1e-12 against the dense LU solution: 1e-10.
* indicator: chi_h within 1e-12 absolute (values are O(1)); chi equal
  wherever |chi_h - 1/2| > 1e-9 (closer than that the threshold is decided
  by rounding, and both answers are valid).
* near-boundary values: 1e-12 relative to max |u|, element by element.
  Which nodes are replaced, and which boundary points and branch each uses,
  are decided by the same IEEE operations on both sides, so the set of
  replaced nodes must agree exactly.
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def gpu(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device=DEV)


def host(t):
    return t.detach().cpu().numpy()


def poisson_circle(n=128):
    return geometry.circle(n, 0.3, spacing=0.75, kappa=np.inf)


def poisson_star(n=256):
    return geometry.star(n, 0.3, 0.2, 5, kappa=np.inf)


def exp_exterior(n, L):
    """Sec. 6.3 on the box [-L/2, L/2)^2 (geometry, forcing, U_b)."""
    g, gt, ub, _ = configs.poisson_exterior(n, L)
    return g, gt, ub


# ---- Poisson limit ---------------------------------------------------------


@pytest.mark.parametrize("make", [poisson_circle, poisson_star])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_poisson_matvec_parity(make, prec, tol):
    g = make()
    q = np.random.default_rng(3).standard_normal(g.m)
    ref = O.Operator(g, configs.DIRICHLET).apply(q)
    G = pkg.Geometry.from_workload(g, bc=configs.DIRICHLET, precision=prec)
    y = torch.empty(g.m, dtype=torch.float64, device=DEV)
    G.apply(gpu(q), y, precision=prec)
    assert_parity(host(y), ref, tol)
    G.close()


@pytest.mark.parametrize("engine", [0, 1])
def test_poisson_solve_matches_dense_lu(engine):
    g = poisson_circle(128)
    Xc = g.X - np.array(g.center)
    ub = Xc[:, 0] ** 2 - Xc[:, 1] ** 2
    qstar = O.solve_dense(g, configs.DIRICHLET, ub)
    G = pkg.Geometry.from_workload(g, bc=configs.DIRICHLET)
    q = torch.zeros(g.m, dtype=torch.float64, device=DEV)
    info = G.solve(gpu(ub), q, tol=1e-12, engine=engine)
    assert info["status"] == 0
    assert_parity(host(q), qstar, 1e-10)
    # the field away from Gamma is the harmonic polynomial (Sec. 5.4, first order)
    u = torch.empty(g.n * g.n, dtype=torch.float64, device=DEV)
    G.evaluate(q, u)
    uo = O.Operator(g, configs.DIRICHLET).evaluate(host(q)).reshape(-1)
    assert_parity(host(u), uo, 1e-12)
    G.close()


def test_poisson_forcing_and_refined_solve():
    g = poisson_star(128)
    rng = np.random.default_rng(7)
    ub = rng.standard_normal(g.m)
    gt = rng.standard_normal((g.n, g.n))
    gt -= gt.mean()
    qstar = O.solve_dense(g, configs.DIRICHLET, ub, g_grid=gt)
    G = pkg.Geometry.from_workload(g, bc=configs.DIRICHLET, precision=ibdl.FP32_REFINED)
    q = torch.zeros(g.m, dtype=torch.float64, device=DEV)
    info = G.solve(gpu(ub), q, g_grid=gpu(gt), tol=1e-10)
    assert info["status"] == 0
    assert_parity(host(q), qstar, 1e-8)
    G.close()


def test_poisson_neumann_is_unsupported():
    g = poisson_circle(64)
    with pytest.raises(ibdl.IbdlError) as e:
        pkg.Geometry.from_workload(g, bc=configs.NEUMANN)
    assert e.value.status == 8


# ---- completed system (App. C) ---------------------------------------------


@pytest.mark.parametrize("n,L", [(128, 1.0), (256, 8.0)])
def test_completed_apply_parity(n, L):
    g, _, _ = exp_exterior(n, L)
    z = np.random.default_rng(11).standard_normal(g.m + 1)
    ref = O.CompletedOperator(g, 10.0).apply(z)
    G = pkg.Geometry.from_workload(g, bc=configs.DIRICHLET, eta=10.0)
    assert G.nsys == g.m + 1
    y = torch.empty(g.m + 1, dtype=torch.float64, device=DEV)
    G.apply(gpu(z), y)
    assert_parity(host(y), ref, 1e-12)
    # in place: q and y alias
    zz = gpu(z)
    G.apply(zz, zz)
    assert_parity(host(zz), ref, 1e-12)
    G.close()


def _completed_lu(op, b):
    M = op.m + 1
    A = np.zeros((M, M))
    e = np.zeros(M)
    for i in range(M):
        e[i] = 1.0
        A[:, i] = op.apply(e)
        e[i] = 0.0
    return np.linalg.solve(A, b)


@pytest.mark.parametrize("prec,tol,rtol", [(0, 1e-12, 1e-10), (1, 1e-10, 1e-8)])
def test_completed_solve_matches_dense_lu(prec, tol, rtol):
    g, gt, ub = exp_exterior(256, 8.0)
    op = O.CompletedOperator(g, 10.0)
    zstar = _completed_lu(op, op.rhs(ub, gt))
    G = pkg.Geometry.from_workload(g, bc=configs.DIRICHLET, precision=prec, eta=10.0)
    z = torch.zeros(g.m + 1, dtype=torch.float64, device=DEV)
    info = G.solve(gpu(ub), z, g_grid=gpu(gt), tol=tol)
    assert info["status"] == 0
    assert_parity(host(z), zstar, rtol)
    u = torch.empty(g.n * g.n, dtype=torch.float64, device=DEV)
    G.evaluate(gpu(zstar), u, g_grid=gpu(gt))
    assert_parity(host(u), op.evaluate(zstar, gt).reshape(-1), 1e-12)
    G.close()


def test_completed_geometry_rules():
    g, _, _ = exp_exterior(64, 1.0)
    with pytest.raises(ibdl.IbdlError) as e:   # eta needs the Poisson limit
        pkg.Geometry.from_workload(geometry.circle(64, 0.3, kappa=1e-2), eta=1.0)
    assert e.value.status == 1
    G = pkg.Geometry.from_workload(g, eta=10.0)
    b = ibdl.Batch(4)
    ub = gpu(np.ones(g.m))
    q = torch.zeros(g.m + 1, dtype=torch.float64, device=DEV)
    with pytest.raises(ibdl.IbdlError) as e:
        b.solve([G], [ub], [q])
    assert e.value.status == 8
    b.close()
    G.close()


# ---- indicator (App. D) ----------------------------------------------------


def _indicator_case(name):
    if name == "star256":
        return geometry.star(256, 0.3, 0.2, 5, kappa=1e-3)
    if name == "wrap":
        return geometry.circle(64, 0.35, center=(-0.25, 1.95), box_len=2.0, origin=(-0.3, 0.1),
                               kappa=5e-2)
    return geometry.sphere(64, 0.3, kappa=1e-2)


@pytest.mark.parametrize("name", ["star256", "wrap", "sphere64"])
def test_indicator_parity(name):
    g = _indicator_case(name)
    chi_h_ref, chi_ref = O.indicator(g)
    G = pkg.Geometry.from_workload(g)
    nd = g.n ** g.dim
    chi_h = torch.empty(nd, dtype=torch.float64, device=DEV)
    chi = torch.empty(nd, dtype=torch.uint8, device=DEV)
    G.indicator(chi_h, chi)
    ch = host(chi_h)
    assert np.max(np.abs(ch - chi_h_ref.reshape(-1))) <= 1e-12
    clear = np.abs(chi_h_ref.reshape(-1) - 0.5) > 1e-9
    assert np.array_equal(host(chi)[clear], chi_ref.reshape(-1)[clear])
    # host outputs, one at a time (a second solve: the spread accumulates in
    # shared memory in no fixed order, so the two calls agree to rounding)
    hc = np.empty(nd, dtype=np.uint8)
    G.indicator(None, hc)
    assert np.array_equal(hc[clear], host(chi)[clear])
    hh = np.empty(nd)
    G.indicator(hh, None)
    assert np.max(np.abs(hh - ch)) <= 1e-12
    G.close()


# ---- near-boundary values (App. A) -----------------------------------------


def _field(g, seed):
    P = configs.grid_nodes(g)
    r = np.random.default_rng(seed)
    u = np.sin(3 * P[:, 0] + 1) * np.cos(2 * P[:, 1]) + 0.01 * r.standard_normal(len(P))
    return u.reshape(g.n, g.n), r.standard_normal(g.m)


@pytest.mark.parametrize("m1,m2", [(6, 8.0), (1, 3.0), (12, 14.5)])
@pytest.mark.parametrize("which", ["star128", "exterior128", "sparse128"])
def test_near_boundary_parity(which, m1, m2):
    """sparse128: boundary points 3h apart, so the third nearest point often
    lies outside the searched cells and the full scan decides."""
    if which == "star128":
        g = geometry.star(128, 0.3, 0.2, 5, kappa=1e-2)
        inside = O.indicator(g)[1]
    elif which == "sparse128":
        g = geometry.circle(128, 0.3, spacing=3.0, kappa=1e-2)
        inside = O.indicator(geometry.circle(128, 0.3, spacing=0.75, kappa=1e-2))[1]
    else:
        g = geometry.exterior(geometry.circle(128, 0.25, spacing=0.75, kappa=np.inf))
        inside = (1 - O.indicator(geometry.circle(128, 0.25, spacing=0.75, kappa=1.0))[1])
        inside = inside.astype(np.uint8)
    u, ub = _field(g, 5)
    ref = O.near_boundary_values(g, u, ub, inside, m1, m2)
    G = pkg.Geometry.from_workload(g, bc=configs.DIRICHLET)
    out = torch.empty(g.n * g.n, dtype=torch.float64, device=DEV)
    G.near_boundary(gpu(u.reshape(-1)), gpu(ub), gpu(inside.reshape(-1), torch.uint8), m1, m2,
                    out)
    o = host(out).reshape(g.n, g.n)
    assert np.max(np.abs(o - ref)) <= 1e-12 * np.max(np.abs(u))
    assert np.array_equal(o != u, ref != u)
    assert (ref != u).sum() > 0
    # host arrays give the same bytes
    ho = np.empty(g.n * g.n)
    G.near_boundary(np.ascontiguousarray(u.reshape(-1)), ub,
                    np.ascontiguousarray(inside.reshape(-1)), m1, m2, ho)
    assert np.array_equal(ho, host(out))
    G.close()


def test_near_boundary_full_c2_sampled():
    """The C2 star (N = 1024, M = 3525): all nodes on the GPU, a sample of
    2000 nodes near Gamma (and 500 anywhere) through the oracle."""
    g = configs.c2().geom
    G = pkg.Geometry.from_workload(g)
    nn = g.n * g.n
    chi = torch.empty(nn, dtype=torch.uint8, device=DEV)
    G.indicator(None, chi)
    inside = host(chi).reshape(g.n, g.n)
    u, ub = _field(g, 9)
    out = torch.empty(nn, dtype=torch.float64, device=DEV)
    G.near_boundary(gpu(u.reshape(-1)), gpu(ub), chi, 6, 8.0, out)
    o = host(out)
    rho, rad = configs.star_radius_at(g, configs.grid_nodes(g))
    band = np.nonzero(np.abs(rho - rad) < 8 * g.h)[0]
    r = np.random.default_rng(1)
    sample = np.concatenate([r.choice(band, 2000, replace=False), r.choice(nn, 500)])
    ref = O.near_boundary_values(g, u, ub, inside, 6, 8.0, nodes=sample).reshape(-1)
    assert np.max(np.abs(o[sample] - ref[sample])) <= 1e-12 * np.max(np.abs(u))
    assert np.array_equal(o[sample] != u.reshape(-1)[sample],
                          ref[sample] != u.reshape(-1)[sample])
    G.close()


def test_near_boundary_edge_cases():
    g = geometry.star(64, 0.3, 0.2, 5, kappa=1e-2)
    G = pkg.Geometry.from_workload(g)
    u, ub = _field(g, 2)
    uin = gpu(u.reshape(-1))
    out = torch.empty_like(uin)
    none = torch.zeros(g.n * g.n, dtype=torch.uint8, device=DEV)
    G.near_boundary(uin, gpu(ub), none, 6, 8.0, out)      # no node of Omega
    assert torch.equal(out, uin)
    with pytest.raises(ibdl.IbdlError) as e:             # in place
        G.near_boundary(uin, gpu(ub), none, 6, 8.0, uin)
    assert e.value.status == 1
    for m1, m2 in ((0, 2.0), (g.n, 2.0), (3, 0.0), (3, float("nan"))):
        with pytest.raises(ibdl.IbdlError) as e:
            G.near_boundary(uin, gpu(ub), none, m1, m2, out)
        assert e.value.status == 1
    G.close()


def _sphere_band(g, r, m1):
    """Nodes whose distance to the sphere is below (m1 + 1) h: a superset of
    the nodes within m1 h of a boundary point."""
    rho = np.linalg.norm(configs.grid_nodes(g) - np.array(g.center), axis=1)
    return np.nonzero(np.abs(rho - r) < (m1 + 1) * g.h)[0], rho


@pytest.mark.parametrize("n,r,m1,m2,center", [(32, 0.3, 3, 5.0, (0.5, 0.5, 0.5)),
                                              (64, 0.27, 6, 8.0, (0.47, 0.52, 0.5)),
                                              (64, 0.3, 1, 3.0, (0.5, 0.5, 0.5))])
def test_near_boundary_3d_parity(n, r, m1, m2, center):
    """Sec. 6.7's 3D near-boundary step against the oracle, every node (the
    oracle visits a band that holds every near node; the others must be
    untouched on both sides)."""
    g = geometry.sphere(n, r, center=center, kappa=1e-2)
    band, rho = _sphere_band(g, r, m1)
    inside = (rho < r).astype(np.uint8)
    P = configs.grid_nodes(g)
    rr = np.random.default_rng(3)
    u = (np.sin(3 * P[:, 0] + 1) * np.cos(2 * P[:, 1]) * np.cos(P[:, 2])
         + 0.01 * rr.standard_normal(len(P)))
    ub = rr.standard_normal(g.m)
    ref = O.near_boundary_values_3d(g, u.reshape(n, n, n), ub, inside.reshape(n, n, n), m1, m2,
                                    nodes=band).reshape(-1)
    G = pkg.Geometry.from_workload(g)
    out = torch.empty(n ** 3, dtype=torch.float64, device=DEV)
    G.near_boundary(gpu(u), gpu(ub), gpu(inside, torch.uint8), m1, m2, out)
    o = host(out)
    assert np.max(np.abs(o - ref)) <= 1e-12 * np.max(np.abs(u))
    assert np.array_equal(o != u, ref != u)
    assert (ref != u).sum() > 0
    ho = np.empty(n ** 3)
    G.near_boundary(u, ub, inside, m1, m2, ho)
    assert np.array_equal(ho, o)
    G.close()
