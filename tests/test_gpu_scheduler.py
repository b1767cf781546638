"""The persistent solver's work-item choices and its trace.

* Every admissible number of pencils per solve-pass item (set per geometry
  with ibdl_geometry_set_solver_pencils, per element type) gives the same
  batched Dirichlet + Neumann solves as the oracle's GMRES, element-wise,
  for float64 solves (bound 1e-9) and float32-refined ones (1e-8).  The
  rule's choice for a few-instance 2D launch (float32 items of 4 pencils)
  is among them.
* Inadmissible choices are refused and leave the geometry as it was.
* The work-item trace of a batched launch has one record per item and per
  phase hand-off, with start <= end on the GPU timer, blocks below the
  launch's grid, the launch's instances, and the phase kinds the solver
  runs; every hand-off but an instance's last names the next phase.
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


def gpu(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def pair():
    g = geometry.star(256, 0.3, 0.2, 5, spacing=1.0 / 1.5, kappa=1e-3)
    rng = np.random.default_rng(71)
    probs = [(configs.DIRICHLET, rng.standard_normal(g.m)), (configs.NEUMANN, rng.standard_normal(g.m))]
    refs = [O.solve(g, bc, b, tol=1e-13).x for bc, b in probs]
    return g, probs, refs


def solve_pair(g, probs, prec, pencils):
    gs = [pkg.Geometry.from_workload(g, bc=bc, precision=prec) for bc, _ in probs]
    for G in gs:
        G.set_solver_pencils(*pencils)
    bs = [gpu(b) for _, b in probs]
    qs = [torch.zeros(g.m, dtype=torch.float64, device=DEV) for _ in probs]
    batch = ibdl.Batch(2)
    try:
        infos = batch.solve(gs, bs, qs, tol=1e-10)
    finally:
        batch.close()
        for G in gs:
            G.close()
    return infos, [q.cpu().numpy() for q in qs]


@pytest.mark.parametrize("prec,pencils", [
    (0, (0, 0, 0)), (0, (1, 0, 0)), (0, (4, 0, 0)), (0, (8, 0, 0)),
    (1, (0, 0, 0)), (1, (0, 1, 1)), (1, (0, 2, 2)), (1, (0, 4, 0)), (1, (0, 8, 4)),
    (1, (0, 16, 0)),
])
def test_solver_pencils_choices_match_oracle(pair, prec, pencils):
    g, probs, refs = pair
    infos, qs = solve_pair(g, probs, prec, pencils)
    for k in range(2):
        assert infos[k]["status"] == ibdl.OK and infos[k]["rel_residual"] <= 1e-10, infos[k]
        assert_parity(qs[k], refs[k], 1e-8 if prec else 1e-9, f"prec {prec} pencils {pencils}")


def test_solver_pencils_rejects_inadmissible():
    g = geometry.star(256, 0.3, 0.2, 5, kappa=1e-3)
    G = pkg.Geometry.from_workload(g, bc=configs.DIRICHLET, precision=1)
    try:
        for bad in ((3, 0, 0), (0, 32, 0), (0, 0, 6), (-1, 0, 0)):
            with pytest.raises(ibdl.IbdlError) as e:
                G.set_solver_pencils(*bad)
            assert e.value.status == ibdl.ERR_INVALID_ARG
        # the geometry still solves (and as before)
        b = gpu(np.random.default_rng(72).standard_normal(g.m))
        q = torch.zeros(g.m, dtype=torch.float64, device=DEV)
        info = G.solve(b, q, tol=1e-8)
        assert info["rel_residual"] <= 1e-8
    finally:
        G.close()


def test_work_item_trace_records():
    g = geometry.star(256, 0.3, 0.2, 5, kappa=1e-3)
    rng = np.random.default_rng(73)
    gs = [pkg.Geometry.from_workload(g, bc=bc, precision=1)
          for bc in (configs.DIRICHLET, configs.NEUMANN)]
    bs = [gpu(rng.standard_normal(g.m)) for _ in gs]
    qs = [torch.zeros(g.m, dtype=torch.float64, device=DEV) for _ in gs]
    batch = ibdl.Batch(2)
    with pytest.raises(ibdl.IbdlError):
        ibdl.profile_trace(True)  # profiling is off
    try:
        ibdl.profile_enable(True)
        ibdl.profile_trace(True)
        infos = batch.solve(gs, bs, qs, tol=1e-8)
        rec, k = ibdl.profile_trace_read()
        ibdl.profile_trace(False)
        again, k2 = ibdl.profile_trace_read()
    finally:
        ibdl.profile_enable(False)
        batch.close()
        for G in gs:
            G.close()
    assert k == len(rec) > 0 and k2 == 0
    r = rec.astype(np.int64)
    t0, t1, meta = r[:, 0], r[:, 1], r[:, 2]
    blk, inst = meta >> 40, (meta >> 24) & 0xFFFF
    ph, item = (meta >> 20) & 15, meta & 0x3FFFF
    assert (t0 > 0).all() and (t1 >= t0).all()
    assert blk.max() < 2 * 152 * 4 and set(np.unique(inst)) == {0, 1}
    assert set(np.unique(ph)) <= {0, 2, 4, 5, 6, 7, 15}
    for k_ in (0, 1):
        m = inst == k_
        ho = ph[m] == 15
        # every hand-off but the instance's last publishes a phase the solver runs
        nxt = item[m][ho][np.argsort(t0[m][ho])]
        assert nxt[-1] == 15 and set(np.unique(nxt[:-1])) <= {0, 2, 4, 5, 6, 7}
        # matvec phases carry their item indices (x tiles: rows per tile 4 -> 64 tiles)
        items0 = item[m & (ph == 0)]
        assert items0.min() == 0 and items0.max() < 512
    for info in infos:
        assert info["rel_residual"] <= 1e-8
