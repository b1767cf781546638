"""The continuous-batching server (ibdl_server_*): requests that arrive
while others are being solved are admitted as slots and memory free up, and
every result equals the same problem solved alone (and the float64 oracle)
within the float32-refined path's tolerance."""
import numpy as np
import pytest
from parity_util import assert_parity

torch = pytest.importorskip("torch")

from oracle import ibdl_oracle as O  # noqa: E402
from workloads import configs, data, geometry  # noqa: E402

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2203_12126_gb300 as pkg
    from paper_2203_12126_gb300 import ibdl
    DEV = torch.device("cuda:0")

TOL = 1e-10          # solver tolerance of every request
STATED = 1e-8        # float32-refined result vs float64: relative error bound


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def stream():
    """Mixed problems: dim, n, m, kappa and bc all differ."""
    rng = np.random.default_rng(51)
    geoms = [
        (geometry.star(128, 0.3, 0.2, 5, kappa=1e-2), configs.DIRICHLET),
        (geometry.star(256, 0.25, 0.15, 3, kappa=1e-3), configs.NEUMANN),
        (geometry.sphere(32, 0.3, kappa=3e-2), configs.DIRICHLET),
        (geometry.ellipsoid(32, (0.3, 0.22, 0.26), kappa=1e-2), configs.NEUMANN),
        (geometry.circle(64, 0.3, kappa=5e-2), configs.NEUMANN),
        (geometry.star(512, 0.2, 0.25, 7, kappa=2e-4), configs.DIRICHLET),
    ]
    out = []
    for g, bc in geoms:
        p = configs.exp_problem(g, bc, data.random_direction(rng, g.dim))
        out.append(p)
    return out


def drain(srv, results, limit=10000):
    for _ in range(limit):
        st = srv.stats()
        if st["queued"] == 0 and st["active"] == 0 and st["finished"] == 0:
            return
        for rid in srv.step():
            results[rid] = srv.take(rid, results.pop(rid))
    raise AssertionError("server did not drain")


def test_mixed_stream_matches_alone_and_oracle():
    probs = stream()
    srv = pkg.Server(max_active=4, rounds_per_step=2, reserve_sms=8, tol=TOL)
    ids, results = {}, {}
    # three requests first; the rest arrive while those are being solved
    for k, p in enumerate(probs[:3]):
        ids[k] = srv.submit(p.geom, p.bdata, bc=p.bc)
        results[ids[k]] = p.geom.m
    for rid in srv.step():
        results[rid] = srv.take(rid, results.pop(rid))
    assert srv.stats()["active"] >= 1
    for k, p in enumerate(probs[3:], start=3):
        ids[k] = srv.submit(p.geom, p.bdata, bc=p.bc)
        results[ids[k]] = p.geom.m
    drain(srv, results)
    st = srv.stats()
    assert st["launches"] >= 3 and st["bytes_in_use"] == 0
    for k, p in enumerate(probs):
        q_mix, rec = results[ids[k]]
        assert rec["status"] == ibdl.OK, rec
        assert rec["rel_residual"] <= TOL, rec
        assert rec["t_arrival"] <= rec["t_admit"] <= rec["t_done"]
        # the same problem alone through ibdl_solve
        G = pkg.Geometry.from_workload(p.geom, bc=p.bc, precision=ibdl.FP32_REFINED)
        q = torch.empty(p.geom.m, dtype=torch.float64, device=DEV)
        G.solve(torch.tensor(p.bdata, device=DEV), q, tol=TOL)
        q_alone = q.cpu().numpy()
        G.close()
        ref = O.solve(p.geom, p.bc, p.bdata, tol=1e-13).x
        assert_parity(q_mix, q_alone, STATED, str((k, rel(q_mix, q_alone))))
        assert_parity(q_mix, ref, STATED, str((k, rel(q_mix, ref))))
        assert_parity(q_alone, ref, STATED, str((k, rel(q_alone, ref))))
    srv.close()


def test_admission_respects_the_memory_budget():
    probs = [configs.exp_problem(geometry.star(256, 0.2 + 0.02 * i, 0.1, 4, kappa=1e-3),
                                 configs.DIRICHLET, np.array([1.0, 0.0])) for i in range(5)]
    # measure one request's footprint, then allow about two at a time
    probe = pkg.Server(max_active=8, tol=1e-8)
    rid = probe.submit(probs[0].geom, probs[0].bdata)
    res = {rid: probs[0].geom.m}
    drain(probe, res)
    one = res[rid][1]["device_bytes"]
    probe.close()
    budget = int(2.6 * one)
    srv = pkg.Server(memory_budget=budget, max_active=8, rounds_per_step=2, tol=1e-8)
    results = {}
    for p in probs:
        results[srv.submit(p.geom, p.bdata)] = p.geom.m
    first = srv.stats()
    srv.step()
    assert srv.stats()["active"] <= 2 < first["queued"]
    drain(srv, results)
    st = srv.stats()
    assert 0 < st["peak_bytes"] <= budget
    for q, rec in results.values():
        assert rec["status"] == ibdl.OK and rec["rel_residual"] <= 1e-8
    srv.close()


def test_request_larger_than_the_budget_fails_alone():
    small = configs.exp_problem(geometry.circle(64, 0.3, kappa=1e-2), configs.DIRICHLET,
                                np.array([0.0, 1.0]))
    big = configs.exp_problem(geometry.star(1024, 0.3, 0.2, 5, kappa=1e-3),
                              configs.DIRICHLET, np.array([0.0, 1.0]))
    srv = pkg.Server(memory_budget=8 << 20, max_active=4, tol=1e-8)
    r_big = srv.submit(big.geom, big.bdata)
    r_small = srv.submit(small.geom, small.bdata)
    results = {r_big: big.geom.m, r_small: small.geom.m}
    drain(srv, results)
    assert results[r_big][1]["status"] == ibdl.ERR_OOM
    assert results[r_small][1]["status"] == ibdl.OK
    with pytest.raises(ibdl.IbdlError):
        srv.take(r_big, big.geom.m)
    srv.close()
