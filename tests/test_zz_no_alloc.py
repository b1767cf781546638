"""The allocation-free Helmholtz entry point, for callers that cannot
allocate device memory (code inside a host callback or a plugin whose host
application owns every device allocation), against the float64 oracle and
the allocating ibdl_helmholtz.

Collected last on purpose: it shares nothing with the other tests, and a
failure here leaves every other test already run.  The calls run in a row
with different inputs and sizes, small to large and back (64, 256, 64,
512), so the shared static scratch must carry no state from one call into
the next, whichever call came before.  After a warm-up call, further calls
must leave the device's free memory unchanged: that is the entry point's
promise.
"""
import numpy as np
import pytest
from parity_util import assert_parity

torch = pytest.importorskip("torch")

from oracle import ibdl_oracle as O  # noqa: E402
from workloads import geometry  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = ((64, 2.0, 5e-2), (256, 1.0, 1e-3), (64, 1.0, 1e-1), (512, 1.0, 1e-3))


def test_noalloc_matches_oracle_and_allocating_solve_on_calls_in_a_row():
    import paper_2203_12126_gb300 as pkg
    from paper_2203_12126_gb300 import ibdl
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(21)
    for n, box, kappa in CASES:
        fh = rng.standard_normal((n, n))
        f = torch.tensor(fh, device=dev)
        out = torch.full_like(f, np.nan)
        ibdl.helmholtz_2d_noalloc(n, box, kappa, f, out)
        torch.cuda.synchronize()
        # the oracle: v = kappa L'^{-1} f on the same periodic box (5-point stencil)
        ref = kappa * O.helmholtz_solve(O.Box(2, n, box, (0.0, 0.0)), kappa, fh)
        assert_parity(out.cpu().numpy(), ref, 1e-12, f"noalloc vs oracle n={n}")
        # and the allocating entry point on a geometry of the same grid
        g = geometry.circle(n, 0.3 * box, center=(0.5 * box, 0.5 * box), box_len=box,
                            kappa=kappa)
        G = pkg.Geometry.from_workload(g)
        alloc = torch.empty_like(f)
        G.helmholtz(f, alloc)
        torch.cuda.synchronize()
        assert_parity(out.cpu().numpy(), alloc.cpu().numpy(), 1e-12, f"noalloc vs alloc n={n}")
        G.close()


def test_noalloc_call_leaves_device_memory_unchanged():
    from paper_2203_12126_gb300 import ibdl
    dev = torch.device("cuda:0")
    n = 512
    f = torch.tensor(np.random.default_rng(22).standard_normal((n, n)), device=dev)
    out = torch.empty_like(f)
    # warm-up: the first call on a device may load the library's module
    # (which places the static scratch) and size the kernels' local memory
    ibdl.helmholtz_2d_noalloc(n, 1.0, 1e-3, f, out)
    ibdl.helmholtz_2d_noalloc(64, 1.0, 1e-3, f, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for nn in (64, 512, 128):
        ibdl.helmholtz_2d_noalloc(nn, 1.0, 1e-3, f, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2203_12126_gb300 import ibdl
    f = torch.zeros((1024, 1024), dtype=torch.float64, device="cuda:0")
    with pytest.raises(ibdl.IbdlError) as e:
        ibdl.helmholtz_2d_noalloc(1024, 1.0, 1e-3, f, f)
    assert e.value.status == ibdl.ERR_INVALID_ARG and "512" in str(e.value)
    with pytest.raises(ibdl.IbdlError):
        ibdl.helmholtz_2d_noalloc(256, 1.0, 1e-3, np.zeros(256 * 256), np.zeros(256 * 256))
