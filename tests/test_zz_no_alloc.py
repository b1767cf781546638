"""The allocation-free Helmholtz entry point (for callers that cannot
allocate device memory) against the allocating ibdl_helmholtz.

Collected last on purpose: it shares nothing with the other tests, and a
failure here leaves every other test already run.  Two calls in a row with
different inputs and sizes check that the shared static scratch carries no
state from one call into the next.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import geometry  # noqa: E402

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_allocating_solve_on_two_calls_in_a_row():
    import paper_2203_12126_gb300 as pkg
    from paper_2203_12126_gb300 import ibdl
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(21)
    for n, box, kappa in ((256, 1.0, 1e-3), (64, 2.0, 5e-2)):
        g = geometry.circle(n, 0.3 * box, center=(0.5 * box, 0.5 * box), box_len=box,
                            kappa=kappa)
        G = pkg.Geometry.from_workload(g)
        f = torch.tensor(rng.standard_normal((n, n)), device=dev)
        ref = torch.empty_like(f)
        G.helmholtz(f, ref)
        out = torch.full_like(f, np.nan)
        ibdl.helmholtz_2d_noalloc(n, box, kappa, f, out)
        torch.cuda.synchronize()
        # same kernels and tables up to the last bit of the twiddles:
        # float64 parity tolerance of the component tests
        assert rel(out.cpu().numpy(), ref.cpu().numpy()) <= 1e-12
        G.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2203_12126_gb300 import ibdl
    f = torch.zeros((1024, 1024), dtype=torch.float64, device="cuda:0")
    with pytest.raises(ibdl.IbdlError) as e:
        ibdl.helmholtz_2d_noalloc(1024, 1.0, 1e-3, f, f)
    assert e.value.status == ibdl.ERR_INVALID_ARG and "512" in str(e.value)
    with pytest.raises(ibdl.IbdlError):
        ibdl.helmholtz_2d_noalloc(256, 1.0, 1e-3, np.zeros(256 * 256), np.zeros(256 * 256))
