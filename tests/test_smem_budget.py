"""Shared-memory bookkeeping of the persistent solver, on the CPU (the query
runs the library's host code; no GPU is touched).

For every supported grid size, dimension, x-pass tiling and element type,
every work item's dynamic shared memory (the row tiles of the x passes, the
pencil items of each layout) must fit in what a solver launch over that
geometry reserves, each element type sized from its own FFT plan and
layout; the twiddle table must have the plan's length (a first pass of
radix 16, then passes of radix <= 16 as even as possible), and sizes outside
the supported range must be refused rather than sized as another size.
"""
import os

import pytest

import paper_2203_12126_gb300 as pkg
from paper_2203_12126_gb300 import ibdl


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(ibdl.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return pkg.load()


def plan_radices(lg, variant=0):
    """Radix of each pass: 16 first (n itself below 16), then the remaining
    bits split as evenly as possible, larger radices first (variant 0), or
    radix-16 passes first and the remainder last (variant 1)."""
    if lg <= 4:
        return [1 << lg]
    rest = lg - 4
    npass = (rest + 3) // 4
    out = [16]
    if variant == 1:
        return out + [16] * (npass - 1) + [1 << (rest - 4 * (npass - 1))]
    for s in range(npass):
        out.append(1 << (rest // npass + (1 if s < rest % npass else 0)))
    return out


def twiddle_count(lg, variant=0):
    ns, tot = 1, 0
    for r in plan_radices(lg, variant):
        tot += ns * r
        ns *= r
    return tot


def table_capacity(lg, elem):
    """Entries a twiddle buffer holds: float32 tables (elem 1) may be of
    either plan variant where two exist (lg 9, 10), so they are sized for
    the larger."""
    if elem == 1 and lg in (9, 10):
        return max(twiddle_count(lg, 0), twiddle_count(lg, 1))
    return twiddle_count(lg)


def tilings(dim, n):
    """The fixed rule and every tiling the autotuner may pick (a float64 row
    tile within 100 KB)."""
    lg = n.bit_length() - 1
    rule = 8 if dim == 3 else (2 if n >= 2048 else 4)
    out = {rule}
    r = 2
    while r <= 32:
        tile64 = (2 * (r // 2) * (n + n // 16 + 1) + twiddle_count(lg)) * 16
        if n // r >= 4 and r <= n - 5 and tile64 <= 100 * 1024:
            out.add(r)
        r *= 2
    return sorted(x for x in out if x <= n)


CASES = [(2, 1 << lg) for lg in range(4, 12)] + [(3, 1 << lg) for lg in range(4, 10)]


@pytest.mark.parametrize("dim,n", CASES)
def test_every_item_fits_the_launch(lib, dim, n):
    lg = n.bit_length() - 1
    for rows in tilings(dim, n):
        budgets = set()
        for elem in (0, 1, 2):
            q = ibdl.solver_smem_query(dim, n, rows, elem)
            budgets.add(q["budget"])
            assert q["twiddles"] == twiddle_count(lg)
            assert q["need"][0] > 0 and q["need"][1] > 0
            assert (q["need"][2] > 0) == (dim == 3)
            for k, need in enumerate(q["need"]):
                assert need <= q["budget"], (dim, n, rows, elem, k, need, q["budget"])
            # a row tile holds two pencil buffers of rows/2 packed rows and the
            # twiddle table, in the element type's complex size
            csize = 8 if elem == 1 else 16
            pen_stride = n + n // 16 + 1
            assert q["need"][0] == (2 * (rows // 2) * pen_stride
                                    + table_capacity(lg, elem)) * csize
        assert len(budgets) == 1      # one reservation per geometry
        # the reservation fits an SM's shared memory (227 KB per block)
        assert budgets.pop() <= 227 * 1024


def test_plan_twiddle_counts_by_hand():
    # 1024 = 16 * 8 * 8: 16 + 16*8 + 128*8 entries; 256 = 16 * 16
    assert plan_radices(10) == [16, 8, 8] and twiddle_count(10) == 16 + 128 + 1024
    assert plan_radices(8) == [16, 16] and twiddle_count(8) == 16 + 256
    assert plan_radices(12) == [16, 16, 16] and twiddle_count(12) == 16 + 256 + 4096
    # the radix-16-first variant: 1024 = 16 * 16 * 4, 512 = 16 * 16 * 2
    assert plan_radices(10, 1) == [16, 16, 4] and twiddle_count(10, 1) == 16 + 256 + 1024
    assert plan_radices(9, 1) == [16, 16, 2] and twiddle_count(9, 1) == 16 + 256 + 512
    # elsewhere the two variants coincide (only lg 9 and 10 offer variant 1)
    for lg in (4, 5, 6, 7, 8, 11, 12):
        assert plan_radices(lg, 1) == plan_radices(lg)


@pytest.mark.parametrize("n,plan", [(1024, 1), (512, 1), (1024, 0), (2048, 0)])
def test_plan_pins_are_checked_on_the_host(lib, n, plan):
    # a float32-refined 2D kind accepts any plan offered for its size (the
    # pin touches no GPU memory; without a device it reports the CUDA error)
    try:
        ibdl.tuning_set_plan(2, n, ibdl.FP32_REFINED, plan)
        ibdl.tuning_set_plan(2, n, ibdl.FP32_REFINED, -1)
    except ibdl.IbdlError as e:
        assert e.status == ibdl.ERR_CUDA


@pytest.mark.parametrize("dim,n,prec,plan", [(2, 256, 1, 1), (2, 2048, 1, 1), (3, 512, 1, 1),
                                             (2, 1024, 0, 1), (2, 1024, 1, 2), (2, 1000, 1, 0)])
def test_plan_pins_outside_the_offered_set_are_refused(lib, dim, n, prec, plan):
    with pytest.raises(ibdl.IbdlError) as e:
        ibdl.tuning_set_plan(dim, n, prec, plan)
    assert e.value.status == ibdl.ERR_INVALID_ARG


@pytest.mark.parametrize("dim,n,rows,elem", [(2, 8, 4, 0), (2, 4096, 2, 0), (3, 1024, 8, 0),
                                             (2, 1000, 4, 0), (2, 1024, 3, 0),
                                             (2, 1024, 4, 3), (4, 64, 4, 0)])
def test_unsupported_sizes_are_refused(lib, dim, n, rows, elem):
    with pytest.raises(ibdl.IbdlError) as e:
        ibdl.solver_smem_query(dim, n, rows, elem)
    assert e.value.status == ibdl.ERR_INVALID_ARG
