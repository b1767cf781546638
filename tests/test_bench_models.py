"""The benchmark's measurement arithmetic, on the CPU: the matvec byte model
behind the roofline fractions, the per-launch field-solve count of the
headline pair, and the work-item trace summary (phase spans, hand-offs,
start gaps, busy share) -- each against values worked out by hand."""
import numpy as np
import pytest

import bench


def test_matvec_byte_model_by_hand():
    # B = 9 p N^d + p M (4^d + 2d + 4): the grid term is 9 passes of N^d
    # values of p bytes, the point term the taps and point I/O
    assert bench.model_matvec_bytes(2, 1024, 3525, 4) == 9 * 4 * 1024 ** 2 + 4 * 3525 * 24
    assert bench.model_matvec_bytes(3, 256, 38039, 4) == 9 * 4 * 256 ** 3 + 4 * 38039 * 74
    # C2 float32: 37.75 MB of grid passes plus 0.34 MB of point traffic
    assert abs(bench.model_matvec_bytes(2, 1024, 3525, 4) / 1e6 - 38.087) < 1e-3
    # C3 float32: 604 MB of grid passes dominate
    assert abs(bench.model_matvec_bytes(3, 256, 38039, 4) / 1e6 - 615.24) < 1e-2
    # float64 doubles every term
    assert bench.model_matvec_bytes(2, 128, 242, 8) == 2 * bench.model_matvec_bytes(2, 128, 242, 4)


def _info(iters, matvecs, updates):
    return {"iters": iters, "matvecs": matvecs, "residual_updates": updates}


def test_pair_launch_field_solves_refined():
    # the benchmark's step: a Dirichlet and a Neumann refined solve, 7 inner
    # iterations each, one float64-grade residual and one float32 update
    # each (matvecs = 7 + 2); the Neumann right-hand side is float32
    infos = [_info(7, 9, 1), _info(7, 9, 1)]
    mv64, mv32, B = bench.launch_field_solves(infos, 2, True, [False, True], 1024, 3525)
    assert mv64 == 2 and mv32 == 14 + 2 + 1
    expect = 2 * bench.model_matvec_bytes(2, 1024, 3525, 8) + \
        17 * bench.model_matvec_bytes(2, 1024, 3525, 4)
    assert B == pytest.approx(expect)
    assert B / 1e6 == pytest.approx(799.83, abs=0.01)


def test_pair_launch_field_solves_float64_and_old_counts():
    # plain float64: every matvec and the Neumann right-hand side at p = 8
    infos = [_info(6, 7, 0), _info(6, 7, 0)]
    mv64, mv32, _ = bench.launch_field_solves(infos, 2, False, [False, True], 1024, 3525)
    assert (mv64, mv32) == (15, 0)
    # solve infos without the update count read as no updates
    infos = [{"iters": 7, "matvecs": 9}, {"iters": 7, "matvecs": 9}]
    mv64, mv32, _ = bench.launch_field_solves(infos, 2, True, [False, True], 1024, 3525)
    assert (mv64, mv32) == (4, 15)


def _rec(t0, t1, blk, inst, phase, prec, item):
    meta = (blk << 40) | (inst << 24) | (phase << 20) | (prec << 18) | item
    return [t0, t1, meta]


def test_trace_summary_by_hand():
    # one instance on two blocks: phase x_fwd (0) with two items, a hand-off
    # (phase 15), then phase E (6) with one item; times in ns
    rec = np.array([
        _rec(1000, 4000, 0, 0, 0, 1, 0),      # x_fwd item 0, 3 us
        _rec(1500, 5000, 1, 0, 0, 1, 1),      # x_fwd item 1, 3.5 us
        _rec(5000, 7000, 1, 0, 15, 1, 6),     # hand-off: 2 us, published at 7000
        _rec(7500, 9500, 1, 0, 6, 1, 0),      # E item, starts 0.5 us later
    ], dtype=np.uint64)
    out = bench.trace_summary(rec)
    assert out["span_us"] == pytest.approx(8.5)          # 1000 .. 9500
    assert out["blocks"] == 2
    busy = (3000 + 3500 + 2000) / (8500 * 2)               # hand-offs are not items
    assert out["busy_share"] == pytest.approx(busy)
    inst = out["instances"][0]
    assert inst["phases"] == 2
    assert inst["handoff_us_median"] == pytest.approx(2.0)
    assert inst["start_gap_us_median"] == pytest.approx(0.5)
    kinds = inst["by_kind"]
    assert kinds["x_fwd_f32"]["span_us_median"] == pytest.approx(4.0)    # 1000 .. 5000
    assert kinds["x_fwd_f32"]["item_us_median"] == pytest.approx(3.25)
    assert kinds["E_f32"]["span_us_median"] == pytest.approx(2.0)
