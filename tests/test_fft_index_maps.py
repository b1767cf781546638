"""Index arithmetic of the shared-memory FFT passes, mirrored on the CPU.

The pencil transforms run a Stockham FFT whose plan (radices per pass),
butterfly indexing and twiddle exponents are compile-time functions of
lg = log2 n.  This file restates them in numpy and checks:

* the plan covers lg bits with radices <= 16, and the last pass has as many
  butterflies as its stride (NB = NS), so its outputs are j + p NS;
* a forward (inverse) transform built from those index maps equals
  np.fft.fft (n * np.fft.ifft) for n = 16 ... 4096;
* the passes that read or write global memory (the first and last, in the
  contiguous and the strided thread order) touch every element of an item's
  pencils exactly once and nothing outside them, also for a partial item
  (npl < c), and a warp's accesses for one butterfly input are contiguous
  runs;
* the x inverse pass's row writes (two real rows per pencil) cover the
  tile's R rows exactly once.

CPU only.
"""
import numpy as np
import pytest


def plan_npass(lg):
    return 1 if lg <= 4 else 1 + (lg - 1) // 4


def plan_lr(lg, s):
    if s == 0:
        return lg if lg < 4 else 4
    np_ = plan_npass(lg)
    return (lg - 4) // (np_ - 1) + (1 if s - 1 < (lg - 4) % (np_ - 1) else 0)


def plan_lgns(lg, s):
    return 0 if s == 0 else plan_lgns(lg, s - 1) + plan_lr(lg, s - 1)


def pass_shape(lg, s):
    lr, lgns = plan_lr(lg, s), plan_lgns(lg, s)
    return 1 << lr, 1 << (lg - lr), 1 << lgns  # R, NB, NS


LGS = range(4, 13)


@pytest.mark.parametrize("lg", LGS)
def test_plan_covers_the_bits(lg):
    npass = plan_npass(lg)
    lrs = [plan_lr(lg, s) for s in range(npass)]
    assert sum(lrs) == lg and all(1 <= r <= 4 for r in lrs)
    assert lrs[0] == min(lg, 4)
    assert npass <= 3
    R, NB, NS = pass_shape(lg, npass - 1)
    assert NB == NS and R * NS == 1 << lg


def stockham(x, inverse):
    """The pass sequence of the kernels: butterfly j of pass s reads inputs
    j + q NB, multiplies input q by w^(q k) (w = exp(-+2 pi i / (NS R)),
    k = j mod NS), does an R-point DFT and writes output p to o + p NS,
    o = (j - k) R + k."""
    n = x.size
    lg = n.bit_length() - 1
    sign = 1.0 if inverse else -1.0
    for s in range(plan_npass(lg)):
        R, NB, NS = pass_shape(lg, s)
        j = np.arange(NB)
        k = j & (NS - 1)
        q = np.arange(R)
        a = x[j[:, None] + q[None, :] * NB]
        a = a * np.exp(sign * 2j * np.pi * np.outer(k, q) / (NS * R))
        p = np.arange(R)
        dft = np.exp(sign * 2j * np.pi * np.outer(q, p) / R)  # [q, p]
        out = a @ dft
        o = ((j - k) * R) + k
        y = np.empty_like(x)
        y[o[:, None] + p[None, :] * NS] = out
        x = y
    return x


@pytest.mark.parametrize("lg", LGS)
def test_stockham_index_maps_give_the_dft(lg):
    n = 1 << lg
    rng = np.random.default_rng(lg)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.allclose(stockham(x, False), np.fft.fft(x), rtol=0, atol=1e-10 * n)
    assert np.allclose(stockham(x, True), n * np.fft.ifft(x), rtol=0, atol=1e-10 * n)


def global_pass_accesses(lg, s, c, npl, strided, last):
    """(thread e, pencil, element) of every global access of pass s: the
    first pass reads elements j + q NB, the last writes o + p NS."""
    lgc = c.bit_length() - 1
    R, NB, NS = pass_shape(lg, s)
    e = np.arange(c * NB)
    if strided:
        pen, j = e & (c - 1), e >> lgc
    else:
        pen, j = e >> (lg - plan_lr(lg, s)), e & (NB - 1)
    keep = pen < npl
    e, pen, j = e[keep], pen[keep], j[keep]
    r = np.arange(R)
    if last:
        k = j & (NS - 1)
        t = (((j - k) * R) + k)[:, None] + r[None, :] * NS
    else:
        t = j[:, None] + r[None, :] * NB
    return (np.repeat(e, R).reshape(-1, R), np.repeat(pen, R).reshape(-1, R), t)


@pytest.mark.parametrize("lg", LGS)
@pytest.mark.parametrize("c", [1, 2, 4, 16])
@pytest.mark.parametrize("strided", [False, True])
@pytest.mark.parametrize("last", [False, True])
def test_global_passes_touch_each_element_once(lg, c, strided, last):
    if strided and c < 2:
        pytest.skip("strided items hold at least two pencils")
    n = 1 << lg
    s = plan_npass(lg) - 1 if last else 0
    for npl in sorted({c, max(1, c - 1)}):
        e, pen, t = global_pass_accesses(lg, s, c, npl, strided, last)
        # address of element t of pencil pen relative to the item's base
        addr = t * n + pen if strided else pen * n + t
        span = n * n if strided else n * c  # the item's pencils lie in [0, span)
        assert addr.min() >= 0 and addr.max() < span
        count = np.bincount(addr.ravel(), minlength=span)
        want = np.zeros(span, dtype=int)
        if strided:
            want[(np.arange(n)[:, None] * n + np.arange(npl)[None, :]).ravel()] = 1
        else:
            want[: npl * n] = 1
        assert np.array_equal(count, want)


@pytest.mark.parametrize("lg", [7, 8, 10, 12])
@pytest.mark.parametrize("strided", [False, True])
@pytest.mark.parametrize("last", [False, True])
def test_warp_accesses_are_contiguous_runs(lg, strided, last):
    """For one butterfly input (or output) index, the 32 threads of a warp
    touch contiguous runs: whole rows of 16 consecutive pencils (strided,
    c = 16) or min(32, NB) consecutive elements of a pencil (contiguous)."""
    n, c = 1 << lg, 16
    s = plan_npass(lg) - 1 if last else 0
    e, pen, t = global_pass_accesses(lg, s, c, c, strided, last)
    addr = t * n + pen if strided else pen * n + t
    run = 16 if strided else min(32, pass_shape(lg, s)[1])
    for w0 in range(0, e.shape[0], 32):
        for col in range(addr.shape[1]):
            a = np.sort(addr[w0:w0 + 32, col])
            runs = np.split(a, np.nonzero(np.diff(a) != 1)[0] + 1)
            assert all(len(r) == run for r in runs)


@pytest.mark.parametrize("lg", LGS)
@pytest.mark.parametrize("rows", [2, 4, 8, 16, 32])
def test_row_writes_of_the_x_inverse_pass(lg, rows):
    """The last inverse pass writes pencil pen as rows 2 pen (real parts)
    and 2 pen + 1 (imaginary parts): the tile's R rows, each element once."""
    n, npen = 1 << lg, rows // 2
    e, pen, t = global_pass_accesses(lg, plan_npass(lg) - 1, npen, npen, False, True)
    real = (2 * pen) * n + t
    imag = (2 * pen + 1) * n + t
    count = np.bincount(np.concatenate([real.ravel(), imag.ravel()]), minlength=rows * n)
    assert count.size == rows * n and np.all(count == 1)
