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


# ---- the radix-16 first pass split over two threads (fft_pass16_split) ----

# exponent of w16 for register (q2l, r) of half h: the table in the kernel
SPLIT_TW = {(0, 0): (0, 4), (0, 1): (0, 6), (0, 2): (0, 0), (0, 3): (0, 2),
            (1, 0): (0, 6), (1, 1): (1, 9), (1, 2): (2, 0), (1, 3): (3, 3)}


def dft4(v, sign):
    w = np.exp(sign * 2j * np.pi * np.outer(np.arange(4), np.arange(4)) / 4)
    return v @ w


def split_radix16(x, inverse):
    """Both halves of one split butterfly, step by step as the kernel takes
    them: returns the 16 outputs each half stores, by output index."""
    sign = 1.0 if inverse else -1.0
    w16 = lambda e: np.exp(sign * 2j * np.pi * e / 16)
    regs = {}
    for h in (0, 1):
        reg = np.zeros((2, 4), complex)
        for q2l in range(2):
            v = np.array([x[2 * h + q2l + 4 * q1] for q1 in range(4)])
            if h:
                v[1::2] = -v[1::2]          # rotates the DFT-4 outputs by two
            reg[q2l] = dft4(v, sign)
            for r in range(4):
                reg[q2l, r] *= w16(SPLIT_TW[(q2l, r)][h])
        regs[h] = reg
    out = {}
    for h in (0, 1):
        own, other = regs[h], regs[1 - h]
        for r in range(2):
            y = dft4(np.array([own[0, r], own[1, r], other[0, r + 2], other[1, r + 2]]), sign)
            if h:
                y[1::2] = -y[1::2]
            for p2 in range(4):
                p = 2 * h + r + 4 * p2
                assert p not in out
                out[p] = y[p2]
    return np.array([out[p] for p in range(16)])


@pytest.mark.parametrize("inverse", [False, True])
def test_split_radix16_butterfly_is_the_16_point_dft(inverse):
    rng = np.random.default_rng(16 + inverse)
    for _ in range(4):
        x = rng.standard_normal(16) + 1j * rng.standard_normal(16)
        ref = 16 * np.fft.ifft(x) if inverse else np.fft.fft(x)
        assert np.allclose(split_radix16(x, inverse), ref, rtol=0, atol=1e-12)


def test_split_twiddle_table_is_p1_times_q2():
    # register (q2l, r) of half h holds p1 = (r + 2h) mod 4 of q2 = 2h + q2l
    for (q2l, r), (e0, e1) in SPLIT_TW.items():
        for h, e in ((0, e0), (1, e1)):
            assert e % 16 == (((r + 2 * h) % 4) * (2 * h + q2l)) % 16


@pytest.mark.parametrize("lg", [5, 6, 8, 10, 11])
@pytest.mark.parametrize("npen", [1, 2, 4, 16])
@pytest.mark.parametrize("strided", [False, True])
def test_split_first_pass_threads_cover_each_butterfly_half_once(lg, npen, strided):
    """Thread e < 2 total takes half h = (e >> 4) & 1 of butterfly
    b = ((e >> 5) << 4) | (e & 15); lanes l and l ^ 16 hold the two halves
    of one butterfly, and every (pencil, j, h) is taken once."""
    nb = 1 << (lg - 4)
    total = npen * nb
    if total % 16:
        pytest.skip("the kernel keeps the plain pass unless total % 16 == 0")
    lgc = npen.bit_length() - 1
    seen = set()
    for e in range(2 * total):
        h = (e >> 4) & 1
        b = ((e >> 5) << 4) | (e & 15)
        assert b < total
        pen, j = ((b & (npen - 1), b >> lgc) if strided else (b >> (lg - 4), b & (nb - 1)))
        assert (pen, j, h) not in seen
        seen.add((pen, j, h))
        partner = e ^ 16
        assert partner < 2 * total and partner >> 5 == e >> 5
        assert ((partner >> 5) << 4) | (partner & 15) == b and (partner >> 4) & 1 != h
    assert len(seen) == 2 * total
