"""CPU mirror of the interpolation's x-tap loads (k_points.cu, row_taps):
away from the row's end the four taps x0 .. x0 + 3 come from the aligned
vectors that cover them (4 floats or 2 doubles per vector) and a selection by
x0's offset in its vector; near the end (and for a grid that is not 16-byte
aligned) one load per tap with the periodic wrap.  Both must give
row[(x0 + k) mod n] for every x0, including a base index of -1 or n - 1
(reduced mod n first), and the vectors must stay inside the row."""
import numpy as np
import pytest


def taps_float(row, x0, n, vec=True):
    x0 &= n - 1
    a0, sh = x0 & ~3, x0 & 3
    if vec and a0 + 8 <= n:
        u = row[a0:a0 + 4]
        assert a0 % 4 == 0 and a0 + 4 <= n
        if sh == 0:
            return list(u)
        w = row[a0 + 4:a0 + 8]
        assert a0 + 8 <= n
        v = list(u) + list(w)
        return [v[k + 1] if sh == 1 else (v[k + 2] if sh == 2 else v[k + 3]) for k in range(4)]
    return [row[(x0 + k) & (n - 1)] for k in range(4)]


def taps_double(row, x0, n, vec=True):
    x0 &= n - 1
    a0, sh = x0 & ~1, x0 & 1
    if vec and a0 + 6 <= n:
        u, w = row[a0:a0 + 2], row[a0 + 2:a0 + 4]
        if sh == 0:
            return [u[0], u[1], w[0], w[1]]
        z = row[a0 + 4:a0 + 6]
        assert a0 + 6 <= n
        return [u[1], w[0], w[1], z[0]]
    return [row[(x0 + k) & (n - 1)] for k in range(4)]


@pytest.mark.parametrize("n", [16, 32, 64, 256])
@pytest.mark.parametrize("taps", [taps_float, taps_double])
@pytest.mark.parametrize("vec", [True, False])
def test_row_taps_match_the_periodic_taps(n, taps, vec):
    row = np.arange(n) * 10.0 + 1.0
    for x0 in range(-1, n + 1):
        want = [row[(x0 + k) % n] for k in range(4)]
        assert taps(row, x0, n, vec) == want, (n, x0)
