"""Seeded synthetic boundary geometries for IBDL solves.

Each generator returns a :class:`Geometry`: the periodic box and grid, the
immersed-boundary points X_i, their unit normals n_i (pointing out of the PDE
domain Omega, as the double-layer spread requires, Sec. 4.1) and the quadrature
weights Delta s_i (arclength, Sec. 5.2) or dA_i (area, Sec. 6.7).

This module holds none of the method's arithmetic (no delta function, spread,
interpolation or Helmholtz solve): it only places points.  Both the CUDA
path's tests and the CPU oracle draw their inputs from here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN_ANGLE = math.pi * (3.0 - math.sqrt(5.0))


@dataclass
class Geometry:
    """A boundary discretisation inside a periodic box.

    Grid nodes sit at ``origin + j*h`` for j = 0..n-1 on every axis
    (node-centred, the reading used for Sec. 5.1), with ``h = box_len / n``.
    Arrays are float64: ``X`` and ``normals`` are (M, dim) with columns
    (x, y[, z]); ``weights`` is (M,).
    """

    dim: int
    n: int
    box_len: float
    origin: tuple
    X: np.ndarray
    normals: np.ndarray
    weights: np.ndarray
    kappa: float
    delta: str = "peskin4"
    # Curve parameter per point (polar angle theta in 2D; polar angle about
    # the centre in 3D) and the shape's centre, for boundary data.
    param: np.ndarray | None = None
    center: tuple = (0.5, 0.5)
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def h(self) -> float:
        return self.box_len / self.n

    @property
    def m(self) -> int:
        return int(self.X.shape[0])

    @property
    def k(self) -> float:
        """Helmholtz wavenumber of Delta u - k^2 u = 0, with k^2 = 1/kappa."""
        return 1.0 / math.sqrt(self.kappa)


# ---------------------------------------------------------------------------
# 2D curves
# ---------------------------------------------------------------------------

def circle_points(center, r, m):
    """M equispaced points on a circle, theta_i = 2 pi i / M, CCW."""
    th = 2.0 * np.pi * np.arange(m) / m
    c, s = np.cos(th), np.sin(th)
    X = np.stack([center[0] + r * c, center[1] + r * s], axis=1)
    nrm = np.stack([c, s], axis=1)
    w = np.full(m, 2.0 * np.pi * r / m)
    return X, nrm, w, th


class StarCurve:
    """r(theta) = r0 (1 + amp cos(lobes*theta)) about ``center``, CCW."""

    def __init__(self, center, r0, amp, lobes, n_modes=4096):
        self.center = center
        self.r0, self.amp, self.lobes = float(r0), float(amp), int(lobes)
        # Fourier coefficients of the speed |X'(theta)| on a fine periodic
        # grid; the speed is analytic, so the trapezoid rule is spectrally
        # accurate and the arclength integrates term by term.
        t = 2.0 * np.pi * np.arange(n_modes) / n_modes
        c = np.fft.fft(self.speed(t)) / n_modes
        # modes below 1e-15 |c_0| are FFT rounding noise: the real harmonics
        # of the speed decay geometrically well before that
        keep = max(8, int(np.max(np.nonzero(np.abs(c[: n_modes // 2]) > 1e-15 * abs(c[0]))[0])) + 1)
        self._c0 = c[0].real
        mm = np.arange(1, keep)
        # the speed depends on theta only through lobes*theta, so only the
        # harmonics that are multiples of `lobes` are non-zero; the others
        # hold FFT rounding noise and are dropped
        if self.lobes > 1 and self.amp != 0.0:
            mm = mm[mm % self.lobes == 0]
        self._cm = c[mm]
        self._mm = mm

    def radius(self, t):
        return self.r0 * (1.0 + self.amp * np.cos(self.lobes * t))

    def dradius(self, t):
        return -self.r0 * self.amp * self.lobes * np.sin(self.lobes * t)

    def speed(self, t):
        return np.hypot(self.radius(t), self.dradius(t))

    @property
    def perimeter(self) -> float:
        return 2.0 * np.pi * self._c0

    def arclength(self, t):
        """s(theta) = integral_0^theta |X'|, from the Fourier series."""
        t = np.asarray(t, dtype=np.float64)
        e = np.exp(1j * np.outer(t, self._mm)) - 1.0
        # the real speed has c_{-m} = conj(c_m): the sum is 2 Re(...)
        s = self._c0 * t + 2.0 * np.real(e @ (self._cm / (1j * self._mm)))
        return s

    def points(self, m):
        """M points equispaced in arclength, starting at theta = 0."""
        P = self.perimeter
        target = P * np.arange(m) / m
        t = 2.0 * np.pi * np.arange(m) / m
        for _ in range(60):
            dt = (self.arclength(t) - target) / self.speed(t)
            t = t - dt
            # Newton converges quadratically; below 1e-13 the next step only
            # moves t by rounding noise
            if np.max(np.abs(dt)) < 1e-13:
                break
        r, dr = self.radius(t), self.dradius(t)
        c, s = np.cos(t), np.sin(t)
        X = np.stack([self.center[0] + r * c, self.center[1] + r * s], axis=1)
        tx, ty = dr * c - r * s, dr * s + r * c       # tangent X'(theta), CCW
        sp = np.hypot(tx, ty)
        nrm = np.stack([ty / sp, -tx / sp], axis=1)   # outward for a CCW curve
        w = np.full(m, P / m)
        return X, nrm, w, t


def circle(n, r, m=None, spacing=1.0, center=(0.5, 0.5), box_len=1.0,
           origin=(0.0, 0.0), kappa=1e-2, delta="peskin4", name="circle"):
    """Circle with M = ceil(2 pi r / (spacing*h)) points unless M is given."""
    h = box_len / n
    if m is None:
        m = int(math.ceil(2.0 * math.pi * r / (spacing * h)))
    X, nrm, w, th = circle_points(center, r, m)
    return Geometry(2, n, box_len, tuple(origin), X, nrm, w, kappa, delta,
                    th, tuple(center), name, {"r": r})


def star(n, r0, amp, lobes, spacing=1.0 / 1.5, m=None, center=(0.5, 0.5),
         box_len=1.0, origin=(0.0, 0.0), kappa=1e-3, delta="peskin4",
         name="star"):
    """Star curve with M = ceil(P / (spacing*h)) arclength-equispaced points."""
    h = box_len / n
    sc = StarCurve(center, r0, amp, lobes)
    if m is None:
        m = int(math.ceil(sc.perimeter / (spacing * h)))
    X, nrm, w, th = sc.points(m)
    return Geometry(2, n, box_len, tuple(origin), X, nrm, w, kappa, delta,
                    th, tuple(center), name,
                    {"r0": r0, "amp": amp, "lobes": lobes,
                     "perimeter": sc.perimeter})


# ---------------------------------------------------------------------------
# 3D surfaces
# ---------------------------------------------------------------------------

def sphere_count(r, h, spacing=1.5):
    """Points for a mean triangulation edge of spacing*h on a sphere:
    M = ceil(4 pi r^2 / ((sqrt(3)/2) (spacing h)^2))."""
    return int(math.ceil(4.0 * math.pi * r * r /
                         ((math.sqrt(3.0) / 2.0) * (spacing * h) ** 2)))


def fibonacci_unit(m):
    """Fibonacci lattice on the unit sphere: z_i = 1-(2i+1)/M, golden-angle
    longitudes."""
    i = np.arange(m, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / m
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    lon = GOLDEN_ANGLE * i
    return np.stack([rho * np.cos(lon), rho * np.sin(lon), z], axis=1)


def sphere(n, r, m=None, spacing=1.5, center=(0.5, 0.5, 0.5), box_len=1.0,
           origin=(0.0, 0.0, 0.0), kappa=1e-3, delta="peskin4", name="sphere"):
    h = box_len / n
    if m is None:
        m = sphere_count(r, h, spacing)
    u = fibonacci_unit(m)
    X = np.asarray(center)[None, :] + r * u
    w = np.full(m, 4.0 * math.pi * r * r / m)
    polar = np.arccos(np.clip(u[:, 2], -1.0, 1.0))
    return Geometry(3, n, box_len, tuple(origin), X, u.copy(), w, kappa, delta,
                    polar, tuple(center), name, {"r": r})


def ellipsoid(n, axes, m=None, spacing=1.5, center=(0.5, 0.5, 0.5),
              box_len=1.0, origin=(0.0, 0.0, 0.0), kappa=1e-3,
              delta="peskin4", name="ellipsoid"):
    """The sphere lattice mapped by diag(a, b, c); weights are the mapped
    area elements (4 pi / M) * abc * |D^{-1} u|, normals ~ D^{-1} u."""
    a, b, c = (float(v) for v in axes)
    h = box_len / n
    if m is None:
        # area of the ellipsoid by Thomsen's formula (input sizing only)
        p = 1.6075
        area = 4 * math.pi * (((a * b) ** p + (a * c) ** p + (b * c) ** p) / 3) ** (1 / p)
        m = int(math.ceil(area / ((math.sqrt(3.0) / 2.0) * (spacing * h) ** 2)))
    u = fibonacci_unit(m)
    D = np.array([a, b, c])
    X = np.asarray(center)[None, :] + u * D[None, :]
    g = u / D[None, :]
    gn = np.linalg.norm(g, axis=1)
    nrm = g / gn[:, None]
    w = (4.0 * math.pi / m) * a * b * c * gn
    polar = np.arccos(np.clip(u[:, 2], -1.0, 1.0))
    return Geometry(3, n, box_len, tuple(origin), X, nrm, w, kappa, delta,
                    polar, tuple(center), name, {"axes": (a, b, c)})


def exterior(geom):
    """The same points for the exterior domain: normals negated (they point
    out of Omega, i.e. into the curve)."""
    import dataclasses
    return dataclasses.replace(geom, normals=-geom.normals, name=geom.name + "-exterior",
                               extra=dict(geom.extra, exterior=True))
