"""The synthetic IBDL workloads, each built from a seed.

* ``c1``: 2D circle r=0.3 at (1/2,1/2), N=128, M=ceil(2 pi r / h)=242,
  cosine 4-point delta, kappa=1e-2, Dirichlet U_b=sin(2 theta) with exact
  interior solution I_2(10 rho) sin(2 theta)/I_2(3); GMRES(30), tol 1e-10.
* ``c2``: 2D star r(theta)=0.3(1+0.2 cos 5 theta), N=1024, M=ceil(1.5 P/h)
  =3525, Peskin 4-point delta, kappa=1e-3, 10-mode seeded Fourier data;
  Dirichlet (seed 0) and Neumann (seed 1).
* ``c3``: 3D sphere r=0.3, N=256, Fibonacci lattice at triangulation edge
  1.5h (M=38038), kappa=1e-3, Neumann data du/dn = k i_1'(kR) cos(vartheta).
* ``c4``: 256 2D star instances (seed 2): N in {128,256,512}, lobes in
  [3,8], amplitude U[0,0.25], r0 U[0.15,0.35], log10 kappa U[-4,-1].
* ``table1``: the circle of Sec. 6.1 (r=0.25, box [-1/2,1/2)^2, k=1,
  U_b = sin 2 theta) at spacing factor c = Delta s / Delta x.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import data, geometry

DIRICHLET, NEUMANN = 0, 1


@dataclass
class Problem:
    geom: geometry.Geometry
    bc: int                 # DIRICHLET or NEUMANN
    bdata: np.ndarray       # U_b (Dirichlet) or V_b (Neumann), float64 (M,)
    tol: float = 1e-10
    restart: int = 30
    name: str = ""
    exact: object = None    # callable(points (K,d)) -> exact u, or None


def c1(n=128):
    g = geometry.circle(n, 0.3, kappa=1e-2, delta="cos4", name="c1-circle")
    ub = np.sin(2.0 * g.param)
    k = g.k
    ex = (lambda P: data.disk_bessel_exact(P[:, 0], P[:, 1], g.center, 0.3, k))
    return Problem(g, DIRICHLET, ub, 1e-10, 30, "c1", ex)


def c2(n=1024, bc=DIRICHLET, seed=None):
    g = geometry.star(n, 0.3, 0.2, 5, spacing=1.0 / 1.5, kappa=1e-3,
                      delta="peskin4", name="c2-star")
    if seed is None:
        seed = 0 if bc == DIRICHLET else 1
    b = data.fourier_data(g.param, seed)
    return Problem(g, bc, b, 1e-8, 30, "c2-" + ("dirichlet" if bc == DIRICHLET else "neumann"))


def c3(n=256, m=None):
    g = geometry.sphere(n, 0.3, m=m, spacing=1.5, kappa=1e-3, name="c3-sphere")
    k = g.k
    vb = data.ball_bessel_neumann(0.3, k, g.param)
    ex = (lambda P: data.ball_bessel_exact(P[:, 0], P[:, 1], P[:, 2], g.center, k))
    return Problem(g, NEUMANN, vb, 1e-8, 30, "c3", ex)


def table1(n, spacing, r=0.25, kappa=1.0, delta="peskin4"):
    """Sec. 6.1 / Table 1: circle r=0.25 centred in [-1/2,1/2)^2, k=1."""
    g = geometry.circle(n, r, spacing=spacing, center=(0.0, 0.0), box_len=1.0,
                        origin=(-0.5, -0.5), kappa=kappa, delta=delta,
                        name="table1-circle")
    ub = np.sin(2.0 * g.param)
    k = g.k
    ex = (lambda P: data.disk_bessel_exact(P[:, 0], P[:, 1], (0.0, 0.0), r, k))
    return Problem(g, DIRICHLET, ub, 1e-8, 30, "table1", ex)


def exp_problem(geom, bc, direction):
    """Closed-form data u = exp(k d.(x-c)) for any geometry."""
    k = geom.k
    c = np.asarray(geom.center)
    if bc == DIRICHLET:
        b = data.exp_exact(geom.X, c, k, direction)
    else:
        b = data.exp_neumann(geom.X, geom.normals, c, k, direction)
    ex = (lambda P: data.exp_exact(P, c, k, direction))
    return Problem(geom, bc, b, 1e-10, 30, "exp", ex)


def c4_instances(count=256, seed=2, sizes=(128, 256, 512)):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        lobes = int(rng.integers(3, 9))
        amp = float(rng.uniform(0.0, 0.25))
        r0 = float(rng.uniform(0.15, 0.35))
        kappa = float(10.0 ** rng.uniform(-4.0, -1.0))
        g = geometry.star(n, r0, amp, lobes, spacing=1.0 / 1.5, kappa=kappa,
                          name=f"c4-{i}")
        b = data.fourier_data(g.param, seed * 100000 + i)
        out.append(Problem(g, DIRICHLET, b, 1e-8, 30, f"c4-{i}"))
    return out


@dataclass
class Request:
    t: float                # arrival offset in seconds
    problem: Problem
    kind: str


def c5_requests(count=300, seed=3, rate=2000.0, sizes2d=(256, 512, 1024),
                sizes3d=(64, 128, 256), frac3d=0.2):
    """The mixed serving stream: Poisson arrivals (mean ``rate`` per second);
    80% 2D stars (N ~ U{sizes2d}, lobes 3-8, amplitude U[0,0.25], r0
    U[0.15,0.35]) and 20% 3D spheres (r ~ U[0.2,0.35]) or ellipsoids (axes ~
    U[0.2,0.35]), 50/50; log10 kappa ~ U[-4,-1]; Dirichlet/Neumann 50/50 with
    the closed-form data u = exp(k d.(x - c)), d a random unit vector."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        kappa = float(10.0 ** rng.uniform(-4.0, -1.0))
        bc = DIRICHLET if rng.uniform() < 0.5 else NEUMANN
        if rng.uniform() < frac3d:
            n = int(rng.choice(sizes3d))
            if rng.uniform() < 0.5:
                r = float(rng.uniform(0.2, 0.35))
                g = geometry.sphere(n, r, kappa=kappa, name=f"c5-{i}-sphere")
                kind = f"3d-sphere-n{n}"
            else:
                axes = tuple(float(a) for a in rng.uniform(0.2, 0.35, size=3))
                g = geometry.ellipsoid(n, axes, kappa=kappa, name=f"c5-{i}-ellipsoid")
                kind = f"3d-ellipsoid-n{n}"
        else:
            n = int(rng.choice(sizes2d))
            lobes = int(rng.integers(3, 9))
            amp = float(rng.uniform(0.0, 0.25))
            r0 = float(rng.uniform(0.15, 0.35))
            g = geometry.star(n, r0, amp, lobes, spacing=1.0 / 1.5, kappa=kappa,
                              name=f"c5-{i}-star")
            kind = f"2d-star-n{n}"
        d = data.random_direction(rng, g.dim)
        p = exp_problem(g, bc, d)
        p.tol = 1e-8
        p.name = f"c5-{i}"
        out.append(Request(t, p, kind + ("-dirichlet" if bc == DIRICHLET else "-neumann")))
    return out


def poisson_exterior(n, L, spacing=0.75):
    """Sec. 6.3: Delta u = g outside a circle of radius 0.25 centred in the
    periodic box [-L/2, L/2)^2, exact u = exp(sin 2 pi x).  Returns the
    exterior geometry (kappa = inf, normals into the circle), the forcing g~
    on the grid (g = Delta u outside, g_e = 0 inside), U_b at the points and
    the exact u at the grid nodes."""
    g = geometry.exterior(geometry.circle(n, 0.25, spacing=spacing, center=(0.0, 0.0),
                                          origin=(-L / 2, -L / 2), box_len=L,
                                          kappa=float("inf")))
    P = grid_nodes(g)
    s, c = np.sin(2 * np.pi * P[:, 0]), np.cos(2 * np.pi * P[:, 0])
    lap = np.exp(s) * ((2 * np.pi * c) ** 2 - 4 * np.pi ** 2 * s)
    gt = np.where(np.linalg.norm(P, axis=1) > 0.25, lap, 0.0).reshape(n, n)
    return g, gt, np.exp(np.sin(2 * np.pi * g.X[:, 0])), np.exp(s)


def grid_nodes(geom):
    """(n^d, d) coordinates of all grid nodes in memory order (x fastest)."""
    h = geom.h
    ax = [geom.origin[c] + h * np.arange(geom.n) for c in range(geom.dim)]
    mesh = np.meshgrid(*ax[::-1], indexing="ij")  # slowest axis first
    cols = [m.reshape(-1) for m in mesh[::-1]]     # back to (x, y[, z])
    return np.stack(cols, axis=1)


def interior_mask_circle(geom, R, margin):
    """Grid nodes inside the disk and farther than ``margin`` from the circle."""
    P = grid_nodes(geom)
    rho = np.linalg.norm(P - np.asarray(geom.center)[None, :], axis=1)
    return rho < R - margin


def star_radius_at(geom, P):
    e = geom.extra
    d = P - np.asarray(geom.center)[None, :]
    th = np.arctan2(d[:, 1], d[:, 0])
    return np.hypot(d[:, 0], d[:, 1]), e["r0"] * (1 + e["amp"] * np.cos(e["lobes"] * th))


def fmt_m(geom):
    return f"N={geom.n}^{geom.dim} M={geom.m}"


_ = math  # keep math imported for callers that extend configs
