"""Boundary data and closed-form solutions for the synthetic IBDL problems.

All closed forms solve the homogeneous PDE Delta u - k^2 u = 0 (Sec. 2,
eq. (pde) with g = 0), k^2 = 1/kappa:

* 2D disk, Dirichlet: u = I_2(k rho) sin(2 theta) / I_2(k R)  (Sec. 6.1).
* 3D ball, Neumann:   u = i_1(k rho) cos(vartheta), the modified spherical
  Bessel solution; du/dn = k i_1'(k R) cos(vartheta) on the sphere.
* Any shape:          u = exp(k d.(x - c)) for a unit vector d; du/dn =
  k (d.n) u.
* Seeded Fourier data: U(theta) = sum_{m=1}^{10} a_m cos(m theta) +
  b_m sin(m theta), a_m, b_m ~ N(0, 1) from numpy's default_rng(seed).

None of the method's own arithmetic lives here.
"""
from __future__ import annotations

import numpy as np
from scipy import special


def fourier_data(theta, seed, modes=10):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(modes)
    b = rng.standard_normal(modes)
    mm = np.arange(1, modes + 1)
    return np.cos(np.outer(theta, mm)) @ a + np.sin(np.outer(theta, mm)) @ b


def disk_bessel_exact(x, y, center, R, k, order=2):
    """I_order(k rho) sin(order*theta) / I_order(k R)."""
    dx, dy = x - center[0], y - center[1]
    rho = np.hypot(dx, dy)
    th = np.arctan2(dy, dx)
    return special.iv(order, k * rho) * np.sin(order * th) / special.iv(order, k * R)


def ball_bessel_exact(x, y, z, center, k):
    """i_1(k rho) cos(vartheta) (vartheta: polar angle about the centre)."""
    dx, dy, dz = x - center[0], y - center[1], z - center[2]
    rho = np.sqrt(dx * dx + dy * dy + dz * dz)
    with np.errstate(invalid="ignore", divide="ignore"):
        c = np.where(rho > 0, dz / np.where(rho > 0, rho, 1.0), 0.0)
    return special.spherical_in(1, k * rho) * c


def ball_bessel_neumann(R, k, polar):
    """du/dn on the sphere of radius R for u = i_1(k rho) cos(vartheta)."""
    return k * special.spherical_in(1, k * R, derivative=True) * np.cos(polar)


def exp_exact(X, center, k, direction):
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return np.exp(k * ((X - np.asarray(center)[None, :]) @ d))


def exp_neumann(X, normals, center, k, direction):
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return k * (normals @ d) * exp_exact(X, center, k, d)


def random_direction(rng, dim):
    v = rng.standard_normal(dim)
    return v / np.linalg.norm(v)
