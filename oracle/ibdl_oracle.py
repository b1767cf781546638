"""Plain, slow FP64 CPU oracle of the IBDL hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module; the library never does.
It shares no code with the CUDA path: inputs come from ``workloads`` (point
placement and boundary data only).

Every function follows a passage of Leathers & Guy, "Immersed Boundary Double
Layer method" (arXiv:2203.12126):

* delta function          Sec. 5.2, eq. (delta eqn 1)-(delta eqn 2)
* spread S                Sec. 5.2, eq. (spread operator again2)
* interpolation S*        Sec. 5.2, eq. (interpolation again)
* S~Q = div(S Q n)        Sec. 4.1 (ibdl), Sec. 5.2 eq. (Stilde): spread each
                          component of Q n, then centred differences
* 5/7-point Laplacian     Sec. 5.1 (five-point; its 3D analogue, Sec. 6.7)
* Dirichlet system        Sec. 5.3, eq. (ibdl schur again)
* Neumann system          Sec. 4.4, eq. (Neumann saddle point)
* field evaluation        Sec. 4.1 step 2, eq. (ibdl 1 again); eq. (ib neumann 1)
* GMRES                   Sec. 5.3 (unpreconditioned, relative residual)
* Poisson limit           Sec. 5.4, App. C: kappa = inf (k = 0); the mean-zero
                          inverse Delta_0^{-1} replaces -kappa L'^{-1}
* completed IBDL          Sec. 5.4 eq. (ibdl completed), App. C: unknowns
                          (Q, u_bar), single layer eta S Q added
* interior indicator      App. D: Delta u + S~ 1 = 0, mean-zero solve, shift by
                          the box-corner value, threshold at 1/2
* near-boundary values    Sec. 5.5, App. A (2D): linear interpolation between
                          the chord point x_A and a point x_B m2 h inside; its
                          3D generalisation (Sec. 6.7) on the triangle of the
                          three nearest points
* Fourier-spectral        Sec. 5.1-5.2, Sec. 6.2.1, Sec. 6.7: spectral Laplacian
  discretisation          and (matching it, Sec. 5.2) spectral divergence in S~

Conventions.  The paper writes the operator as L_p = Delta_h - k^2.  This
oracle uses L' = I - kappa Delta_h with kappa = 1/k^2, so L_p = -(1/kappa) L'
and L_p^{-1} = -kappa L'^{-1}; the Dirichlet operator of eq. (ibdl schur
again), -S* L_p^{-1} S~ + I/2, becomes A_D = I/2 + kappa S* L'^{-1} S~ and
the Neumann one becomes A_N = kappa S* L'^{-1} S~ - I/2.  Grid fields are
numpy arrays of shape (n,)*d indexed [.., y, x] (x fastest in memory); grid
node j sits at origin + j h.  Forcing g~ is given in the paper's convention
Delta u - k^2 u = g.

Parity pins live in tests/test_oracle_*.py; functions without a pin say so.
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------
# Regularised delta function, Sec. 5.2
# ---------------------------------------------------------------------------


def phi_peskin4(r):
    """Peskin's 4-point kernel, eq. (delta eqn 2): two branches in |r|."""
    a = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(a)
    inner = a <= 1.0
    outer = (a > 1.0) & (a < 2.0)
    ai = a[inner]
    out[inner] = (3.0 - 2.0 * ai + np.sqrt(1.0 + 4.0 * ai - 4.0 * ai * ai)) / 8.0
    ao = a[outer]
    out[outer] = (5.0 - 2.0 * ao - np.sqrt(np.maximum(0.0, -7.0 + 12.0 * ao - 4.0 * ao * ao))) / 8.0
    return out


def phi_cos4(r):
    """Cosine 4-point kernel (1 + cos(pi r / 2)) / 4 on |r| < 2."""
    a = np.abs(np.asarray(r, dtype=np.float64))
    return np.where(a < 2.0, 0.25 * (1.0 + np.cos(0.5 * np.pi * a)), 0.0)


PHI = {"peskin4": phi_peskin4, "cos4": phi_cos4}


class Box:
    """Periodic box [origin, origin + L)^d with n nodes per axis."""

    def __init__(self, dim, n, box_len, origin):
        self.d = int(dim)
        self.n = int(n)
        self.L = float(box_len)
        self.o = np.asarray(origin, dtype=np.float64)[: self.d]
        self.h = self.L / self.n

    @classmethod
    def of(cls, geom):
        return cls(geom.dim, geom.n, geom.box_len, geom.origin)

    @property
    def shape(self):
        return (self.n,) * self.d

    def axis(self, c):
        """numpy array axis of spatial direction c (0 = x)."""
        return self.d - 1 - c


def _tap_table(box, X, delta):
    """For every point and axis: the 4 node indices j whose |x_j - X| < 2h
    (before periodic wrap) and phi((x_j - X)/h) there.

    Nodes at origin + j h; with s = (X - origin)/h the support of phi(j - s)
    is s-2 < j < s+2, i.e. j = floor(s)-1 .. floor(s)+2.
    """
    phi = PHI[delta]
    s = (X - box.o[None, :]) / box.h                      # (M, d)
    base = np.floor(s).astype(np.int64) - 1               # (M, d)
    j = base[:, :, None] + np.arange(4)[None, None, :]    # (M, d, 4)
    wt = phi(j - s[:, :, None])                           # (M, d, 4)
    return j % box.n, wt


def spread(box, X, F, w, delta="peskin4"):
    """(S F)_j = sum_i F_i w_i delta_h(x_j - X_i), eq. (spread operator
    again2), delta_h = h^{-d} prod_c phi((x_c - X_c)/h), eq. (delta eqn 1)."""
    M = X.shape[0]
    jj, wt = _tap_table(box, X, delta)
    out = np.zeros(box.shape)
    amp = F * w / box.h ** box.d
    taps = np.indices((4,) * box.d).reshape(box.d, -1).T   # all 4^d tap tuples
    for t in taps:
        val = amp.copy()
        idx = [None] * box.d
        for c in range(box.d):
            val = val * wt[:, c, t[c]]
            idx[box.axis(c)] = jj[:, c, t[c]]
        np.add.at(out, tuple(idx), val)
    assert val.shape == (M,)
    return out


def interp(box, X, u, delta="peskin4"):
    """(S* u)(X_i) = sum_j u_j delta_h(x_j - X_i) h^d, eq. (interpolation
    again): the h^{-d} of delta_h cancels the h^d cell volume."""
    jj, wt = _tap_table(box, X, delta)
    out = np.zeros(X.shape[0])
    taps = np.indices((4,) * box.d).reshape(box.d, -1).T
    for t in taps:
        val = np.ones(X.shape[0])
        idx = [None] * box.d
        for c in range(box.d):
            val = val * wt[:, c, t[c]]
            idx[box.axis(c)] = jj[:, c, t[c]]
        out += val * u[tuple(idx)]
    return out


def central_diff(box, g, c):
    """(D_c g)_j = (g_{j+e_c} - g_{j-e_c}) / (2h), periodic (Sec. 5.2)."""
    a = box.axis(c)
    return (np.roll(g, -1, axis=a) - np.roll(g, 1, axis=a)) / (2.0 * box.h)


def spread_div(box, X, nrm, w, Q, delta="peskin4"):
    """S~ Q = div_h (S (Q n)), eq. (Stilde): spread each component Q n_c,
    then sum the centred differences."""
    out = np.zeros(box.shape)
    for c in range(box.d):
        out += central_diff(box, spread(box, X, Q * nrm[:, c], w, delta), c)
    return out


# ---------------------------------------------------------------------------
# Periodic Helmholtz solve, Sec. 5.1
# ---------------------------------------------------------------------------


def laplacian(box, u):
    """Standard 5-point (2D) / 7-point (3D) Laplacian, periodic."""
    out = -2.0 * box.d * u
    for a in range(box.d):
        out = out + np.roll(u, 1, axis=a) + np.roll(u, -1, axis=a)
    return out / box.h ** 2


def apply_Lprime(box, kappa, u):
    """L' u = u - kappa Delta_h u (explicit stencil, used by pins)."""
    return u - kappa * laplacian(box, u)


def symbol(box, kappa):
    """Eigenvalues of L' on the Fourier modes exp(2 pi i k.j / n):
    sigma(k) = 1 + (4 kappa / h^2) sum_c sin^2(pi k_c / n)."""
    k = np.arange(box.n)
    s2 = np.sin(np.pi * k / box.n) ** 2
    sig = np.ones(box.shape)
    for a in range(box.d):
        shp = [1] * box.d
        shp[a] = box.n
        sig = sig + (4.0 * kappa / box.h ** 2) * s2.reshape(shp)
    return sig


def helmholtz_solve(box, kappa, f):
    """v = L'^{-1} f by diagonalising the periodic stencil with the FFT."""
    F = np.fft.fftn(f)
    return np.real(np.fft.ifftn(F / symbol(box, kappa)))


def laplace_symbol(box):
    """Eigenvalues of -Delta_h on the Fourier modes:
    lambda(k) = (4 / h^2) sum_c sin^2(pi k_c / n); zero only at k = 0."""
    k = np.arange(box.n)
    s2 = np.sin(np.pi * k / box.n) ** 2
    lam = np.zeros(box.shape)
    for a in range(box.d):
        shp = [1] * box.d
        shp[a] = box.n
        lam = lam + (4.0 / box.h ** 2) * s2.reshape(shp)
    return lam


def laplace_inverse0(box, f):
    """Delta_0^{-1} f of Sec. 5.4 / App. C: the mean-zero u with
    Delta_h u = f - mean(f) (the k = 0 mode of f is dropped)."""
    lam = laplace_symbol(box)
    F = np.fft.fftn(f)
    F.reshape(-1)[0] = 0.0
    lam.reshape(-1)[0] = 1.0
    return np.real(np.fft.ifftn(-F / lam))


def green(box, kappa, f, disc="fd"):
    """The grid solve every operator below uses: kappa L'^{-1} f for finite
    kappa (= -L_p^{-1} f with L_p = Delta_h - k^2), and its k = 0 limit
    -Delta_0^{-1} f for kappa = inf (the Poisson equation, Sec. 5.4).
    disc = "spectral" uses the Fourier-spectral Laplacian instead of the
    5/7-point stencil."""
    if disc == "spectral":
        lam = spectral_laplace_symbol(box)
        F = np.fft.fftn(f)
        if np.isinf(kappa):
            F.reshape(-1)[0] = 0.0
            lam.reshape(-1)[0] = 1.0
            return np.real(np.fft.ifftn(F / lam))
        return np.real(np.fft.ifftn(kappa * F / (1.0 + kappa * lam)))
    if np.isinf(kappa):
        return -laplace_inverse0(box, f)
    return kappa * helmholtz_solve(box, kappa, f)


# ---------------------------------------------------------------------------
# Fourier-spectral discretisation (Sec. 5.1, Sec. 6.2.1, Sec. 6.7)
# ---------------------------------------------------------------------------


def wavenumbers(box):
    """Signed integer wavenumbers of the n-point grid in FFT order:
    0, 1, ..., n/2 - 1, -n/2, ..., -1."""
    return np.fft.fftfreq(box.n, d=1.0 / box.n)


def spectral_derivative(box, g, c):
    """d/dx_c of the trigonometric interpolant: mode k times i 2 pi k / L;
    the Nyquist mode (k = -n/2) is set to zero so real data stays real."""
    a = box.axis(c)
    k = wavenumbers(box)
    fac = 2j * np.pi * k / box.L
    fac[box.n // 2] = 0.0
    shp = [1] * box.d
    shp[a] = box.n
    return np.real(np.fft.ifft(np.fft.fft(g, axis=a) * fac.reshape(shp), axis=a))


def spectral_laplace_symbol(box):
    """Eigenvalues of the spectral -Delta: sum_c (2 pi k_c / L)^2 (the
    Nyquist mode keeps (pi n / L)^2)."""
    k = wavenumbers(box)
    k2 = (2.0 * np.pi * k / box.L) ** 2
    lam = np.zeros(box.shape)
    for a in range(box.d):
        shp = [1] * box.d
        shp[a] = box.n
        lam = lam + k2.reshape(shp)
    return lam


def spread_div_spectral(box, X, nrm, w, Q, delta="peskin4"):
    """S~ Q with the spectral divergence: sum_c D_c S(Q n_c) (Sec. 5.2: the
    divergence matches the PDE's discretisation)."""
    out = np.zeros(box.shape)
    for c in range(box.d):
        out += spectral_derivative(box, spread(box, X, Q * nrm[:, c], w, delta), c)
    return out


def helmholtz_dense(box, kappa):
    """Dense matrix of L' (tiny grids only): column j = L' e_j."""
    n = box.n ** box.d
    A = np.zeros((n, n))
    e = np.zeros(box.shape)
    for j in range(n):
        e.reshape(-1)[j] = 1.0
        A[:, j] = apply_Lprime(box, kappa, e).reshape(-1)
        e.reshape(-1)[j] = 0.0
    return A


# ---------------------------------------------------------------------------
# The boundary operators, Sec. 4.1, 4.4 and 5.3
# ---------------------------------------------------------------------------

DIRICHLET, NEUMANN = 0, 1


class Operator:
    """A_D Q = Q/2 + kappa S* L'^{-1} S~ Q         (eq. (ibdl schur again))
    A_N U = kappa S* L'^{-1} S~ U - U/2          (eq. (Neumann saddle point))

    kappa = inf is the Poisson equation (Sec. 5.4, App. C with eta = 0):
    A_D Q = Q/2 - S* Delta_0^{-1} S~ Q (Dirichlet only).
    """

    def __init__(self, geom, bc, kappa=None, delta=None, disc="fd"):
        self.box = Box.of(geom)
        self.disc = disc
        self.X = np.asarray(geom.X, dtype=np.float64)
        self.nrm = np.asarray(geom.normals, dtype=np.float64)
        self.w = np.asarray(geom.weights, dtype=np.float64)
        self.kappa = float(geom.kappa if kappa is None else kappa)
        self.delta = geom.delta if delta is None else delta
        self.bc = int(bc)
        self.matvecs = 0
        if np.isinf(self.kappa) and self.bc != DIRICHLET:
            raise ValueError("the Poisson limit is defined for the Dirichlet problem only")

    @property
    def m(self):
        return self.X.shape[0]

    def div(self, Q):
        """S~ Q with the divergence of the chosen discretisation."""
        sd = spread_div_spectral if self.disc == "spectral" else spread_div
        return sd(self.box, self.X, self.nrm, self.w, Q, self.delta)

    def layer(self, Q):
        """v = kappa L'^{-1} S~ Q on the grid (-Delta_0^{-1} S~ Q if kappa = inf)."""
        return green(self.box, self.kappa, self.div(Q), self.disc)

    def apply(self, Q):
        self.matvecs += 1
        Q = np.asarray(Q, dtype=np.float64)
        y = interp(self.box, self.X, self.layer(Q), self.delta)
        return y + 0.5 * Q if self.bc == DIRICHLET else y - 0.5 * Q

    __call__ = apply

    def rhs(self, bdata, g_grid=None):
        """Right-hand side of the boundary system.

        Dirichlet: U_b - S* L_p^{-1} g~ = U_b + kappa S* L'^{-1} g~.
        Neumann:   S* L_p^{-1} S V_b - S* L_p^{-1} g~
                   = kappa S* L'^{-1} (g~ - S V_b).
        """
        b = np.asarray(bdata, dtype=np.float64)
        if self.bc == DIRICHLET:
            out = b.copy()
            if g_grid is not None:
                out += interp(self.box, self.X, green(self.box, self.kappa, g_grid, self.disc),
                              self.delta)
            return out
        src = -spread(self.box, self.X, b, self.w, self.delta)
        if g_grid is not None:
            src = src + g_grid
        return interp(self.box, self.X, green(self.box, self.kappa, src, self.disc), self.delta)

    def evaluate(self, Q, vb=None, g_grid=None):
        """Grid solution, step 2 of Sec. 4.1: L_p u + S~Q = g~ gives
        u = kappa L'^{-1}(S~Q - g~); Neumann (eq. (ib neumann 1)) adds S V_b."""
        src = self.div(Q)
        if self.bc == NEUMANN and vb is not None:
            src = src + spread(self.box, self.X, vb, self.w, self.delta)
        if g_grid is not None:
            src = src - g_grid
        return green(self.box, self.kappa, src, self.disc)

    def dense(self):
        """Assemble A column by column, A[:, i] = A e_i."""
        M = self.m
        A = np.zeros((M, M))
        e = np.zeros(M)
        for i in range(M):
            e[i] = 1.0
            A[:, i] = self.apply(e)
            e[i] = 0.0
        return A


# ---------------------------------------------------------------------------
# GMRES, Sec. 5.3 (textbook restarted GMRES(m), modified Gram-Schmidt)
# ---------------------------------------------------------------------------


class GmresResult:
    def __init__(self, x, iters, rel_res, history, converged):
        self.x, self.iters, self.rel_res = x, iters, rel_res
        self.history, self.converged = history, converged


def gmres(A, b, tol=1e-8, restart=30, maxiter=1000, x0=None):
    """Solve A x = b until ||b - A x|| / ||b|| <= tol, x0 = 0 by default.

    Arnoldi with modified Gram-Schmidt builds an orthonormal basis of the
    Krylov space; Givens rotations keep the Hessenberg matrix triangular, so
    |g_{j+1}| is the residual norm of the least-squares iterate.  ``iters``
    counts inner iterations (matrix-vector products after the first
    residual), as the paper's tables do.
    """
    b = np.asarray(b, dtype=np.float64)
    M = b.shape[0]
    x = np.zeros(M) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return GmresResult(np.zeros(M), 0, 0.0, [], True)
    total = 0
    history = []
    while True:
        r = b - A(x) if np.any(x) else b.copy()
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol:
            return GmresResult(x, total, beta / bnorm, history, True)
        if total >= maxiter:
            return GmresResult(x, total, beta / bnorm, history, False)
        m = restart
        V = np.zeros((m + 1, M))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        V[0] = r / beta
        g[0] = beta
        k = 0
        for j in range(m):
            w = A(V[j])
            total += 1
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            hnext = np.linalg.norm(w)
            H[j + 1, j] = hnext
            if hnext > 0.0:
                V[j + 1] = w / hnext
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or total >= maxiter or hnext == 0.0:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + V[:k].T @ y


def solve(geom, bc, bdata, tol=1e-10, restart=30, maxiter=1000, g_grid=None,
          kappa=None, disc="fd"):
    """Step 1 of Sec. 4.1 (or Sec. 4.4): GMRES on the boundary system."""
    op = Operator(geom, bc, kappa, disc=disc)
    b = op.rhs(bdata, g_grid)
    res = gmres(op, b, tol, restart, maxiter)
    res.matvecs = op.matvecs
    res.op = op
    res.b = b
    return res


def solve_dense(geom, bc, bdata, g_grid=None, kappa=None, disc="fd"):
    """Exact discrete solution Q* = A^{-1} b by LU (small M only)."""
    op = Operator(geom, bc, kappa, disc=disc)
    b = op.rhs(bdata, g_grid)
    return np.linalg.solve(op.dense(), b)


# ---------------------------------------------------------------------------
# Completed IBDL for the Poisson equation, Sec. 5.4 and App. C
# ---------------------------------------------------------------------------


class CompletedOperator:
    """The completed system of App. C on z = (Q, u_bar), length M + 1:

      Q/2 - S* Delta_0^{-1} (S~ + eta S) Q + u_bar 1 = U_b - S* Delta_0^{-1} g~
      eta sum_i w_i Q_i                               = h^d sum_j g~_j

    The second row is the solvability condition eta int_Gamma Q ds =
    int_C g~; with per-point weights w_i it reads sum_i w_i Q_i (the paper's
    Delta s 1^T Q for uniform spacing).  Dirichlet only.
    """

    def __init__(self, geom, eta, delta=None):
        self.box = Box.of(geom)
        self.X = np.asarray(geom.X, dtype=np.float64)
        self.nrm = np.asarray(geom.normals, dtype=np.float64)
        self.w = np.asarray(geom.weights, dtype=np.float64)
        self.delta = geom.delta if delta is None else delta
        self.eta = float(eta)
        self.matvecs = 0

    @property
    def m(self):
        return self.X.shape[0]

    def source(self, Q):
        """(S~ + eta S) Q on the grid."""
        return (spread_div(self.box, self.X, self.nrm, self.w, Q, self.delta)
                + self.eta * spread(self.box, self.X, Q, self.w, self.delta))

    def apply(self, z):
        self.matvecs += 1
        z = np.asarray(z, dtype=np.float64)
        Q, ubar = z[:self.m], z[self.m]
        top = (0.5 * Q - interp(self.box, self.X, laplace_inverse0(self.box, self.source(Q)),
                                self.delta) + ubar)
        return np.concatenate([top, [self.eta * np.dot(self.w, Q)]])

    __call__ = apply

    def rhs(self, ub, g_grid=None):
        top = np.array(ub, dtype=np.float64)
        last = 0.0
        if g_grid is not None:
            top -= interp(self.box, self.X, laplace_inverse0(self.box, g_grid), self.delta)
            last = self.box.h ** self.box.d * float(np.sum(g_grid))
        return np.concatenate([top, [last]])

    def evaluate(self, z, g_grid=None):
        """u = -Delta_0^{-1} (S~ + eta S) Q + Delta_0^{-1} g~ + u_bar."""
        Q, ubar = np.asarray(z[:self.m]), float(z[self.m])
        u = -laplace_inverse0(self.box, self.source(Q)) + ubar
        if g_grid is not None:
            u = u + laplace_inverse0(self.box, g_grid)
        return u


def solve_completed(geom, eta, ub, g_grid=None, tol=1e-10, restart=30, maxiter=1000):
    """GMRES on the completed system; returns the result with x = (Q, u_bar)."""
    op = CompletedOperator(geom, eta)
    b = op.rhs(ub, g_grid)
    res = gmres(op, b, tol, restart, maxiter)
    res.matvecs = op.matvecs
    res.op = op
    res.b = b
    return res


# ---------------------------------------------------------------------------
# Interior indicator, App. D
# ---------------------------------------------------------------------------


def indicator(geom):
    """App. D: Delta u + S~ 1 = 0 solved for the mean-zero u, i.e.
    u = -Delta_0^{-1} S~ 1; chi_h = u - u(box corner node); the indicator is
    chi = 1 where chi_h > 1/2, else 0.  Returns (chi_h, chi as uint8)."""
    box = Box.of(geom)
    f = spread_div(box, geom.X, geom.normals, geom.weights, np.ones(geom.m), geom.delta)
    u = -laplace_inverse0(box, f)
    chi_h = u - u.reshape(-1)[0]
    return chi_h, (chi_h > 0.5).astype(np.uint8)


# ---------------------------------------------------------------------------
# Near-boundary values, Sec. 5.5 and App. A (2D)
# ---------------------------------------------------------------------------


def near_boundary_values(geom, u, ub, inside, m1, m2, nodes=None):
    """Replace u at the nodes of Omega within m1 meshwidths of Gamma (App. A).

    For a node x_p with inside = 1 whose nearest boundary point is closer than
    m1 h:
      1. x_1, x_2 = the two nearest boundary points (ties: lower index first);
      2. x_A = the orthogonal projection of x_p on the line x_2 + t (x_1 - x_2);
         if t is outside [0, 1], take the third nearest point and use the two
         of the three that lie farthest apart, with t clamped to [0, 1];
      3. u(x_A) = U_b(x_1)|x_A - x_2| / |x_2 - x_1| + U_b(x_2)|x_A - x_1| / |x_2 - x_1|;
      4. x_B = x_A + m2 h (x_p - x_A) / |x_p - x_A|;
      5. u(x_B) = the bilinear interpolation of u on the cell holding x_B;
      6. u(x_p) = u(x_A)|x_B - x_p| / |x_B - x_A| + u(x_B)|x_A - x_p| / |x_B - x_A|.
    A node on the chord (|x_p - x_A| = 0) takes u(x_A).  Other nodes keep
    their value.  u: grid (n, n); ub: boundary values (the data U_b for
    Dirichlet, the solved U for Neumann); inside: (n, n) 0/1.  ``nodes``
    (flat indices iy * n + ix) restricts the work to a sample of nodes; the
    others are returned unchanged."""
    box = Box.of(geom)
    assert box.d == 2
    n, h = box.n, box.h
    X = np.asarray(geom.X, dtype=np.float64)
    ub = np.asarray(ub, dtype=np.float64)
    uin = np.asarray(u, dtype=np.float64).reshape(n, n)
    out = uin.copy()
    ins = np.asarray(inside).reshape(n, n)
    thresh = (m1 * h) * (m1 * h)
    ox, oy = float(box.o[0]), float(box.o[1])
    todo = range(n * n) if nodes is None else sorted(int(j) for j in nodes)
    for j in todo:
        iy, ix = divmod(j, n)
        if not ins[iy, ix]:
            continue
        py = oy + iy * h
        dy = py - X[:, 1]
        px = ox + ix * h
        dx = px - X[:, 0]
        d2 = dx * dx + dy * dy
        order = np.argsort(d2, kind="stable")
        if not d2[order[0]] < thresh:
            continue
        a, b = int(order[0]), int(order[1])
        p = np.array([px, py])
        t = _chord_t(p, X[a], X[b])
        if not (0.0 <= t <= 1.0):
            c = int(order[2])
            best = -1.0
            for ia, ib in ((a, b), (a, c), (b, c)):
                e = X[ia] - X[ib]
                sep = e[0] * e[0] + e[1] * e[1]
                if sep > best:
                    best, pa, pb = sep, ia, ib
            a, b = pa, pb
            t = min(max(_chord_t(p, X[a], X[b]), 0.0), 1.0)
        x1, x2 = X[a], X[b]
        xA = x2 + t * (x1 - x2)
        L12 = np.linalg.norm(x2 - x1)
        uA = ub[a] * np.linalg.norm(xA - x2) / L12 + ub[b] * np.linalg.norm(xA - x1) / L12
        dA = np.linalg.norm(p - xA)
        if dA == 0.0:
            out[iy, ix] = uA
            continue
        xB = xA + (p - xA) / dA * (m2 * h)
        rx, ry = (xB[0] - ox) / h, (xB[1] - oy) / h
        jx, jy = math.floor(rx), math.floor(ry)
        fx, fy = rx - jx, ry - jy
        u00 = uin[jy % n, jx % n]
        u10 = uin[jy % n, (jx + 1) % n]
        u01 = uin[(jy + 1) % n, jx % n]
        u11 = uin[(jy + 1) % n, (jx + 1) % n]
        uB = (fx * fy * u11 + fy * (1.0 - fx) * u01 + fx * (1.0 - fy) * u10
              + (1.0 - fx - fy + fx * fy) * u00)
        LAB = np.linalg.norm(xB - xA)
        out[iy, ix] = uA * np.linalg.norm(xB - p) / LAB + uB * dA / LAB
    return out


def near_boundary_values_3d(geom, u, ub, inside, m1, m2, nodes=None):
    """The 3D near-boundary step of Sec. 6.7 ("a direct generalization" of
    App. A), read as: for a node x_p of Omega whose nearest boundary point is
    closer than m1 h,
      1. x_1, x_2, x_3 = its three nearest boundary points (ties: lower index);
      2. x_A = the orthogonal foot of x_p on their plane, with barycentric
         coordinates (l_1, l_2, l_3) clamped to >= 0 and renormalised to sum 1
         (the point of the triangle, or of its edges, nearest in that sense);
         a degenerate triangle (zero area) takes x_A = x_1;
      3. u(x_A) = sum l_k U_b(x_k);
      4. x_B = x_A + m2 h (x_p - x_A) / |x_p - x_A|;
      5. u(x_B) = the trilinear interpolation of u on the cell holding x_B;
      6. u(x_p) = u(x_A)|x_B - x_p| / |x_B - x_A| + u(x_B)|x_A - x_p| / |x_B - x_A|.
    A node at x_A takes u(x_A).  u, inside: grids (n, n, n) indexed [z, y, x]."""
    box = Box.of(geom)
    assert box.d == 3
    n, h = box.n, box.h
    X = np.asarray(geom.X, dtype=np.float64)
    ub = np.asarray(ub, dtype=np.float64)
    uin = np.asarray(u, dtype=np.float64).reshape(n, n, n)
    out = uin.copy()
    ins = np.asarray(inside).reshape(n, n, n)
    thresh = (m1 * h) * (m1 * h)
    ox, oy, oz = float(box.o[0]), float(box.o[1]), float(box.o[2])
    todo = range(n ** 3) if nodes is None else sorted(int(j) for j in nodes)
    for j in todo:
        iz, r = divmod(j, n * n)
        iy, ix = divmod(r, n)
        if not ins[iz, iy, ix]:
            continue
        px, py, pz = ox + ix * h, oy + iy * h, oz + iz * h
        dx, dy, dz = px - X[:, 0], py - X[:, 1], pz - X[:, 2]
        d2 = dx * dx + dy * dy + dz * dz
        order = np.argsort(d2, kind="stable")
        if not d2[order[0]] < thresh:
            continue
        i1, i2, i3 = (int(k) for k in order[:3])
        p = np.array([px, py, pz])
        lam = _barycentric_clamped(p, X[i1], X[i2], X[i3])
        if lam is None:
            xA, uA = X[i1].copy(), ub[i1]
        else:
            xA = lam[0] * X[i1] + lam[1] * X[i2] + lam[2] * X[i3]
            uA = lam[0] * ub[i1] + lam[1] * ub[i2] + lam[2] * ub[i3]
        dA = np.linalg.norm(p - xA)
        if dA == 0.0:
            out[iz, iy, ix] = uA
            continue
        xB = xA + (p - xA) / dA * (m2 * h)
        rr = [(xB[0] - ox) / h, (xB[1] - oy) / h, (xB[2] - oz) / h]
        jj = [math.floor(v) for v in rr]
        ff = [rr[c] - jj[c] for c in range(3)]
        uB = 0.0
        for cz in (0, 1):
            for cy in (0, 1):
                for cx in (0, 1):
                    wgt = ((ff[0] if cx else 1.0 - ff[0]) * (ff[1] if cy else 1.0 - ff[1])
                           * (ff[2] if cz else 1.0 - ff[2]))
                    uB += wgt * uin[(jj[2] + cz) % n, (jj[1] + cy) % n, (jj[0] + cx) % n]
        LAB = np.linalg.norm(xB - xA)
        out[iz, iy, ix] = uA * np.linalg.norm(xB - p) / LAB + uB * dA / LAB
    return out


def _barycentric_clamped(p, a, b, c):
    """Barycentric coordinates of the orthogonal foot of p on the plane of
    the triangle (a, b, c), clamped to >= 0 and renormalised; None for a
    degenerate triangle."""
    e1, e2, w = b - a, c - a, p - a
    d11, d12, d22 = _dot3(e1, e1), _dot3(e1, e2), _dot3(e2, e2)
    w1, w2 = _dot3(w, e1), _dot3(w, e2)
    det = d11 * d22 - d12 * d12
    if not det > 0.0:
        return None
    l2 = (d22 * w1 - d12 * w2) / det
    l3 = (d11 * w2 - d12 * w1) / det
    lam = [max(1.0 - l2 - l3, 0.0), max(l2, 0.0), max(l3, 0.0)]
    sm = lam[0] + lam[1] + lam[2]
    return [lam[0] / sm, lam[1] / sm, lam[2] / sm]


def _dot3(u, v):
    """u . v summed left to right (so every rounding is fixed)."""
    return float(u[0] * v[0] + u[1] * v[1] + u[2] * v[2])


def _chord_t(p, x1, x2):
    """Parameter t of the orthogonal projection of p on x_2 + t (x_1 - x_2)."""
    e = x1 - x2
    return float(((p[0] - x2[0]) * e[0] + (p[1] - x2[1]) * e[1]) / (e[0] * e[0] + e[1] * e[1]))
