"""Plain FP64 Krylov solvers (Sec. 4: CG, multishift CG) and helpers.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

All inner products are <a, b> = sum conj(a) b over every component; residuals
are the non-squared relative residual ||b - A x|| / ||b|| of the system solved.
"""
from __future__ import annotations

import numpy as np


def dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def norm2(a):
    return float(np.real(np.vdot(a.ravel(), a.ravel())))


def cg(apply_A, b, tol=1e-10, maxiter=100000, x0=None):
    """Textbook conjugate gradient on a hermitian positive definite A.

    Stops when the iterated residual satisfies ||r|| <= tol ||b||.
    Returns (x, iterations).
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_A(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = norm2(r)
    stop = tol * tol * norm2(b)
    k = 0
    while rr > stop and k < maxiter:
        Ap = apply_A(p)
        alpha = rr / np.real(dot(p, Ap))
        x += alpha * p
        r -= alpha * Ap
        rr_new = norm2(r)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        k += 1
    return x, k


def multishift_cg(apply_A, b, shifts, tol=1e-10, maxiter=100000):
    """Multishift CG (Jegerlehner): solves (A + sigma_k) x_k = b for all shifts
    from one Krylov space, built on the smallest shift.

    Recurrences (sigma_0 = smallest shift, d_k = sigma_k - sigma_0):
      CG on A + sigma_0:  alpha_n = rr_n / <p, (A+sigma_0) p>,  beta_n = rr_{n+1}/rr_n
      zeta_k^{n+1} = zeta_k^n zeta_k^{n-1} alpha_{n-1} /
                     (alpha_n beta_{n-1} (zeta_k^{n-1} - zeta_k^n)
                      + zeta_k^{n-1} alpha_{n-1} (1 + d_k alpha_n))
      alpha_k = alpha_n zeta_k^{n+1} / zeta_k^n,   x_k += alpha_k p_k
      beta_k  = beta_n (zeta_k^{n+1} / zeta_k^n)^2
      p_k     = zeta_k^{n+1} r_{n+1} + beta_k p_k
    with zeta^{-1} = zeta^0 = 1, alpha_{-1} = 1, beta_{-1} = 0.  A shift stops
    updating once its residual zeta_k ||r|| drops below tol ||b||.
    Returns (xs, iterations).
    """
    shifts = np.asarray(shifts, dtype=np.float64)
    order = np.argsort(shifts)
    s0 = shifts[order[0]]
    n = len(shifts)
    xs = [np.zeros_like(b) for _ in range(n)]
    ps = [b.copy() for _ in range(n)]
    r = b.copy()
    p = b.copy()
    rr = norm2(r)
    bb = rr
    zeta = np.ones(n)
    zeta_old = np.ones(n)
    alpha_old = 1.0
    beta_old = 0.0
    active = np.ones(n, dtype=bool)
    k = 0
    while k < maxiter and active.any():
        Ap = apply_A(p) + s0 * p
        alpha = rr / np.real(dot(p, Ap))
        r_new = r - alpha * Ap
        rr_new = norm2(r_new)
        beta = rr_new / rr
        for i in range(n):
            if not active[i]:
                continue
            d = shifts[i] - s0
            zn = zeta[i] * zeta_old[i] * alpha_old / (
                alpha * beta_old * (zeta_old[i] - zeta[i])
                + zeta_old[i] * alpha_old * (1.0 + d * alpha))
            ai = alpha * zn / zeta[i]
            xs[i] += ai * ps[i]
            bi = beta * (zn / zeta[i]) ** 2
            ps[i] = zn * r_new + bi * ps[i]
            zeta_old[i] = zeta[i]
            zeta[i] = zn
            if zn * zn * rr_new <= tol * tol * bb:
                active[i] = False
        p = r_new + beta * p
        r = r_new
        rr = rr_new
        alpha_old = alpha
        beta_old = beta
        k += 1
    return xs, k


def power_iteration(apply_A, v0, iters=100):
    """Largest eigenvalue of a hermitian positive semi-definite A:
    v <- A v / ||A v||, estimate <v, A v> / <v, v>."""
    v = v0 / np.sqrt(norm2(v0))
    lam = 0.0
    for _ in range(iters):
        w = apply_A(v)
        lam = float(np.real(dot(v, w)))
        v = w / np.sqrt(norm2(w))
    return lam


def dense_matrix(apply_op, n_sites, inner_shape):
    """Column-by-column dense matrix of a linear operator on (n_sites, *inner)."""
    ncomp = n_sites * int(np.prod(inner_shape))
    M = np.empty((ncomp, ncomp), dtype=np.complex128)
    e = np.zeros(ncomp, dtype=np.complex128)
    for j in range(ncomp):
        e[:] = 0
        e[j] = 1
        M[:, j] = apply_op(e.reshape((n_sites,) + tuple(inner_shape))).ravel()
    return M


def rel_residual(apply_A, x, b):
    return np.sqrt(norm2(b - apply_A(x)) / norm2(b))
