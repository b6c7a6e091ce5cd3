"""Rational approximation of A^-1/2 for the non-degenerate doublet, and its
correction term, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 4.2 runs the heavy doublet through a rational approximation in partial
fractions (one multishift solve per application) and a correction term for
its error (Fig. 4's heatbath and acceptance timings).  The paper does not print
the approximation; this module takes Zolotarev's optimal one and the binomial
series of the correction, as readings of that setting.

* Coefficients.  On [eps, 1], the best approximation of type (n, n) to x^-1/2
  in the relative sense has its poles and zeros at
      x = -eps c_{2l-1}  and  x = -eps c_{2l},
      c_j = sn^2(j K / (2n + 1); k) / (1 - sn^2(j K / (2n + 1); k)),
  with k = sqrt(1 - eps) and K = K(k) the complete elliptic integral
  (Zolotarev).  The constant factor makes the relative error sqrt(x) r(x) - 1
  equioscillate symmetrically about zero; delta is its maximum.  sn and K are
  evaluated by the arithmetic-geometric mean (Abramowitz and Stegun 16.4).  A
  range [lo, hi] is mapped to [eps, 1] with eps = lo / hi.
* Partial fractions.  r(x) = a0 + sum_l a_l / (x + sigma_l), the form a
  multishift solve applies.
* Correction.  With R = r(A), Z = A R^2 - 1 has norm at most about 2 delta on the
  spectrum, and the correction factor (1 + Z)^p is its binomial series in Z:
  heatbath p = -1/4, acceptance p = 1/2.
"""
from __future__ import annotations

import math

import numpy as np


def _agm_sn(u, k):
    """sn(u | k) by the arithmetic-geometric mean (A&S 16.4.3)."""
    a = [1.0]
    c = [k]
    b = math.sqrt(1.0 - k * k)
    while abs(c[-1]) > 1e-18 and len(a) < 80:
        a_next = 0.5 * (a[-1] + b)
        c.append(0.5 * (a[-1] - b))
        b = math.sqrt(a[-1] * b)
        a.append(a_next)
    n = len(a) - 1
    phi = (2.0 ** n) * a[n] * u
    for i in range(n, 0, -1):
        phi = 0.5 * (phi + math.asin(c[i] / a[i] * math.sin(phi)))
    return math.sin(phi)


def _ellip_k(k):
    """Complete elliptic integral of the first kind, K(k) = pi / (2 AGM(1, k'))."""
    a, b = 1.0, math.sqrt(1.0 - k * k)
    for _ in range(80):
        a, b = 0.5 * (a + b), math.sqrt(a * b)
        if abs(a - b) <= 1e-17 * a:
            break
    return math.pi / (2.0 * a)


def zolotarev_inv_sqrt(n: int, lo: float, hi: float, grid: int = 200001):
    """(a0, a[n], sigma[n], delta): r(x) = a0 + sum a_l / (x + sigma_l) ~ x^-1/2 on
    [lo, hi] with max relative error delta."""
    eps = lo / hi
    k = math.sqrt(1.0 - eps)
    K = _ellip_k(k)
    c = np.empty(2 * n)
    for j in range(1, 2 * n + 1):
        s = _agm_sn(j * K / (2 * n + 1), k)
        c[j - 1] = s * s / (1.0 - s * s)
    poles = eps * c[0::2]       # sigma_l on [eps, 1]
    zeros = eps * c[1::2]       # r has factors (x + zeros_l)
    # constant factor: symmetric relative error over [eps, 1]
    x = np.exp(np.linspace(math.log(eps), 0.0, grid))
    g = np.sqrt(x) * np.prod((x[:, None] + zeros[None]) / (x[:, None] + poles[None]), axis=1)
    gmax, gmin = g.max(), g.min()
    d = 2.0 / (gmax + gmin)
    delta = (gmax - gmin) / (gmax + gmin)
    # partial fractions of d prod (x + z)/(x + p) on [eps, 1]
    a = np.empty(n)
    for l in range(n):
        num = np.prod(zeros - poles[l])
        den = np.prod(np.delete(poles, l) - poles[l])
        a[l] = d * num / den
    a0 = d
    # map [eps, 1] -> [lo, hi]: r_hi(x) = hi^-1/2 r(x / hi)
    s = 1.0 / math.sqrt(hi)
    return a0 * s, a * hi * s, poles * hi, delta


def evaluate(a0, a, sigma, x):
    x = np.asarray(x, dtype=np.float64)
    return a0 + np.sum(np.asarray(a)[None] / (x[..., None] + np.asarray(sigma)[None]), axis=-1)


def rational_apply(apply_shifted_inverse, a0, a, sigma, b):
    """y = a0 b + sum_l a_l (A + sigma_l)^-1 b, with the shifted inverses supplied
    by the caller (a dense solve, or CG)."""
    y = a0 * b
    for al, sl in zip(a, sigma):
        y = y + al * apply_shifted_inverse(sl, b)
    return y


def binomial_series(p: float, apply_Z, b, tol=1e-14, max_terms=40):
    """(1 + Z)^p b = sum_j binom(p, j) Z^j b, summed until a term's norm falls
    below tol ||b||.  Returns (y, number of Z applications)."""
    y = b.copy()
    t = b.copy()
    coef = 1.0
    nb = np.linalg.norm(b)
    napply = 0
    for j in range(1, max_terms + 1):
        t = apply_Z(t)
        napply += 1
        coef *= (p - (j - 1)) / j
        term = coef * t
        y = y + term
        if np.linalg.norm(term) <= tol * nb:
            break
    return y, napply
