"""Seeded synthetic inputs: SU(3) gauge fields and complex-Gaussian spinors.

This module makes INPUTS only.  It holds none of the twisted-mass operator's
arithmetic (no hopping term, no clover term, no solver), so that both the CPU
oracle and the CUDA path can be fed the same fields without sharing any of the
method's code.

Recipe (the paper measures on ETMC ensembles that are not available here;
these seeded fields stand in for them):

* links      U_mu(x) = reunitarise(exp(i * eps * H)),  H = sum_a h_a lambda_a,
             h_a ~ N(0,1) i.i.d. per link, lambda_a the Gell-Mann matrices
             (tr lambda_a lambda_b = 2 delta_ab); eps = EPS_PLAQ_059 gives a mean
             plaquette of 0.590 for uncorrelated links.
* spinors    complex Gaussian, real and imaginary parts ~ N(0,1) i.i.d.
* generator  numpy's Philox counter-based bit generator, keyed by (seed, chunk).

Canonical host layouts (C order, complex128):
  gauge        [t][z][y][x][mu][3][3]            mu = 0:x 1:y 2:z 3:t
  full spinor  [t][z][y][x][spin 4][colour 3]
  odd spinor   [site_o][spin 4][colour 3]         site_o = lex // 2 over odd sites
  heavy spinor [site_o][flavour 2][spin 4][colour 3]
"""
from __future__ import annotations

import os

import numpy as np

# Calibrated so that the mean plaquette of independent links is 0.590 (see
# tests/test_synth.py); for uncorrelated links <P> = c^4 with c = <Re tr U>/3.
EPS_PLAQ_059 = 0.2197


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def gell_mann() -> np.ndarray:
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return lam


def reunitarise(u: np.ndarray) -> np.ndarray:
    """Project onto SU(3): Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1)."""
    u = np.array(u, dtype=np.complex128, copy=True)
    r0 = u[..., 0, :]
    r0 /= np.sqrt(np.sum(np.abs(r0) ** 2, axis=-1, keepdims=True))
    r1 = u[..., 1, :]
    r1 -= np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 /= np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1, keepdims=True))
    u[..., 0, :] = r0
    u[..., 1, :] = r1
    u[..., 2, :] = np.conj(np.cross(r0, r1))
    return u


def _expm_i(h: np.ndarray) -> np.ndarray:
    """exp(i h) for a stack of hermitian 3x3 matrices (scaling and squaring,
    Taylor series of order 14 on h/16)."""
    a = 1j * h / 16.0
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), a.shape)
    term = eye.copy()
    out = eye.copy()
    for n in range(1, 15):
        term = term @ a / n
        out = out + term
    for _ in range(4):
        out = out @ out
    return out


def random_su3(n: int, eps: float, gen: np.random.Generator) -> np.ndarray:
    """n links U = reunitarise(exp(i eps H)), H = sum_a h_a lambda_a, h_a ~ N(0,1)."""
    h = gen.standard_normal((n, 8))
    H = np.einsum("na,aij->nij", h, gell_mann())
    return reunitarise(_expm_i(eps * H))


_LINK_CHUNK = 1 << 18


def _link_chunk(args):
    """Links [c*_LINK_CHUNK, c*_LINK_CHUNK + n) from the generator keyed (seed, c)."""
    seed, c, n, eps = args
    gen = np.random.Generator(np.random.Philox(key=(int(seed) << 32) | int(c)))
    return random_su3(n, eps, gen)


def gauge_field(dims, seed: int, eps: float = EPS_PLAQ_059, workers: int | None = None) -> np.ndarray:
    """Canonical gauge field [t][z][y][x][mu][3][3] complex128.  dims = (X,Y,Z,T).

    Links are made in chunks of 2^18, chunk c from its own Philox stream keyed
    (seed, c), so the field does not depend on how many processes make it.
    Large fields use a spawn-context process pool (safe after CUDA is up)."""
    X, Y, Z, T = dims
    n = X * Y * Z * T * 4
    tasks = [(seed, c, min(_LINK_CHUNK, n - c * _LINK_CHUNK), eps)
             for c in range((n + _LINK_CHUNK - 1) // _LINK_CHUNK)]
    if workers is None:
        workers = min(len(tasks), os.cpu_count() or 1, 32)
    if workers > 1 and len(tasks) >= 8:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.map(_link_chunk, tasks, chunksize=1)
    else:
        parts = [_link_chunk(t) for t in tasks]
    return np.concatenate(parts).reshape(T, Z, Y, X, 4, 3, 3)


def unit_gauge(dims) -> np.ndarray:
    X, Y, Z, T = dims
    u = np.zeros((T, Z, Y, X, 4, 3, 3), dtype=np.complex128)
    u[..., :, :] = np.eye(3)
    return u


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """Site-local SU(3) matrices g(x), [t][z][y][x][3][3], far from unity."""
    X, Y, Z, T = dims
    g = random_su3(X * Y * Z * T, 1.5, rng(seed))
    return g.reshape(T, Z, Y, X, 3, 3)


def _roll_site(f: np.ndarray, mu: int, d: int) -> np.ndarray:
    """f(x + d*mu_hat) on the periodic torus, for a [t][z][y][x]... array."""
    return np.roll(f, -d, axis=3 - mu)


def gauge_transform_links(u: np.ndarray, g: np.ndarray) -> np.ndarray:
    """U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dagger."""
    out = np.empty_like(u)
    for mu in range(4):
        gp = _roll_site(g, mu, 1)
        out[..., mu, :, :] = g @ u[..., mu, :, :] @ np.conj(np.swapaxes(gp, -1, -2))
    return out


def pure_gauge(g: np.ndarray) -> np.ndarray:
    """U_mu(x) = g(x) g(x+mu)^dagger (zero field strength)."""
    T, Z, Y, X = g.shape[:4]
    return gauge_transform_links(unit_gauge((X, Y, Z, T)), g)


def abelian_flux(dims, mu: int, nu: int, n: int, charges=(1.0, -1.0, 0.0)) -> np.ndarray:
    """Constant U(1) flux in the (mu,nu) plane embedded as diag(e^{i q phi}) with
    integer charges q summing to zero (default (1,-1,0)): every plaquette in that plane carries the phase
    Phi = 2 pi n / (L_mu L_nu) (times q).  Uses the standard torus gauge:
      U_nu(x)  = exp(i q Phi x_mu)
      U_mu(x)  = exp(-i q Phi L_mu x_nu)  on x_mu = L_mu - 1, else 1."""
    X, Y, Z, T = dims
    L = [X, Y, Z, T]
    phi = 2 * np.pi * n / (L[mu] * L[nu])
    q = np.asarray(charges, dtype=np.float64)
    coords = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    xc = [coords[3], coords[2], coords[1], coords[0]]
    u = unit_gauge(dims)
    ph_nu = np.exp(1j * phi * xc[mu][..., None] * q)
    u[..., nu, :, :] = 0
    for c in range(3):
        u[..., nu, c, c] = ph_nu[..., c]
    edge = xc[mu] == L[mu] - 1
    ph_mu = np.where(edge[..., None], np.exp(-1j * phi * L[mu] * xc[nu][..., None] * q), 1.0)
    u[..., mu, :, :] = 0
    for c in range(3):
        u[..., mu, c, c] = ph_mu[..., c]
    return u


def plaquette(u: np.ndarray) -> float:
    """Mean plaquette (1/3) Re tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
    over all sites and the 6 planes (input calibration only)."""
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            a = u[..., mu, :, :]
            b = _roll_site(u[..., nu, :, :], mu, 1)
            c = np.conj(np.swapaxes(_roll_site(u[..., mu, :, :], nu, 1), -1, -2))
            d = np.conj(np.swapaxes(u[..., nu, :, :], -1, -2))
            tot += np.real(np.trace(a @ b @ c @ d, axis1=-2, axis2=-1)).mean() / 3.0
    return tot / 6.0


def spinor(shape, seed: int) -> np.ndarray:
    """Complex Gaussian field; re, im ~ N(0,1)."""
    gen = rng(seed)
    re = gen.standard_normal(shape)
    im = gen.standard_normal(shape)
    return re + 1j * im


def odd_spinor(dims, seed: int, nflavour: int = 1) -> np.ndarray:
    X, Y, Z, T = dims
    vh = X * Y * Z * T // 2
    shape = (vh, 4, 3) if nflavour == 1 else (vh, nflavour, 4, 3)
    return spinor(shape, seed)
