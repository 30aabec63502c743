"""Test-side helpers: lattice coordinates, plane waves, dense assembly,
gauge transformations.  Independent of both the oracle and the CUDA path."""
from __future__ import annotations

import numpy as np


def coords(dims) -> np.ndarray:
    """(V, 4) integer coordinates, x0 slowest, x3 fastest."""
    T, L1, L2, L3 = dims
    g = np.stack(np.meshgrid(np.arange(T), np.arange(L1), np.arange(L2), np.arange(L3), indexing="ij"), -1)
    return g.reshape(-1, 4)


def site_index(dims, c) -> np.ndarray:
    T, L1, L2, L3 = dims
    c = np.asarray(c)
    return c[..., 3] + L3 * (c[..., 2] + L2 * (c[..., 1] + L1 * c[..., 0]))


def shift(dims, mu, d=1) -> np.ndarray:
    """index of x + d*mu for every site x (periodic)."""
    c = coords(dims).copy()
    c[:, mu] = (c[:, mu] + d) % dims[mu]
    return site_index(dims, c)


def parity(dims) -> np.ndarray:
    return coords(dims).sum(axis=1) % 2


def even_odd_sites(dims):
    p = parity(dims)
    return np.nonzero(p == 0)[0], np.nonzero(p == 1)[0]


def relerr(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    d = np.linalg.norm((a - b).ravel())
    n = np.linalg.norm(b.ravel())
    return d / n if n > 0 else d


def dense(apply, n_sites: int) -> np.ndarray:
    """Dense matrix of a linear map on spinor fields of n_sites sites."""
    N = 12 * n_sites
    M = np.empty((N, N), dtype=np.complex128)
    e = np.zeros(N, dtype=np.complex128)
    for j in range(N):
        e[:] = 0
        e[j] = 1
        M[:, j] = np.asarray(apply(e.reshape(n_sites, 4, 3))).ravel()
    return M


def gauge_transform(dims, U, g):
    """U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag."""
    Ug = np.empty_like(U)
    for mu in range(4):
        xp = shift(dims, mu, +1)
        Ug[:, mu] = g @ U[:, mu] @ g[xp].conj().transpose(0, 2, 1)
    return Ug


def colour_rotate(g, psi):
    """(g psi)(x) = g(x) psi(x) on colour."""
    return np.einsum("xab,xsb->xsa", g, psi)


def plaquette(dims, U) -> float:
    """(1/3) Re tr of the 1x1 Wilson loop, averaged over sites and the 6 planes."""
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            xpm = shift(dims, mu, 1)
            xpn = shift(dims, nu, 1)
            P = U[:, mu] @ U[xpm, nu] @ U[xpn, mu].conj().transpose(0, 2, 1) @ U[:, nu].conj().transpose(0, 2, 1)
            tot += np.trace(P, axis1=1, axis2=2).real.mean() / 3.0
    return tot / 6.0


def rng_spinor(n, seed):
    from paper_1011_0911_gb300 import synth
    return synth.gaussian_spinor(n, seed)
