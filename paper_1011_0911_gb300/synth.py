"""Seeded synthetic inputs: gauge links, Gaussian spinor sources, random
gauge transformations.

This module is the ONE piece shared by the CUDA path's callers and the CPU
oracle's tests.  It holds none of the solver's arithmetic (no Dirac operator,
no clover term, no plaquette): it only turns a seed into arrays.

Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), written here from its published
definition and checked against the published known-answer vectors.  Gaussian
variates use the Box-Muller transform.

Links follow the synthetic-field recipe of the benchmark workloads: U = exp(i eps H)
with H = sum_a h_a lambda_a / 2, h_a ~ N(0,1), lambda_a the Gell-Mann
matrices.  The distribution of H is invariant under conjugation, so
E[U] = c 1 with c = E[(1/3) Re tr U], and for independent links the mean
plaquette is c^4.  eps is therefore tuned (by bisection on a fixed sample) so
that c^4 = 0.55, the normalised average plaquette <U_P>/3 ~ 1.651/3 of Table 2.
"""
from __future__ import annotations

import functools
import os

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)

# stream identifiers (second key word) for the different kinds of input
STREAM_LINKS = 1
STREAM_SOURCE = 2
STREAM_GAUGE_TRANSFORM = 3
STREAM_EPS_SAMPLE = 4
STREAM_SUBSPACE = 5
STREAM_NET = 6


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32 with 10 rounds.  ctr: (N, 4) uint32, key: two uint32 words."""
    c = [ctr[:, i].astype(np.uint64) for i in range(4)]
    k0 = np.uint32(key[0])
    k1 = np.uint32(key[1])
    for r in range(10):
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
        if r < 9:
            k0 = np.uint32((int(k0) + int(_W0)) & 0xFFFFFFFF)
            k1 = np.uint32((int(k1) + int(_W1)) & 0xFFFFFFFF)
    return np.stack(c, axis=1).astype(np.uint32)


def uniforms(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniform doubles in (0, 1) with 53 random bits, two per Philox block."""
    nblk = (n + 1) // 2
    ctr = np.zeros((nblk, 4), dtype=np.uint32)
    idx = np.arange(offset, offset + nblk, dtype=np.uint64)
    ctr[:, 0] = (idx & _MASK).astype(np.uint32)
    ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
    w = philox4x32_10(ctr, (seed & 0xFFFFFFFF, stream & 0xFFFFFFFF)).astype(np.uint64)
    a = ((w[:, 0] >> np.uint64(5)) << np.uint64(26)) | (w[:, 1] >> np.uint64(6))
    b = ((w[:, 2] >> np.uint64(5)) << np.uint64(26)) | (w[:, 3] >> np.uint64(6))
    u = np.empty(2 * nblk, dtype=np.float64)
    u[0::2] = (a.astype(np.float64) + 0.5) / 2.0**53
    u[1::2] = (b.astype(np.float64) + 0.5) / 2.0**53
    return u[:n]


def gaussians(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal doubles (Box-Muller on pairs of uniforms)."""
    m = n + (n % 2)
    u = uniforms(seed, stream, m)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    t = 2.0 * np.pi * u[1::2]
    g = np.empty(m)
    g[0::2] = r * np.cos(t)
    g[1::2] = r * np.sin(t)
    return g[:n]


def gell_mann() -> np.ndarray:
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3.0)
    return lam


def _hermitian_from_normals(h: np.ndarray) -> np.ndarray:
    """H = sum_a h_a lambda_a / 2 for h of shape (N, 8)."""
    return np.einsum("na,aij->nij", h, gell_mann()) * 0.5


def _expi(H: np.ndarray, eps: float) -> np.ndarray:
    """exp(i eps H) for Hermitian traceless H (N,3,3): scaling and squaring of a
    Taylor series, then the rows are re-orthonormalised and the third row set to
    the conjugate cross product of the first two (exact SU(3) structure)."""
    X = 1j * eps * H
    nrm = np.abs(X).sum(axis=2).max() if X.shape[0] else 0.0
    s = max(0, int(np.ceil(np.log2(max(nrm, 1e-300) / 0.25))))
    X = X / (2.0**s)
    out = np.broadcast_to(np.eye(3, dtype=np.complex128), X.shape).copy()
    term = out.copy()
    for k in range(1, 13):
        term = term @ X / k
        out += term
    for _ in range(s):
        out = out @ out
    r0 = out[:, 0]
    r0 = r0 / np.sqrt((np.abs(r0) ** 2).sum(axis=1))[:, None]
    r1 = out[:, 1]
    r1 = r1 - (r0.conj() * r1).sum(axis=1)[:, None] * r0
    r1 = r1 / np.sqrt((np.abs(r1) ** 2).sum(axis=1))[:, None]
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=1)


@functools.lru_cache(maxsize=None)
def tuned_eps(target_plaquette: float = 0.55, nsample: int = 1 << 16) -> float:
    """eps such that c(eps)^4 = target, c = E[(1/3) Re tr exp(i eps H)],
    estimated on a fixed sample of H from the eigenvalues of H."""
    h = gaussians(0x5EED, STREAM_EPS_SAMPLE, 8 * nsample).reshape(nsample, 8)
    w = np.linalg.eigvalsh(_hermitian_from_normals(h))
    target_c = target_plaquette ** 0.25

    def c_of(eps):
        return np.cos(eps * w).sum(axis=1).mean() / 3.0

    lo, hi = 0.0, 1.2
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if c_of(mid) > target_c:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def su3_links(dims, seed: int, eps: float | None = None, cache: bool = True) -> np.ndarray:
    """Gauge field U[site][mu][3][3] (complex128), site = x3 + L3*(x2 + L2*(x1 + L1*x0)).

    Deterministic in (dims, seed, eps); large fields are cached on disk under
    $LQCD_SYNTH_CACHE (default /tmp/lqcd_synth_cache) to skip regeneration."""
    T, L1, L2, L3 = dims
    V = T * L1 * L2 * L3
    if eps is None:
        eps = tuned_eps()
    path = None
    if cache and V >= 1 << 16:
        d = os.environ.get("LQCD_SYNTH_CACHE", "/tmp/lqcd_synth_cache")
        path = os.path.join(d, f"links_{T}x{L1}x{L2}x{L3}_s{seed}_e{eps:.17g}.npy")
        if os.path.exists(path):
            try:
                U = np.load(path)
                if U.shape == (V, 4, 3, 3):
                    return U
            except (OSError, ValueError):
                pass
    n = 4 * V
    out = np.empty((n, 3, 3), dtype=np.complex128)
    chunk = 1 << 18
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        # each link owns 8 normals: counters for link j start at 4*j (2 normals per counter)
        h = _gaussians_range(seed, STREAM_LINKS, 8 * s, 8 * e).reshape(e - s, 8)
        out[s:e] = _expi(_hermitian_from_normals(h), eps)
    U = out.reshape(V, 4, 3, 3)
    if path is not None:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".{os.getpid()}.tmp.npy"
            np.save(tmp, U)
            os.replace(tmp, path)
        except OSError:
            pass
    return U


def _gaussians_range(seed: int, stream: int, start: int, stop: int) -> np.ndarray:
    """Normals with global indices [start, stop) of the (seed, stream) sequence (start even)."""
    assert start % 2 == 0
    m = stop - start
    m += m % 2
    u = uniforms(seed, stream, m, offset=start // 2)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    t = 2.0 * np.pi * u[1::2]
    g = np.empty(m)
    g[0::2] = r * np.cos(t)
    g[1::2] = r * np.sin(t)
    return g[: stop - start]


def unit_links(dims) -> np.ndarray:
    T, L1, L2, L3 = dims
    V = T * L1 * L2 * L3
    return np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()


def gaussian_spinor(nsites: int, seed: int, stream: int = STREAM_SOURCE) -> np.ndarray:
    """Complex Gaussian spinor field [nsites][4][3], real and imaginary parts N(0,1)."""
    g = gaussians(seed, stream, 24 * nsites)
    return (g[0::2] + 1j * g[1::2]).reshape(nsites, 4, 3)


def random_su3(n: int, seed: int, stream: int = STREAM_GAUGE_TRANSFORM, eps: float = 2.0) -> np.ndarray:
    """n random SU(3) matrices exp(i eps H) (for gauge-covariance checks)."""
    h = gaussians(seed, stream, 8 * n).reshape(n, 8)
    return _expi(_hermitian_from_normals(h), eps)


def lattice_volume(dims) -> int:
    T, L1, L2, L3 = dims
    return T * L1 * L2 * L3
