"""ctypes front end of the plain FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and
by the benchmark's CPU-baseline leg, never by the product path.  Arrays are
numpy complex128 in the canonical layouts:
    full spinor  [V][4][3], even/odd spinor [V/2][4][3] (rank among the sites
    of that parity, lexicographic order), links [V][4][3][3].
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build_oracle

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = C.CDLL(path)
        P = C.c_void_p
        D = C.c_double
        I = C.c_int
        LG = C.c_long
        IP = C.POINTER(C.c_int)
        DP = C.POINTER(C.c_double)
        sig = {
            "or_create": (P, [I, I, I, I, I]),
            "or_destroy": (None, [P]),
            "or_set_gauge": (None, [P, P]),
            "or_set_params": (I, [P, D, D]),
            "or_gamma": (None, [I, P]),
            "or_fhat_site": (None, [P, LG, I, I, P]),
            "or_clover_site": (None, [P, LG, P]),
            "or_clover_inv_site": (None, [P, LG, P]),
            "or_logdet": (D, [P, I]),
            "or_hop": (None, [P, P, P]),
            "or_apply_clover": (None, [P, I, P, P]),
            "or_apply_D": (None, [P, P, P]),
            "or_apply_Dhat": (None, [P, P, P]),
            "or_apply_W": (None, [P, C.c_double, P, P]),
            "or_apply_Dhat_dag": (None, [P, P, P]),
            "or_apply_gamma5": (None, [LG, P, P]),
            "or_dhat_site": (None, [P, P, LG, P]),
            "or_d_site": (None, [P, P, LG, P]),
            "or_even_rank_to_site": (LG, [P, I, LG]),
            "or_cgnr": (I, [P, P, P, D, I, IP]),
            "or_sap": (None, [P, IP, I, I, P, P]),
            "or_sap_block_solve": (None, [P, IP, LG, I, P, P]),
            "or_gcr": (I, [P, I, IP, I, I, I, I, D, P, P, IP, DP]),
            "or_block_dhat": (None, [P, IP, P, P]),
            "or_dD_apply": (None, [P, LG, I, I, P, P]),
            "or_force_dD": (None, [P, P, P, P]),
            "or_force_logdet": (None, [P, I, P]),
            "or_gauge_action": (D, [P, D]),
            "or_grad_gauge": (None, [P, D, P]),
            "or_block_bicgstab": (I, [P, IP, P, P, D, I, IP, DP]),
            "or_dfl_build": (I, [P, IP, I, I, I, I, P]),
            "or_dfl_project": (None, [P, P, P]),
            "or_dfl_expand": (None, [P, P, P]),
            "or_dfl_little": (None, [P, P]),
            "or_dfl_little_apply": (None, [P, P, P]),
            "or_dfl_coarse_solve": (I, [P, P, P, D, I, I, IP]),
            "or_dfl_precond": (None, [P, IP, I, I, D, P, P]),
            "or_dfl_subspace": (None, [P, P]),
            "or_num_threads": (I, []),
            "or_ptc_transport": (None, [P, I, P, P]),
            "or_ptc_forward": (None, [P, I, IP, P, P, P, P]),
            "or_ptc_backward": (None, [P, I, IP, P, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def num_threads() -> int:
    """OpenMP threads used by the oracle's site loops."""
    return lib().or_num_threads()


def gamma(mu: int) -> np.ndarray:
    """gamma_mu (mu = 0..3) or gamma5 (mu = 4) of the oracle's chiral basis."""
    g = np.zeros((4, 4), dtype=np.complex128)
    lib().or_gamma(mu, _p(g))
    return g


def gamma5(x: np.ndarray) -> np.ndarray:
    x = _c(x)
    out = np.empty_like(x)
    lib().or_apply_gamma5(x.size // 12, _p(x), _p(out))
    return out


class Oracle:
    """One lattice with its gauge field and clover term (all FP64)."""

    def __init__(self, dims, U: np.ndarray, kappa: float, csw: float, antiperiodic_t: bool = True):
        self.dims = tuple(int(d) for d in dims)
        T, L1, L2, L3 = self.dims
        self.V = T * L1 * L2 * L3
        self.Vh = self.V // 2
        self._o = lib().or_create(T, L1, L2, L3, 1 if antiperiodic_t else 0)
        if not self._o:
            raise ValueError(f"bad lattice {dims}")
        self._U = _c(U).reshape(self.V, 4, 3, 3)
        lib().or_set_gauge(self._o, _p(self._U))
        self.status = lib().or_set_params(self._o, float(kappa), float(csw))
        self.kappa, self.csw = kappa, csw

    def __del__(self):
        if getattr(self, "_o", None):
            lib().or_destroy(self._o)
            self._o = None

    # ---- geometry
    def even_sites(self) -> np.ndarray:
        return np.array([lib().or_even_rank_to_site(self._o, 0, r) for r in range(self.Vh)])

    def odd_sites(self) -> np.ndarray:
        return np.array([lib().or_even_rank_to_site(self._o, 1, r) for r in range(self.Vh)])

    # ---- operators
    def _apply(self, fn, x, n):
        x = _c(x).reshape(n, 4, 3)
        out = np.empty_like(x)
        fn(self._o, _p(x), _p(out))
        return out

    def hop(self, x):
        return self._apply(lib().or_hop, x, self.V)

    def D(self, x):
        return self._apply(lib().or_apply_D, x, self.V)

    def Dhat(self, x):
        return self._apply(lib().or_apply_Dhat, x, self.Vh)

    def W(self, x, dm):
        """Hasenbusch operator W(dm) = Q_S + dm on an even field (Eq. 3)."""
        x = _c(x).reshape(self.Vh, 4, 3)
        out = np.empty_like(x)
        lib().or_apply_W(self._o, float(dm), _p(x), _p(out))
        return out

    def Dhat_dag(self, x):
        return self._apply(lib().or_apply_Dhat_dag, x, self.Vh)

    def clover(self, x, inverse=False):
        x = _c(x).reshape(self.V, 4, 3)
        out = np.empty_like(x)
        lib().or_apply_clover(self._o, 1 if inverse else 0, _p(x), _p(out))
        return out

    def clover_site(self, x: int, inverse=False) -> np.ndarray:
        A = np.empty((12, 12), dtype=np.complex128)
        (lib().or_clover_inv_site if inverse else lib().or_clover_site)(self._o, int(x), _p(A))
        return A

    def fhat_site(self, x: int, mu: int, nu: int) -> np.ndarray:
        F = np.empty((3, 3), dtype=np.complex128)
        lib().or_fhat_site(self._o, int(x), mu, nu, _p(F))
        return F

    def logdet(self, parity: int) -> float:
        return lib().or_logdet(self._o, parity)

    def dhat_site(self, x_e, re: int) -> np.ndarray:
        x_e = _c(x_e).reshape(self.Vh, 4, 3)
        out = np.empty((4, 3), dtype=np.complex128)
        lib().or_dhat_site(self._o, _p(x_e), int(re), _p(out))
        return out

    def d_site(self, x, site: int) -> np.ndarray:
        x = _c(x).reshape(self.V, 4, 3)
        out = np.empty((4, 3), dtype=np.complex128)
        lib().or_d_site(self._o, _p(x), int(site), _p(out))
        return out

    # ---- solvers
    def cgnr(self, eta_e, tol=1e-10, maxit=10000):
        eta_e = _c(eta_e).reshape(self.Vh, 4, 3)
        psi = np.empty_like(eta_e)
        it = C.c_int(0)
        st = lib().or_cgnr(self._o, _p(eta_e), _p(psi), tol, maxit, C.byref(it))
        return psi, st, it.value

    @staticmethod
    def _bs(bs):
        return (C.c_int * 4)(*[int(b) for b in bs])

    def sap(self, eta, bs=(4, 4, 4, 4), ncy=4, nmr=5):
        eta = _c(eta).reshape(self.V, 4, 3)
        psi = np.empty_like(eta)
        lib().or_sap(self._o, self._bs(bs), ncy, nmr, _p(eta), _p(psi))
        return psi

    def sap_block_solve(self, r, blk, bs=(4, 4, 4, 4), nmr=5):
        r = _c(r).reshape(self.V, 4, 3)
        chi = np.zeros_like(r)
        lib().or_sap_block_solve(self._o, self._bs(bs), int(blk), nmr, _p(r), _p(chi))
        return chi

    # ---- Lie derivatives and MD force gradients (Sec. 2, Eq. 4)
    # A link moves along U_mu(x) -> exp(eps T_a) U_mu(x), T_a = i lambda_a / 2; gradients
    # are dS/d eps in arrays [V][4][8] (the MD force is minus the gradient).
    def dD_apply(self, x, site, mu, a):
        """(dD/d eps) x for the link (site, mu) moved along T_a (full fields)."""
        x = _c(x).reshape(self.V, 4, 3)
        out = np.empty_like(x)
        lib().or_dD_apply(self._o, int(site), int(mu), int(a), _p(x), _p(out))
        return out

    def force_dD(self, X, Y):
        """Re <Y, (dD/d eps) X> for every link and generator."""
        X = _c(X).reshape(self.V, 4, 3)
        Y = _c(Y).reshape(self.V, 4, 3)
        g = np.empty((self.V, 4, 8))
        lib().or_force_dD(self._o, _p(X), _p(Y), _p(g))
        return g

    def grad_logdet(self, parity):
        """d log|det A_parity| / d eps (the clover term of Eq. 4 is -2 x this, summed over parities)."""
        g = np.empty((self.V, 4, 8))
        lib().or_force_logdet(self._o, int(parity), _p(g))
        return g

    def _full(self, xe, xo=None):
        f = np.zeros((self.V, 4, 3), dtype=np.complex128)
        f[self.even_sites()] = np.asarray(xe).reshape(self.Vh, 4, 3)
        if xo is not None:
            f[self.odd_sites()] = np.asarray(xo).reshape(self.Vh, 4, 3)
        return f

    def _g5(self, x):
        y = np.array(x, dtype=np.complex128, copy=True)
        y[..., 2:, :] *= -1
        return y

    def _complete_x(self, xe):
        """(x_e, -A_oo^-1 H_oe x_e): D of it is (Dhat x_e, 0)."""
        h = self.hop(self._full(xe))
        t = np.zeros_like(h)
        t[self.odd_sites()] = h[self.odd_sites()]
        xo = -self.clover(t, inverse=True)[self.odd_sites()]
        return self._full(xe, xo)

    def _complete_y(self, ye):
        """(y_e, -A_oo^-1 H_eo^dag y_e), with H^dag = gamma5 H gamma5: <y, dD x> = <y_e, dDhat x_e>."""
        h = self._g5(self.hop(self._g5(self._full(ye))))
        t = np.zeros_like(h)
        t[self.odd_sites()] = h[self.odd_sites()]
        yo = -self.clover(t, inverse=True)[self.odd_sites()]
        return self._full(ye, yo)

    def dhat_inv(self, eta_e, tol=1e-13):
        psi, st, _ = self.cgnr(eta_e, tol=tol, maxit=100000)
        assert st == 0
        return psi

    def grad_pf(self, phi_e):
        """d/d eps |Dhat^-1 phi_e|^2 = -2 Re <Y, dDhat X>, X = Dhat^-1 phi, Y = Dhat^-dag X."""
        xe = self.dhat_inv(phi_e)
        ye = self._g5(self.dhat_inv(self._g5(xe)))
        return -2.0 * self.force_dD(self._complete_x(xe), self._complete_y(ye))

    # W(dm) = A_ee^-1 Dhat + dm (Eq. 3) and its adjoint Dhat^dag A_ee^-1 + dm on even fields
    def _aee(self, xe, inverse=False):
        return self.clover(self._full(xe), inverse=inverse)[self.even_sites()]

    def _w_dag(self, xe, dm):
        return self._g5(self.Dhat(self._g5(self._aee(xe, inverse=True)))) + dm * np.asarray(xe).reshape(self.Vh, 4, 3)

    def w_inv(self, eta_e, dm, tol=1e-13, maxit=100000):
        """W(dm)^-1 eta by CG on W^dag W (plain, for the force pins)."""
        b = self._w_dag(eta_e, dm).ravel()
        x = np.zeros_like(b)
        r = b.copy()
        p = r.copy()
        rr = np.vdot(r, r).real
        b2 = rr
        for _ in range(maxit):
            if rr <= tol * tol * b2:
                break
            q = self._w_dag(self.W(p, dm), dm).ravel()
            al = rr / np.vdot(p, q).real
            x += al * p
            r -= al * q
            rn = np.vdot(r, r).real
            p = r + (rn / rr) * p
            rr = rn
        return x.reshape(self.Vh, 4, 3)

    def w_dag_inv(self, eta_e, dm):
        """W(dm)^-dag eta = W (W^dag W)^-1 eta, by CG on W^dag W (plain, for the force pins)."""
        b = np.asarray(eta_e, dtype=np.complex128).ravel()
        y = np.zeros_like(b)
        r = b.copy()
        p = r.copy()
        rr = np.vdot(r, r).real
        b2 = rr
        for _ in range(100000):
            if rr <= 1e-26 * b2:
                break
            q = self._w_dag(self.W(p, dm), dm).ravel()
            al = rr / np.vdot(p, q).real
            y += al * p
            r -= al * q
            rn = np.vdot(r, r).real
            p = r + (rn / rr) * p
            rr = rn
        return self.W(y.reshape(self.Vh, 4, 3), dm)

    def _grad_qs(self, u, z):
        """Re <z, dQ_S u> for even fields, Q_S = A_ee^-1 Dhat:
        dQ_S = A_ee^-1 (dDhat - dA_ee Q_S), so <z, dQ_S u> = <A_ee^-1 z, dDhat u> - <A_ee^-1 z, dA_ee Q_S u>."""
        zz = self._aee(z, inverse=True)
        v = self.W(u, 0.0)
        return (self.force_dD(self._complete_x(u), self._complete_y(zz))
                - self.force_dD(self._full(v), self._full(zz)))

    def grad_w1(self, phi_e, dm):
        """d/d eps |W(dm)^-1 phi|^2 (the F1 term of Eq. 4) = -2 Re <W^-dag X, dQ_S X>, X = W^-1 phi."""
        x = self.w_inv(phi_e, dm)
        return -2.0 * self._grad_qs(x, self.w_dag_inv(x, dm))

    def grad_w2(self, phi_e, dm):
        """d/d eps |(1 + dm / Q_S) phi|^2 (the F2 term of Eq. 4): with u = Q_S^-1 phi, v = W(dm) u,
        dv = -dm Q_S^-1 dQ_S u, so the gradient is -2 dm Re <Q_S^-dag v, dQ_S u>."""
        u = self.w_inv(phi_e, 0.0)
        v = self.W(u, dm)
        return -2.0 * dm * self._grad_qs(u, self.w_dag_inv(v, 0.0))

    def gauge_action(self, beta):
        """Wilson gauge action beta sum_P (1 - Re tr U_P / 3)."""
        return lib().or_gauge_action(self._o, float(beta))

    def grad_gauge(self, beta):
        g = np.empty((self.V, 4, 8))
        lib().or_grad_gauge(self._o, float(beta), _p(g))
        return g

    # ---- DD-HMC block solves (Sec. 3)
    def nblocks(self, bs):
        n = 1
        for L, b in zip(self.dims, bs):
            n *= L // b
        return n

    def block_dhat(self, x_e, bs):
        """Dhat_blk x_e on every Dirichlet block of extents bs (even half fields)."""
        x_e = _c(x_e).reshape(self.Vh, 4, 3)
        out = np.empty_like(x_e)
        lib().or_block_dhat(self._o, self._bs(bs), _p(x_e), _p(out))
        return out

    def block_bicgstab(self, eta_e, bs, tol=1e-10, maxit=1000):
        """BiCGstab on every block: (psi_e, status, iters[nblk], relres[nblk])."""
        eta_e = _c(eta_e).reshape(self.Vh, 4, 3)
        psi = np.empty_like(eta_e)
        nb = self.nblocks(bs)
        its = np.zeros(nb, dtype=np.int32)
        rr = np.zeros(nb)
        st = lib().or_block_bicgstab(self._o, self._bs(bs), _p(eta_e), _p(psi), tol, maxit,
                                     its.ctypes.data_as(C.POINTER(C.c_int)),
                                     rr.ctypes.data_as(C.POINTER(C.c_double)))
        return psi, st, its, rr

    def gcr(self, eta, precond=1, bs=(4, 4, 4, 4), ncy=4, nmr=5, nkv=16, nmx=2048, tol=1e-10):
        eta = _c(eta).reshape(self.V, 4, 3)
        psi = np.empty_like(eta)
        it = C.c_int(0)
        rr = C.c_double(0)
        st = lib().or_gcr(self._o, precond, self._bs(bs), ncy, nmr, nkv, nmx, tol, _p(eta), _p(psi),
                          C.byref(it), C.byref(rr))
        return psi, st, it.value, rr.value

    # ---- deflation
    def dfl_build(self, v0, bs=(4, 4, 4, 4), ninv=4, ncy=4, nmr=4):
        v0 = _c(v0)
        Ns = v0.size // (12 * self.V)
        self.Ns = Ns
        self.dfl_bs = tuple(bs)
        nb = 1
        for L, b in zip(self.dims, bs):
            nb *= L // b
        self.nblk = nb
        return lib().or_dfl_build(self._o, self._bs(bs), Ns, ninv, ncy, nmr, _p(v0))

    def dfl_subspace(self):
        out = np.empty((self.Ns, self.V, 4, 3), dtype=np.complex128)
        lib().or_dfl_subspace(self._o, _p(out))
        return out

    def dfl_project(self, x):
        x = _c(x).reshape(self.V, 4, 3)
        c = np.empty(self.nblk * self.Ns, dtype=np.complex128)
        lib().or_dfl_project(self._o, _p(x), _p(c))
        return c

    def dfl_expand(self, c):
        c = _c(c)
        out = np.empty((self.V, 4, 3), dtype=np.complex128)
        lib().or_dfl_expand(self._o, _p(c), _p(out))
        return out

    def dfl_little(self):
        N = self.nblk * self.Ns
        A = np.empty((N, N), dtype=np.complex128)
        lib().or_dfl_little(self._o, _p(A))
        return A

    def dfl_little_apply(self, c):
        c = _c(c)
        out = np.empty_like(c)
        lib().or_dfl_little_apply(self._o, _p(c), _p(out))
        return out

    def dfl_coarse_solve(self, b, tol=1e-8, nkv=16, nmx=4096):
        b = _c(b)
        x = np.empty_like(b)
        it = C.c_int(0)
        st = lib().or_dfl_coarse_solve(self._o, _p(b), _p(x), tol, nkv, nmx, C.byref(it))
        return x, st, it.value

    def dfl_precond(self, rho, bs=(4, 4, 4, 4), ncy=4, nmr=5, ctol=1e-8):
        rho = _c(rho).reshape(self.V, 4, 3)
        out = np.empty_like(rho)
        lib().or_dfl_precond(self._o, self._bs(bs), ncy, nmr, ctol, _p(rho), _p(out))
        return out


def chrono_guess(o: Oracle, xs, eta):
    """Chronological initial guess (Sec. 2, the method of Brower et al.):
    x0 = sum_i c_i x_i over the stored solutions x_i with c minimising
    |eta - Dhat x0|, solved here by a least-squares routine on the dense
    columns Dhat x_i.  Returns (x0, c)."""
    xs = [np.asarray(x, dtype=np.complex128).reshape(o.Vh, 4, 3) for x in xs]
    Y = np.stack([o.Dhat(x).ravel() for x in xs], axis=1)
    c = np.linalg.lstsq(Y, np.asarray(eta, dtype=np.complex128).ravel(), rcond=None)[0]
    x0 = sum(ci * x for ci, x in zip(c, xs))
    return x0, c


def ptc_weight_count(chans) -> int:
    """complex weights of a network with channel counts chans[0..nl]"""
    return sum(chans[l] * chans[l + 1] * 9 * 16 for l in range(len(chans) - 1))


def ptc_transport(o: Oracle, d: int, f: np.ndarray) -> np.ndarray:
    f = _c(f).reshape(o.V, 4, 3)
    out = np.empty_like(f)
    lib().or_ptc_transport(o._o, d, _p(f), _p(out))
    return out


def ptc_forward(o: Oracle, chans, W: np.ndarray, x: np.ndarray, keep_acts=False):
    """N(x) for input fields x [chans[0]][V][4][3]; weights W flat complex."""
    chans = [int(c) for c in chans]
    nl = len(chans) - 1
    ch = (C.c_int * len(chans))(*chans)
    W = _c(W)
    x = _c(x).reshape(chans[0], o.V, 4, 3)
    out = np.empty((chans[-1], o.V, 4, 3), dtype=np.complex128)
    acts = np.empty((sum(chans[:-1]), o.V, 4, 3), dtype=np.complex128) if keep_acts else None
    lib().or_ptc_forward(o._o, nl, ch, _p(W), _p(x), _p(out), _p(acts) if keep_acts else None)
    return (out, acts) if keep_acts else out


def ptc_backward(o: Oracle, chans, W: np.ndarray, acts: np.ndarray, gout: np.ndarray):
    """(dW, g_in) for the conjugate gradient gout at the output."""
    chans = [int(c) for c in chans]
    nl = len(chans) - 1
    ch = (C.c_int * len(chans))(*chans)
    W = _c(W)
    dW = np.empty_like(W)
    gout = _c(gout).reshape(chans[-1], o.V, 4, 3)
    gin = np.empty((chans[0], o.V, 4, 3), dtype=np.complex128)
    lib().or_ptc_backward(o._o, nl, ch, _p(W), _p(_c(acts)), _p(gout), _p(dW), _p(gin))
    return dW, gin


def even_odd_split(o: Oracle, x: np.ndarray):
    """(x_e, x_o) of a full field in the oracle's even/odd rank order."""
    x = np.asarray(x).reshape(o.V, 4, 3)
    return x[o.even_sites()], x[o.odd_sites()]


# ---------------------------------------------------------------- MD step
# The molecular-dynamics step of the two-flavour HMC (Sec. 2): links U, momenta
# p^a per link (P = sum_a p^a T_a, T_a = i lambda_a / 2, kinetic energy
# sum p^2 / 2), action S = S_g + |Dhat^-1 phi|^2 - 2 log|det A_oo| (the
# even-odd factorisation of det(D^dag D) with the clover term, Eq. 2 and 4).
# Equations of motion: dU/dt = P U, dp^a/dt = -dS/d eps_a.  Leapfrog (the
# paper's integrator): p -= dt/2 g, U <- exp(dt P) U, p -= dt/2 g.

def _gell_mann_T():
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return 0.5j * lam


GENERATORS = _gell_mann_T()


def md_action(dims, U, phi_e, kappa, csw, beta):
    o = Oracle(dims, U, kappa, csw)
    x = o.dhat_inv(phi_e)
    return o.gauge_action(beta) + float(np.vdot(x, x).real) - 2.0 * o.logdet(1)


def md_gradient(dims, U, phi_e, kappa, csw, beta):
    o = Oracle(dims, U, kappa, csw)
    return o.grad_gauge(beta) + o.grad_pf(phi_e) - 2.0 * o.grad_logdet(1)


def hamiltonian(dims, U, p, phi_e, kappa, csw, beta):
    return 0.5 * float(np.sum(p * p)) + md_action(dims, U, phi_e, kappa, csw, beta)


def _move_links(U, p, dt):
    from scipy.linalg import expm
    P = np.einsum("xma,aij->xmij", p, GENERATORS)
    V = np.empty_like(U)
    for x in range(U.shape[0]):
        for mu in range(4):
            V[x, mu] = expm(dt * P[x, mu]) @ U[x, mu]
    return V


def leapfrog(dims, U, p, phi_e, kappa, csw, beta, dt, nsteps):
    """nsteps leapfrog steps of size dt: returns (U, p)."""
    U = np.array(U, copy=True)
    p = np.array(p, dtype=np.float64, copy=True)
    for _ in range(nsteps):
        p -= 0.5 * dt * md_gradient(dims, U, phi_e, kappa, csw, beta)
        U = _move_links(U, p, dt)
        p -= 0.5 * dt * md_gradient(dims, U, phi_e, kappa, csw, beta)
    return U, p
