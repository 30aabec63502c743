"""Pins of the oracle's Lie derivatives for the molecular-dynamics forces
(Sec. 2, Eq. 4).  Every gradient is checked against central finite
differences of its action, evaluated by the oracle's operators and solvers on
gauge fields with one link moved to exp(+-eps T_a) U (scipy's matrix
exponential), so a dropped clover leaf, a wrong sign or adjoint, or a wrong
generator normalisation fails.  The force of the pseudofermion action is also
checked for gauge covariance, and the clover log det has no force at c_sw = 0."""
import numpy as np
import pytest

scipy_linalg = pytest.importorskip("scipy.linalg")

import oracle as orc
from paper_1011_0911_gb300 import synth
from tests import util

KAPPA, CSW, DM = 0.1355, 1.9, 0.09
EPS = 1e-5


def gell_mann():
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return 0.5j * lam   # T_a = i lambda_a / 2


T = gell_mann()


def moved(U, x, mu, a, eps):
    V = U.copy()
    V[x, mu] = scipy_linalg.expm(eps * T[a]) @ U[x, mu]
    return V


def fd(dims, U, x, mu, a, action, csw=CSW):
    sp = action(orc.Oracle(dims, moved(U, x, mu, a, +EPS), KAPPA, csw))
    sm = action(orc.Oracle(dims, moved(U, x, mu, a, -EPS), KAPPA, csw))
    return (sp - sm) / (2 * EPS)


def links_to_check(dims):
    """a few links: the time boundary, bulk links, every direction and generator"""
    V = int(np.prod(dims))
    rng = np.random.default_rng(5)
    out = [(V - 1, 0, 3), (0, 0, 7), (1, 3, 0)]
    for _ in range(5):
        out.append((int(rng.integers(V)), int(rng.integers(4)), int(rng.integers(8))))
    return out


DIMS = [(2, 2, 2, 2), (4, 2, 2, 2)]


@pytest.mark.parametrize("dims", DIMS)
def test_dD_is_the_derivative_of_D(dims):
    U = synth.su3_links(dims, 0)
    o = orc.Oracle(dims, U, KAPPA, CSW)
    X = synth.gaussian_spinor(o.V, 3)
    for x, mu, a in links_to_check(dims):
        Dp = orc.Oracle(dims, moved(U, x, mu, a, +EPS), KAPPA, CSW).D(X)
        Dm = orc.Oracle(dims, moved(U, x, mu, a, -EPS), KAPPA, CSW).D(X)
        assert util.relerr(o.dD_apply(X, x, mu, a), (Dp - Dm) / (2 * EPS)) < 1e-7


@pytest.mark.parametrize("dims", DIMS)
def test_force_dD_is_the_inner_product(dims):
    U = synth.su3_links(dims, 1)
    o = orc.Oracle(dims, U, KAPPA, CSW)
    X, Y = synth.gaussian_spinor(o.V, 4), synth.gaussian_spinor(o.V, 5)
    g = o.force_dD(X, Y)
    for x, mu, a in links_to_check(dims):
        ref = np.vdot(Y, o.dD_apply(X, x, mu, a)).real
        assert abs(g[x, mu, a] - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("parity", [0, 1])
def test_grad_logdet(parity):
    dims = (4, 2, 2, 2)
    U = synth.su3_links(dims, 2)
    o = orc.Oracle(dims, U, KAPPA, CSW)
    g = o.grad_logdet(parity)
    for x, mu, a in links_to_check(dims):
        ref = fd(dims, U, x, mu, a, lambda q: q.logdet(parity))
        assert abs(g[x, mu, a] - ref) <= 1e-7 * max(1.0, abs(ref))
    assert np.abs(g).max() > 1e-3


def test_no_clover_force_without_clover_term():
    dims = (2, 2, 2, 2)
    o = orc.Oracle(dims, synth.su3_links(dims, 3), KAPPA, 0.0)
    assert np.all(o.grad_logdet(0) == 0) and np.all(o.grad_logdet(1) == 0)


@pytest.mark.parametrize("dims", DIMS)
def test_grad_pseudofermion(dims):
    """S = |Dhat^-1 phi|^2."""
    U = synth.su3_links(dims, 4)
    o = orc.Oracle(dims, U, KAPPA, CSW)
    phi = synth.gaussian_spinor(o.Vh, 6)
    g = o.grad_pf(phi)

    def S(q):
        return float(np.vdot(q.dhat_inv(phi), q.dhat_inv(phi)).real)

    for x, mu, a in links_to_check(dims):
        ref = fd(dims, U, x, mu, a, S)
        assert abs(g[x, mu, a] - ref) <= 1e-6 * max(1.0, abs(ref))


def test_grad_hasenbusch_terms():
    """S1 = |W(dm)^-1 phi1|^2 and S2 = |(1 + dm / Q_S) phi2|^2 of Eq. 4."""
    dims = (4, 2, 2, 2)
    U = synth.su3_links(dims, 5)
    o = orc.Oracle(dims, U, KAPPA, CSW)
    p1, p2 = synth.gaussian_spinor(o.Vh, 7), synth.gaussian_spinor(o.Vh, 8)
    g1, g2 = o.grad_w1(p1, DM), o.grad_w2(p2, DM)

    def S1(q):
        x = q.w_inv(p1, DM)
        return float(np.vdot(x, x).real)

    def S2(q):
        v = q.W(q.w_inv(p2, 0.0), DM)
        return float(np.vdot(v, v).real)

    for x, mu, a in links_to_check(dims)[:5]:
        r1 = fd(dims, U, x, mu, a, S1)
        r2 = fd(dims, U, x, mu, a, S2)
        assert abs(g1[x, mu, a] - r1) <= 1e-6 * max(1.0, abs(r1))
        assert abs(g2[x, mu, a] - r2) <= 1e-6 * max(1.0, abs(r2))


def test_force_is_gauge_covariant():
    """M(x, mu) = sum_a g^a T_a transforms as g(x) M g(x)^dag when the links
    and the source are gauge transformed (the action is invariant)."""
    dims = (4, 2, 2, 2)
    U = synth.su3_links(dims, 6)
    o = orc.Oracle(dims, U, KAPPA, CSW)
    phi = synth.gaussian_spinor(o.Vh, 9)
    G = synth.random_su3(o.V, 11)
    og = orc.Oracle(dims, util.gauge_transform(dims, U, G), KAPPA, CSW)
    ev = o.even_sites()
    phig = util.colour_rotate(G[ev], phi.reshape(o.Vh, 4, 3))
    M = np.einsum("xma,aij->xmij", o.grad_pf(phi), T)
    Mg = np.einsum("xma,aij->xmij", og.grad_pf(phig), T)
    ref = np.einsum("xij,xmjk,xlk->xmil", G, M, G.conj())
    assert util.relerr(Mg, ref) < 1e-9
