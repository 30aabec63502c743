"""Pins of the oracle's Lie derivatives for the molecular-dynamics forces
(Sec. 2, Eq. 4).  Every gradient is checked against central finite
differences of its action, evaluated by the oracle's operators and solvers on
gauge fields with one link moved to exp(+-eps T_a) U (scipy's matrix
exponential), so a dropped clover leaf, a wrong sign or adjoint, or a wrong
generator normalisation fails.  The force of the pseudofermion action is also
checked for gauge covariance, the clover log det has no force at c_sw = 0, and
the link-by-link derivative equals the local formulation of the force (spin-
summed outer products for the hops, staples through every clover leaf)."""
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


def gammas():
    s = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    z = np.zeros((2, 2))
    g = [np.block([[z, -np.eye(2)], [-np.eye(2), z]])]
    for k in range(3):
        g.append(np.block([[z, -1j * s[k]], [1j * s[k], z]]))
    return [np.asarray(m, dtype=np.complex128) for m in g]


def force_local(dims, U, X, Y, csw, bc_t=-1.0):
    """Re <Y, dD X> per link and generator from local colour matrices: the two
    hops give M = -1/2 s_f U B1 + 1/2 s_b B2 U^dag (B1, B2 spin-summed outer
    products of the projected X with Y), and every clover leaf through the
    link gives (c_sw / 8) U B Om A (or -B Om A U^dag for an adjoint factor),
    Om = Lam - Lam^dag, Lam = (i/4) sum sigma X Y^dag; the gradient is Re tr(T_a M)."""
    V = U.shape[0]
    c = util.coords(dims)
    G = gammas()
    one = np.eye(4)
    M = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    X, Y = X.reshape(V, 4, 3), Y.reshape(V, 4, 3)
    fw = [util.shift(dims, m, +1) for m in range(4)]
    bw = [util.shift(dims, m, -1) for m in range(4)]
    for x in range(V):
        for mu in range(4):
            y = fw[mu][x]
            sf = bc_t if (mu == 0 and c[x, 0] == dims[0] - 1) else 1.0
            sb = bc_t if (mu == 0 and c[y, 0] == 0) else 1.0
            a = (one - G[mu]) @ X[y]
            b = (one + G[mu]) @ X[x]
            B1 = np.einsum("sk,si->ki", a, Y[x].conj())
            B2 = np.einsum("sk,si->ki", b, Y[y].conj())
            M[x, mu] += -0.5 * sf * U[x, mu] @ B1 + 0.5 * sb * B2 @ U[x, mu].conj().T
    for yy in range(V):
        for mu in range(4):
            for nu in range(4):
                if mu == nu:
                    continue
                sig = 0.5j * (G[mu] @ G[nu] - G[nu] @ G[mu])
                lam = 0.25j * np.einsum("ab,bk,ai->ki", sig, X[yy], Y[yy].conj())
                om = lam - lam.conj().T
                pm, pn, mm, mn = fw[mu][yy], fw[nu][yy], bw[mu][yy], bw[nu][yy]
                leaves = [[(yy, mu, 0), (pm, nu, 0), (pn, mu, 1), (yy, nu, 1)],
                          [(yy, nu, 0), (fw[nu][mm], mu, 1), (mm, nu, 1), (mm, mu, 0)],
                          [(mm, mu, 1), (bw[nu][mm], nu, 1), (bw[nu][mm], mu, 0), (mn, nu, 0)],
                          [(mn, nu, 1), (mn, mu, 0), (fw[mu][mn], nu, 0), (yy, mu, 1)]]
                for leaf in leaves:
                    f = [U[s, d].conj().T if dg else U[s, d] for s, d, dg in leaf]
                    for i, (s, d, dg) in enumerate(leaf):
                        A = np.eye(3, dtype=np.complex128)
                        for k in range(i):
                            A = A @ f[k]
                        B = np.eye(3, dtype=np.complex128)
                        for k in range(i + 1, 4):
                            B = B @ f[k]
                        if dg:
                            M[s, d] += -(csw / 8.0) * B @ om @ A @ U[s, d].conj().T
                        else:
                            M[s, d] += (csw / 8.0) * U[s, d] @ B @ om @ A
    return np.einsum("aij,xmji->xma", T, M).real


@pytest.mark.parametrize("dims", DIMS)
def test_force_from_local_outer_products_and_staples(dims):
    """The local formulation of the force (the one a per-link kernel uses)
    equals the oracle's link-by-link derivative of D."""
    U = synth.su3_links(dims, 7)
    o = orc.Oracle(dims, U, KAPPA, CSW)
    X, Y = synth.gaussian_spinor(o.V, 9), synth.gaussian_spinor(o.V, 10)
    assert util.relerr(force_local(dims, U, X, Y, CSW), o.force_dD(X, Y)) < 1e-12
