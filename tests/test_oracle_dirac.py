"""Pins of the CPU oracle's operators (Eq. 1 and Eq. 2) against facts that do
not come from the oracle itself: Clifford algebra, free-field closed forms,
gamma5-hermiticity, gauge covariance, closed forms of the clover term, library
determinants and inverses, and the Schur identities of Eq. 2 / Eq. 5."""
import numpy as np
import pytest

import oracle as orc
from paper_1011_0911_gb300 import synth
from tests import util

KAPPA, CSW = 0.1355, 1.9


def make(dims, U=None, kappa=KAPPA, csw=CSW, seed=0, antiperiodic=True):
    if U is None:
        U = synth.su3_links(dims, seed)
    return orc.Oracle(dims, U, kappa, csw, antiperiodic), U


# ---------------------------------------------------------------- gamma algebra

def test_gamma_clifford_algebra():
    g = [orc.gamma(mu) for mu in range(4)]
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2 * (mu == nu) * np.eye(4), atol=1e-15)
    g5 = orc.gamma(4)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]), atol=1e-15)
    assert np.allclose(g5, g[0] @ g[1] @ g[2] @ g[3], atol=1e-15)
    for mu in range(4):
        for nu in range(4):
            s = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
            assert np.allclose(s, s.conj().T)
            assert np.allclose(s @ g5, g5 @ s)  # chirality blocks


# ---------------------------------------------------------------- free field

def _plane_wave(dims, p, u):
    x = util.coords(dims)
    ph = np.exp(1j * (x @ np.asarray(p)))
    return ph[:, None, None] * u[None]


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 4)])
def test_free_field_plane_wave(dims):
    """Unit links: D e^{ipx} u = [m0 + sum(1-cos p) + i sum gamma sin p] e^{ipx} u,
    p_k = 2 pi n_k / L_k, p_0 = (2 n_0 + 1) pi / T (antiperiodic time)."""
    o, _ = make(dims, synth.unit_links(dims), csw=1.9)
    m0 = 1 / (2 * KAPPA) - 4
    g = [orc.gamma(mu) for mu in range(4)]
    rng = np.random.default_rng(1)
    for n in [(0, 0, 0, 0), (1, 1, 0, 1), (2, 3, 1, 0), (-1, 2, 1, 3)]:
        p = np.array([(2 * n[0] + 1) * np.pi / dims[0]] + [2 * np.pi * n[k] / dims[k] for k in (1, 2, 3)])
        M = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        psi = _plane_wave(dims, p, u)
        out = o.D(psi)
        expect = _plane_wave(dims, p, M @ u)
        assert util.relerr(out, expect) < 1e-14
        # basis-independent eigenvalues m0 + sum(1-cos p) +- i sqrt(sum sin^2 p), 6-fold each
        ev = np.linalg.eigvals(np.kron(M, np.eye(3)))
        a, b = m0 + np.sum(1 - np.cos(p)), np.sqrt(np.sum(np.sin(p) ** 2))
        assert np.allclose(ev.real, a, atol=1e-13)
        assert np.allclose(np.sort(ev.imag), [-b] * 6 + [b] * 6, atol=1e-13)


def test_free_field_dhat_closed_form():
    """Unit links: Dhat = (4+m0) - H_eo H_oe / (4+m0); on the even restriction of
    a plane wave H_eo H_oe acts as M_H(p)^2, M_H(p) = sum(-cos p + i gamma sin p)."""
    dims = (4, 4, 4, 4)
    o, _ = make(dims, synth.unit_links(dims))
    m0 = 1 / (2 * KAPPA) - 4
    g = [orc.gamma(mu) for mu in range(4)]
    ev, _ = util.even_odd_sites(dims)
    rng = np.random.default_rng(2)
    for n in [(0, 1, 0, 0), (1, 2, 3, 1)]:
        p = np.array([(2 * n[0] + 1) * np.pi / dims[0]] + [2 * np.pi * n[k] / dims[k] for k in (1, 2, 3)])
        MH = sum(-np.cos(p[mu]) * np.eye(4) + 1j * g[mu] * np.sin(p[mu]) for mu in range(4))
        Mhat = (4 + m0) * np.eye(4) - MH @ MH / (4 + m0)
        u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        psi_e = _plane_wave(dims, p, u)[ev]
        expect = _plane_wave(dims, p, Mhat @ u)[ev]
        assert util.relerr(o.Dhat(psi_e), expect) < 1e-14


# ---------------------------------------------------------------- structure

@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 4, 4, 4)])
def test_gamma5_hermiticity(dims):
    o, _ = make(dims)
    chi = synth.gaussian_spinor(o.V, 11)
    psi = synth.gaussian_spinor(o.V, 12)
    lhs = np.vdot(chi, o.D(psi))
    rhs = np.conj(np.vdot(psi, orc.gamma5(o.D(orc.gamma5(chi)))))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    ce, pe = chi[: o.Vh], psi[: o.Vh]
    lhs = np.vdot(ce, o.Dhat(pe))
    rhs = np.conj(np.vdot(pe, orc.gamma5(o.Dhat(orc.gamma5(ce)))))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # Dhat_dag is the adjoint of Dhat
    assert abs(np.vdot(ce, o.Dhat(pe)) - np.conj(np.vdot(pe, o.Dhat_dag(ce)))) < 1e-12 * abs(lhs)


def test_gauge_covariance():
    """D[U^g](g psi) = g D[U] psi and Fhat[U^g] = g Fhat[U] g^dag."""
    dims = (4, 4, 4, 4)
    o, U = make(dims)
    g = synth.random_su3(o.V, 77)
    Ug = util.gauge_transform(dims, U, g)
    og = orc.Oracle(dims, Ug, KAPPA, CSW)
    psi = synth.gaussian_spinor(o.V, 5)
    lhs = og.D(util.colour_rotate(g, psi))
    rhs = util.colour_rotate(g, o.D(psi))
    assert util.relerr(lhs, rhs) < 1e-13
    for x in (0, 17, 200):
        for mu, nu in ((0, 1), (2, 3), (3, 0)):
            F = o.fhat_site(x, mu, nu)
            Fg = og.fhat_site(x, mu, nu)
            assert np.allclose(Fg, g[x] @ F @ g[x].conj().T, atol=1e-13)
    # Dhat is covariant on the even sublattice
    ev, _ = util.even_odd_sites(dims)
    pe = psi[ev]
    lhs = og.Dhat(util.colour_rotate(g[ev], pe))
    rhs = util.colour_rotate(g[ev], o.Dhat(pe))
    assert util.relerr(lhs, rhs) < 1e-13


def test_eo_rank_order():
    dims = (4, 2, 4, 6)
    o, _ = make(dims)
    ev, od = util.even_odd_sites(dims)
    assert np.array_equal(o.even_sites(), ev)
    assert np.array_equal(o.odd_sites(), od)


# ---------------------------------------------------------------- clover term

def test_clover_unit_links_vanishes():
    dims = (4, 4, 4, 4)
    o, _ = make(dims, synth.unit_links(dims))
    m0 = 1 / (2 * KAPPA) - 4
    for x in (0, 5, 255):
        assert np.allclose(o.clover_site(x), (4 + m0) * np.eye(12), atol=1e-15)
        for mu in range(4):
            for nu in range(4):
                assert np.abs(o.fhat_site(x, mu, nu)).max() < 1e-15


def test_clover_structure_random_field():
    dims = (4, 4, 4, 4)
    o, _ = make(dims)
    for x in (0, 33, 254):
        A = o.clover_site(x)
        assert np.allclose(A, A.conj().T, atol=1e-14)
        assert np.abs(A[:6, 6:]).max() < 1e-15 and np.abs(A[6:, :6]).max() < 1e-15
        Ai = o.clover_site(x, inverse=True)
        assert np.abs(A @ Ai - np.eye(12)).max() < 1e-14
        for mu in range(4):
            for nu in range(4):
                F = o.fhat_site(x, mu, nu)
                assert np.allclose(F, -F.conj().T, atol=1e-15)
                assert np.allclose(F, -o.fhat_site(x, nu, mu), atol=1e-15)
    # log|det A| summed over each parity, against a library determinant
    ev, od = util.even_odd_sites(dims)
    for par, sites in ((0, ev), (1, od)):
        ld = sum(np.linalg.slogdet(o.clover_site(x))[1] for x in sites)
        assert abs(ld - o.logdet(par)) < 1e-10 * abs(ld)


def test_clover_single_link_closed_form():
    """Unit links except U_mu(x0) = W.  In the (mu,nu) plane the two plaquettes
    through the link are W (at x0) and W^dag (at x0-nu); transported to their
    corners they give Fhat_{mu nu} = (W - W^dag)/8 at x0+nu, x0+mu+nu,
    -(W - W^dag)/8 at x0-nu, x0+mu-nu, and 0 at x0, x0+mu (the two leaves cancel)
    and everywhere else."""
    dims = (4, 4, 4, 4)
    V = util.coords(dims).shape[0]
    W = synth.random_su3(1, 3)[0]
    x0c = np.array([1, 2, 0, 3])
    for mu in range(4):
        U = synth.unit_links(dims)
        x0 = util.site_index(dims, x0c)
        U[x0, mu] = W
        o, _ = make(dims, U)
        F0 = (W - W.conj().T) / 8
        for nu in range(4):
            if nu == mu:
                continue
            expect = {}
            def at(dmu, dnu):
                c = x0c.copy()
                c[mu] = (c[mu] + dmu) % 4
                c[nu] = (c[nu] + dnu) % 4
                return int(util.site_index(dims, c))
            expect[at(0, 1)] = F0
            expect[at(1, 1)] = F0
            expect[at(0, -1)] = -F0
            expect[at(1, -1)] = -F0
            for x in range(V):
                F = o.fhat_site(x, mu, nu)
                assert np.allclose(F, expect.get(x, np.zeros((3, 3))), atol=1e-15), (mu, nu, x)
            # planes without mu carry no field strength
            for a in range(4):
                for b in range(4):
                    if mu not in (a, b):
                        for x in (at(0, 1), at(1, -1), x0):
                            assert np.abs(o.fhat_site(x, a, b)).max() < 1e-15


def test_clover_constant_abelian_flux():
    """Constant flux phi = 2 pi / (T L1) in the (0,1) plane along T3 = diag(1,-1,0):
    every plaquette in that plane is exp(i phi T3), so Fhat_01 = i sin(phi) T3 and
    c_sw (i/4) sum sigma Fhat = -(c_sw/2) sin(phi) sigma_01 T3, whose eigenvalues
    are +-(c_sw/2) sin(phi) (4-fold each) and 0 (4-fold)."""
    dims = (4, 4, 2, 2)
    T, L1 = dims[0], dims[1]
    phi = 2 * np.pi / (T * L1)
    T3 = np.diag([1.0, -1.0, 0.0])
    x = util.coords(dims)
    U = synth.unit_links(dims)
    for s in range(len(x)):
        x0, x1 = x[s, 0], x[s, 1]
        U[s, 0] = np.diag(np.exp(-1j * phi * x1 * np.diag(T3)))
        if x1 == L1 - 1:
            U[s, 1] = np.diag(np.exp(1j * phi * L1 * x0 * np.diag(T3)))
    o, _ = make(dims, U, csw=1.9)
    m0 = 1 / (2 * KAPPA) - 4
    a = 1.9 / 2 * np.sin(phi)
    expect = np.sort(np.array([4 + m0 + a] * 4 + [4 + m0 - a] * 4 + [4 + m0] * 4))
    for s in (0, 7, 31, 63):
        assert np.allclose(o.fhat_site(s, 0, 1), 1j * np.sin(phi) * T3, atol=1e-15)
        ev = np.sort(np.linalg.eigvalsh(o.clover_site(s)))
        assert np.allclose(ev, expect, atol=1e-14)


def test_boundary_sign_is_a_hop_sign():
    """Folding the antiperiodic sign into the time links at x0 = T-1 and running
    periodic gives the same D; the clover term (closed loops) is unchanged."""
    dims = (4, 4, 2, 4)
    o, U = make(dims)
    Uf = U.copy()
    x = util.coords(dims)
    Uf[x[:, 0] == dims[0] - 1, 0] *= -1
    of = orc.Oracle(dims, Uf, KAPPA, CSW, antiperiodic_t=False)
    psi = synth.gaussian_spinor(o.V, 9)
    assert util.relerr(of.D(psi), o.D(psi)) < 1e-14
    for s in (0, 40, 127):
        assert np.allclose(of.clover_site(s), o.clover_site(s), atol=1e-14)
    # and the sign matters: periodic without folding differs
    op = orc.Oracle(dims, U, KAPPA, CSW, antiperiodic_t=False)
    assert util.relerr(op.D(psi), o.D(psi)) > 1e-3


def _abelian_flux_links(dims):
    T, L1 = dims[0], dims[1]
    phi = 2 * np.pi / (T * L1)
    t3 = np.array([1.0, -1.0, 0.0])
    x = util.coords(dims)
    U = synth.unit_links(dims)
    for s in range(len(x)):
        U[s, 0] = np.diag(np.exp(-1j * phi * x[s, 1] * t3))
        if x[s, 1] == L1 - 1:
            U[s, 1] = np.diag(np.exp(1j * phi * L1 * x[s, 0] * t3))
    return U, phi


def test_singular_clover_reported():
    """With the constant abelian flux the clover eigenvalue 4 + m0 - (c_sw/2) sin(phi)
    vanishes for c_sw = 2 (4+m0) / sin(phi): the inversion must report it."""
    dims = (4, 4, 2, 2)
    U, phi = _abelian_flux_links(dims)
    csw = 2 * (1 / (2 * KAPPA)) / np.sin(phi)
    o = orc.Oracle(dims, U, KAPPA, csw)
    assert o.status == 4
    o2 = orc.Oracle(dims, U, KAPPA, 0.9 * csw)
    assert o2.status == 0


# ---------------------------------------------------------------- dense checks

@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_schur_identities_dense(dims):
    """(D^-1)_ee = Dhat^-1 (Eq. 5) and log|det D| = log|det A_oo| + log|det Dhat| (Eq. 2)."""
    o, _ = make(dims)
    ev, od = util.even_odd_sites(dims)
    D = util.dense(o.D, o.V)
    Dh = util.dense(o.Dhat, o.Vh)
    idx_e = (12 * ev[:, None] + np.arange(12)[None]).ravel()
    Dinv = np.linalg.inv(D)
    assert util.relerr(Dinv[np.ix_(idx_e, idx_e)], np.linalg.inv(Dh)) < 1e-12
    ld_D = np.linalg.slogdet(D)[1]
    ld_h = np.linalg.slogdet(Dh)[1]
    assert abs(ld_D - (o.logdet(1) + ld_h)) < 1e-9 * abs(ld_D)
    # the dense D is the matrix-free D; gamma5 D is Hermitian
    g5 = np.kron(np.eye(o.V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    assert np.abs(g5 @ D - (g5 @ D).conj().T).max() < 1e-13


def test_dense_d_hops_only_nearest_neighbours():
    """Brute-force structure on 4^4: the block of D coupling x to y is non-zero
    only for y = x or y = x +- mu, and equals -1/2 (1 -+ gamma_mu) (x) U."""
    dims = (4, 4, 4, 4)
    o, U = make(dims)
    D = util.dense(o.D, o.V)
    g = [orc.gamma(mu) for mu in range(4)]
    x = 37
    c = util.coords(dims)[x]
    nz = set(np.nonzero(np.abs(D[12 * x:12 * x + 12]).reshape(12, o.V, 12).max(axis=(0, 2)))[0])
    nb = {x}
    for mu in range(4):
        for d in (1, -1):
            cc = c.copy()
            cc[mu] = (cc[mu] + d) % 4
            y = int(util.site_index(dims, cc))
            nb.add(y)
            blk = D[12 * x:12 * x + 12, 12 * y:12 * y + 12]
            sign = -1.0 if (mu == 0 and ((d == 1 and c[0] == 3) or (d == -1 and c[0] == 0))) else 1.0
            if d == 1:
                expect = -0.5 * sign * np.kron(np.eye(4) - g[mu], U[x, mu])
            else:
                expect = -0.5 * sign * np.kron(np.eye(4) + g[mu], U[y, mu].conj().T)
            assert np.allclose(blk, expect, atol=1e-15)
    assert nz == nb


def test_dhat_site_sampler_matches_full():
    dims = (4, 4, 4, 4)
    o, _ = make(dims)
    pe = synth.gaussian_spinor(o.Vh, 3)
    full = o.Dhat(pe)
    for r in (0, 1, 50, 127):
        assert np.allclose(o.dhat_site(pe, r), full[r], atol=1e-13)
    psi = synth.gaussian_spinor(o.V, 4)
    fullD = o.D(psi)
    for s in (0, 99, 255):
        assert np.allclose(o.d_site(psi, s), fullD[s], atol=1e-13)


# ---------------------------------------------------------------- generator

def test_generator_links_su3_and_plaquette():
    """For independent links with a conjugation-invariant law E[U] = c 1, so the
    mean plaquette is c^4 = 0.55 (Table 2: <U_P>/3 ~ 0.5504)."""
    dims = (8, 8, 8, 8)
    U = synth.su3_links(dims, 0)
    u = U.reshape(-1, 3, 3)
    assert np.abs(u @ u.conj().transpose(0, 2, 1) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(u) - 1).max() < 1e-14
    P = util.plaquette(dims, U)
    # 6 V = 24576 plaquettes, per-plaquette std ~0.2 -> statistical error ~0.002
    assert abs(P - 0.55) < 0.01
