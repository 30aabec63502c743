"""Pins of the oracle's molecular-dynamics step (the HMC of Sec. 2): the Wilson
gauge action and its gradient against an independent numpy plaquette and
finite differences, free flow U(t) = exp(tP) U when the action vanishes,
reversibility of the leapfrog, and its second-order energy error."""
import numpy as np
import pytest

pytest.importorskip("scipy.linalg")

import oracle as orc
from paper_1011_0911_gb300 import synth
from tests import util

DIMS = (2, 2, 2, 2)
KAPPA, CSW, BETA = 0.1355, 1.9, 5.3


def momenta(V, seed):
    return np.random.default_rng(seed).standard_normal((V, 4, 8))


def test_gauge_action_and_gradient():
    dims = (4, 2, 2, 2)
    U = synth.su3_links(dims, 0)
    o = orc.Oracle(dims, U, KAPPA, CSW)
    V = o.V

    def S(Uq):
        return BETA * 6 * V * (1.0 - util.plaquette(dims, Uq))

    assert abs(o.gauge_action(BETA) - S(U)) <= 1e-12 * S(U)
    from scipy.linalg import expm
    g = o.grad_gauge(BETA)
    eps = 1e-5
    for x, mu, a in [(0, 0, 0), (V - 1, 3, 7), (5, 1, 4), (9, 2, 2)]:
        up, um = U.copy(), U.copy()
        up[x, mu] = expm(eps * orc.GENERATORS[a]) @ U[x, mu]
        um[x, mu] = expm(-eps * orc.GENERATORS[a]) @ U[x, mu]
        ref = (S(up) - S(um)) / (2 * eps)
        assert abs(g[x, mu, a] - ref) <= 1e-7 * max(1.0, abs(ref))


def test_free_flow_when_the_action_vanishes():
    """beta = 0, c_sw = 0 and phi = 0: no force, so n steps give exp(n dt P) U."""
    from scipy.linalg import expm
    U = synth.su3_links(DIMS, 1)
    V = U.shape[0]
    p = momenta(V, 2)
    phi = np.zeros((V // 2, 4, 3), dtype=np.complex128)
    U1, p1 = orc.leapfrog(DIMS, U, p, phi, KAPPA, 0.0, 0.0, 0.1, 3)
    assert np.array_equal(p1, p)
    P = np.einsum("xma,aij->xmij", p, orc.GENERATORS)
    ref = np.array([[expm(0.3 * P[x, mu]) @ U[x, mu] for mu in range(4)] for x in range(V)])
    assert util.relerr(U1, ref) < 1e-13


def test_leapfrog_is_reversible():
    U = synth.su3_links(DIMS, 3)
    V = U.shape[0]
    p = momenta(V, 4)
    phi = synth.gaussian_spinor(V // 2, 5)
    U1, p1 = orc.leapfrog(DIMS, U, p, phi, KAPPA, CSW, BETA, 0.05, 3)
    assert util.relerr(U1, U) > 1e-3
    U2, p2 = orc.leapfrog(DIMS, U1, -p1, phi, KAPPA, CSW, BETA, 0.05, 3)
    assert util.relerr(U2, U) < 1e-10
    assert util.relerr(-p2, p) < 1e-10


def test_energy_error_is_second_order():
    """|dH| over a fixed trajectory falls about 4x when the step is halved."""
    U = synth.su3_links(DIMS, 6)
    V = U.shape[0]
    p = momenta(V, 7)
    phi = synth.gaussian_spinor(V // 2, 8)
    H0 = orc.hamiltonian(DIMS, U, p, phi, KAPPA, CSW, BETA)
    dH = []
    for dt, n in ((0.04, 5), (0.02, 10)):
        U1, p1 = orc.leapfrog(DIMS, U, p, phi, KAPPA, CSW, BETA, dt, n)
        dH.append(orc.hamiltonian(DIMS, U1, p1, phi, KAPPA, CSW, BETA) - H0)
    ratio = abs(dH[0]) / abs(dH[1])
    assert 3.0 < ratio < 5.0, (dH, ratio)
    assert abs(dH[1]) < 0.05
