"""Pins of the oracle's Hasenbusch operator W(dm) = Q_S + dm (Eq. 3), with
Q_S = 1 - Q_ee^-1 Q_eo Q_oo^-1 Q_oe and Q = gamma5 D (Eq. 2), built from the
dense gamma5 D by block algebra (independent of the matrix-free code path):
the Schur factorisation of det Q (Eq. 2), the inverse identity
Q_S^-1 = P_e Q^-1 Q_ee P_e of Eq. 5, and linearity in dm."""
import numpy as np
import pytest

import oracle as orc
from paper_1011_0911_gb300 import synth
from tests import util

KAPPA, CSW = 0.1355, 1.9


def make(dims, seed=0):
    U = synth.su3_links(dims, seed)
    return orc.Oracle(dims, U, KAPPA, CSW)


def blocks(o, dims):
    """Dense Q = gamma5 D and its even / odd index sets (canonical site order)."""
    D = util.dense(o.D, o.V)
    g5 = np.kron(np.eye(o.V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    Q = g5 @ D
    ev, od = util.even_odd_sites(dims)
    ie = (12 * ev[:, None] + np.arange(12)[None]).ravel()
    io = (12 * od[:, None] + np.arange(12)[None]).ravel()
    return Q, ie, io


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 2)])
def test_W_is_the_block_formula(dims):
    o = make(dims)
    Q, ie, io = blocks(o, dims)
    Qee, Qeo, Qoe, Qoo = Q[np.ix_(ie, ie)], Q[np.ix_(ie, io)], Q[np.ix_(io, ie)], Q[np.ix_(io, io)]
    QS = np.eye(len(ie)) - np.linalg.solve(Qee, Qeo @ np.linalg.solve(Qoo, Qoe))
    for dm in (0.0, 0.09):
        W = util.dense(lambda x: o.W(x, dm), o.Vh)
        assert util.relerr(W, QS + dm * np.eye(len(ie))) < 1e-13


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 2)])
def test_det_factorisation_eq2(dims):
    """log|det Q| = log|det Q_ee| + log|det Q_oo| + log|det Q_S|, Q_S = W(0)."""
    o = make(dims)
    Q, ie, io = blocks(o, dims)
    W0 = util.dense(lambda x: o.W(x, 0.0), o.Vh)
    lhs = np.linalg.slogdet(Q)[1]
    rhs = (np.linalg.slogdet(Q[np.ix_(ie, ie)])[1] + np.linalg.slogdet(Q[np.ix_(io, io)])[1]
           + np.linalg.slogdet(W0)[1])
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    # the clover blocks give log|det Q_ee| (gamma5 has |det| = 1)
    assert abs(np.linalg.slogdet(Q[np.ix_(ie, ie)])[1] - o.logdet(0)) < 1e-10 * abs(o.logdet(0))


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 2)])
def test_inverse_identity_eq5(dims):
    """Q_S^-1 = P_e Q^-1 Q_ee P_e."""
    o = make(dims)
    Q, ie, io = blocks(o, dims)
    W0 = util.dense(lambda x: o.W(x, 0.0), o.Vh)
    rhs = np.linalg.inv(Q)[np.ix_(ie, ie)] @ Q[np.ix_(ie, ie)]
    assert util.relerr(np.linalg.inv(W0), rhs) < 1e-11


def test_linear_in_dm_and_free_field():
    o = make((4, 4, 4, 4))
    x = synth.gaussian_spinor(o.Vh, 3)
    a, b = o.W(x, 0.0), o.W(x, 0.25)
    assert util.relerr(b - a, 0.25 * x.reshape(a.shape)) < 1e-14
    # unit links, c_sw = 0: Q_S = 1 - H_eo H_oe / (4 + m0)^2, and on a constant
    # field H_eo H_oe = 4 (the two projectors (1 -+ g) add up to 2 per direction)
    dims = (4, 4, 4, 4)
    U = synth.unit_links(dims)
    of = orc.Oracle(dims, U, KAPPA, 0.0, antiperiodic_t=False)
    c = np.zeros((of.Vh, 4, 3), dtype=np.complex128)
    c[:, 0, 0] = 1.0
    m = 4 + (1 / (2 * KAPPA) - 4)
    assert util.relerr(of.W(c, 0.0), (1 - 16.0 / m ** 2) * c) < 1e-14
