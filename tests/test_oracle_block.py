"""Pins of the oracle's DD-HMC block solves (Sec. 3: the inversions on the
blocks for the block force use BiCGstab).  The block operator is checked
against the even-odd Schur complement of the dense Dirac matrix with every
entry coupling two different blocks removed (dense algebra, independent of the
matrix-free code), one block covering the lattice gives back the global Dhat,
and BiCGstab is checked against a dense solve, block by block."""
import numpy as np
import pytest

import oracle as orc
from paper_1011_0911_gb300 import synth
from tests import util

KAPPA, CSW = 0.1355, 1.9


def make(dims, seed=0):
    return orc.Oracle(dims, synth.su3_links(dims, seed), KAPPA, CSW)


def dense_block_dhat(o, dims, bs):
    """Schur complement of D restricted to the blocks (Dirichlet), even sites in rank order."""
    D = util.dense(o.D, o.V)
    c = util.coords(dims)
    blk = np.zeros(len(c), dtype=np.int64)
    for mu in range(4):
        blk = blk * (dims[mu] // bs[mu]) + c[:, mu] // bs[mu]
    same = blk[:, None] == blk[None, :]
    Db = D * np.kron(same, np.ones((12, 12)))
    ev, od = util.even_odd_sites(dims)
    ie = (12 * ev[:, None] + np.arange(12)[None]).ravel()
    io = (12 * od[:, None] + np.arange(12)[None]).ravel()
    Dee, Deo, Doe, Doo = Db[np.ix_(ie, ie)], Db[np.ix_(ie, io)], Db[np.ix_(io, ie)], Db[np.ix_(io, io)]
    return Dee - Deo @ np.linalg.solve(Doo, Doe), blk[ev]


@pytest.mark.parametrize("dims,bs", [((4, 4, 2, 2), (2, 2, 2, 2)), ((4, 2, 4, 2), (4, 2, 2, 2))],
                         ids=["2x2x1x1-blocks", "1x1x2x1-blocks"])
def test_block_dhat_is_dense_schur_of_masked_D(dims, bs):
    """Dirichlet blocks: hops leaving a block dropped; a block spanning a whole
    direction keeps the wrapped hop (the mask keeps every in-block entry)."""
    o = make(dims)
    ref, _ = dense_block_dhat(o, dims, bs)
    got = util.dense(lambda x: o.block_dhat(x, bs), o.Vh)
    assert util.relerr(got, ref) < 1e-13
    # it differs from the global Dhat (the blocks are really cut)
    assert util.relerr(got, util.dense(o.Dhat, o.Vh)) > 1e-3


def test_one_block_is_the_global_dhat():
    dims = (4, 4, 4, 2)
    o = make(dims, 1)
    x = synth.gaussian_spinor(o.Vh, 5)
    assert util.relerr(o.block_dhat(x, dims), o.Dhat(x)) < 1e-14


def test_bicgstab_solves_each_block():
    dims, bs = (4, 4, 2, 2), (2, 4, 2, 2)
    o = make(dims, 2)
    A, blk = dense_block_dhat(o, dims, bs)
    eta = synth.gaussian_spinor(o.Vh, 6)
    psi, st, its, rr = o.block_bicgstab(eta, bs, tol=1e-12, maxit=500)
    assert st == 0
    assert len(its) == o.nblocks(bs) == 2 and np.all(its > 0)
    assert np.all(rr <= 1e-12)
    ref = np.linalg.solve(A, eta.ravel())
    assert util.relerr(psi.ravel(), ref) < 1e-9
    # the residual of every block, from the dense operator
    r = (eta.ravel() - A @ psi.ravel()).reshape(o.Vh, 12)
    e = eta.reshape(o.Vh, 12)
    for b in range(2):
        assert np.linalg.norm(r[blk == b]) <= 1e-12 * np.linalg.norm(e[blk == b]) * 1.01


def test_blocks_are_independent_and_zero_sources():
    """A source on one block leaves the others at zero (zero iterations there)."""
    dims, bs = (4, 4, 2, 2), (2, 2, 2, 2)
    o = make(dims, 3)
    _, blk = dense_block_dhat(o, dims, bs)
    eta = synth.gaussian_spinor(o.Vh, 7)
    eta[blk != 1] = 0
    psi, st, its, rr = o.block_bicgstab(eta, bs, tol=1e-11)
    assert st == 0
    assert np.all(psi[blk != 1] == 0)
    assert np.all(its[np.arange(len(its)) != 1] == 0) and its[1] > 0
    assert rr[1] <= 1e-11


def test_iteration_limit_reported():
    dims, bs = (4, 4, 2, 2), (4, 4, 2, 2)
    o = make(dims, 4)
    eta = synth.gaussian_spinor(o.Vh, 8)
    psi, st, its, rr = o.block_bicgstab(eta, bs, tol=1e-14, maxit=3)
    assert st == 5 and its[0] == 3 and rr[0] > 1e-14
