"""GPU DD-HMC block solves (Sec. 3: BiCGstab on the Dirichlet blocks) against
the oracle: the block Schur operator per application, the solution of every
block, and at 48x24^3 with the paper's 6^2 x 12^2 blocks the residual of all
128 blocks recomputed by the oracle's own block operator."""
import numpy as np
import pytest
import torch

from paper_1011_0911_gb300 import lqcd, synth
from tests import util
from tests.gpu_util import Pair, relerr, to_gpu

pytestmark = pytest.mark.gpu


def block_ids(dims, bs):
    """block number of every even site (rank order), as the library numbers them"""
    ev, _ = util.even_odd_sites(dims)
    c = util.coords(dims)[ev]
    b = np.zeros(len(ev), dtype=np.int64)
    for mu in range(4):
        b = b * (dims[mu] // bs[mu]) + c[:, mu] // bs[mu]
    return b


@pytest.mark.parametrize("dims,bs", [((8, 8, 8, 8), (4, 4, 4, 4)), ((8, 4, 4, 8), (4, 4, 4, 4)),
                                     ((12, 8, 4, 4), (6, 4, 4, 2))],
                         ids=["8x8x8x8", "8x4x4x8-wrapping", "12x8x4x4-6x4x4x2"])
def test_block_dhat_parity(dims, bs):
    P = Pair(dims, kappa=0.1355)
    x = synth.gaussian_spinor(P.Vh, 11)
    got = P.ctx.apply_Dhat_block(to_gpu(x), bs)
    assert relerr(got, P.o.block_dhat(x, bs)) < 1e-13


def test_one_block_is_the_global_dhat():
    dims = (8, 4, 4, 8)
    P = Pair(dims)
    x = to_gpu(synth.gaussian_spinor(P.Vh, 12))
    a = P.ctx.apply_Dhat_block(x, dims)
    b = P.ctx.apply_Dhat(x, prec=lqcd.F64)
    assert util.relerr(a.cpu().numpy(), b.cpu().numpy()) < 1e-15


@pytest.mark.parametrize("dims,bs", [((8, 8, 8, 8), (4, 4, 4, 4)), ((12, 8, 4, 4), (6, 4, 4, 2))],
                         ids=["16-blocks", "odd-time-blocks"])
def test_block_solve_parity(dims, bs):
    """Same iteration per block as the oracle: solutions agree, every block's
    recomputed residual is below tol, iteration counts within one step."""
    P = Pair(dims, kappa=0.1355)
    eta = synth.gaussian_spinor(P.Vh, 13)
    psi, st, its, rr, sts = P.ctx.block_solve(to_gpu(eta), bs, tol=1e-10, nmx=500)
    ref, st_o, its_o, rr_o = P.o.block_bicgstab(eta, bs, tol=1e-10, maxit=500)
    assert st == 0 and st_o == 0 and np.all(sts == 0)
    assert len(its) == P.o.nblocks(bs)
    x = psi.cpu().numpy()
    assert util.relerr(x, ref) < 1e-8
    assert np.all(rr <= 1e-10) and np.all(np.abs(its - its_o) <= 1)
    # the residual per block from the oracle's operator
    r = (eta - P.o.block_dhat(x, bs)).reshape(P.Vh, 12)
    e = eta.reshape(P.Vh, 12)
    blk = block_ids(dims, bs)
    for b in range(len(its)):
        assert np.linalg.norm(r[blk == b]) <= 1.01e-10 * np.linalg.norm(e[blk == b])


def test_block_solve_edges():
    """Zero sources on some blocks (no steps there, psi = 0), an iteration limit
    that stops every block (status 5 per block), extents that do not tile."""
    dims, bs = (8, 8, 8, 8), (4, 4, 4, 4)
    P = Pair(dims, kappa=0.1355)
    blk = block_ids(dims, bs)
    eta = synth.gaussian_spinor(P.Vh, 14)
    eta[blk % 3 == 0] = 0
    psi, st, its, rr, sts = P.ctx.block_solve(to_gpu(eta), bs, tol=1e-10, nmx=500)
    assert st == 0
    x = psi.cpu().numpy()
    assert np.all(x[blk % 3 == 0] == 0)
    nb = len(its)
    assert np.all(its[np.arange(nb) % 3 == 0] == 0) and np.all(its[np.arange(nb) % 3 != 0] > 0)
    psi, st, its, rr, sts = P.ctx.block_solve(to_gpu(eta), bs, tol=1e-10, nmx=2, check=False)
    assert st == 5
    assert np.all(sts[np.arange(nb) % 3 != 0] == 5) and np.all(its[np.arange(nb) % 3 != 0] == 2)
    assert P.ctx.block_count((4, 4, 4, 3)) == -1
    with pytest.raises(lqcd.LqcdError):
        P.ctx.block_solve(to_gpu(eta), (4, 4, 6, 4))


def test_block_solve_48x24_paper_blocks():
    """The paper's DD-HMC blocks 6^2 x 12^2 on the 48x24^3 lattice (kappa =
    0.13625): all 128 blocks to 1e-10, the residual of each recomputed by the
    oracle's block operator."""
    dims, bs = (48, 24, 24, 24), (6, 6, 12, 12)
    U = synth.su3_links(dims, 0)
    P = Pair(dims, kappa=0.13625, U=U)
    eta = synth.gaussian_spinor(P.Vh, 15)
    psi, st, its, rr, sts = P.ctx.block_solve(to_gpu(eta), bs, tol=1e-10, nmx=1000)
    assert st == 0 and len(its) == 128
    x = psi.cpu().numpy()
    r = (eta - P.o.block_dhat(x, bs)).reshape(P.Vh, 12)
    e = eta.reshape(P.Vh, 12)
    blk = block_ids(dims, bs)
    nr = np.bincount(blk, weights=np.sum(np.abs(r) ** 2, axis=1), minlength=128)
    ne = np.bincount(blk, weights=np.sum(np.abs(e) ** 2, axis=1), minlength=128)
    assert np.all(np.sqrt(nr / ne) <= 1.01e-10)
