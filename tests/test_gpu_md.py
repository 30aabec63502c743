"""GPU molecular-dynamics forces and the leapfrog step (Sec. 2, Eq. 4) against
the oracle's link-by-link derivatives (themselves pinned by finite
differences, gauge covariance and the local force formulation in
test_oracle_force.py): Re <Y, dD X>, the clover log det gradient, the Wilson
gauge action and force, the pseudofermion force with its two solves, and two
leapfrog steps."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1011_0911_gb300 import lqcd, synth
from tests import util
from tests.gpu_util import Pair, to_gpu

pytestmark = pytest.mark.gpu

KAPPA, BETA = 0.1355, 5.3
DIMS = [(4, 2, 2, 2), (4, 4, 4, 2)]


def cpu(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("csw", [0.0, 1.9])
@pytest.mark.parametrize("dims", DIMS, ids=lambda d: "x".join(map(str, d)))
def test_force_dD(dims, csw):
    P = Pair(dims, kappa=KAPPA, csw=csw, seed=7)
    X, Y = synth.gaussian_spinor(P.V, 9), synth.gaussian_spinor(P.V, 10)
    g = cpu(P.ctx.force_dD(to_gpu(X), to_gpu(Y)))
    ref = P.o.force_dD(X, Y)
    assert util.relerr(g, ref) < 1e-12


@pytest.mark.parametrize("dims", DIMS, ids=lambda d: "x".join(map(str, d)))
def test_force_logdet(dims):
    P = Pair(dims, kappa=KAPPA, csw=1.9, seed=2)
    for parity in (0, 1):
        assert util.relerr(cpu(P.ctx.force_logdet(parity)), P.o.grad_logdet(parity)) < 1e-12
    Q = Pair(dims, kappa=KAPPA, csw=0.0, seed=2)
    assert torch.count_nonzero(Q.ctx.force_logdet(1)).item() == 0


@pytest.mark.parametrize("dims", DIMS, ids=lambda d: "x".join(map(str, d)))
def test_gauge_action_and_force(dims):
    P = Pair(dims, kappa=KAPPA, csw=1.9, seed=3)
    S = P.ctx.gauge_action(BETA)
    assert abs(S - P.o.gauge_action(BETA)) <= 1e-12 * abs(S)
    assert util.relerr(cpu(P.ctx.force_gauge(BETA)), P.o.grad_gauge(BETA)) < 1e-12


@pytest.mark.parametrize("dims", DIMS, ids=lambda d: "x".join(map(str, d)))
def test_force_pseudofermion(dims):
    P = Pair(dims, kappa=KAPPA, csw=1.9, seed=4)
    phi = synth.gaussian_spinor(P.Vh, 6)
    sp = P.ctx.md_solver(solver=lqcd.SOLVER_CGNR, tol=1e-13, nmx=100000)
    g, info = P.ctx.force_pf(to_gpu(phi), sp)
    assert all(i["status"] == 0 for i in info)
    assert util.relerr(cpu(g), P.o.grad_pf(phi)) < 1e-9


def test_force_dD_sampled_8x4():
    """8^4 (the workload lattice of the CGNR solve): sampled links and
    generators against the oracle's derivative of D applied link by link."""
    P = Pair((8, 8, 8, 8), kappa=KAPPA, csw=1.9, seed=5)
    X, Y = synth.gaussian_spinor(P.V, 11), synth.gaussian_spinor(P.V, 12)
    g = cpu(P.ctx.force_dD(to_gpu(X), to_gpu(Y)))
    rng = np.random.default_rng(3)
    samples = [(P.V - 1, 0, 3), (0, 0, 7), (17, 2, 4)]
    samples += [(int(rng.integers(P.V)), int(rng.integers(4)), int(rng.integers(8))) for _ in range(13)]
    for x, mu, a in samples:
        ref = np.vdot(Y, P.o.dD_apply(X, x, mu, a)).real
        assert abs(g[x, mu, a] - ref) <= 1e-12 * max(1.0, abs(ref)), (x, mu, a)


def test_md_gradient_and_leapfrog():
    """Two leapfrog steps of the HMC's MD on the GPU against the oracle's
    leapfrog (links moved by scipy's matrix exponential, exact solves)."""
    dims = (4, 2, 2, 2)
    P = Pair(dims, kappa=KAPPA, csw=1.9, seed=8)
    phi = synth.gaussian_spinor(P.Vh, 13)
    sp = P.ctx.md_solver(solver=lqcd.SOLVER_CGNR, tol=1e-13, nmx=100000)
    g, S = P.ctx.md_gradient(to_gpu(phi), BETA, sp)
    assert util.relerr(cpu(g), orc.md_gradient(dims, P.U, phi, KAPPA, 1.9, BETA)) < 1e-9
    assert abs(S - orc.md_action(dims, P.U, phi, KAPPA, 1.9, BETA)) <= 1e-9 * abs(S)
    p0 = np.random.default_rng(4).standard_normal((P.V, 4, 8))
    U = torch.from_numpy(P.U.copy()).cuda()
    p = torch.from_numpy(p0.copy()).cuda()
    P.ctx.md_leapfrog(U, p, to_gpu(phi), BETA, 0.02, 2, sp)
    Uref, pref = orc.leapfrog(dims, P.U, p0, phi, KAPPA, 1.9, BETA, 0.02, 2)
    assert util.relerr(cpu(U), Uref) < 1e-10
    assert util.relerr(cpu(p), pref) < 1e-10
    # the context now holds the evolved field
    o2 = orc.Oracle(dims, Uref, KAPPA, 1.9)
    x = synth.gaussian_spinor(P.Vh, 14)
    assert util.relerr(cpu(P.ctx.apply_Dhat(to_gpu(x))), o2.Dhat(x)) < 1e-12
