"""GPU parity of the Hasenbusch operator W(dm) = Q_S + dm (Eq. 3) against the
oracle, and its solves (the pseudofermion solve of Eq. 4) to a true FP64
W-residual of 1e-10; the clover term of D is unchanged afterwards."""
import numpy as np
import pytest
import torch

from paper_1011_0911_gb300 import lqcd, synth
from tests import util
from tests.gpu_util import TOL, Pair, relerr, rounded, to_gpu

pytestmark = pytest.mark.gpu

DM = 0.09   # the mass shift of Sec. 2


@pytest.fixture(scope="module")
def pair():
    return Pair((8, 8, 8, 8))


@pytest.mark.parametrize("prec", [lqcd.F64, lqcd.F32], ids=["f64", "f32"])
@pytest.mark.parametrize("dm", [0.0, DM])
def test_apply_W(pair, prec, dm):
    P = pair
    x = rounded(synth.gaussian_spinor(2 * P.Vh, 31).reshape(2, P.Vh, 4, 3), prec)
    out = P.ctx.apply_W(to_gpu(x, prec), dm, prec)
    for k in range(2):
        assert relerr(out[k], P.o.W(x[k], dm)) < TOL[prec]


@pytest.mark.parametrize("solver", [lqcd.SOLVER_SAP_GCR, lqcd.SOLVER_CGNR], ids=["sap_gcr", "cgnr"])
def test_solve_W(pair, solver):
    P = pair
    eta = synth.gaussian_spinor(2 * P.Vh, 32).reshape(2, P.Vh, 4, 3)
    psi, info, st = P.ctx.solve_W(to_gpu(eta), DM, solver=solver, tol=1e-10, nmx=20000)
    assert st == 0
    x = psi.cpu().numpy()
    for k in range(2):
        assert util.relerr(P.o.W(x[k], DM), eta[k]) <= 1e-10
        assert info[k]["relres_dhat"] <= 1e-10
    # D is restored: Dhat still matches the oracle
    pe = synth.gaussian_spinor(P.Vh, 33)
    assert relerr(P.ctx.apply_Dhat(to_gpu(pe)), P.o.Dhat(pe)) < TOL[lqcd.F64]


def test_solve_W_mixed_and_shift_helps(pair):
    """FP32 SAP inside the FP64 GCR reaches the same residual; the shifted
    operator needs fewer GCR steps than Dhat itself (the point of Eq. 3)."""
    P = pair
    eta = synth.gaussian_spinor(P.Vh, 34)
    _, iw, st = P.ctx.solve_W(to_gpu(eta), 0.5, tol=1e-10, sap_prec=lqcd.F32, inner=lqcd.F32)
    assert st == 0 and iw[0]["relres_dhat"] <= 1e-10
    _, i0, st0 = P.ctx.solve_dhat(to_gpu(eta), tol=1e-10, sap_prec=lqcd.F32, inner=lqcd.F32)
    assert st0 == 0
    assert iw[0]["iters"] < i0[0]["iters"]


def test_solve_W_rejects_deflated_solver(pair):
    with pytest.raises(lqcd.LqcdError):
        pair.ctx.solve_W(to_gpu(synth.gaussian_spinor(pair.Vh, 35)), DM, solver=lqcd.SOLVER_DFL_SAP_GCR)
