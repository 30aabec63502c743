"""The chronological initial guess on the GPU against the oracle's
least-squares definition, and solves started from it: same 1e-10 true
residual, fewer GCR steps along a slowly varying sequence of sources."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1011_0911_gb300 import lqcd, synth
from tests import util
from tests.gpu_util import Pair, to_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pair():
    return Pair((8, 8, 8, 8))


def test_guess_matches_oracle(pair):
    P = pair
    xs = [synth.gaussian_spinor(P.Vh, 70 + i) for i in range(5)]
    eta = synth.gaussian_spinor(P.Vh, 80)
    P.ctx.chrono_reset(4)
    for x in xs:                      # ring of 4: the first one drops out
        P.ctx.chrono_add(to_gpu(x))
    x0, n = P.ctx.chrono_guess(to_gpu(eta))
    ref, _ = orc.chrono_guess(P.o, xs[1:], eta)
    assert n == 4
    assert util.relerr(x0.cpu().numpy(), ref) < 1e-10


def test_guess_is_exact_in_the_image_and_zero_when_empty(pair):
    P = pair
    xs = [synth.gaussian_spinor(P.Vh, 90 + i) for i in range(3)]
    P.ctx.chrono_reset(8)
    x0, n = P.ctx.chrono_guess(to_gpu(xs[0]))
    assert n == 0 and torch.count_nonzero(x0) == 0
    for x in xs:
        P.ctx.chrono_add(to_gpu(x))
    P.ctx.chrono_add(to_gpu(xs[0] + xs[1]))      # dependent: dropped from the solve
    eta = P.o.Dhat(0.5 * xs[0] - 2j * xs[2])
    x0, n = P.ctx.chrono_guess(to_gpu(eta))
    assert n == 3
    assert util.relerr(P.o.Dhat(x0.cpu().numpy()), eta) < 1e-10


def test_sequence_of_solves_with_guesses(pair):
    """eta_t = cos(t) a + sin(t) b: each solve starts from the guess of the
    previous solutions and needs fewer steps than from zero."""
    P = pair
    a, b = synth.gaussian_spinor(P.Vh, 100), synth.gaussian_spinor(P.Vh, 101)
    P.ctx.chrono_reset(4)
    cold, warm = [], []
    for t in np.linspace(0.0, 0.3, 6):
        eta = to_gpu(np.cos(t) * a + np.sin(t) * b)
        _, i0, s0 = P.ctx.solve_dhat(eta, sap_prec=lqcd.F32, inner=lqcd.F32)
        x0, _ = P.ctx.chrono_guess(eta)
        psi, i1, s1 = P.ctx.solve_dhat_guess(eta, x0, sap_prec=lqcd.F32, inner=lqcd.F32)
        assert s0 == 0 and s1 == 0
        assert util.relerr(P.o.Dhat(psi.cpu().numpy()), eta.cpu().numpy()) <= 1e-10
        P.ctx.chrono_add(psi)
        cold.append(i0[0]["iters"])
        warm.append(i1[0]["iters"])
    assert warm[0] == cold[0]                      # nothing stored yet
    assert sum(warm[2:]) < 0.7 * sum(cold[2:]), (cold, warm)


def test_guessed_solve_rejects_cgnr(pair):
    e = to_gpu(synth.gaussian_spinor(pair.Vh, 110))
    with pytest.raises(lqcd.LqcdError):
        pair.ctx.solve_dhat_guess(e, torch.zeros_like(e), solver=lqcd.SOLVER_CGNR)
