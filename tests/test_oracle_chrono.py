"""Pins of the oracle's chronological initial guess: a source in the image of
the stored solutions is solved exactly, the residual is orthogonal to the
images Dhat x_i (least-squares optimality), and no stored solution (nor zero)
gives a smaller residual."""
import numpy as np

import oracle as orc
from paper_1011_0911_gb300 import synth
from tests import util


def make(dims=(4, 4, 4, 4)):
    return orc.Oracle(dims, synth.su3_links(dims, 0), 0.1355, 1.9)


def test_exact_when_eta_in_the_image():
    o = make()
    xs = [synth.gaussian_spinor(o.Vh, 40 + i) for i in range(4)]
    a = np.array([0.3 - 0.1j, -1.2, 0.0, 0.7j])
    eta = o.Dhat(sum(ai * x for ai, x in zip(a, xs)))
    x0, c = orc.chrono_guess(o, xs, eta)
    assert np.allclose(c, a, atol=1e-12)
    assert util.relerr(o.Dhat(x0), eta) < 1e-12


def test_residual_orthogonal_and_minimal():
    o = make()
    xs = [synth.gaussian_spinor(o.Vh, 50 + i) for i in range(5)]
    eta = synth.gaussian_spinor(o.Vh, 60)
    x0, _ = orc.chrono_guess(o, xs, eta)
    r = eta.ravel() - o.Dhat(x0).ravel()
    for x in xs:
        y = o.Dhat(x).ravel()
        assert abs(np.vdot(y, r)) < 1e-11 * np.linalg.norm(y) * np.linalg.norm(r)
    rn = np.linalg.norm(r)
    assert rn <= np.linalg.norm(eta) + 1e-12
    for x in xs:
        # the best multiple of one stored solution is no better either
        y = o.Dhat(x).ravel()
        best = np.linalg.norm(eta.ravel() - (np.vdot(y, eta.ravel()) / np.vdot(y, y)) * y)
        assert rn <= best + 1e-12
