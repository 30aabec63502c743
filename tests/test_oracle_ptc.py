"""Pins of the oracle's parallel-transport network: adjointness of the
transports, gauge equivariance, identity weights, the Wilson hop term as a
special case, and central finite differences of the loss gradient."""
import numpy as np

import oracle as orc
from paper_1011_0911_gb300 import synth
from tests import util

DIMS = (4, 4, 4, 4)
CHANS = (1, 2, 2, 1)


def make(dims=DIMS, kappa=0.1355, csw=1.9, seed=0):
    U = synth.su3_links(dims, seed)
    return orc.Oracle(dims, U, kappa, csw), U


def rand_weights(chans, seed, scale=0.3):
    n = orc.ptc_weight_count(chans)
    g = synth.gaussians(seed, synth.STREAM_NET, 2 * n)
    return scale * (g[0::2] + 1j * g[1::2])


def test_transport_adjoint():
    o, _ = make()
    f = synth.gaussian_spinor(o.V, 1)
    g = synth.gaussian_spinor(o.V, 2)
    for d in range(1, 9):
        dd = d + 1 if d % 2 else d - 1
        lhs = np.vdot(g, orc.ptc_transport(o, d, f))
        rhs = np.vdot(orc.ptc_transport(o, dd, g), f)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_equivariance():
    """N[U^g](g rho) = g N[U](rho) for a random gauge transformation g."""
    o, U = make()
    W = rand_weights(CHANS, 5)
    g = synth.random_su3(o.V, 9)
    og = orc.Oracle(DIMS, util.gauge_transform(DIMS, U, g), 0.1355, 1.9)
    rho = synth.gaussian_spinor(o.V, 3)
    lhs = orc.ptc_forward(og, CHANS, W, util.colour_rotate(g, rho)[None])[0]
    rhs = util.colour_rotate(g, orc.ptc_forward(o, CHANS, W, rho[None])[0])
    assert util.relerr(lhs, rhs) < 1e-13


def test_identity_weights():
    o, _ = make()
    W = np.zeros(orc.ptc_weight_count(CHANS), dtype=np.complex128)
    off = 0
    for l in range(3):
        cin, cout = CHANS[l], CHANS[l + 1]
        w = W[off:off + cout * cin * 144].reshape(cout, cin, 9, 4, 4)
        w[0, 0, 0] = np.eye(4)   # channel 0 -> channel 0, identity path
        off += cout * cin * 144
    rho = synth.gaussian_spinor(o.V, 4)
    assert util.relerr(orc.ptc_forward(o, CHANS, W, rho[None])[0], rho) < 1e-15


def test_wilson_weights_reproduce_D():
    """One 1->1 layer with W_0 = (4+m0), W_+mu = -(1-g_mu)/2, W_-mu = -(1+g_mu)/2 is D at c_sw = 0."""
    kappa = 0.1355
    o, U = make(csw=0.0, kappa=kappa)
    m0 = 1 / (2 * kappa) - 4
    W = np.zeros((9, 4, 4), dtype=np.complex128)
    W[0] = (4 + m0) * np.eye(4)
    for mu in range(4):
        gm = orc.gamma(mu)
        W[1 + 2 * mu] = -0.5 * (np.eye(4) - gm)
        W[2 + 2 * mu] = -0.5 * (np.eye(4) + gm)
    rho = synth.gaussian_spinor(o.V, 6)
    out = orc.ptc_forward(o, (1, 1), W.ravel(), rho[None])[0]
    assert util.relerr(out, o.D(rho)) < 1e-14


def _loss(o, W, rho, t):
    n = orc.ptc_forward(o, CHANS, W, rho[None])[0]
    return np.linalg.norm(n - t) ** 2 / np.linalg.norm(t) ** 2


def test_gradient_finite_differences():
    """dL/dRe W + i dL/dIm W from the backward pass against central differences
    (h = 1e-6) of L = |N(rho) - t|^2 / |t|^2."""
    o, _ = make()
    W = rand_weights(CHANS, 7)
    rho = synth.gaussian_spinor(o.V, 8)
    t = synth.gaussian_spinor(o.V, 9)
    out, acts = orc.ptc_forward(o, CHANS, W, rho[None], keep_acts=True)
    gout = 2 * (out[0] - t) / np.linalg.norm(t) ** 2
    dW, gin = orc.ptc_backward(o, CHANS, W, acts, gout[None])
    rng = np.random.default_rng(0)
    h = 1e-6
    for j in rng.integers(0, W.size, 12):
        for part, unit in ((0, 1.0), (1, 1j)):
            Wp, Wm = W.copy(), W.copy()
            Wp[j] += h * unit
            Wm[j] -= h * unit
            fd = (_loss(o, Wp, rho, t) - _loss(o, Wm, rho, t)) / (2 * h)
            an = dW[j].real if part == 0 else dW[j].imag
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(fd)) + 1e-7 * np.abs(dW).max(), (j, part, fd, an)
    # input gradient against a directional finite difference
    v = synth.gaussian_spinor(o.V, 10)
    fd = (_loss(o, W, rho + h * v, t) - _loss(o, W, rho - h * v, t)) / (2 * h)
    an = np.real(np.vdot(gin[0], v))
    assert abs(fd - an) < 1e-6 * abs(fd)
