"""GPU parity of the clover term, D (Eq. 1) and Dhat (Eq. 2) against the FP64
CPU oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_1011_0911_gb300 import lqcd, synth
from tests import util
from tests.gpu_util import TOL, Pair, relerr, rounded, to_gpu

pytestmark = pytest.mark.gpu

# several CTAs of 128 sites with ragged tails (Vh = 432, 720), L = 2 directions
# (forward and backward neighbour coincide), and the 8^4 workload
DIMS = [(6, 6, 6, 4), (10, 6, 4, 6), (8, 8, 8, 8), (4, 2, 4, 2), (2, 2, 2, 2)]


@pytest.fixture(scope="module", params=DIMS, ids=lambda d: "x".join(map(str, d)))
def pair(request):
    return Pair(request.param)


def test_clover_and_inverse(pair):
    P = pair
    ld_e, ld_o = P.logdet
    assert abs(ld_e - P.o.logdet(0)) <= 1e-12 * abs(P.o.logdet(0))
    assert abs(ld_o - P.o.logdet(1)) <= 1e-12 * abs(P.o.logdet(1))
    for parity, sites in ((0, P.ev), (1, P.od)):
        x = synth.gaussian_spinor(P.Vh, 7 + parity)
        for inverse in (False, True):
            out = P.ctx.apply_clover(parity, inverse, to_gpu(x))
            ref = np.stack([P.o.clover_site(s, inverse) @ x[i].ravel() for i, s in enumerate(sites)])
            assert relerr(out, ref.reshape(x.shape)) < 1e-14


@pytest.mark.parametrize("prec", [lqcd.F64, lqcd.F32, lqcd.F16S], ids=["f64", "f32", "f16s"])
def test_D(pair, prec):
    P = pair
    psi = rounded(synth.gaussian_spinor(P.V, 3), prec)
    out = P.ctx.apply_D(to_gpu(psi, prec), prec)
    assert relerr(out, P.o.D(psi)) < TOL[prec]


@pytest.mark.parametrize("prec", [lqcd.F64, lqcd.F32, lqcd.F16S], ids=["f64", "f32", "f16s"])
def test_Dhat(pair, prec):
    P = pair
    pe = rounded(synth.gaussian_spinor(P.Vh, 4), prec)
    out = P.ctx.apply_Dhat(to_gpu(pe, prec), prec)
    assert relerr(out, P.o.Dhat(pe)) < TOL[prec]


@pytest.mark.parametrize("prec", [lqcd.F64, lqcd.F32, lqcd.F16S], ids=["f64", "f32", "f16s"])
@pytest.mark.parametrize("nrhs", [3, 12])
@pytest.mark.parametrize("kind", ["hop", "mr", "sm"])
def test_multi_rhs_matches_single(pair, prec, nrhs, kind, monkeypatch):
    """The multi-RHS kernel forms (one field per thread; two fields per thread
    in registers, with a partial last group for 3 fields; the operator staged
    in shared memory per tile of sites) compute each field exactly as the
    single-field launch."""
    P = pair
    monkeypatch.setenv("LQCD_HOP_KIND", kind)
    pe = rounded(synth.gaussian_spinor(nrhs * P.Vh, 5).reshape(nrhs, P.Vh, 4, 3), prec)
    g = to_gpu(pe, prec)
    many = P.ctx.apply_Dhat(g, prec)
    for k in range(nrhs):
        one = P.ctx.apply_Dhat(g[k].contiguous(), prec)
        assert torch.equal(one, many[k])
    k = nrhs - 1
    assert relerr(many[k], P.o.Dhat(pe[k])) < TOL[prec]


def test_native_roundtrip_and_bad_args(pair):
    P = pair
    x = synth.gaussian_spinor(2 * P.Vh, 9).reshape(2, P.Vh, 4, 3)
    for prec in (lqcd.F64, lqcd.F32):
        g = to_gpu(x, prec)
        n = P.ctx.pack(g, prec, 1)
        back = P.ctx.unpack(n, prec, 1, 2)
        assert torch.equal(back.reshape(g.shape), g)
    with pytest.raises(lqcd.LqcdError) as e:   # bfloat16 is the network's storage only
        P.ctx.apply_Dhat(to_gpu(x[0]), prec=lqcd.BF16)
    assert e.value.status == 1


def test_f16s_storage_roundtrip(pair):
    """Half precision with a per-site scale: every site is reproduced to the
    FP16 rounding of its own largest component; zero sites stay zero."""
    P = pair
    x = synth.gaussian_spinor(2 * P.Vh, 21).reshape(2, P.Vh, 4, 3).astype(np.complex64)
    x[1, ::3] *= 1e-30          # tiny sites keep their relative precision
    x[0, 1] = 0
    g = torch.from_numpy(x).cuda()
    back = P.ctx.unpack(P.ctx.pack(g, lqcd.F16S, 1), lqcd.F16S, 1, 2).cpu().numpy()
    site_max = np.abs(np.stack([x.real, x.imag], -1)).reshape(2, P.Vh, -1).max(-1)
    err = np.abs(np.stack([(back - x).real, (back - x).imag], -1)).reshape(2, P.Vh, -1).max(-1)
    assert np.all(err <= 2.0 ** -11 * site_max * (1 + 1e-6))
    assert np.all(back[0, 1] == 0)


def test_unit_links_free_field_on_gpu():
    """Closed form on the GPU too: unit links, plane wave with antiperiodic p0."""
    dims = (4, 4, 4, 4)
    P = Pair(dims, U=synth.unit_links(dims))
    x = util.coords(dims)
    p = np.array([np.pi / 4, 2 * np.pi / 4, 0, 2 * np.pi * 3 / 4])
    u = np.arange(12).reshape(4, 3) + 1j
    psi = np.exp(1j * x @ p)[:, None, None] * u[None]
    out = P.ctx.apply_D(to_gpu(psi))
    assert relerr(out, P.o.D(psi)) < 1e-14


def test_dhat_full_size_sampled():
    """48x24^3 (the production lattice of Sec. 3), FP32 and FP64 Dhat in the
    launch configuration the benchmark times, checked at sampled sites against
    the oracle's one-site evaluation of the definition."""
    dims = (48, 24, 24, 24)
    P = Pair(dims, kappa=0.13625)
    rng = np.random.default_rng(0)
    sample = np.concatenate([[0, 1, P.Vh - 1], rng.integers(0, P.Vh, 61)])
    for prec in (lqcd.F32, lqcd.F64, lqcd.F16S):
        pe = rounded(synth.gaussian_spinor(P.Vh, 11), prec)
        g = to_gpu(pe, prec)
        nin = P.ctx.pack(g, prec, 1)
        nout = P.ctx.native_empty(prec, 1, 1)
        P.ctx.apply_Dhat_native(nin, nout, prec, 1)
        out = P.ctx.unpack(nout, prec, 1, 1).reshape(P.Vh, 4, 3).cpu().numpy().astype(np.complex128)
        ref = np.stack([P.o.dhat_site(pe, int(r)) for r in sample])
        assert util.relerr(out[sample], ref) < TOL[prec]


def test_dhat_12_fields_full_size_sampled(monkeypatch):
    """The benchmarked launch: 12 FP32 fields at 48x24^3 through the native
    entry point, in the launch shape the autotuner picks for it, checked at 64
    sampled sites of every field against the oracle's one-site evaluation of
    Eq. 2 (FP32 bound 1e-6; measured 1.0e-7).  Every kernel form the tuner may
    pick is bitwise equal to the tuned one, so the check covers whichever form
    the benchmark times; F16S (bound 3e-3) goes through the same launch."""
    dims = (48, 24, 24, 24)
    P = Pair(dims, kappa=0.13625)
    nrhs = 12
    rng = np.random.default_rng(1)
    pe = np.stack([synth.gaussian_spinor(P.Vh, 11 + k) for k in range(nrhs)])
    for prec in (lqcd.F32, lqcd.F16S):
        per = rounded(pe, prec)
        nin = P.ctx.pack(to_gpu(per, prec), prec, 1)
        nout = P.ctx.native_empty(prec, 1, nrhs)
        P.ctx.apply_Dhat_native(nin, nout, prec, nrhs)
        out = P.ctx.unpack(nout, prec, 1, nrhs).reshape(nrhs, P.Vh, 4, 3).cpu().numpy().astype(np.complex128)
        for k in range(nrhs):
            sample = np.concatenate([[0, 1, P.Vh - 1], rng.integers(0, P.Vh, 61)])
            ref = np.stack([P.o.dhat_site(per[k], int(r)) for r in sample])
            assert util.relerr(out[k][sample], ref) < TOL[prec], (prec, k)
        for kind in ("hop", "mr", "sm"):
            monkeypatch.setenv("LQCD_HOP_KIND", kind)
            alt = P.ctx.native_empty(prec, 1, nrhs)
            P.ctx.apply_Dhat_native(nin, alt, prec, nrhs)
            assert torch.equal(alt, nout), (prec, kind)
        monkeypatch.delenv("LQCD_HOP_KIND")
