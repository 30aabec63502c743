"""The batched multi-lattice SAP-GCR: lattices of different sizes and kappa
solved together to a true Dhat residual of 1e-10 each (checked by the FP64
oracle), agreement with the single-lattice solver, graph replay against eager
launches, converged lattices dropping out, and the bounded device-side wait."""
import numpy as np
import pytest
import torch

from paper_1011_0911_gb300 import lqcd, synth
from tests import util
from tests.gpu_util import Pair, to_gpu

pytestmark = pytest.mark.gpu

# uneven batch: 3 blocks along time in 12x8x8x8 (same-colour blocks touch
# across the wrap); kappa differs per lattice
LATS = [((8, 8, 8, 8), 0.1350, 1), ((16, 8, 8, 8), 0.1360, 2), ((12, 8, 8, 8), 0.1355, 3), ((8, 8, 8, 16), 0.1358, 4)]


@pytest.fixture(scope="module")
def pairs():
    return [Pair(d, kappa=k, seed=s) for d, k, s in LATS]


def sources(pairs, seed=700):
    return [synth.gaussian_spinor(P.Vh, seed + i) for i, P in enumerate(pairs)]


@pytest.mark.parametrize("sap_prec", [lqcd.F16S, lqcd.F32], ids=["f16s", "f32"])
def test_batch_solves_every_lattice(pairs, sap_prec):
    B = lqcd.Batch([P.ctx for P in pairs], nkv=16, tol=1e-10, sap_prec=sap_prec)
    eta = sources(pairs)
    psi, info, st = B.solve_dhat([to_gpu(e) for e in eta])
    assert st == 0, (st, B.last_error(), info)
    for P, e, x, inf in zip(pairs, eta, psi, info):
        xs = x.cpu().numpy()
        assert util.relerr(P.o.Dhat(xs), e) <= 1e-10
        assert inf["relres_dhat"] <= 1e-10 and inf["status"] == 0
        assert inf["iters"] > 0
        # the single-lattice solver reaches the same solution
        ref, _, st1 = P.ctx.solve_dhat(to_gpu(e), solver=lqcd.SOLVER_SAP_GCR, tol=1e-10, sap_prec=lqcd.F32,
                                       inner=lqcd.F32)
        assert st1 == 0
        assert util.relerr(xs, ref.cpu().numpy()) < 1e-7
    s = B.stats()
    assert s["cycles"] >= 1 and s["graph_replays"] == max(0, s["cycles"] - 1)


def test_graph_replay_matches_eager(pairs):
    eta = [to_gpu(e) for e in sources(pairs, 800)]
    Bg = lqcd.Batch([P.ctx for P in pairs], use_graph=True)
    Be = lqcd.Batch([P.ctx for P in pairs], use_graph=False)
    xg, ig, sg = Bg.solve_dhat(eta)
    xe, ie, se = Be.solve_dhat(eta)
    assert sg == 0 and se == 0
    assert Be.stats()["graph_replays"] == 0
    for a, b, i, j in zip(xg, xe, ig, ie):
        assert i["iters"] == j["iters"]
        assert torch.equal(a, b)


def test_converged_lattice_drops_out(pairs):
    """A zero source is solved at once (psi = 0); the others still converge."""
    eta = sources(pairs, 900)
    eta[1] = np.zeros_like(eta[1])
    B = lqcd.Batch([P.ctx for P in pairs])
    psi, info, st = B.solve_dhat([to_gpu(e) for e in eta])
    assert st == 0
    assert info[1]["iters"] == 0 and torch.count_nonzero(psi[1]) == 0
    for k in (0, 2, 3):
        assert util.relerr(pairs[k].o.Dhat(psi[k].cpu().numpy()), eta[k]) <= 1e-10


def test_bounded_wait_reports_timeout(pairs):
    """A grid barrier that waits for a CTA that does not exist ends by its time
    limit with LQCD_ERR_TIMEOUT; the batch and its contexts stay usable."""
    ctxs = [P.ctx for P in pairs[:2]]
    eta = [to_gpu(e) for e in sources(pairs[:2], 1000)]
    Bs = lqcd.Batch(ctxs, wait_timeout_s=0.05, stall_test=True, use_graph=False)
    _, _, st = Bs.solve_dhat(eta)
    assert st == 8, Bs.last_error()
    B = lqcd.Batch(ctxs)
    psi, info, st = B.solve_dhat(eta)
    assert st == 0
    for P, e, x in zip(pairs[:2], eta, psi):
        assert util.relerr(P.o.Dhat(x.cpu().numpy()), e.cpu().numpy()) <= 1e-10


def test_batch_rejects_mixed_block_shapes():
    P = Pair((6, 6, 6, 6))
    Q = Pair((8, 8, 8, 8))
    with pytest.raises(lqcd.LqcdError):
        lqcd.Batch([P.ctx, Q.ctx])
