"""The allocation-free Dhat entry point (odd-site intermediate in the library's
fixed device array) against lqcd_apply_Dhat_native, which takes the
intermediate from the context's workspace: two calls in a row, each compared
with the workspace path on the same input.  Both launch the same kernels with
the same tuned shapes, so the results must be bitwise equal; one case is also
checked against the oracle.  Collected last on purpose, so that it also runs
after every other test has used the library in this process."""
import numpy as np
import pytest
import torch

from paper_1011_0911_gb300 import lqcd, synth
from tests.gpu_util import TOL, Pair, rounded
from tests import util

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 32 << 20


def native_even(P, prec, nrhs, seed):
    x = np.stack([synth.gaussian_spinor(P.Vh, seed + k) for k in range(nrhs)])
    x = rounded(x, prec)
    dt = torch.complex128 if prec == lqcd.F64 else torch.complex64
    return x, P.ctx.pack(torch.from_numpy(x).to(dt).cuda(), prec, 1)


@pytest.mark.parametrize("prec", [lqcd.F32, lqcd.F64, lqcd.F16S], ids=["f32", "f64", "f16s"])
@pytest.mark.parametrize("dims,nrhs", [((8, 8, 8, 8), 1), ((16, 8, 8, 8), 3)])
def test_static_scratch_matches_workspace_path(dims, nrhs, prec):
    P = Pair(dims)
    ctx = P.ctx
    for call, seed in enumerate((300, 400)):
        x, xn = native_even(P, prec, nrhs, seed)
        ref = ctx.native_empty(prec, 1, nrhs)
        got = ctx.native_empty(prec, 1, nrhs)
        ctx.apply_Dhat_native(xn, ref, prec, nrhs)
        ctx.apply_Dhat_native_static(xn, got, prec, nrhs)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), call
        if call == 1 and nrhs == 3:
            k = nrhs - 1
            out = ctx.unpack(got, prec, 1, nrhs)[k].cpu().numpy().astype(np.complex128)
            assert util.relerr(out.reshape(P.Vh, 4, 3), P.o.Dhat(x[k])) < TOL[prec]


def test_static_scratch_rejects_oversize_request():
    """More right-hand sides than the fixed array holds: LQCD_ERR_ARG, no launch."""
    P = Pair((16, 8, 8, 8))
    per_rhs = 12 * 16 * P.Vh                 # FP64 odd half-field bytes
    nrhs = SCRATCH_BYTES // per_rhs + 1
    x = P.ctx.native_empty(lqcd.F64, 1, nrhs)
    y = P.ctx.native_empty(lqcd.F64, 1, nrhs)
    with pytest.raises(lqcd.LqcdError) as e:
        P.ctx.apply_Dhat_native_static(x, y, lqcd.F64, nrhs)
    assert e.value.status == 1
    with pytest.raises(lqcd.LqcdError) as e:   # bfloat16 is the network's storage only
        P.ctx.apply_Dhat_native_static(x, y, lqcd.BF16, 1)
    assert e.value.status == 1
    # the largest request that fits still runs
    n_ok = SCRATCH_BYTES // per_rhs
    x = P.ctx.native_empty(lqcd.F64, 1, n_ok).zero_()
    y = P.ctx.native_empty(lqcd.F64, 1, n_ok)
    P.ctx.apply_Dhat_native_static(x, y, lqcd.F64, n_ok)
    torch.cuda.synchronize()
    assert torch.count_nonzero(y).item() == 0
