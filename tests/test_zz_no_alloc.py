"""The allocation-free Dhat entry point (odd-site intermediate in the library's
fixed device array) against lqcd_apply_Dhat_native, which takes the
intermediate from the context's workspace: two calls in a row, each compared
with the workspace path on the same input.  Collected last on purpose, so that
it also runs after every other test has used the library in this process."""
import numpy as np
import pytest
import torch

from paper_1011_0911_gb300 import lqcd, synth
from tests.gpu_util import TOL, Pair

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 32 << 20


def native_even(P, prec, nrhs, seed):
    x = np.stack([synth.gaussian_spinor(P.Vh, seed + k) for k in range(nrhs)])
    return P.ctx.pack(torch.from_numpy(x).cuda(), prec, 1)


@pytest.mark.parametrize("prec", [lqcd.F32, lqcd.F64])
@pytest.mark.parametrize("dims,nrhs", [((8, 8, 8, 8), 1), ((16, 8, 8, 8), 3)])
def test_static_scratch_matches_workspace_path(dims, nrhs, prec):
    P = Pair(dims)
    ctx = P.ctx
    for call, seed in enumerate((300, 400)):
        x = native_even(P, prec, nrhs, seed)
        ref = ctx.native_empty(prec, 1, nrhs)
        got = ctx.native_empty(prec, 1, nrhs)
        ctx.apply_Dhat_native(x, ref, prec, nrhs)
        ctx.apply_Dhat_native_static(x, got, prec, nrhs)
        torch.cuda.synchronize()
        a = ctx.unpack(got, prec, 1, nrhs).to(torch.complex128)
        b = ctx.unpack(ref, prec, 1, nrhs).to(torch.complex128)
        err = (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()
        assert err <= TOL[prec], (call, err)


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
    # the largest request that fits still runs
    n_ok = SCRATCH_BYTES // per_rhs
    x = P.ctx.native_empty(lqcd.F64, 1, n_ok).zero_()
    y = P.ctx.native_empty(lqcd.F64, 1, n_ok)
    P.ctx.apply_Dhat_native_static(x, y, lqcd.F64, n_ok)
    torch.cuda.synchronize()
