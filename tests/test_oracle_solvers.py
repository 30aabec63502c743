"""Pins of the oracle's solvers and deflation against brute force (dense LU of
the assembled operator) and against exact algebraic identities."""
import numpy as np
import pytest

import oracle as orc
from paper_1011_0911_gb300 import synth
from tests import util

KAPPA, CSW = 0.1355, 1.9


def make(dims, kappa=KAPPA, csw=CSW, seed=0):
    U = synth.su3_links(dims, seed)
    return orc.Oracle(dims, U, kappa, csw), U


def test_cgnr_matches_dense_solution():
    dims = (4, 4, 4, 4)
    o, _ = make(dims)
    Dh = util.dense(o.Dhat, o.Vh)
    eta = synth.gaussian_spinor(o.Vh, 21)
    x_ref = np.linalg.solve(Dh, eta.ravel())
    psi, st, it = o.cgnr(eta, tol=1e-12)
    assert st == 0 and it > 5
    assert util.relerr(psi.ravel(), x_ref) < 1e-9
    assert util.relerr(o.Dhat(psi), eta) <= 1e-12


def test_cgnr_8x4_true_residual():
    dims = (8, 8, 8, 8)
    o, _ = make(dims)
    eta = synth.gaussian_spinor(o.Vh, 1)
    psi, st, it = o.cgnr(eta, tol=1e-10)
    assert st == 0
    assert util.relerr(o.Dhat(psi), eta) <= 1e-10


def test_gcr_identity_and_sap_match_dense_solution():
    dims = (4, 4, 4, 4)
    o, _ = make(dims)
    D = util.dense(o.D, o.V)
    eta = synth.gaussian_spinor(o.V, 22)
    x_ref = np.linalg.solve(D, eta.ravel())
    for precond, bs in ((0, (4, 4, 4, 4)), (1, (2, 2, 2, 2)), (1, (4, 2, 2, 2))):
        psi, st, it, rr = o.gcr(eta, precond=precond, bs=bs, ncy=2, nmr=4, nkv=8, nmx=500, tol=1e-11)
        assert st == 0, (precond, bs, it)
        assert rr <= 1e-11
        assert util.relerr(psi.ravel(), x_ref) < 1e-8
        assert util.relerr(o.D(psi), eta) <= 1.01e-11


def test_schur_solution_from_full_solve():
    """Eq. 5: the even part of D^-1 (eta_e, 0) solves Dhat psi_e = eta_e."""
    dims = (8, 8, 8, 8)
    o, _ = make(dims)
    ev, od = util.even_odd_sites(dims)
    eta_e = synth.gaussian_spinor(o.Vh, 3)
    full = np.zeros((o.V, 4, 3), dtype=np.complex128)
    full[ev] = eta_e
    psi, st, it, rr = o.gcr(full, precond=1, ncy=4, nmr=5, nkv=16, tol=1e-12)
    assert st == 0
    psi_c, st2, _ = o.cgnr(eta_e, tol=1e-12)
    assert util.relerr(psi[ev], psi_c) < 1e-8
    assert util.relerr(o.Dhat(psi[ev]), eta_e) < 1e-10


def test_sap_single_block_is_inverse():
    """One block covering the whole lattice with many MinRes steps gives the exact
    inverse (heavy quark so that MinRes converges)."""
    dims = (4, 4, 4, 4)
    o, _ = make(dims, kappa=0.11)
    eta = synth.gaussian_spinor(o.V, 4)
    x_ref = np.linalg.solve(util.dense(o.D, o.V), eta.ravel())
    psi = o.sap(eta, bs=dims, ncy=1, nmr=120)
    assert util.relerr(psi.ravel(), x_ref) < 1e-10


def test_sap_exact_blocks_leave_zero_residual_on_last_colour():
    """With (nearly) exact block solves the residual vanishes on the blocks of the
    colour updated last: this pins the Dirichlet block operator P D P."""
    dims = (8, 8, 8, 8)
    o, _ = make(dims, kappa=0.11)
    eta = synth.gaussian_spinor(o.V, 8)
    psi = o.sap(eta, bs=(4, 4, 4, 4), ncy=1, nmr=80)
    r = eta - o.D(psi)
    c = util.coords(dims) // 4
    colour = c.sum(axis=1) % 2
    assert np.linalg.norm(r[colour == 1]) < 1e-10 * np.linalg.norm(eta)
    assert np.linalg.norm(r[colour == 0]) > 1e-3 * np.linalg.norm(eta)


def test_sap_block_solve_equals_dense_block_restriction():
    """One block solve with many MinRes steps equals the dense inverse of the
    block restriction P D P applied to r on that block."""
    dims = (8, 4, 4, 4)
    o, _ = make(dims, kappa=0.11)
    D = util.dense(o.D, o.V)
    r = synth.gaussian_spinor(o.V, 9)
    c = util.coords(dims) // 4
    blk = c[:, 3] + 1 * (c[:, 2] + 1 * (c[:, 1] + 1 * c[:, 0]))
    for b in (0, 1):
        sites = np.nonzero(blk == b)[0]
        idx = (12 * sites[:, None] + np.arange(12)).ravel()
        Db = D[np.ix_(idx, idx)]
        x = np.linalg.solve(Db, r[sites].ravel())
        chi = o.sap_block_solve(r, b, bs=(4, 4, 4, 4), nmr=100)
        assert util.relerr(chi[sites].ravel(), x) < 1e-10
        others = np.nonzero(blk != b)[0]
        assert np.abs(chi[others]).max() == 0


@pytest.fixture(scope="module")
def dfl8():
    dims = (8, 8, 8, 8)
    o, _ = make(dims)
    Ns = 4
    v0 = synth.gaussian_spinor(Ns * o.V, 100, synth.STREAM_SUBSPACE).reshape(Ns, o.V, 4, 3)
    st = o.dfl_build(v0, bs=(4, 4, 4, 4), ninv=2, ncy=2, nmr=4)
    assert st == 0
    return o, Ns


def test_dfl_block_orthonormal(dfl8):
    o, Ns = dfl8
    phi = o.dfl_subspace()
    c = util.coords(o.dims) // 4
    blk = c[:, 3] + 2 * (c[:, 2] + 2 * (c[:, 1] + 2 * c[:, 0]))
    for b in (0, 5, 15):
        m = phi[:, blk == b].reshape(Ns, -1)
        assert np.abs(m.conj() @ m.T - np.eye(Ns)).max() < 1e-13


def test_dfl_little_operator_is_dense_projection(dfl8):
    """A = Pi^dag D Pi, with Pi assembled densely from the subspace fields."""
    o, Ns = dfl8
    phi = o.dfl_subspace()
    c = util.coords(o.dims) // 4
    blk = c[:, 3] + 2 * (c[:, 2] + 2 * (c[:, 1] + 2 * c[:, 0]))
    nblk = 16
    Pi = np.zeros((o.V * 12, nblk * Ns), dtype=np.complex128)
    for b in range(nblk):
        for k in range(Ns):
            f = np.zeros((o.V, 4, 3), dtype=np.complex128)
            f[blk == b] = phi[k, blk == b]
            Pi[:, b * Ns + k] = f.ravel()
    DPi = np.stack([o.D(Pi[:, j].reshape(o.V, 4, 3)).ravel() for j in range(nblk * Ns)], axis=1)
    A_ref = Pi.conj().T @ DPi
    A = o.dfl_little()
    assert util.relerr(A, A_ref) < 1e-13
    # Pi^dag and Pi
    rho = synth.gaussian_spinor(o.V, 31)
    assert util.relerr(o.dfl_project(rho), Pi.conj().T @ rho.ravel()) < 1e-13
    cc = synth.gaussian_spinor(nblk * Ns // 12 + 1, 32).ravel()[: nblk * Ns]
    assert util.relerr(o.dfl_expand(cc).ravel(), Pi @ cc) < 1e-13
    assert util.relerr(o.dfl_little_apply(cc), A_ref @ cc) < 1e-13
    # projector identities with P_L = 1 - D Pi A^-1 Pi^dag
    Ainv = np.linalg.inv(A_ref)
    x = rho.ravel()
    PLx = x - DPi @ (Ainv @ (Pi.conj().T @ x))
    assert np.linalg.norm(Pi.conj().T @ PLx) < 1e-12 * np.linalg.norm(x)
    PLPLx = PLx - DPi @ (Ainv @ (Pi.conj().T @ PLx))
    assert util.relerr(PLPLx, PLx) < 1e-12
    # coarse solve
    xs, st, it = o.dfl_coarse_solve(cc, tol=1e-12)
    assert st == 0
    assert util.relerr(xs, Ainv @ cc) < 1e-9


def test_dfl_gcr_converges_and_reduces_iterations(dfl8):
    o, Ns = dfl8
    eta = synth.gaussian_spinor(o.V, 40)
    psi, st, it_d, rr = o.gcr(eta, precond=2, ncy=4, nmr=5, nkv=16, tol=1e-10)
    assert st == 0 and rr <= 1e-10
    assert util.relerr(o.D(psi), eta) <= 1.01e-10
    psi2, st2, it_s, rr2 = o.gcr(eta, precond=1, ncy=4, nmr=5, nkv=16, tol=1e-10)
    assert st2 == 0
    assert util.relerr(psi, psi2) < 1e-7
    assert it_d <= it_s


def _block_ids(dims, bs):
    c = util.coords(dims) // np.asarray(bs)
    nb = [L // b for L, b in zip(dims, bs)]
    return c[:, 3] + nb[3] * (c[:, 2] + nb[2] * (c[:, 1] + nb[1] * c[:, 0])), int(np.prod(nb))


def _block_qr(v, blk, nblk):
    """Per block, the orthonormal factor of the QR decomposition of the Ns
    columns v[l] restricted to the block, with the phases fixed so that R has a
    positive real diagonal -- the unique factor that Gram-Schmidt produces."""
    Ns = v.shape[0]
    out = np.zeros_like(v)
    for b in range(nblk):
        m = blk == b
        M = v[:, m].reshape(Ns, -1).T
        Q, R = np.linalg.qr(M)
        ph = np.diag(R) / np.abs(np.diag(R))
        Q = Q * ph[None, :]
        out[:, m] = Q.T.reshape((Ns,) + v[:, m].shape[1:])
    return out


@pytest.mark.parametrize("ninv", [0, 1, 2])
def test_dfl_build_is_block_qr_of_sap_iterates(ninv):
    """Subspace generation (Sec. 4, locally deflated SAP-GCR; the inverse-iteration
    reading of the design notes): after ninv passes v <- M_sap v / |M_sap v| the
    block-orthonormal fields are the per-block QR factors of the iterates.  M_sap is
    positively homogeneous (the MinRes coefficients are scale free), so the
    normalisation does not change the directions; the oracle's SAP is pinned on
    its own (dense block inverse, one-block limit, vanishing residual)."""
    dims, bs, Ns, ncy, nmr = (8, 8, 8, 8), (4, 4, 4, 4), 4, 2, 4
    o, _ = make(dims)
    v0 = synth.gaussian_spinor(Ns * o.V, 100, synth.STREAM_SUBSPACE).reshape(Ns, o.V, 4, 3)
    assert o.dfl_build(v0, bs=bs, ninv=ninv, ncy=ncy, nmr=nmr) == 0
    v = v0.copy()
    for _ in range(ninv):
        v = np.stack([o.sap(v[l], bs=bs, ncy=ncy, nmr=nmr) for l in range(Ns)])
    blk, nblk = _block_ids(dims, bs)
    ref = _block_qr(v, blk, nblk)
    phi = o.dfl_subspace()
    assert util.relerr(phi, ref) < 1e-12
    if ninv > 0:   # the iterates differ from the Gaussian start
        assert util.relerr(_block_qr(v0, blk, nblk), ref) > 0.1


def test_dfl_precond_is_sap_on_deflated_residual_plus_coarse_correction(dfl8):
    """M_dfl rho = M_sap(P_L rho) + Pi A^-1 Pi^dag rho (Sec. 4, deflated SAP),
    with Pi and A = Pi^dag D Pi assembled densely in numpy and A^-1 by LU; the
    oracle's coarse solve runs to 1e-13 so both sides see the same P_L rho."""
    o, Ns = dfl8
    bs, ncy, nmr = (4, 4, 4, 4), 3, 4
    phi = o.dfl_subspace()
    blk, nblk = _block_ids(o.dims, bs)
    Pi = np.zeros((o.V * 12, nblk * Ns), dtype=np.complex128)
    for b in range(nblk):
        for k in range(Ns):
            f = np.zeros((o.V, 4, 3), dtype=np.complex128)
            f[blk == b] = phi[k, blk == b]
            Pi[:, b * Ns + k] = f.ravel()
    DPi = np.stack([o.D(Pi[:, j].reshape(o.V, 4, 3)).ravel() for j in range(nblk * Ns)], axis=1)
    A = Pi.conj().T @ DPi
    rho = synth.gaussian_spinor(o.V, 41)
    e = np.linalg.solve(A, Pi.conj().T @ rho.ravel())
    PL = rho.ravel() - DPi @ e
    ref = o.sap(PL.reshape(o.V, 4, 3), bs=bs, ncy=ncy, nmr=nmr).ravel() + Pi @ e
    got = o.dfl_precond(rho, bs=bs, ncy=ncy, nmr=nmr, ctol=1e-13).ravel()
    assert util.relerr(got, ref) < 1e-10
    # either half alone is far from the whole
    assert util.relerr(Pi @ e, ref) > 1e-2
    assert util.relerr(ref - Pi @ e, ref) > 1e-2
    # closed form: on the image of D Pi the deflated residual vanishes, M_sap(0) = 0
    # and M_dfl returns the coarse preimage, M_dfl (D Pi c) = Pi c
    c = synth.gaussian_spinor(nblk * Ns // 12 + 1, 42).ravel()[: nblk * Ns]
    got = o.dfl_precond((DPi @ c).reshape(o.V, 4, 3), bs=bs, ncy=ncy, nmr=nmr, ctol=1e-13).ravel()
    assert util.relerr(got, Pi @ c) < 1e-10
