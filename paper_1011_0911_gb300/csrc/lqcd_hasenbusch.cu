// Hasenbusch mass preconditioning (Eq. 3-4): W(dm) = Q_S + dm with
// Q_S = 1 - Q_ee^-1 Q_eo Q_oo^-1 Q_oe (Eq. 2), Q = gamma5 D.  gamma5 is
// diagonal on sites and cancels pairwise, so Q_S = A_ee^-1 Dhat and
//   W(dm) = A_ee^-1 Dhat + dm.
// The solve uses A_ee W(dm) = (1 + dm) A_ee - H_eo A_oo^-1 H_oe, the Schur
// complement of D' = D with its even-site clover blocks scaled by 1 + dm:
//   W(dm)^-1 eta = Dhat'^-1 (A_ee eta)
// (and, with Eq. 5, Q_S^-1 = P_e Q^-1 Q_ee P_e at dm = 0).
#include <cmath>
#include <vector>

#include "lqcd_stencil.cuh"

namespace {

using namespace stencil;

// out = A_ee^-1 dh + dm psi on even sites (out may alias dh)
template <class R, class SP, class CL>
__global__ void k_w_finish(long Vh, int nrhs, long rs, const SP *dh, const SP *psi, SP *out, const CL *Ai, R dm)
{
    const long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (r >= Vh || k >= nrhs) return;
    Spinor<R> v, w, p;
    load_spinor(dh + k * rs, Vh, (int)r, v);
    load_spinor(psi + k * rs, Vh, (int)r, p);
    clover_apply<R, CL>(Ai, Vh, (int)r, v, w);
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < 3; c++) w.s[s][c] = w.s[s][c] + dm * p.s[s][c];
    store_spinor(out + k * rs, Vh, (int)r, w);
}

// out = W(dm) in on native even fields of precision p
lqcd_status apply_W_native(lqcd_ctx *c, lqcd_prec p, double dm, const void *in, void *out, int nrhs)
{
    void *tmp;
    LQCD_TRY(ws_get(c, WS_TMP_O, native_half_bytes(c, p) * nrhs, &tmp));
    LQCD_TRY(dirac_dhat(c, p, in, out, tmp, nrhs));
    const long Vh = c->g.Vh;
    dim3 grid(div_up(Vh, 128), nrhs);
    if (p == LQCD_F64)
        k_w_finish<double, double2, double2><<<grid, 128, 0, c->stream>>>(
            Vh, nrhs, 12 * Vh, (const double2 *)out, (const double2 *)in, (double2 *)out, c->Ai64[0], dm);
    else
        k_w_finish<float, float4, float4><<<grid, 128, 0, c->stream>>>(
            Vh, nrhs, 6 * Vh, (const float4 *)out, (const float4 *)in, (float4 *)out, c->Ai32[0], (float)dm);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

}  // namespace

extern "C" {

lqcd_status lqcd_apply_W(lqcd_ctx *c, lqcd_prec p, double dm, const void *in, void *out, int nrhs)
{
    if (!c || !in || !out || nrhs < 1) return set_err(c, LQCD_ERR_ARG, "bad argument");
    if (p != LQCD_F64 && p != LQCD_F32) return set_err(c, LQCD_ERR_ARG, "precision %d", (int)p);
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    const size_t hb = native_half_bytes(c, p) * nrhs;
    void *a, *b;
    LQCD_TRY(ws_get(c, WS_PACK_IN, hb, &a));
    LQCD_TRY(ws_get(c, WS_PACK_OUT, hb, &b));
    LQCD_TRY(pack_field(c, p, 1, in, a, nrhs, false));
    LQCD_TRY(apply_W_native(c, p, dm, a, b, nrhs));
    return pack_field(c, p, 1, out, b, nrhs, true);
}

lqcd_status lqcd_solve_W(lqcd_ctx *c, const lqcd_solver_params *sp, double dm, const double *eta, double *psi,
                         int nrhs, lqcd_solve_info *info)
{
    if (!c || !sp || !eta || !psi || nrhs < 1) return set_err(c, LQCD_ERR_ARG, "bad argument");
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    if (sp->solver != LQCD_SOLVER_CGNR && sp->solver != LQCD_SOLVER_SAP_GCR)
        return set_err(c, LQCD_ERR_ARG, "W(dm) solves use CGNR or SAP-GCR (subspace and network belong to D)");
    if (!(dm > -1.0)) return set_err(c, LQCD_ERR_ARG, "dm must exceed -1");
    const long Vh = c->g.Vh;
    const size_t cb = (size_t)12 * Vh * nrhs * sizeof(double2);   // canonical even fields
    void *buf;
    LQCD_TRY(ws_get(c, WS_HASEN, 2 * cb, &buf));
    double *rhs = (double *)buf, *res = (double *)((char *)buf + cb);
    // rhs = A_ee eta with the unshifted clover term
    for (int k = 0; k < nrhs; k++)
        LQCD_TRY(lqcd_apply_clover(c, 0, 0, eta + (size_t)k * 24 * Vh, rhs + (size_t)k * 24 * Vh));
    std::vector<double> e2(nrhs), r2(nrhs);
    for (int k = 0; k < nrhs; k++) LQCD_TRY(blas_norm2(c, 24 * Vh, eta + (size_t)k * 24 * Vh, &e2[k]));
    const double kappa = c->kappa, csw = c->csw;
    lqcd_solver_params q = *sp;
    q.tol = 0.25 * sp->tol;
    lqcd_status st = LQCD_OK, worst = LQCD_OK;
    for (int attempt = 0; attempt < 3; attempt++) {
        // solve Dhat' psi = A_ee eta on D' (even clover blocks scaled by 1 + dm), then restore D
        st = clover_build(c, kappa, csw, nullptr, nullptr, 1.0 + dm);
        if (st == LQCD_OK) st = lqcd_solve_dhat(c, &q, rhs, psi, nrhs, info);
        const lqcd_status rs = clover_build(c, kappa, csw, nullptr, nullptr, 1.0);
        if (rs != LQCD_OK) return rs;
        if (st != LQCD_OK && st != LQCD_ERR_NOT_CONVERGED) return st;
        worst = st;
        // the W residual in FP64 on the restored operator
        LQCD_TRY(lqcd_apply_W(c, LQCD_F64, dm, psi, res, nrhs));
        LQCD_TRY(blas_sub(c, 24 * Vh * nrhs, eta, res, res));
        bool again = false;
        for (int k = 0; k < nrhs; k++) {
            LQCD_TRY(blas_norm2(c, 24 * Vh, res + (size_t)k * 24 * Vh, &r2[k]));
            const double rel = e2[k] > 0 ? std::sqrt(r2[k] / e2[k]) : 0.0;
            if (info) info[k].relres_dhat = rel;
            if (rel > sp->tol) again = true;
        }
        if (!again || st != LQCD_OK) break;
        q.tol *= 0.1;
    }
    if (worst == LQCD_OK)
        for (int k = 0; k < nrhs; k++)
            if (e2[k] > 0 && std::sqrt(r2[k] / e2[k]) > sp->tol) worst = LQCD_ERR_NOT_CONVERGED;
    return worst;
}

}  // extern "C"
