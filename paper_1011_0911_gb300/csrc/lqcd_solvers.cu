// Outer solvers: even-odd CGNR on Dhat (Eq. 2) and the flexible GCR of
// Sec. 3-4 on the full operator, preconditioned by SAP or deflated SAP; the
// solution of Dhat psi_e = eta_e is the even part of D^-1 (eta_e, 0) (Eq. 5).
//
// Precision: all Krylov bookkeeping is FP64 (Gram-Schmidt, residual, solution
// update).  The preconditioner and D phi_k may run in FP32 ("inner"
// precision); the recursive residual then carries FP32-level errors, so a
// cycle stops once it has gained ~1e-5 and the next cycle restarts from the
// FP64 true residual eta - D psi.
#include <chrono>
#include <cmath>
#include <vector>

#include "lqcd_internal.cuh"

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Cplx {
    double re, im;
};
inline Cplx cmul(Cplx a, Cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline Cplx cdiv(Cplx a, double b) { return {a.re / b, a.im / b}; }

// ---------------------------------------------------------------- CGNR
lqcd_status cgnr_native(lqcd_ctx *c, const double2 *eta, double2 *x, double tol, int nmx, lqcd_solve_info *info)
{
    const long Vh = c->g.Vh;
    const long n2 = 24 * Vh;   // doubles in one even field
    const size_t hb = native_half_bytes(c, LQCD_F64);
    void *buf;
    LQCD_TRY(ws_get(c, WS_CGNR, 5 * hb, &buf));
    double2 *r = (double2 *)buf, *z = r + 12 * Vh, *p = z + 12 * Vh, *w = p + 12 * Vh, *t = w + 12 * Vh;
    void *tmp_o;
    LQCD_TRY(ws_get(c, WS_TMP_O, hb, &tmp_o));
    auto dhat = [&](const double2 *in, double2 *out) { return dirac_dhat(c, LQCD_F64, in, out, tmp_o, 1); };
    auto dhat_dag = [&](const double2 *in, double2 *out) -> lqcd_status {
        LQCD_TRY(blas_gamma5_native64(c, 1, in, t));
        LQCD_TRY(dirac_dhat(c, LQCD_F64, t, out, tmp_o, 1));
        return blas_gamma5_native64(c, 1, out, out);
    };
    double t0 = now_s();
    LQCD_TRY(blas_zero(c, hb, x));
    LQCD_TRY(blas_copy(c, n2, (const double *)eta, (double *)r));
    double eta2;
    LQCD_TRY(blas_norm2(c, n2, (const double *)eta, &eta2));
    int it = 0;
    lqcd_status st = LQCD_ERR_NOT_CONVERGED;
    double rr = eta2;
    if (eta2 == 0) {
        st = LQCD_OK;
    } else if (!std::isfinite(eta2)) {
        st = LQCD_ERR_NAN;
    } else {
        LQCD_TRY(dhat_dag(r, z));
        LQCD_TRY(blas_copy(c, n2, (const double *)z, (double *)p));
        double zz;
        LQCD_TRY(blas_norm2(c, n2, (const double *)z, &zz));
        while (it < nmx) {
            LQCD_TRY(dhat(p, w));
            double ww;
            LQCD_TRY(blas_norm2(c, n2, (const double *)w, &ww));
            if (!std::isfinite(ww)) {
                st = LQCD_ERR_NAN;
                break;
            }
            if (ww == 0) {
                st = LQCD_ERR_BREAKDOWN;
                break;
            }
            double alpha = zz / ww;
            LQCD_TRY(blas_axpy(c, n2, alpha, 0, (const double *)p, (double *)x));
            LQCD_TRY(blas_axpy(c, n2, -alpha, 0, (const double *)w, (double *)r));
            it++;
            LQCD_TRY(blas_norm2(c, n2, (const double *)r, &rr));
            if (rr <= tol * tol * eta2) {
                // recompute the residual before accepting
                LQCD_TRY(dhat(x, w));
                LQCD_TRY(blas_sub(c, n2, (const double *)eta, (const double *)w, (double *)r));
                LQCD_TRY(blas_norm2(c, n2, (const double *)r, &rr));
                if (rr <= tol * tol * eta2) {
                    st = LQCD_OK;
                    break;
                }
                LQCD_TRY(dhat_dag(r, z));
                LQCD_TRY(blas_copy(c, n2, (const double *)z, (double *)p));
                LQCD_TRY(blas_norm2(c, n2, (const double *)z, &zz));
                continue;
            }
            LQCD_TRY(dhat_dag(r, z));
            double zz1;
            LQCD_TRY(blas_norm2(c, n2, (const double *)z, &zz1));
            LQCD_TRY(blas_xpay(c, n2, (const double *)z, zz1 / zz, (double *)p));
            zz = zz1;
        }
    }
    // final true residual
    LQCD_TRY(dhat(x, w));
    LQCD_TRY(blas_sub(c, n2, (const double *)eta, (const double *)w, (double *)r));
    LQCD_TRY(blas_norm2(c, n2, (const double *)r, &rr));
    if (info) {
        info->iters = it;
        info->restarts = 0;
        info->relres_dhat = eta2 > 0 ? std::sqrt(rr / eta2) : 0;
        info->true_relres = info->relres_dhat;
        info->seconds = now_s() - t0;
        info->status = st;
    }
    return st;
}

// ---------------------------------------------------------------- GCR
struct GcrParams {
    const lqcd_solver_params *sp;
    double tol;
};

// phi = M rho (all native full FP64)
lqcd_status precond(lqcd_ctx *c, const lqcd_solver_params *sp, const double2 *rho, double2 *phi)
{
    const lqcd_sap_params &sap = sp->sap;
    if (sp->solver == LQCD_SOLVER_DFL_SAP_GCR) return dfl_precond_native(c, &sap, rho, phi);
    if (sap.prec == LQCD_F64) return sap_apply(c, &sap, rho, phi);
    void *a, *b;
    size_t fb = 2 * native_half_bytes(c, sap.prec);
    LQCD_TRY(ws_get(c, WS_SAP_IN, fb, &a));
    LQCD_TRY(ws_get(c, WS_SAP_PSI, fb, &b));
    LQCD_TRY(convert_native(c, LQCD_F64, sap.prec, rho, a, 2));
    LQCD_TRY(sap_apply(c, &sap, a, b));
    return convert_native(c, sap.prec, LQCD_F64, b, phi, 2);
}

// chi = D phi in the inner precision, result FP64
lqcd_status apply_D_inner(lqcd_ctx *c, lqcd_prec inner, const double2 *phi, double2 *chi)
{
    if (inner == LQCD_F64) return dirac_D(c, LQCD_F64, phi, chi, 1);
    void *a, *b;
    size_t fb = 2 * native_half_bytes(c, inner);
    LQCD_TRY(ws_get(c, WS_MISC, fb, &a));
    LQCD_TRY(ws_get(c, WS_MISC2, fb, &b));
    LQCD_TRY(convert_native(c, LQCD_F64, inner, phi, a, 2));
    LQCD_TRY(dirac_D(c, inner, a, b, 1));
    return convert_native(c, inner, LQCD_F64, b, chi, 2);
}

// flexible GCR on D psi = eta, warm start from psi; native full FP64 fields
lqcd_status gcr_native(lqcd_ctx *c, const lqcd_solver_params *sp, double tol, const double2 *eta, double2 *psi,
                       int *iters, int *restarts, double *relres, int nmx)
{
    const long Vh = c->g.Vh;
    const long n2 = 48 * Vh;   // doubles in one full field
    const long nf = 24 * Vh;   // double2 in one full field
    const int nkv = sp->nkv;
    if (nkv < 1 || nkv > 64) return set_err(c, LQCD_ERR_ARG, "nkv=%d", nkv);
    void *buf;
    LQCD_TRY(ws_get(c, WS_SOLVER, (size_t)(2 * nkv + 2) * nf * sizeof(double2), &buf));
    double2 *phi = (double2 *)buf, *chi = phi + nkv * nf, *rho = chi + nkv * nf, *w = rho + nf;
    const double inner_gain = sp->inner == LQCD_F64 ? 0.0 : 1e-5;
    double eta2;
    LQCD_TRY(blas_norm2(c, n2, (const double *)eta, &eta2));
    double eta_n = std::sqrt(eta2);
    // rho = eta - D psi
    LQCD_TRY(dirac_D(c, LQCD_F64, psi, w, 1));
    LQCD_TRY(blas_sub(c, n2, (const double *)eta, (const double *)w, (double *)rho));
    double rn2;
    LQCD_TRY(blas_norm2(c, n2, (const double *)rho, &rn2));
    double res = std::sqrt(rn2);
    if (!std::isfinite(res)) return set_err(c, LQCD_ERR_NAN, "non-finite residual");
    int it = 0, rs = 0;
    std::vector<Cplx> a(nkv * nkv), cc(nkv), alpha(nkv);
    std::vector<double> b(nkv);
    std::vector<double> dots(2 * 64), coef(2 * 64);
    lqcd_status st = LQCD_ERR_NOT_CONVERGED;
    if (eta_n == 0 || res <= tol * eta_n) st = LQCD_OK;
    while (st != LQCD_OK && it < nmx) {
        int nk = 0;
        double cycle_start = res;
        for (int k = 0; k < nkv && it < nmx; k++) {
            double2 *ph = phi + k * nf, *ch = chi + k * nf;
            LQCD_TRY(precond(c, sp, rho, ph));
            LQCD_TRY(apply_D_inner(c, sp->inner, ph, ch));
            for (int i = 0; i < k; i++) a[i * nkv + k] = {0, 0};
            for (int pass = 0; pass < 2 && k > 0; pass++) {
                LQCD_TRY(blas_dot(c, n2, (const double *)chi, (const double *)ch, k, n2, dots.data()));
                for (int i = 0; i < k; i++) {
                    a[i * nkv + k].re += dots[2 * i];
                    a[i * nkv + k].im += dots[2 * i + 1];
                }
                LQCD_TRY(blas_multi_axpy(c, n2, k, dots.data(), (const double *)chi, n2, (double *)ch, -1.0));
            }
            double bb;
            LQCD_TRY(blas_norm2(c, n2, (const double *)ch, &bb));
            b[k] = std::sqrt(bb);
            if (!std::isfinite(b[k])) return set_err(c, LQCD_ERR_NAN, "non-finite Krylov vector");
            if (b[k] == 0) {
                st = LQCD_ERR_BREAKDOWN;
                break;
            }
            LQCD_TRY(blas_scal(c, n2, 1.0 / b[k], 0, (double *)ch));
            LQCD_TRY(blas_dot(c, n2, (const double *)ch, (const double *)rho, 1, 0, dots.data()));
            cc[k] = {dots[0], dots[1]};
            LQCD_TRY(blas_axpy(c, n2, -cc[k].re, -cc[k].im, (const double *)ch, (double *)rho));
            it++;
            nk = k + 1;
            double r2;
            LQCD_TRY(blas_norm2(c, n2, (const double *)rho, &r2));
            double rr = std::sqrt(r2);
            if (rr <= tol * eta_n || rr <= inner_gain * cycle_start) break;
        }
        if (st == LQCD_ERR_BREAKDOWN && nk == 0) break;
        for (int j = nk - 1; j >= 0; j--) {
            Cplx s = cc[j];
            for (int i = j + 1; i < nk; i++) {
                Cplx t = cmul(a[j * nkv + i], alpha[i]);
                s.re -= t.re;
                s.im -= t.im;
            }
            alpha[j] = cdiv(s, b[j]);
        }
        for (int j = 0; j < nk; j++) {
            coef[2 * j] = alpha[j].re;
            coef[2 * j + 1] = alpha[j].im;
        }
        LQCD_TRY(blas_multi_axpy(c, n2, nk, coef.data(), (const double *)phi, n2, (double *)psi, 1.0));
        // restart from the FP64 true residual
        LQCD_TRY(dirac_D(c, LQCD_F64, psi, w, 1));
        LQCD_TRY(blas_sub(c, n2, (const double *)eta, (const double *)w, (double *)rho));
        LQCD_TRY(blas_norm2(c, n2, (const double *)rho, &rn2));
        res = std::sqrt(rn2);
        rs++;
        if (!std::isfinite(res)) {
            st = LQCD_ERR_NAN;
            break;
        }
        if (res <= tol * eta_n) st = LQCD_OK;
        else if (st == LQCD_ERR_BREAKDOWN)
            break;
    }
    if (iters) *iters += it;
    if (restarts) *restarts += rs;
    if (relres) *relres = eta_n > 0 ? res / eta_n : 0;
    return st;
}

// even-odd helpers on native fields: even half of a full field is its first half
lqcd_status dhat_relres(lqcd_ctx *c, const double2 *eta_e, const double2 *psi_e, double *out)
{
    const long Vh = c->g.Vh;
    const long n2 = 24 * Vh;
    void *b, *tmp_o;
    LQCD_TRY(ws_get(c, WS_MISC, 2 * native_half_bytes(c, LQCD_F64), &b));
    LQCD_TRY(ws_get(c, WS_TMP_O, native_half_bytes(c, LQCD_F64), &tmp_o));
    double2 *w = (double2 *)b, *r = w + 12 * Vh;
    LQCD_TRY(dirac_dhat(c, LQCD_F64, psi_e, w, tmp_o, 1));
    LQCD_TRY(blas_sub(c, n2, (const double *)eta_e, (const double *)w, (double *)r));
    double rr, ee;
    LQCD_TRY(blas_norm2(c, n2, (const double *)r, &rr));
    LQCD_TRY(blas_norm2(c, n2, (const double *)eta_e, &ee));
    *out = ee > 0 ? std::sqrt(rr / ee) : 0;
    return LQCD_OK;
}

lqcd_status check_params(lqcd_ctx *c, const lqcd_solver_params *p, int nrhs)
{
    if (!p || nrhs < 1) return set_err(c, LQCD_ERR_ARG, "bad solver arguments");
    if (!(p->tol > 0)) return set_err(c, LQCD_ERR_ARG, "tol must be > 0");
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    if (p->solver == LQCD_SOLVER_DFL_SAP_GCR && !c->dfl)
        return set_err(c, LQCD_ERR_STATE, "deflation subspace not built");
    if (p->solver != LQCD_SOLVER_CGNR && (p->inner != LQCD_F64 && p->inner != LQCD_F32))
        return set_err(c, LQCD_ERR_ARG, "inner precision %d", (int)p->inner);
    return LQCD_OK;
}

lqcd_status worst(lqcd_status a, lqcd_status b) { return a != LQCD_OK ? a : b; }

}  // namespace

extern "C" {

lqcd_status lqcd_solve_dhat(lqcd_ctx *c, const lqcd_solver_params *p, const double *eta, double *psi, int nrhs,
                            lqcd_solve_info *info)
{
    if (!c || !eta || !psi) return set_err(c, LQCD_ERR_ARG, "null argument");
    LQCD_TRY(check_params(c, p, nrhs));
    const long Vh = c->g.Vh;
    const size_t hb = native_half_bytes(c, LQCD_F64);
    lqcd_status all = LQCD_OK;
    for (int k = 0; k < nrhs; k++) {
        const double *eta_k = eta + (size_t)k * 24 * Vh;
        double *psi_k = psi + (size_t)k * 24 * Vh;
        lqcd_solve_info li{};
        double t0 = now_s();
        void *io;
        LQCD_TRY(ws_get(c, WS_SOLVE_IO, 4 * hb, &io));
        double2 *eta_f = (double2 *)io, *psi_f = eta_f + 24 * Vh;   // full native fields
        LQCD_TRY(blas_zero(c, 4 * hb, io));
        LQCD_TRY(pack_field(c, LQCD_F64, 1, eta_k, eta_f, 1, false));   // even half, odd = 0
        lqcd_status st;
        if (p->solver == LQCD_SOLVER_CGNR) {
            st = cgnr_native(c, eta_f, psi_f, p->tol, p->nmx, &li);
        } else {
            double tol = p->tol;
            int iters = 0, restarts = 0;
            double rel = 0, rh = 0;
            st = LQCD_OK;
            for (int attempt = 0; attempt < 4; attempt++) {
                st = gcr_native(c, p, tol, eta_f, psi_f, &iters, &restarts, &rel, p->nmx - iters);
                if (st != LQCD_OK) break;
                LQCD_TRY(dhat_relres(c, eta_f, psi_f, &rh));
                if (rh <= p->tol) break;
                // the Dhat residual r_e - H_eo A_oo^-1 r_o is not bounded by |r|: tighten
                tol = tol * std::max(0.05, 0.5 * p->tol / rh);
            }
            if (st == LQCD_OK && rh > p->tol) st = LQCD_ERR_NOT_CONVERGED;
            li.iters = iters;
            li.restarts = restarts;
            li.true_relres = rel;
            li.relres_dhat = rh;
            li.status = st;
            li.seconds = now_s() - t0;
        }
        LQCD_TRY(pack_field(c, LQCD_F64, 1, psi_k, psi_f, 1, true));
        if (info) info[k] = li;
        all = worst(all, st);
    }
    if (all != LQCD_OK && all != LQCD_ERR_CUDA) set_err(c, all, "solve did not converge (status %d)", (int)all);
    return all;
}

lqcd_status lqcd_solve_D(lqcd_ctx *c, const lqcd_solver_params *p, const double *eta, double *psi, int nrhs,
                         lqcd_solve_info *info)
{
    if (!c || !eta || !psi) return set_err(c, LQCD_ERR_ARG, "null argument");
    LQCD_TRY(check_params(c, p, nrhs));
    if (p->solver == LQCD_SOLVER_CGNR) return set_err(c, LQCD_ERR_ARG, "CGNR solves Dhat only");
    const long Vh = c->g.Vh;
    const size_t hb = native_half_bytes(c, LQCD_F64);
    lqcd_status all = LQCD_OK;
    for (int k = 0; k < nrhs; k++) {
        void *io;
        LQCD_TRY(ws_get(c, WS_SOLVE_IO, 4 * hb, &io));
        double2 *eta_f = (double2 *)io, *psi_f = eta_f + 24 * Vh;
        double t0 = now_s();
        LQCD_TRY(pack_field(c, LQCD_F64, 2, eta + (size_t)k * 48 * Vh, eta_f, 1, false));
        LQCD_TRY(blas_zero(c, 2 * hb, psi_f));
        lqcd_solve_info li{};
        int iters = 0, restarts = 0;
        double rel = 0;
        lqcd_status st = gcr_native(c, p, p->tol, eta_f, psi_f, &iters, &restarts, &rel, p->nmx);
        LQCD_TRY(pack_field(c, LQCD_F64, 2, psi + (size_t)k * 48 * Vh, psi_f, 1, true));
        li.iters = iters;
        li.restarts = restarts;
        li.true_relres = rel;
        li.relres_dhat = -1;
        li.status = st;
        li.seconds = now_s() - t0;
        if (info) info[k] = li;
        all = worst(all, st);
    }
    return all;
}

}  // extern "C"
