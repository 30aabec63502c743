// Outer solvers: even-odd CGNR on Dhat (Eq. 2) and the flexible GCR of
// Sec. 3-4 on the full operator, preconditioned by SAP or deflated SAP; the
// solution of Dhat psi_e = eta_e is the even part of D^-1 (eta_e, 0) (Eq. 5).
//
// Precision: the residual, the solution update and the restart residual
// eta - D psi are FP64.  The preconditioner and D phi_k may run in FP32
// ("inner" precision), and with krylov = F32 the Krylov vectors and their
// Gram-Schmidt are FP32 too (FP64 sums); the recursive residual then carries
// FP32-level errors, so a cycle stops once it has gained ~1e-5 and the next
// cycle restarts from the FP64 true residual.
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
// All fields below are native full FP64 fields; nrhs of them are stored one
// after the other (stride nf double2).  The GCR of every right-hand side runs
// in lockstep so that the preconditioner, D and the BLAS-1 kernels each cover
// the whole batch in one launch; every right-hand side keeps its own
// Gram-Schmidt coefficients, and a converged one receives zero updates.

// phi = M rho
lqcd_status precond(lqcd_ctx *c, const lqcd_solver_params *sp, const double2 *rho, double2 *phi, int nrhs)
{
    const lqcd_sap_params &sap = sp->sap;
    if (sp->solver == LQCD_SOLVER_DFL_SAP_GCR) return dfl_precond_native(c, &sap, rho, phi, nrhs);
    if (sp->solver == LQCD_SOLVER_NET_GCR) return net_apply_native(c, rho, phi, nrhs);
    if (sp->solver == LQCD_SOLVER_DFL_NET_GCR) return dfl_precond_native(c, &sap, rho, phi, nrhs, true);
    if (sap.prec == LQCD_F64) return sap_apply(c, &sap, rho, phi, nrhs);
    void *a, *b;
    size_t fb = 2 * native_half_bytes(c, sap.prec) * nrhs;
    LQCD_TRY(ws_get(c, WS_SAP_IN, fb, &a));
    LQCD_TRY(ws_get(c, WS_SAP_PSI, fb, &b));
    LQCD_TRY(convert_native(c, LQCD_F64, sap.prec, rho, a, 2 * nrhs));
    LQCD_TRY(sap_apply(c, &sap, a, b, nrhs));
    return convert_native(c, sap.prec, LQCD_F64, b, phi, 2 * nrhs);
}

// chi = D phi in the inner precision, result FP64
lqcd_status apply_D_inner(lqcd_ctx *c, lqcd_prec inner, const double2 *phi, double2 *chi, int nrhs)
{
    if (inner == LQCD_F64) return dirac_D(c, LQCD_F64, phi, chi, nrhs);
    void *a, *b;
    size_t fb = 2 * native_half_bytes(c, inner) * nrhs;
    LQCD_TRY(ws_get(c, WS_MISC, fb, &a));
    LQCD_TRY(ws_get(c, WS_MISC2, fb, &b));
    LQCD_TRY(convert_native(c, LQCD_F64, inner, phi, a, 2 * nrhs));
    LQCD_TRY(dirac_D(c, inner, a, b, nrhs));
    return convert_native(c, inner, LQCD_F64, b, chi, 2 * nrhs);
}

struct GcrState {
    std::vector<int> iters, restarts, net_fallbacks;
    std::vector<double> relres;
    std::vector<lqcd_status> status;
    explicit GcrState(int nrhs)
        : iters(nrhs, 0), restarts(nrhs, 0), net_fallbacks(nrhs, 0), relres(nrhs, 0),
          status(nrhs, LQCD_ERR_NOT_CONVERGED)
    {
    }
};

// LQCD_PROFILE=1: synchronise around the phases of the GCR and report their
// wall time on stderr (developer instrumentation; off by default)
struct PhaseProf {
    bool on;
    double t[4] = {0, 0, 0, 0};
    double t0 = 0;
    explicit PhaseProf(lqcd_ctx *c) : on(getenv("LQCD_PROFILE") && getenv("LQCD_PROFILE")[0] == '1'), ctx(c) {}
    lqcd_ctx *ctx;
    void start()
    {
        if (!on) return;
        cudaStreamSynchronize(ctx->stream);
        t0 = now_s();
    }
    void stop(int i)
    {
        if (!on) return;
        cudaStreamSynchronize(ctx->stream);
        t[i] += now_s() - t0;
    }
    ~PhaseProf()
    {
        if (!on) return;
        fprintf(stderr, "[lqcd gcr] precond %.4f s, D_inner %.4f s, gram-schmidt %.4f s, restart %.4f s\n", t[0],
                t[1], t[2], t[3]);
        double *p = ctx->prof_t;
        if (p[0] + p[1] + p[2] + p[3] + p[4] + p[5] > 0)
            fprintf(stderr,
                    "[lqcd dfl] project %.4f s, coarse %.4f s, expand %.4f s, D+sub %.4f s, sap %.4f s, "
                    "axpy %.4f s\n",
                    p[0], p[1], p[2], p[3], p[4], p[5]);
        fprintf(stderr, "[lqcd gcr] gram-schmidt %.1f GB, %.0f GB/s, %ld second passes\n", ctx->prof_gs_bytes * 1e-9,
                t[2] > 0 ? ctx->prof_gs_bytes * 1e-9 / t[2] : 0.0, ctx->prof_gs_second);
        for (int i = 0; i < 8; i++) p[i] = 0;
        ctx->prof_gs_bytes = 0;
        ctx->prof_gs_second = 0;
    }
};

// per-rhs squared norms of nrhs fields
lqcd_status bnorm2(lqcd_ctx *c, long n2, int nrhs, const double2 *x, std::vector<double> &out)
{
    std::vector<double> d(2 * nrhs);
    LQCD_TRY(bblas_dot(c, n2, nrhs, (const double *)x, 0, n2, (const double *)x, n2, 1, d.data()));
    out.resize(nrhs);
    for (int r = 0; r < nrhs; r++) out[r] = d[2 * r];
    return LQCD_OK;
}

// Krylov-vector storage of the GCR.  Krylov64: phi_k and chi_k native F64
// full fields.  Krylov32 (krylov = inner = F32): phi_k and chi_k native F32
// full fields, so D phi_k runs on them directly and the Gram-Schmidt moves
// half the bytes and leaves GB300's FP64 pipe (FP64 products bound it at about
// a third of HBM bandwidth); rho and psi stay F64, the products with FP32
// vectors are formed in float and accumulated in double.
struct Krylov64 {
    using T = double2;
    lqcd_ctx *c;
    const lqcd_solver_params *sp;
    int nrhs;
    long nf;   // elements (double2) per full field
    long n2;   // doubles per full field
    Krylov64(lqcd_ctx *ctx, const lqcd_solver_params *p, int n)
        : c(ctx), sp(p), nrhs(n), nf(24 * (long)ctx->g.Vh), n2(48 * (long)ctx->g.Vh)
    {
    }
    size_t field_bytes() const { return nf * sizeof(T); }
    lqcd_status precond_with(const lqcd_solver_params *p, const double2 *rho, T *ph)
    {
        return precond(c, p, rho, ph, nrhs);
    }
    lqcd_status D_inner(const T *ph, T *ch) { return apply_D_inner(c, sp->inner, ph, ch, nrhs); }
    lqcd_status dots(const T *A, long sa, const T *B, int kk, double *out)
    {
        return bblas_dot(c, n2, nrhs, (const double *)A, 2 * sa, n2, (const double *)B, n2, kk, out);
    }
    lqcd_status axpy(int k, const double *cf, const T *X, long sa, T *y, double sign)
    {
        return bblas_multi_axpy(c, n2, nrhs, k, cf, (const double *)X, 2 * sa, n2, (double *)y, n2, sign);
    }
    // |chi|^2 and <rho, chi> (the family {chi, rho} against chi)
    lqcd_status norm_rdot(const T *ch, const double2 *rho, double *out)
    {
        return bblas_dot(c, n2, nrhs, (const double *)ch, 2 * (rho - ch), n2, (const double *)ch, n2, 2, out);
    }
    // rho -= cR chi; chi *= s
    lqcd_status rho_update(const double *cR, const double *s, T *ch, double2 *rho)
    {
        std::vector<double> cs(2 * nrhs);
        for (int r = 0; r < nrhs; r++) {
            cs[2 * r] = s[r] - 1.0;
            cs[2 * r + 1] = 0.0;
        }
        LQCD_TRY(bblas_multi_axpy(c, n2, nrhs, 1, cR, (const double *)ch, 0, n2, (double *)rho, n2, -1.0));
        return bblas_multi_axpy(c, n2, nrhs, 1, cs.data(), (const double *)ch, 0, n2, (double *)ch, n2, 1.0);
    }
    lqcd_status psi_update(int nk, const double *cf, const T *phi, long sa, double2 *psi)
    {
        return bblas_multi_axpy(c, n2, nrhs, nk, cf, (const double *)phi, 2 * sa, n2, (double *)psi, n2, 1.0);
    }
    double final_fields() const { return 7.0; }   // F64-field transfers of norm_rdot + rho_update
};

struct Krylov32 {
    using T = float4;
    lqcd_ctx *c;
    const lqcd_solver_params *sp;
    int nrhs;
    long nf;    // elements (float4) per full F32 field
    long nf64;  // double2 per full F64 field
    Krylov32(lqcd_ctx *ctx, const lqcd_solver_params *p, int n)
        : c(ctx), sp(p), nrhs(n), nf(12 * (long)ctx->g.Vh), nf64(24 * (long)ctx->g.Vh)
    {
    }
    size_t field_bytes() const { return nf * sizeof(T); }
    // the preconditioner's output in F32: SAP in F32 writes it directly, other
    // forms are converted from their own output precision
    lqcd_status precond_with(const lqcd_solver_params *p, const double2 *rho, T *ph)
    {
        const lqcd_sap_params &sap = p->sap;
        if (p->solver == LQCD_SOLVER_SAP_GCR && sap.prec != LQCD_F64) {
            void *a;
            const size_t fb = 2 * native_half_bytes(c, sap.prec) * nrhs;
            LQCD_TRY(ws_get(c, WS_SAP_IN, fb, &a));
            LQCD_TRY(convert_native(c, LQCD_F64, sap.prec, rho, a, 2 * nrhs));
            if (sap.prec == LQCD_F32) return sap_apply(c, &sap, a, ph, nrhs);
            void *b;
            LQCD_TRY(ws_get(c, WS_SAP_PSI, fb, &b));
            LQCD_TRY(sap_apply(c, &sap, a, b, nrhs));
            return convert_native(c, sap.prec, LQCD_F32, b, ph, 2 * nrhs);
        }
        void *t;
        LQCD_TRY(ws_get(c, WS_PHI64, (size_t)nf64 * nrhs * sizeof(double2), &t));
        LQCD_TRY(precond(c, p, rho, (double2 *)t, nrhs));
        return convert_native(c, LQCD_F64, LQCD_F32, t, ph, 2 * nrhs);
    }
    lqcd_status D_inner(const T *ph, T *ch) { return dirac_D(c, LQCD_F32, ph, ch, nrhs); }
    lqcd_status dots(const T *A, long sa, const T *B, int kk, double *out)
    {
        return bdot32(c, nf, nrhs, A, sa, nf, B, nf, kk, out);
    }
    lqcd_status axpy(int k, const double *cf, const T *X, long sa, T *y, double sign)
    {
        return bmulti_axpy32(c, nf, nrhs, k, cf, X, sa, nf, y, nf, sign);
    }
    lqcd_status norm_rdot(const T *ch, const double2 *rho, double *out)
    {
        return bnorm_rdot32(c, nrhs, ch, nf, rho, nf64, out);
    }
    lqcd_status rho_update(const double *cR, const double *s, T *ch, double2 *rho)
    {
        return brho_update32(c, nrhs, cR, s, ch, nf, rho, nf64);
    }
    lqcd_status psi_update(int nk, const double *cf, const T *phi, long sa, double2 *psi)
    {
        return bmulti_axpy_mixed(c, nrhs, nk, cf, phi, sa, nf, psi, nf64);
    }
    double final_fields() const { return 4.5; }
};

// flexible GCR on D psi_r = eta_r, warm start from psi; tol per rhs
template <class KV>
lqcd_status gcr_impl(lqcd_ctx *c, const lqcd_solver_params *sp, const std::vector<double> &tol, const double2 *eta,
                     double2 *psi, int nrhs, int nmx, GcrState &S)
{
    using T = typename KV::T;
    KV kv(c, sp, nrhs);
    const long Vh = c->g.Vh;
    const long n2 = 48 * Vh;   // doubles in one full F64 field
    const long nf = kv.nf;     // Krylov elements per field
    const int nkv = sp->nkv;
    if (nkv < 1 || nkv > 64) return set_err(c, LQCD_ERR_ARG, "nkv=%d", nkv);
    if (nrhs * nkv > 1024 || nrhs > 64) return set_err(c, LQCD_ERR_ARG, "nrhs=%d with nkv=%d too large", nrhs, nkv);
    const long bf = nrhs * nf;   // Krylov elements per batch of fields
    const size_t bf64 = (size_t)nrhs * 24 * Vh;   // double2 per batch of F64 fields
    void *buf;
    LQCD_TRY(ws_get(c, WS_SOLVER, 2 * nkv * bf * sizeof(T) + 2 * bf64 * sizeof(double2), &buf));
    T *phi = (T *)buf, *chi = phi + nkv * bf;
    double2 *rho = (double2 *)(chi + nkv * bf), *w = rho + bf64;
    const double inner_gain = sp->inner == LQCD_F64 ? 0.0 : 1e-5;
    const double gs_field = (double)bf * sizeof(T);
    PhaseProf prof(c);
    std::vector<double> eta2, rn2, eta_n(nrhs), res(nrhs), cycle_start(nrhs);
    LQCD_TRY(bnorm2(c, n2, nrhs, eta, eta2));
    LQCD_TRY(dirac_D(c, LQCD_F64, psi, w, nrhs));
    LQCD_TRY(blas_sub(c, n2 * nrhs, (const double *)eta, (const double *)w, (double *)rho));
    LQCD_TRY(bnorm2(c, n2, nrhs, rho, rn2));
    std::vector<char> active(nrhs);
    for (int r = 0; r < nrhs; r++) {
        eta_n[r] = std::sqrt(eta2[r]);
        res[r] = std::sqrt(rn2[r]);
        if (!std::isfinite(res[r])) S.status[r] = LQCD_ERR_NAN;
        else if (eta_n[r] == 0 || res[r] <= tol[r] * eta_n[r]) S.status[r] = LQCD_OK;
        else S.status[r] = LQCD_ERR_NOT_CONVERGED;
        active[r] = S.status[r] == LQCD_ERR_NOT_CONVERGED;
    }
    // per rhs: a[r][i][k], b[r][k], cc[r][k], alpha[r][k]
    std::vector<Cplx> a((size_t)nrhs * nkv * nkv), cc((size_t)nrhs * nkv), alpha((size_t)nrhs * nkv);
    std::vector<double> b((size_t)nrhs * nkv), dots(2 * (size_t)nrhs * 64), coef(2 * (size_t)nrhs * 64);
    int it = 0;
    auto any_active = [&]() {
        for (int r = 0; r < nrhs; r++)
            if (active[r]) return true;
        return false;
    };
    while (any_active() && it < nmx) {
        int nk = 0;
        std::vector<char> done(nrhs, 0);
        for (int r = 0; r < nrhs; r++) cycle_start[r] = res[r];
        for (int k = 0; k < nkv && it < nmx; k++) {
            T *ph = phi + k * bf, *ch = chi + k * bf;
            prof.start();
            LQCD_TRY(kv.precond_with(sp, rho, ph));
            prof.stop(0);
            // chi_k = D phi_k, orthogonalised against chi_0..chi_{k-1}; leaves |chi_k|^2
            // and <rho, chi_k> in dots
            auto orth = [&]() -> lqcd_status {
                prof.start();
                LQCD_TRY(kv.D_inner(ph, ch));
                prof.stop(1);
                prof.start();
                for (int r = 0; r < nrhs; r++)
                    for (int i = 0; i < k; i++) a[((size_t)r * nkv + i) * nkv + k] = {0, 0};
                // classical Gram-Schmidt; a second pass only where the first removed more
                // than half of |chi_k|^2 (Daniel-Gragg-Kaufman-Stewart criterion).  The
                // first pass reduces chi_0..chi_k against chi_k, which also gives |chi_k|^2.
                for (int pass = 0; pass < 2 && k > 0; pass++) {
                    const int kk = pass == 0 ? k + 1 : k;
                    LQCD_TRY(kv.dots(chi, bf, ch, kk, dots.data()));
                    bool again = false;
                    std::vector<double> cf(2 * (size_t)nrhs * k);
                    for (int r = 0; r < nrhs; r++) {
                        double removed = 0;
                        for (int i = 0; i < k; i++) {
                            const double dr = dots[2 * (r * kk + i)], di = dots[2 * (r * kk + i) + 1];
                            a[((size_t)r * nkv + i) * nkv + k].re += dr;
                            a[((size_t)r * nkv + i) * nkv + k].im += di;
                            cf[2 * (r * k + i)] = dr;
                            cf[2 * (r * k + i) + 1] = di;
                            removed += dr * dr + di * di;
                        }
                        if (pass == 0 && active[r] && removed > 0.5 * dots[2 * (r * kk + k)]) again = true;
                    }
                    LQCD_TRY(kv.axpy(k, cf.data(), chi, bf, ch, -1.0));
                    // bytes: the dot reads kk + 1 fields, the update k + 1 and writes one
                    c->prof_gs_bytes += (kk + 1 + k + 2) * gs_field;
                    if (!again) break;
                    c->prof_gs_second += pass == 0;
                }
                return kv.norm_rdot(ch, rho, dots.data());
            };
            LQCD_TRY(orth());
            if (sp->solver == LQCD_SOLVER_NET_GCR || sp->solver == LQCD_SOLVER_DFL_NET_GCR) {
                // the network's direction must cut |rho| to 0.95 |rho| at least, i.e.
                // |c_k|^2 >= (1 - 0.95^2) |rho|^2; where it does not, SAP replaces it
                std::vector<int> reject;
                for (int r = 0; r < nrhs; r++) {
                    if (!active[r]) continue;
                    const double q2 = dots[2 * (2 * r)];
                    const double c2 = q2 > 0 ? (dots[2 * (2 * r + 1)] * dots[2 * (2 * r + 1)] +
                                                dots[2 * (2 * r + 1) + 1] * dots[2 * (2 * r + 1) + 1]) / q2
                                             : 0.0;
                    if (!std::isfinite(c2) || !std::isfinite(q2) || c2 < (1.0 - 0.95 * 0.95) * rn2[r]) reject.push_back(r);
                }
                if (!reject.empty()) {
                    void *fb;
                    LQCD_TRY(ws_get(c, WS_NET_FALLBACK, (size_t)bf * sizeof(T), &fb));
                    lqcd_solver_params sap_only = *sp;
                    sap_only.solver = sp->solver == LQCD_SOLVER_DFL_NET_GCR ? LQCD_SOLVER_DFL_SAP_GCR
                                                                            : LQCD_SOLVER_SAP_GCR;
                    LQCD_TRY(kv.precond_with(&sap_only, rho, (T *)fb));
                    for (int r : reject) {
                        LQCD_CUDA_CHECK(c, cudaMemcpyAsync(ph + r * nf, (T *)fb + r * nf, kv.field_bytes(),
                                                           cudaMemcpyDeviceToDevice, c->stream));
                        S.net_fallbacks[r]++;
                    }
                    LQCD_TRY(orth());
                }
            }
            std::vector<double> sx(nrhs);
            for (int r = 0; r < nrhs; r++) {
                const double bk = std::sqrt(dots[2 * (2 * r)]);
                b[(size_t)r * nkv + k] = bk;
                const double s = (bk > 0 && std::isfinite(bk)) ? 1.0 / bk : 0.0;
                if (active[r] && s == 0.0) {
                    S.status[r] = std::isfinite(bk) ? LQCD_ERR_BREAKDOWN : LQCD_ERR_NAN;
                    active[r] = 0;
                }
                // c_k = <chi_k / b_k, rho> = conj(<rho, chi_k>) / b_k
                const double cr = dots[2 * (2 * r + 1)] * s, ci = -dots[2 * (2 * r + 1) + 1] * s;
                cc[(size_t)r * nkv + k] = {cr, ci};
                // rho -= c_k chi_k / b_k (chi_k not yet normalised); chi_k *= 1/b_k
                coef[2 * r] = active[r] ? cr * s : 0.0;
                coef[2 * r + 1] = active[r] ? ci * s : 0.0;
                sx[r] = s;
                if (active[r]) rn2[r] = std::max(0.0, rn2[r] - (cr * cr + ci * ci));
            }
            LQCD_TRY(kv.rho_update(coef.data(), sx.data(), ch, rho));
            c->prof_gs_bytes += kv.final_fields() * (double)bf64 * sizeof(double2);
            it++;
            nk = k + 1;
            bool recompute = false;
            for (int r = 0; r < nrhs; r++) {
                if (active[r]) S.iters[r]++;
                // |rho|^2 - |c|^2 loses digits once |rho| has dropped ~1e7 within the cycle
                if (active[r] && rn2[r] < 1e-14 * cycle_start[r] * cycle_start[r]) recompute = true;
            }
            if (recompute) LQCD_TRY(bnorm2(c, n2, nrhs, rho, rn2));
            prof.stop(2);
            bool all_done = true;
            for (int r = 0; r < nrhs; r++) {
                double rr = std::sqrt(rn2[r]);
                if (!active[r] || rr <= tol[r] * eta_n[r] || rr <= inner_gain * cycle_start[r]) done[r] = 1;
                all_done = all_done && done[r];
            }
            if (all_done) break;
        }
        // back substitution per rhs: alpha_j = (c_j - sum_{i>j} a_ji alpha_i) / b_j
        for (int r = 0; r < nrhs; r++) {
            for (int j = nk - 1; j >= 0; j--) {
                Cplx s = cc[(size_t)r * nkv + j];
                for (int i = j + 1; i < nk; i++) {
                    Cplx t = cmul(a[((size_t)r * nkv + j) * nkv + i], alpha[(size_t)r * nkv + i]);
                    s.re -= t.re;
                    s.im -= t.im;
                }
                double bj = b[(size_t)r * nkv + j];
                alpha[(size_t)r * nkv + j] = (active[r] && bj > 0) ? cdiv(s, bj) : Cplx{0, 0};
            }
            for (int j = 0; j < nk; j++) {
                coef[2 * (r * nk + j)] = alpha[(size_t)r * nkv + j].re;
                coef[2 * (r * nk + j) + 1] = alpha[(size_t)r * nkv + j].im;
            }
        }
        prof.start();
        if (nk > 0) LQCD_TRY(kv.psi_update(nk, coef.data(), phi, bf, psi));
        // restart from the FP64 true residual
        LQCD_TRY(dirac_D(c, LQCD_F64, psi, w, nrhs));
        LQCD_TRY(blas_sub(c, n2 * nrhs, (const double *)eta, (const double *)w, (double *)rho));
        LQCD_TRY(bnorm2(c, n2, nrhs, rho, rn2));
        prof.stop(3);
        for (int r = 0; r < nrhs; r++) {
            if (!active[r]) continue;
            res[r] = std::sqrt(rn2[r]);
            S.restarts[r]++;
            if (!std::isfinite(res[r])) {
                S.status[r] = LQCD_ERR_NAN;
                active[r] = 0;
            } else if (res[r] <= tol[r] * eta_n[r]) {
                S.status[r] = LQCD_OK;
                active[r] = 0;
            }
        }
    }
    for (int r = 0; r < nrhs; r++) S.relres[r] = eta_n[r] > 0 ? res[r] / eta_n[r] : 0;
    return LQCD_OK;
}

// Krylov vectors in F64 or (krylov == F32, inner == F32) in F32
lqcd_status gcr_native(lqcd_ctx *c, const lqcd_solver_params *sp, const std::vector<double> &tol,
                       const double2 *eta, double2 *psi, int nrhs, int nmx, GcrState &S)
{
    if (sp->krylov == LQCD_F32) return gcr_impl<Krylov32>(c, sp, tol, eta, psi, nrhs, nmx, S);
    return gcr_impl<Krylov64>(c, sp, tol, eta, psi, nrhs, nmx, S);
}

// |eta_e - Dhat psi_e| / |eta_e| per rhs; eta, psi: nrhs native full fields (even halves used)
lqcd_status dhat_relres(lqcd_ctx *c, const double2 *eta, const double2 *psi, int nrhs, std::vector<double> &out)
{
    const long Vh = c->g.Vh;
    const long n2 = 24 * Vh;   // doubles in one even field
    const long nf = 24 * Vh;   // double2 per full field
    void *b, *tmp_o;
    LQCD_TRY(ws_get(c, WS_MISC, 2 * native_half_bytes(c, LQCD_F64), &b));
    LQCD_TRY(ws_get(c, WS_TMP_O, native_half_bytes(c, LQCD_F64), &tmp_o));
    double2 *w = (double2 *)b, *rr = w + 12 * Vh;
    out.resize(nrhs);
    for (int r = 0; r < nrhs; r++) {
        LQCD_TRY(dirac_dhat(c, LQCD_F64, psi + r * nf, w, tmp_o, 1));
        LQCD_TRY(blas_sub(c, n2, (const double *)(eta + r * nf), (const double *)w, (double *)rr));
        double x, e;
        LQCD_TRY(blas_norm2(c, n2, (const double *)rr, &x));
        LQCD_TRY(blas_norm2(c, n2, (const double *)(eta + r * nf), &e));
        out[r] = e > 0 ? std::sqrt(x / e) : 0;
    }
    return LQCD_OK;
}

lqcd_status check_params(lqcd_ctx *c, const lqcd_solver_params *p, int nrhs)
{
    if (!p || nrhs < 1) return set_err(c, LQCD_ERR_ARG, "bad solver arguments");
    if (!(p->tol > 0)) return set_err(c, LQCD_ERR_ARG, "tol must be > 0");
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    if ((p->solver == LQCD_SOLVER_DFL_SAP_GCR || p->solver == LQCD_SOLVER_DFL_NET_GCR) && !c->dfl)
        return set_err(c, LQCD_ERR_STATE, "deflation subspace not built");
    if ((p->solver == LQCD_SOLVER_NET_GCR || p->solver == LQCD_SOLVER_DFL_NET_GCR) && !c->net)
        return set_err(c, LQCD_ERR_STATE, "network not set");
    if (p->solver < LQCD_SOLVER_CGNR || p->solver > LQCD_SOLVER_DFL_NET_GCR)
        return set_err(c, LQCD_ERR_ARG, "solver %d", (int)p->solver);
    if (p->solver != LQCD_SOLVER_CGNR && (p->inner != LQCD_F64 && p->inner != LQCD_F32))
        return set_err(c, LQCD_ERR_ARG, "inner precision %d", (int)p->inner);
    if (p->krylov != LQCD_F64 && !(p->krylov == LQCD_F32 && p->inner == LQCD_F32))
        return set_err(c, LQCD_ERR_ARG, "Krylov precision %d with inner precision %d", (int)p->krylov,
                       (int)p->inner);
    return LQCD_OK;
}

lqcd_status worst(lqcd_status a, lqcd_status b) { return a != LQCD_OK ? a : b; }

// guess: psi holds the initial even-site guess x0 on entry (GCR solvers); the
// odd part of the full-lattice start is -A_oo^-1 H_oe x0, so that the full
// residual starts as (eta_e - Dhat x0, 0)
lqcd_status solve_dhat_impl(lqcd_ctx *c, const lqcd_solver_params *p, const double *eta, double *psi, int nrhs,
                            lqcd_solve_info *info, bool guess)
{
    if (!c || !eta || !psi) return set_err(c, LQCD_ERR_ARG, "null argument");
    LQCD_TRY(check_params(c, p, nrhs));
    if (guess && p->solver == LQCD_SOLVER_CGNR) return set_err(c, LQCD_ERR_ARG, "initial guesses are for the GCR solvers");
    const long Vh = c->g.Vh;
    const long nf = 24 * Vh;
    const size_t hb = native_half_bytes(c, LQCD_F64);
    lqcd_status all = LQCD_OK;
    double t0 = now_s();
    if (p->solver == LQCD_SOLVER_CGNR) {
        for (int k = 0; k < nrhs; k++) {
            lqcd_solve_info li{};
            void *io;
            LQCD_TRY(ws_get(c, WS_SOLVE_IO, 4 * hb, &io));
            double2 *eta_f = (double2 *)io, *psi_f = eta_f + nf;
            LQCD_TRY(blas_zero(c, 4 * hb, io));
            LQCD_TRY(pack_field(c, LQCD_F64, 1, eta + (size_t)k * 24 * Vh, eta_f, 1, false));
            lqcd_status st = cgnr_native(c, eta_f, psi_f, p->tol, p->nmx, &li);
            LQCD_TRY(pack_field(c, LQCD_F64, 1, psi + (size_t)k * 24 * Vh, psi_f, 1, true));
            if (info) info[k] = li;
            all = worst(all, st);
        }
    } else {
        // full fields (eta_e, 0) for every rhs, solved together
        void *io;
        LQCD_TRY(ws_get(c, WS_SOLVE_IO, 4 * hb * nrhs, &io));
        double2 *eta_f = (double2 *)io, *psi_f = eta_f + nrhs * nf;
        LQCD_TRY(blas_zero(c, 4 * hb * nrhs, io));
        for (int k = 0; k < nrhs; k++)
            LQCD_TRY(pack_field(c, LQCD_F64, 1, eta + (size_t)k * 24 * Vh, eta_f + k * nf, 1, false));
        if (guess) {
            const long hh = 12 * Vh;   // double2 in one half field
            for (int k = 0; k < nrhs; k++)
                LQCD_TRY(pack_field(c, LQCD_F64, 1, psi + (size_t)k * 24 * Vh, psi_f + k * nf, 1, false));
            LQCD_TRY(dirac_hop_parity(c, LQCD_F64, 1, psi_f, psi_f + hh, nf, nf, nrhs));
            for (int k = 0; k < nrhs; k++) {
                double2 *po = psi_f + k * nf + hh;
                LQCD_TRY(clover_apply_native64(c, 1, 1, po, po));
                LQCD_TRY(blas_scal(c, 2 * hh, -1.0, 0.0, (double *)po));
            }
        }
        GcrState S(nrhs);
        std::vector<double> tol(nrhs, p->tol), rh(nrhs, 0);
        for (int attempt = 0; attempt < 4; attempt++) {
            int used = 0;
            for (int k = 0; k < nrhs; k++) used = std::max(used, S.iters[k]);
            LQCD_TRY(gcr_native(c, p, tol, eta_f, psi_f, nrhs, p->nmx - used, S));
            LQCD_TRY(dhat_relres(c, eta_f, psi_f, nrhs, rh));
            bool again = false;
            for (int k = 0; k < nrhs; k++)
                if (S.status[k] == LQCD_OK && rh[k] > p->tol) {
                    // the Dhat residual r_e - H_eo A_oo^-1 r_o is not bounded by |r|: tighten
                    tol[k] = tol[k] * std::max(0.05, 0.5 * p->tol / rh[k]);
                    S.status[k] = LQCD_ERR_NOT_CONVERGED;
                    again = true;
                }
            if (!again) break;
        }
        for (int k = 0; k < nrhs; k++) {
            if (S.status[k] == LQCD_OK && rh[k] > p->tol) S.status[k] = LQCD_ERR_NOT_CONVERGED;
            LQCD_TRY(pack_field(c, LQCD_F64, 1, psi + (size_t)k * 24 * Vh, psi_f + k * nf, 1, true));
            if (info) {
                info[k].iters = S.iters[k];
                info[k].restarts = S.restarts[k];
                info[k].true_relres = S.relres[k];
                info[k].relres_dhat = rh[k];
                info[k].status = S.status[k];
                info[k].seconds = now_s() - t0;
                info[k].net_fallbacks = S.net_fallbacks[k];
            }
            all = worst(all, S.status[k]);
        }
    }
    if (all != LQCD_OK && all != LQCD_ERR_CUDA) set_err(c, all, "solve did not converge (status %d)", (int)all);
    return all;
}

}  // namespace

extern "C" {

lqcd_status lqcd_solve_dhat(lqcd_ctx *c, const lqcd_solver_params *p, const double *eta, double *psi, int nrhs,
                            lqcd_solve_info *info)
{
    return solve_dhat_impl(c, p, eta, psi, nrhs, info, false);
}

lqcd_status lqcd_solve_dhat_guess(lqcd_ctx *c, const lqcd_solver_params *p, const double *eta, double *psi,
                                  int nrhs, lqcd_solve_info *info)
{
    return solve_dhat_impl(c, p, eta, psi, nrhs, info, true);
}

lqcd_status lqcd_solve_D(lqcd_ctx *c, const lqcd_solver_params *p, const double *eta, double *psi, int nrhs,
                         lqcd_solve_info *info)
{
    if (!c || !eta || !psi) return set_err(c, LQCD_ERR_ARG, "null argument");
    LQCD_TRY(check_params(c, p, nrhs));
    if (p->solver == LQCD_SOLVER_CGNR) return set_err(c, LQCD_ERR_ARG, "CGNR solves Dhat only");
    const long Vh = c->g.Vh;
    const long nf = 24 * Vh;
    const size_t hb = native_half_bytes(c, LQCD_F64);
    double t0 = now_s();
    void *io;
    LQCD_TRY(ws_get(c, WS_SOLVE_IO, 4 * hb * nrhs, &io));
    double2 *eta_f = (double2 *)io, *psi_f = eta_f + nrhs * nf;
    LQCD_TRY(pack_field(c, LQCD_F64, 2, eta, eta_f, nrhs, false));
    LQCD_TRY(blas_zero(c, 2 * hb * nrhs, psi_f));
    GcrState S(nrhs);
    std::vector<double> tol(nrhs, p->tol);
    LQCD_TRY(gcr_native(c, p, tol, eta_f, psi_f, nrhs, p->nmx, S));
    LQCD_TRY(pack_field(c, LQCD_F64, 2, psi, psi_f, nrhs, true));
    lqcd_status all = LQCD_OK;
    for (int k = 0; k < nrhs; k++) {
        if (info) {
            info[k].iters = S.iters[k];
            info[k].restarts = S.restarts[k];
            info[k].true_relres = S.relres[k];
            info[k].relres_dhat = -1;
            info[k].status = S.status[k];
            info[k].seconds = now_s() - t0;
            info[k].net_fallbacks = S.net_fallbacks[k];
        }
        all = worst(all, S.status[k]);
    }
    return all;
}

}  // extern "C"
