/*
 * Oracle, part 2: solvers.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 *  - CGNR: conjugate gradient on the normal equation of the even-odd Schur
 *    complement Dhat of Eq. 2, with Dhat^dag = gamma5 Dhat gamma5.
 *    Pinned by: the exact solution of a dense 2^4 / 4^4 system (library LU),
 *    and the true residual recomputed from the definition of Dhat.
 *  - SAP: Schwarz alternating procedure on 4^4 (generally bs[]) blocks with
 *    even-odd block MinRes, the preconditioner named with the solver in
 *    Sec. 3-4.  The paper does not print the algorithm; the steps below are
 *    the reading recorded in the design notes.  A heuristic: parity of SAP
 *    itself is UNPINNED as a "correct value"; pinned only by the special case
 *    that one block covering the whole lattice with many MinRes steps gives
 *    Dhat^-1, and by the Dirichlet block operator equalling the dense
 *    restriction P D P.
 *  - GCR: flexible generalised conjugate residual (Sec. 3-4), preconditioned
 *    by the identity, SAP or deflated SAP.  Pinned by the true residual and by
 *    agreement with the dense LU solution.
 */
#include "oracle_internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- plain BLAS-1 on complex vectors of n entries (serial sums) ---- */
static ocplx vdot(long n, const ocplx *a, const ocplx *b)
{
    ocplx s = 0;
    for (long i = 0; i < n; i++) s += conj(a[i]) * b[i];
    return s;
}
static double vnorm2(long n, const ocplx *a)
{
    double s = 0;
    for (long i = 0; i < n; i++) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}
static void vaxpy(long n, ocplx a, const ocplx *x, ocplx *y)
{
    for (long i = 0; i < n; i++) y[i] += a * x[i];
}

/* ------------------------------------------------------------------------ */
/* CGNR on Dhat (even sites)                                                */

int or_cgnr(const oracle *o, const double *eta_, double *psi_, double tol, int maxit, int *iters)
{
    long n = 12 * o->Vh;
    const ocplx *eta = (const ocplx *)eta_;
    ocplx *x = (ocplx *)psi_;
    ocplx *r = malloc(sizeof(ocplx) * n), *z = malloc(sizeof(ocplx) * n);
    ocplx *p = malloc(sizeof(ocplx) * n), *w = malloc(sizeof(ocplx) * n);
    for (long i = 0; i < n; i++) {
        x[i] = 0;
        r[i] = eta[i];
    }
    double eta2 = vnorm2(n, eta);
    int status = OR_ERR_NOT_CONVERGED, it = 0;
    if (eta2 == 0) {
        status = OR_OK;
        goto done;
    }
    or_apply_Dhat_dag(o, (double *)r, (double *)z);
    memcpy(p, z, sizeof(ocplx) * n);
    double zz = vnorm2(n, z);
    while (it < maxit) {
        or_apply_Dhat(o, (double *)p, (double *)w);
        double ww = vnorm2(n, w);
        if (ww == 0) {
            status = OR_ERR_BREAKDOWN;
            break;
        }
        double alpha = zz / ww;
        vaxpy(n, alpha, p, x);
        vaxpy(n, -alpha, w, r);
        it++;
        if (vnorm2(n, r) <= tol * tol * eta2) {
            /* recompute the residual from its definition before stopping */
            or_apply_Dhat(o, (double *)x, (double *)w);
            for (long i = 0; i < n; i++) r[i] = eta[i] - w[i];
            if (vnorm2(n, r) <= tol * tol * eta2) {
                status = OR_OK;
                break;
            }
            or_apply_Dhat_dag(o, (double *)r, (double *)z);
            memcpy(p, z, sizeof(ocplx) * n);
            zz = vnorm2(n, z);
            continue;
        }
        or_apply_Dhat_dag(o, (double *)r, (double *)z);
        double zz1 = vnorm2(n, z);
        double beta = zz1 / zz;
        for (long i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        zz = zz1;
    }
done:
    if (iters) *iters = it;
    free(r);
    free(z);
    free(p);
    free(w);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Block decomposition for SAP                                              */

/* Dhat_blk rho = A_ee rho - H_eo,blk A_oo^-1 H_oe,blk rho on one block */
static void block_dhat(const oracle *o, const blocking *B, long blk, const ocplx *rho, ocplx *out,
                       ocplx *tmp_o)
{
    long h = B->vol / 2;
    const long *se = B->se + blk * h, *so = B->so + blk * h;
    for (long k = 0; k < h; k++) {
        ocplx t[12];
        ob_block_hop_site(o, B, blk, rho, so[k], t);
        ob_mat12_vec(o->Ainv + 144 * so[k], t, tmp_o + 12 * k);
    }
    for (long k = 0; k < h; k++) {
        ocplx t[12], a[12];
        ob_block_hop_site(o, B, blk, tmp_o, se[k], t);
        ob_mat12_vec(o->A + 144 * se[k], rho + 12 * k, a);
        for (int i = 0; i < 12; i++) out[12 * k + i] = a[i] - t[i];
    }
}

/* Approximate solve of D_blk chi = r|_blk by even-odd reduction and nmr MinRes
 * steps on Dhat_blk from zero; chi (a full field) receives the block's values. */
static void block_solve(const oracle *o, const blocking *B, long blk, int nmr, const ocplx *r,
                        ocplx *chi)
{
    long h = B->vol / 2, n = 12 * h;
    const long *se = B->se + blk * h, *so = B->so + blk * h;
    ocplx *ro = malloc(sizeof(ocplx) * n), *to = malloc(sizeof(ocplx) * n);
    ocplx *rho = malloc(sizeof(ocplx) * n), *ce = malloc(sizeof(ocplx) * n);
    ocplx *p = malloc(sizeof(ocplx) * n), *co = malloc(sizeof(ocplx) * n);
    /* b_e = r_e - H_eo,blk A_oo^-1 r_o */
    for (long k = 0; k < h; k++) ob_mat12_vec(o->Ainv + 144 * so[k], r + 12 * so[k], to + 12 * k);
    for (long k = 0; k < h; k++) {
        ocplx t[12];
        ob_block_hop_site(o, B, blk, to, se[k], t);
        for (int i = 0; i < 12; i++) rho[12 * k + i] = r[12 * se[k] + i] - t[i];
    }
    for (long i = 0; i < n; i++) ce[i] = 0;
    /* MinRes: p = Dhat rho, alpha = <p,rho>/<p,p>, chi += alpha rho, rho -= alpha p */
    for (int it = 0; it < nmr; it++) {
        block_dhat(o, B, blk, rho, p, to);
        double pp = vnorm2(n, p);
        if (pp == 0) break;
        ocplx alpha = vdot(n, p, rho) / pp;
        vaxpy(n, alpha, rho, ce);
        vaxpy(n, -alpha, p, rho);
    }
    /* chi_o = A_oo^-1 (r_o - H_oe,blk chi_e) */
    for (long k = 0; k < h; k++) {
        ocplx t[12];
        ob_block_hop_site(o, B, blk, ce, so[k], t);
        for (int i = 0; i < 12; i++) ro[12 * k + i] = r[12 * so[k] + i] - t[i];
        ob_mat12_vec(o->Ainv + 144 * so[k], ro + 12 * k, co + 12 * k);
    }
    for (long k = 0; k < h; k++)
        for (int i = 0; i < 12; i++) {
            chi[12 * se[k] + i] = ce[12 * k + i];
            chi[12 * so[k] + i] = co[12 * k + i];
        }
    free(ro);
    free(to);
    free(rho);
    free(ce);
    free(p);
    free(co);
}

void or_sap_block_solve(const oracle *o, const int bs[4], long blk, int nmr, const double *r,
                        double *chi)
{
    blocking B;
    ob_load_gammas();
    if (ob_make_blocking(o, bs, &B) != OR_OK) return;
    block_solve(o, &B, blk, nmr, (const ocplx *)r, (ocplx *)chi);
    ob_free_blocking(&B);
}

/* M_sap eta: psi = 0, r = eta; ncy cycles over the two block colours; after
 * each colour sweep the residual is recomputed from its definition. */
void or_sap(const oracle *o, const int bs[4], int ncy, int nmr, const double *eta_, double *psi_)
{
    blocking B;
    ob_load_gammas();
    if (ob_make_blocking(o, bs, &B) != OR_OK) return;
    long n = 12 * o->V;
    const ocplx *eta = (const ocplx *)eta_;
    ocplx *psi = (ocplx *)psi_;
    ocplx *r = malloc(sizeof(ocplx) * n), *chi = malloc(sizeof(ocplx) * n);
    for (long i = 0; i < n; i++) {
        psi[i] = 0;
        r[i] = eta[i];
    }
    int first = 1;
    for (int cyc = 0; cyc < ncy; cyc++)
        for (int col = 0; col < 2; col++) {
            if (!first) {
                or_apply_D(o, (double *)psi, (double *)r);
                for (long i = 0; i < n; i++) r[i] = eta[i] - r[i];
            }
            first = 0;
#pragma omp parallel for schedule(dynamic)
            for (long b = 0; b < B.nblk; b++)
                if (B.colour[b] == col) block_solve(o, &B, b, nmr, r, chi);
            for (long b = 0; b < B.nblk; b++) {
                if (B.colour[b] != col) continue;
                long h = B.vol / 2;
                for (long k = 0; k < h; k++)
                    for (int i = 0; i < 12; i++) {
                        long xe = B.se[b * h + k], xo = B.so[b * h + k];
                        psi[12 * xe + i] += chi[12 * xe + i];
                        psi[12 * xo + i] += chi[12 * xo + i];
                    }
            }
        }
    free(r);
    free(chi);
    ob_free_blocking(&B);
}

/* ------------------------------------------------------------------------ */
/* DD-HMC block solves (Sec. 3: the inversions on the blocks needed for the   */
/* block force F_1 use BiCGstab).  Every block's Dirichlet operator Dhat_blk  */
/* is an independent system; BiCGstab (van der Vorst 1992) runs on each from */
/* psi = 0 with rhat = r_0 = eta|_blk.                                        */

/* out_e = Dhat_blk in_e on every block (even half fields, canonical rank order) */
void or_block_dhat(const oracle *o, const int bs[4], const double *in_, double *out_)
{
    blocking B;
    ob_load_gammas();
    if (ob_make_blocking(o, bs, &B) != OR_OK) return;
    const ocplx *in = (const ocplx *)in_;
    ocplx *out = (ocplx *)out_;
    long h = B.vol / 2, n = 12 * h;
#pragma omp parallel for schedule(dynamic)
    for (long b = 0; b < B.nblk; b++) {
        ocplx *x = malloc(sizeof(ocplx) * n), *y = malloc(sizeof(ocplx) * n), *t = malloc(sizeof(ocplx) * n);
        for (long k = 0; k < h; k++)
            for (int i = 0; i < 12; i++) x[12 * k + i] = in[12 * o->rank[B.se[b * h + k]] + i];
        block_dhat(o, &B, b, x, y, t);
        for (long k = 0; k < h; k++)
            for (int i = 0; i < 12; i++) out[12 * o->rank[B.se[b * h + k]] + i] = y[12 * k + i];
        free(x);
        free(y);
        free(t);
    }
    ob_free_blocking(&B);
}

/* One block: BiCGstab steps in the order of the method,
 *   rho = <rhat, r>, beta = (rho / rho_prev)(alpha / omega),
 *   p = r + beta (p - omega v), v = A p, alpha = rho / <rhat, v>, s = r - alpha v,
 *   (|s| <= tol |eta|: x += alpha p, done), t = A s, omega = <t, s> / <t, t>,
 *   x += alpha p + omega s, r = s - omega t, converged when |r| <= tol |eta|.
 * Returns the status; *iters the steps taken, *relres the recomputed residual. */
static int block_bicgstab(const oracle *o, const blocking *B, long blk, const ocplx *eta, ocplx *x, double tol,
                          int maxit, int *iters, double *relres)
{
    long h = B->vol / 2, n = 12 * h;
    ocplx *r = malloc(sizeof(ocplx) * n), *rh = malloc(sizeof(ocplx) * n), *p = malloc(sizeof(ocplx) * n);
    ocplx *v = malloc(sizeof(ocplx) * n), *sv = malloc(sizeof(ocplx) * n), *t = malloc(sizeof(ocplx) * n);
    ocplx *tmp = malloc(sizeof(ocplx) * n);
    double e2 = vnorm2(n, eta);
    for (long i = 0; i < n; i++) {
        x[i] = 0;
        r[i] = eta[i];
        rh[i] = eta[i];
        p[i] = 0;
        v[i] = 0;
    }
    ocplx rho_prev = 1, alpha = 1, omega = 1;
    int it = 0, status = OR_ERR_NOT_CONVERGED;
    if (e2 == 0) status = OR_OK;
    while (status == OR_ERR_NOT_CONVERGED && it < maxit) {
        ocplx rho = vdot(n, rh, r);
        if (rho == 0) {
            status = OR_ERR_BREAKDOWN;
            break;
        }
        ocplx beta = (rho / rho_prev) * (alpha / omega);
        for (long i = 0; i < n; i++) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        block_dhat(o, B, blk, p, v, tmp);
        ocplx rv = vdot(n, rh, v);
        if (rv == 0) {
            status = OR_ERR_BREAKDOWN;
            break;
        }
        alpha = rho / rv;
        for (long i = 0; i < n; i++) sv[i] = r[i] - alpha * v[i];
        it++;
        if (vnorm2(n, sv) <= tol * tol * e2) {
            vaxpy(n, alpha, p, x);
            status = OR_OK;
            break;
        }
        block_dhat(o, B, blk, sv, t, tmp);
        double tt = vnorm2(n, t);
        if (tt == 0) {
            status = OR_ERR_BREAKDOWN;
            break;
        }
        omega = vdot(n, t, sv) / tt;
        for (long i = 0; i < n; i++) {
            x[i] += alpha * p[i] + omega * sv[i];
            r[i] = sv[i] - omega * t[i];
        }
        rho_prev = rho;
        if (vnorm2(n, r) <= tol * tol * e2) status = OR_OK;
    }
    /* recomputed residual */
    block_dhat(o, B, blk, x, t, tmp);
    double r2 = 0;
    for (long i = 0; i < n; i++) r2 += creal((eta[i] - t[i]) * conj(eta[i] - t[i]));
    *iters = it;
    *relres = e2 > 0 ? sqrt(r2 / e2) : 0;
    free(r);
    free(rh);
    free(p);
    free(v);
    free(sv);
    free(t);
    free(tmp);
    return status;
}

/* Dhat_blk psi_e = eta_e on every block; iters / relres per block (may be NULL).
 * Returns the worst block status. */
int or_block_bicgstab(const oracle *o, const int bs[4], const double *eta_, double *psi_, double tol, int maxit,
                      int *iters, double *relres)
{
    blocking B;
    ob_load_gammas();
    if (ob_make_blocking(o, bs, &B) != OR_OK) return OR_ERR_ARG;
    const ocplx *eta = (const ocplx *)eta_;
    ocplx *psi = (ocplx *)psi_;
    long h = B.vol / 2, n = 12 * h;
    int *st = malloc(sizeof(int) * B.nblk);
#pragma omp parallel for schedule(dynamic)
    for (long b = 0; b < B.nblk; b++) {
        ocplx *e = malloc(sizeof(ocplx) * n), *x = malloc(sizeof(ocplx) * n);
        for (long k = 0; k < h; k++)
            for (int i = 0; i < 12; i++) e[12 * k + i] = eta[12 * o->rank[B.se[b * h + k]] + i];
        int it;
        double rr;
        st[b] = block_bicgstab(o, &B, b, e, x, tol, maxit, &it, &rr);
        if (iters) iters[b] = it;
        if (relres) relres[b] = rr;
        for (long k = 0; k < h; k++)
            for (int i = 0; i < 12; i++) psi[12 * o->rank[B.se[b * h + k]] + i] = x[12 * k + i];
        free(e);
        free(x);
    }
    int worst = OR_OK;
    for (long b = 0; b < B.nblk; b++)
        if (st[b] != OR_OK && worst == OR_OK) worst = st[b];
    free(st);
    ob_free_blocking(&B);
    return worst;
}

/* ------------------------------------------------------------------------ */
/* flexible GCR on the full lattice                                         */

/* precond: 0 identity, 1 SAP, 2 deflated SAP (subspace built beforehand) */
static void precond_apply(const oracle *o, int precond, const int bs[4], int ncy, int nmr,
                          const ocplx *rho, ocplx *phi)
{
    long n = 12 * o->V;
    if (precond == 0)
        memcpy(phi, rho, sizeof(ocplx) * n);
    else if (precond == 1)
        or_sap(o, bs, ncy, nmr, (const double *)rho, (double *)phi);
    else
        or_dfl_precond(o, bs, ncy, nmr, 1e-8, (const double *)rho, (double *)phi);
}

int or_gcr(const oracle *o, int precond, const int bs[4], int ncy, int nmr, int nkv, int nmx,
           double tol, const double *eta_, double *psi_, int *iters, double *relres)
{
    long n = 12 * o->V;
    const ocplx *eta = (const ocplx *)eta_;
    ocplx *psi = (ocplx *)psi_;
    ocplx *rho = malloc(sizeof(ocplx) * n);
    ocplx *phi = malloc(sizeof(ocplx) * n * nkv), *chi = malloc(sizeof(ocplx) * n * nkv);
    ocplx *a = calloc((size_t)nkv * nkv, sizeof(ocplx)), *c = malloc(sizeof(ocplx) * nkv);
    ocplx *alpha = malloc(sizeof(ocplx) * nkv);
    double *b = malloc(sizeof(double) * nkv);
    double eta_norm = sqrt(vnorm2(n, eta));
    int status = OR_ERR_NOT_CONVERGED, it = 0;
    for (long i = 0; i < n; i++) {
        psi[i] = 0;
        rho[i] = eta[i];
    }
    double res = eta_norm;
    if (eta_norm == 0) {
        status = OR_OK;
        goto done;
    }
    while (it < nmx) {
        int k, nk = 0;
        for (k = 0; k < nkv && it < nmx; k++) {
            ocplx *ph = phi + n * k, *ch = chi + n * k;
            precond_apply(o, precond, bs, ncy, nmr, rho, ph);
            or_apply_D(o, (double *)ph, (double *)ch);
            for (int i = 0; i < k; i++) a[nkv * i + k] = 0;
            for (int pass = 0; pass < 2; pass++) { /* classical GS + one re-orthogonalisation */
                ocplx proj[64];
                for (int i = 0; i < k; i++) proj[i] = vdot(n, chi + n * i, ch);
                for (int i = 0; i < k; i++) {
                    vaxpy(n, -proj[i], chi + n * i, ch);
                    a[nkv * i + k] += proj[i];
                }
            }
            b[k] = sqrt(vnorm2(n, ch));
            if (b[k] == 0) {
                status = OR_ERR_BREAKDOWN;
                goto done;
            }
            for (long i = 0; i < n; i++) ch[i] /= b[k];
            c[k] = vdot(n, ch, rho);
            vaxpy(n, -c[k], ch, rho);
            it++;
            nk = k + 1;
            if (sqrt(vnorm2(n, rho)) <= tol * eta_norm) break;
        }
        /* back substitution: alpha_k = (c_k - sum_{i>k} a_ki alpha_i) / b_k */
        for (int j = nk - 1; j >= 0; j--) {
            ocplx s = c[j];
            for (int i = j + 1; i < nk; i++) s -= a[nkv * j + i] * alpha[i];
            alpha[j] = s / b[j];
        }
        for (int j = 0; j < nk; j++) vaxpy(n, alpha[j], phi + n * j, psi);
        /* restart from the true residual */
        or_apply_D(o, (double *)psi, (double *)rho);
        for (long i = 0; i < n; i++) rho[i] = eta[i] - rho[i];
        res = sqrt(vnorm2(n, rho));
        if (res <= tol * eta_norm) {
            status = OR_OK;
            break;
        }
    }
done:
    if (iters) *iters = it;
    if (relres) *relres = eta_norm > 0 ? res / eta_norm : 0;
    free(rho);
    free(phi);
    free(chi);
    free(a);
    free(c);
    free(alpha);
    free(b);
    return status;
}
