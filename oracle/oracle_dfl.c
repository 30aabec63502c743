/*
 * Oracle, part 3: local deflation ("locally deflated" Schwarz-preconditioned
 * GCR, Sec. 3 and Sec. 4, Table 1).  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper names the method but does not print it; the steps here are the
 * reading recorded in the design notes:
 *   1. start from Ns caller-supplied fields v_l (the random numbers are inputs);
 *   2. ninv times: v_l <- M_sap v_l, then v_l <- v_l / |v_l|;
 *   3. on every block Lambda, Gram-Schmidt of {v_l restricted to Lambda} gives
 *      the block-orthonormal fields phi^Lambda_l;
 *   4. the little Dirac operator A_{(L k),(L' l)} = <phi^L_k, D phi^L'_l>;
 *   5. M_dfl rho = M_sap(rho - D Pi A^-1 Pi^dag rho) + Pi A^-1 Pi^dag rho, with
 *      A^-1 applied by plain GCR to a relative residual ctol.
 * Pinned by (tests/test_oracle_solvers.py): block orthonormality; the subspace
 * equal to numpy's per-block QR factor of v0, M_sap v0 and M_sap^2 v0 (ninv = 0,
 * 1, 2); A equal to the dense Pi^dag D Pi; Pi^dag P_L = 0 and P_L^2 = P_L for
 * P_L = 1 - D Pi A^-1 Pi^dag; M_dfl equal to the composition assembled from the
 * dense Pi, an LU solve of A and the (separately pinned) SAP, and
 * M_dfl (D Pi c) = Pi c; the deflated GCR reaching the SAP-GCR solution.
 */
#include "oracle_internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct or_dfl {
    int Ns;
    blocking B;
    ocplx *phi;   /* [Ns][V][12]: phi^Lambda_l is field l restricted to block Lambda */
    long *nbr;    /* [nblk][9]: distinct neighbour blocks (self first), -1 if unused */
    ocplx *A;     /* [nblk][9][Ns][Ns] couplings A[L][j][k][l] = <phi^L_k, D phi^{nbr_j}_l> */
};

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

void or_dfl_free(oracle *o)
{
    if (!o->dfl) return;
    ob_free_blocking(&o->dfl->B);
    free(o->dfl->phi);
    free(o->dfl->nbr);
    free(o->dfl->A);
    free(o->dfl);
    o->dfl = NULL;
}

/* (D P_blk v)(x): D applied to the field v masked to block blk, at site x */
static void d_site_masked(const oracle *o, const blocking *B, long blk, const ocplx *v, long x,
                          ocplx *res)
{
    for (int i = 0; i < 12; i++) res[i] = 0;
    if (B->blk_of[x] == blk) ob_mat12_vec(o->A + 144 * x, v + 12 * x, res);
    int x0 = o->coord[4 * x];
    for (int mu = 0; mu < 4; mu++) {
        ocplx t[12];
        long y = o->fw[4 * x + mu];
        if (B->blk_of[y] == blk) {
            double sf = (mu == 0 && x0 == o->L[0] - 1) ? o->bc_t : 1.0;
            ob_colour_mul(o->U + 9 * (4 * x + mu), 0, v + 12 * y, t);
            ob_add_proj(res, t, mu, -1.0, -0.5 * sf);
        }
        long z = o->bw[4 * x + mu];
        if (B->blk_of[z] == blk) {
            double sb = (mu == 0 && x0 == 0) ? o->bc_t : 1.0;
            ob_colour_mul(o->U + 9 * (4 * z + mu), 1, v + 12 * z, t);
            ob_add_proj(res, t, mu, +1.0, -0.5 * sb);
        }
    }
}

/* the block containing the site reached from block b's origin by one block step */
static long block_step(const blocking *B, long b, int mu, int dir)
{
    int c[4];
    long r = b;
    c[3] = r % B->nb[3];
    r /= B->nb[3];
    c[2] = r % B->nb[2];
    r /= B->nb[2];
    c[1] = r % B->nb[1];
    c[0] = r / B->nb[1];
    c[mu] = (c[mu] + dir + B->nb[mu]) % B->nb[mu];
    return c[3] + B->nb[3] * (c[2] + (long)B->nb[2] * (c[1] + (long)B->nb[1] * c[0]));
}

int or_dfl_build(oracle *o, const int bs[4], int Ns, int ninv, int ncy, int nmr, const double *v0)
{
    or_dfl_free(o);
    ob_load_gammas();
    struct or_dfl *d = calloc(1, sizeof(struct or_dfl));
    if (ob_make_blocking(o, bs, &d->B) != OR_OK) {
        free(d);
        return OR_ERR_ARG;
    }
    d->Ns = Ns;
    long n = 12 * o->V, h = d->B.vol / 2, nblk = d->B.nblk;
    /* steps 1-2: inverse iteration with SAP */
    ocplx *v = malloc(sizeof(ocplx) * n * Ns);
    memcpy(v, v0, sizeof(ocplx) * n * Ns);
    ocplx *t = malloc(sizeof(ocplx) * n);
    for (int pass = 0; pass < ninv; pass++)
        for (int l = 0; l < Ns; l++) {
            or_sap(o, bs, ncy, nmr, (double *)(v + n * l), (double *)t);
            double nrm = sqrt(vnorm2(n, t));
            for (long i = 0; i < n; i++) v[n * l + i] = t[i] / nrm;
        }
    free(t);
    /* step 3: Gram-Schmidt on each block (modified GS, applied twice) */
    d->phi = v;
    int status = OR_OK;
    for (long b = 0; b < nblk; b++) {
        long vol = d->B.vol;
        long *sites = malloc(sizeof(long) * vol);
        for (long k = 0; k < h; k++) {
            sites[k] = d->B.se[b * h + k];
            sites[h + k] = d->B.so[b * h + k];
        }
        for (int l = 0; l < Ns; l++) {
            ocplx *vl = v + n * l;
            for (int pass = 0; pass < 2; pass++)
                for (int k = 0; k < l; k++) {
                    ocplx *vk = v + n * k;
                    ocplx s = 0;
                    for (long j = 0; j < vol; j++)
                        for (int i = 0; i < 12; i++)
                            s += conj(vk[12 * sites[j] + i]) * vl[12 * sites[j] + i];
                    for (long j = 0; j < vol; j++)
                        for (int i = 0; i < 12; i++) vl[12 * sites[j] + i] -= s * vk[12 * sites[j] + i];
                }
            double nn = 0;
            for (long j = 0; j < vol; j++)
                for (int i = 0; i < 12; i++) {
                    ocplx z = vl[12 * sites[j] + i];
                    nn += creal(z) * creal(z) + cimag(z) * cimag(z);
                }
            if (nn == 0) status = OR_ERR_BREAKDOWN;
            double inv = nn > 0 ? 1.0 / sqrt(nn) : 0.0;
            for (long j = 0; j < vol; j++)
                for (int i = 0; i < 12; i++) vl[12 * sites[j] + i] *= inv;
        }
        free(sites);
    }
    /* step 4: little Dirac operator, by its definition, block row by block row */
    d->nbr = malloc(sizeof(long) * nblk * 9);
    d->A = calloc((size_t)nblk * 9 * Ns * Ns, sizeof(ocplx));
    for (long b = 0; b < nblk; b++) {
        int m = 0;
        d->nbr[9 * b + m++] = b;
        for (int mu = 0; mu < 4; mu++)
            for (int dir = 1; dir >= -1; dir -= 2) {
                long c = block_step(&d->B, b, mu, dir);
                int seen = 0;
                for (int j = 0; j < m; j++)
                    if (d->nbr[9 * b + j] == c) seen = 1;
                if (!seen) d->nbr[9 * b + m++] = c;
            }
        for (; m < 9; m++) d->nbr[9 * b + m] = -1;
    }
#pragma omp parallel for schedule(dynamic)
    for (long b = 0; b < nblk; b++) {
        long vol = d->B.vol;
        for (int j = 0; j < 9; j++) {
            long c = d->nbr[9 * b + j];
            if (c < 0) continue;
            for (int l = 0; l < Ns; l++)
                for (long s = 0; s < vol; s++) {
                    long x = s < h ? d->B.se[b * h + s] : d->B.so[b * h + s - h];
                    ocplx w[12];
                    d_site_masked(o, &d->B, c, v + n * l, x, w);
                    for (int k = 0; k < Ns; k++) {
                        ocplx acc = 0;
                        for (int i = 0; i < 12; i++) acc += conj(v[n * k + 12 * x + i]) * w[i];
                        d->A[(((size_t)b * 9 + j) * Ns + k) * Ns + l] += acc;
                    }
                }
        }
    }
    o->dfl = d;
    return status;
}

void or_dfl_subspace(const oracle *o, double *phi)
{
    memcpy(phi, o->dfl->phi, sizeof(ocplx) * 12 * o->V * o->dfl->Ns);
}

/* Pi^dag: c[L*Ns + k] = <phi^L_k, in> */
void or_dfl_project(const oracle *o, const double *in_, double *c_)
{
    const struct or_dfl *d = o->dfl;
    const ocplx *in = (const ocplx *)in_;
    ocplx *c = (ocplx *)c_;
    long n = 12 * o->V, h = d->B.vol / 2;
    for (long b = 0; b < d->B.nblk; b++)
        for (int k = 0; k < d->Ns; k++) {
            ocplx acc = 0;
            for (long s = 0; s < d->B.vol; s++) {
                long x = s < h ? d->B.se[b * h + s] : d->B.so[b * h + s - h];
                for (int i = 0; i < 12; i++) acc += conj(d->phi[n * k + 12 * x + i]) * in[12 * x + i];
            }
            c[b * d->Ns + k] = acc;
        }
}

/* Pi: out(x) = sum_k c[blk(x)*Ns + k] phi_k(x) */
void or_dfl_expand(const oracle *o, const double *c_, double *out_)
{
    const struct or_dfl *d = o->dfl;
    const ocplx *c = (const ocplx *)c_;
    ocplx *out = (ocplx *)out_;
    long n = 12 * o->V;
    for (long x = 0; x < o->V; x++) {
        long b = d->B.blk_of[x];
        for (int i = 0; i < 12; i++) {
            ocplx acc = 0;
            for (int k = 0; k < d->Ns; k++) acc += c[b * d->Ns + k] * d->phi[n * k + 12 * x + i];
            out[12 * x + i] = acc;
        }
    }
}

/* dense little operator, (nblk*Ns)^2, row-major */
void or_dfl_little(const oracle *o, double *Amat_)
{
    const struct or_dfl *d = o->dfl;
    ocplx *Amat = (ocplx *)Amat_;
    long N = d->B.nblk * d->Ns;
    for (long i = 0; i < N * N; i++) Amat[i] = 0;
    for (long b = 0; b < d->B.nblk; b++)
        for (int j = 0; j < 9; j++) {
            long c = d->nbr[9 * b + j];
            if (c < 0) continue;
            for (int k = 0; k < d->Ns; k++)
                for (int l = 0; l < d->Ns; l++)
                    Amat[(b * d->Ns + k) * N + c * d->Ns + l] +=
                        d->A[(((size_t)b * 9 + j) * d->Ns + k) * d->Ns + l];
        }
}

void or_dfl_little_apply(const oracle *o, const double *c_, double *out_)
{
    const struct or_dfl *d = o->dfl;
    const ocplx *c = (const ocplx *)c_;
    ocplx *out = (ocplx *)out_;
    int Ns = d->Ns;
    for (long b = 0; b < d->B.nblk; b++)
        for (int k = 0; k < Ns; k++) {
            ocplx acc = 0;
            for (int j = 0; j < 9; j++) {
                long nb = d->nbr[9 * b + j];
                if (nb < 0) continue;
                for (int l = 0; l < Ns; l++)
                    acc += d->A[(((size_t)b * 9 + j) * Ns + k) * Ns + l] * c[nb * Ns + l];
            }
            out[b * Ns + k] = acc;
        }
}

/* plain (unpreconditioned) GCR on the little operator */
int or_dfl_coarse_solve(const oracle *o, const double *b_, double *c_, double tol, int nkv, int nmx,
                        int *iters)
{
    const struct or_dfl *d = o->dfl;
    long N = d->B.nblk * d->Ns;
    const ocplx *b = (const ocplx *)b_;
    ocplx *x = (ocplx *)c_;
    ocplx *rho = malloc(sizeof(ocplx) * N), *p = malloc(sizeof(ocplx) * N * nkv);
    ocplx *q = malloc(sizeof(ocplx) * N * nkv), *a = calloc((size_t)nkv * nkv, sizeof(ocplx));
    ocplx *cc = malloc(sizeof(ocplx) * nkv), *al = malloc(sizeof(ocplx) * nkv);
    double *bb = malloc(sizeof(double) * nkv);
    double bn = sqrt(vnorm2(N, b));
    for (long i = 0; i < N; i++) {
        x[i] = 0;
        rho[i] = b[i];
    }
    int it = 0, status = OR_ERR_NOT_CONVERGED;
    if (bn == 0) {
        status = OR_OK;
        goto done;
    }
    while (it < nmx) {
        int nk = 0;
        for (int k = 0; k < nkv && it < nmx; k++) {
            ocplx *pk = p + N * k, *qk = q + N * k;
            memcpy(pk, rho, sizeof(ocplx) * N);
            or_dfl_little_apply(o, (double *)pk, (double *)qk);
            for (int i = 0; i < k; i++) a[nkv * i + k] = 0;
            for (int pass = 0; pass < 2; pass++)
                for (int i = 0; i < k; i++) {
                    ocplx s = vdot(N, q + N * i, qk);
                    for (long j = 0; j < N; j++) qk[j] -= s * q[N * i + j];
                    a[nkv * i + k] += s;
                }
            bb[k] = sqrt(vnorm2(N, qk));
            if (bb[k] == 0) {
                status = OR_ERR_BREAKDOWN;
                goto done;
            }
            for (long j = 0; j < N; j++) qk[j] /= bb[k];
            cc[k] = vdot(N, qk, rho);
            for (long j = 0; j < N; j++) rho[j] -= cc[k] * qk[j];
            it++;
            nk = k + 1;
            if (sqrt(vnorm2(N, rho)) <= tol * bn) break;
        }
        for (int j = nk - 1; j >= 0; j--) {
            ocplx s = cc[j];
            for (int i = j + 1; i < nk; i++) s -= a[nkv * j + i] * al[i];
            al[j] = s / bb[j];
        }
        for (int j = 0; j < nk; j++)
            for (long i = 0; i < N; i++) x[i] += al[j] * p[N * j + i];
        or_dfl_little_apply(o, (double *)x, (double *)rho);
        for (long i = 0; i < N; i++) rho[i] = b[i] - rho[i];
        if (sqrt(vnorm2(N, rho)) <= tol * bn) {
            status = OR_OK;
            break;
        }
    }
done:
    if (iters) *iters = it;
    free(rho);
    free(p);
    free(q);
    free(a);
    free(cc);
    free(al);
    free(bb);
    return status;
}

/* M_dfl rho = M_sap(rho - D Pi A^-1 Pi^dag rho) + Pi A^-1 Pi^dag rho */
void or_dfl_precond(const oracle *o, const int bs[4], int ncy, int nmr, double ctol,
                    const double *rho_, double *phi_)
{
    const struct or_dfl *d = o->dfl;
    long n = 12 * o->V, N = d->B.nblk * d->Ns;
    const ocplx *rho = (const ocplx *)rho_;
    ocplx *phi = (ocplx *)phi_;
    ocplx *c = malloc(sizeof(ocplx) * N), *e = malloc(sizeof(ocplx) * N);
    ocplx *u = malloc(sizeof(ocplx) * n), *w = malloc(sizeof(ocplx) * n);
    or_dfl_project(o, rho_, (double *)c);
    or_dfl_coarse_solve(o, (double *)c, (double *)e, ctol, 16, 4096, NULL);
    or_dfl_expand(o, (double *)e, (double *)u);
    or_apply_D(o, (double *)u, (double *)w);
    for (long i = 0; i < n; i++) w[i] = rho[i] - w[i];
    or_sap(o, bs, ncy, nmr, (double *)w, (double *)phi);
    for (long i = 0; i < n; i++) phi[i] += u[i];
    free(c);
    free(e);
    free(u);
    free(w);
}
