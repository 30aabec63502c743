/*
 * Oracle, part 1: lattice geometry, gamma matrices, the clover term and the
 * Wilson-clover operator D of Eq. 1, and the even-odd Schur complement of
 * Eq. 2.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Pinned by (tests/test_oracle_dirac.py): Clifford algebra of the gamma table;
 * the free-field plane-wave closed form of D; gamma5-hermiticity; gauge
 * covariance of D and of Fhat; Fhat = 0 on unit links; the single-plaquette
 * and constant-abelian-flux closed forms of the clover term; independence of
 * the clover term from the fermion boundary sign; A*A^-1 = 1 and log det
 * against a library determinant; the Schur identities of Eq. 2 and Eq. 5 on a
 * dense 4^4 operator.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* gamma[mu] for mu = 0..3, gamma[4] = gamma5 = g0 g1 g2 g3 */
static ocplx G[5][4][4];
static int G_ready = 0;

static void build_gammas(void)
{
    if (G_ready) return;
    memset(G, 0, sizeof(G));
    /* Pauli matrices */
    ocplx s[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    /* gamma_0 = [[0,-1],[-1,0]] in 2x2 blocks */
    for (int a = 0; a < 2; a++) {
        G[0][a][2 + a] = -1;
        G[0][2 + a][a] = -1;
    }
    /* gamma_k = [[0,-i sigma_k],[i sigma_k,0]] */
    for (int k = 1; k <= 3; k++)
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                G[k][a][2 + b] = -I * s[k - 1][a][b];
                G[k][2 + a][b] = I * s[k - 1][a][b];
            }
    /* gamma_5 = g0 g1 g2 g3 (computed, not typed in) */
    ocplx t1[4][4], t2[4][4];
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            ocplx acc = 0;
            for (int k = 0; k < 4; k++) acc += G[0][i][k] * G[1][k][j];
            t1[i][j] = acc;
        }
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            ocplx acc = 0;
            for (int k = 0; k < 4; k++) acc += t1[i][k] * G[2][k][j];
            t2[i][j] = acc;
        }
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            ocplx acc = 0;
            for (int k = 0; k < 4; k++) acc += t2[i][k] * G[3][k][j];
            G[4][i][j] = acc;
        }
    G_ready = 1;
}

void or_gamma(int mu, double *g)
{
    build_gammas();
    ocplx *out = (ocplx *)g;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) out[4 * i + j] = G[mu][i][j];
}

/* ------------------------------------------------------------------------ */
/* geometry                                                                 */

oracle *or_create(int T, int L1, int L2, int L3, int antiperiodic_t)
{
    if (T <= 0 || L1 <= 0 || L2 <= 0 || L3 <= 0) return NULL;
    if (T % 2 || L1 % 2 || L2 % 2 || L3 % 2) return NULL;
    build_gammas();
    oracle *o = calloc(1, sizeof(oracle));
    o->L[0] = T;
    o->L[1] = L1;
    o->L[2] = L2;
    o->L[3] = L3;
    o->V = (long)T * L1 * L2 * L3;
    o->Vh = o->V / 2;
    o->bc_t = antiperiodic_t ? -1.0 : 1.0;
    o->U = calloc((size_t)o->V * 36, sizeof(ocplx));
    o->par = malloc(sizeof(int) * o->V);
    o->rank = malloc(sizeof(long) * o->V);
    o->site_of[0] = malloc(sizeof(long) * o->Vh);
    o->site_of[1] = malloc(sizeof(long) * o->Vh);
    o->fw = malloc(sizeof(long) * 4 * o->V);
    o->bw = malloc(sizeof(long) * 4 * o->V);
    o->coord = malloc(sizeof(int) * 4 * o->V);
    long count[2] = {0, 0};
    for (long x = 0; x < o->V; x++) {
        /* decode the lexicographic index, x3 fastest */
        long r = x;
        int c[4];
        c[3] = (int)(r % L3);
        r /= L3;
        c[2] = (int)(r % L2);
        r /= L2;
        c[1] = (int)(r % L1);
        c[0] = (int)(r / L1);
        for (int mu = 0; mu < 4; mu++) o->coord[4 * x + mu] = c[mu];
        int p = (c[0] + c[1] + c[2] + c[3]) % 2;
        o->par[x] = p;
        o->rank[x] = count[p];
        o->site_of[p][count[p]] = x;
        count[p]++;
    }
    for (long x = 0; x < o->V; x++) {
        for (int mu = 0; mu < 4; mu++) {
            int c[4], d[4];
            for (int nu = 0; nu < 4; nu++) c[nu] = d[nu] = o->coord[4 * x + nu];
            c[mu] = (c[mu] + 1) % o->L[mu];
            d[mu] = (d[mu] - 1 + o->L[mu]) % o->L[mu];
            o->fw[4 * x + mu] = c[3] + (long)L3 * (c[2] + (long)L2 * (c[1] + (long)L1 * c[0]));
            o->bw[4 * x + mu] = d[3] + (long)L3 * (d[2] + (long)L2 * (d[1] + (long)L1 * d[0]));
        }
    }
    return o;
}

void or_destroy(oracle *o)
{
    if (!o) return;
    or_dfl_free(o);
    free(o->U);
    free(o->A);
    free(o->Ainv);
    free(o->par);
    free(o->rank);
    free(o->site_of[0]);
    free(o->site_of[1]);
    free(o->fw);
    free(o->bw);
    free(o->coord);
    free(o);
}

long or_even_rank_to_site(const oracle *o, int parity, long r) { return o->site_of[parity][r]; }

void or_set_gauge(oracle *o, const double *U)
{
    memcpy(o->U, U, sizeof(ocplx) * 36 * (size_t)o->V);
    o->have_clover = 0;
}

/* ------------------------------------------------------------------------ */
/* 3x3 colour algebra                                                       */

static const ocplx *link(const oracle *o, long x, int mu) { return o->U + 9 * (4 * x + mu); }

static void mm(const ocplx *a, const ocplx *b, ocplx *c) /* c = a b */
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            ocplx acc = 0;
            for (int k = 0; k < 3; k++) acc += a[3 * i + k] * b[3 * k + j];
            c[3 * i + j] = acc;
        }
}

static void dag(const ocplx *a, ocplx *b) /* b = a^dag */
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) b[3 * i + j] = conj(a[3 * j + i]);
}

/* product of four 3x3 matrices */
static void mm4(const ocplx *a, const ocplx *b, const ocplx *c, const ocplx *d, ocplx *out)
{
    ocplx t1[9], t2[9];
    mm(a, b, t1);
    mm(t1, c, t2);
    mm(t2, d, out);
}

/* ------------------------------------------------------------------------ */
/* clover field strength Fhat_{mu nu}(x), Eq. 1                             */

void or_fhat_site(const oracle *o, long x, int mu, int nu, double *Fout)
{
    ocplx *F = (ocplx *)Fout;
    if (mu == nu) {
        for (int i = 0; i < 9; i++) F[i] = 0;
        return;
    }
    long xpm = o->fw[4 * x + mu], xpn = o->fw[4 * x + nu];
    long xmm = o->bw[4 * x + mu], xmn = o->bw[4 * x + nu];
    long xmm_pn = o->fw[4 * xmm + nu]; /* x - mu + nu */
    long xmm_mn = o->bw[4 * xmm + nu]; /* x - mu - nu */
    long xmn_pm = o->fw[4 * xmn + mu]; /* x - nu + mu */
    ocplx d1[9], d2[9], d3[9], d4[9];
    ocplx leaf[4][9];
    /* leaf 1: x -> x+mu -> x+mu+nu -> x+nu -> x */
    dag(link(o, xpn, mu), d1);
    dag(link(o, x, nu), d2);
    mm4(link(o, x, mu), link(o, xpm, nu), d1, d2, leaf[0]);
    /* leaf 2: x -> x+nu -> x+nu-mu -> x-mu -> x */
    dag(link(o, xmm_pn, mu), d1);
    dag(link(o, xmm, nu), d2);
    mm4(link(o, x, nu), d1, d2, link(o, xmm, mu), leaf[1]);
    /* leaf 3: x -> x-mu -> x-mu-nu -> x-nu -> x */
    dag(link(o, xmm, mu), d1);
    dag(link(o, xmm_mn, nu), d2);
    mm4(d1, d2, link(o, xmm_mn, mu), link(o, xmn, nu), leaf[2]);
    /* leaf 4: x -> x-nu -> x-nu+mu -> x+mu -> x */
    dag(link(o, xmn, nu), d3);
    dag(link(o, x, mu), d4);
    mm4(d3, link(o, xmn, mu), link(o, xmn_pm, nu), d4, leaf[3]);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            ocplx q = 0, qd = 0;
            for (int l = 0; l < 4; l++) {
                q += leaf[l][3 * a + b];
                qd += conj(leaf[l][3 * b + a]);
            }
            F[3 * a + b] = (q - qd) / 8.0;
        }
}

/* sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu] */
static void sigma(int mu, int nu, ocplx s[4][4])
{
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            ocplx acc = 0;
            for (int k = 0; k < 4; k++) acc += G[mu][i][k] * G[nu][k][j] - G[nu][i][k] * G[mu][k][j];
            s[i][j] = 0.5 * I * acc;
        }
}

/* A(x) = (4+m0) 1 + c_sw sum_{mu,nu} (i/4) sigma_{mu nu} (x) Fhat_{mu nu}(x), 12x12, index 3*spin+colour */
static void clover_site(const oracle *o, long x, ocplx *A)
{
    for (int i = 0; i < 144; i++) A[i] = 0;
    for (int i = 0; i < 12; i++) A[13 * i] = 4.0 + o->m0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = 0; nu < 4; nu++) {
            if (mu == nu) continue;
            ocplx s[4][4], F[9];
            sigma(mu, nu, s);
            or_fhat_site(o, x, mu, nu, (double *)F);
            for (int si = 0; si < 4; si++)
                for (int sj = 0; sj < 4; sj++)
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++)
                            A[12 * (3 * si + a) + 3 * sj + b] +=
                                o->csw * 0.25 * I * s[si][sj] * F[3 * a + b];
        }
}

/* LU with partial pivoting of an n x n matrix; returns 0 or OR_ERR_SINGULAR.
 * inv receives the inverse, *logabsdet the log of |det|. */
static int lu_invert(int n, const ocplx *Ain, ocplx *inv, double *logabsdet)
{
    ocplx a[144], b[144];
    int piv[12];
    double amax = 0;
    for (int i = 0; i < n * n; i++) {
        a[i] = Ain[i];
        if (cabs(a[i]) > amax) amax = cabs(a[i]);
    }
    double ld = 0;
    for (int k = 0; k < n; k++) {
        int p = k;
        for (int i = k + 1; i < n; i++)
            if (cabs(a[n * i + k]) > cabs(a[n * p + k])) p = i;
        if (!(cabs(a[n * p + k]) >= 1e-12 * amax) || amax == 0) return OR_ERR_SINGULAR;
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < n; j++) {
                ocplx t = a[n * k + j];
                a[n * k + j] = a[n * p + j];
                a[n * p + j] = t;
            }
        ld += log(cabs(a[n * k + k]));
        for (int i = k + 1; i < n; i++) {
            ocplx l = a[n * i + k] / a[n * k + k];
            a[n * i + k] = l;
            for (int j = k + 1; j < n; j++) a[n * i + j] -= l * a[n * k + j];
        }
    }
    /* solve A X = 1 column by column */
    for (int i = 0; i < n * n; i++) b[i] = 0;
    for (int i = 0; i < n; i++) b[n * i + i] = 1;
    for (int k = 0; k < n; k++)
        if (piv[k] != k)
            for (int j = 0; j < n; j++) {
                ocplx t = b[n * k + j];
                b[n * k + j] = b[n * piv[k] + j];
                b[n * piv[k] + j] = t;
            }
    for (int j = 0; j < n; j++) {
        for (int i = 0; i < n; i++) { /* forward, unit lower */
            ocplx acc = b[n * i + j];
            for (int k = 0; k < i; k++) acc -= a[n * i + k] * b[n * k + j];
            b[n * i + j] = acc;
        }
        for (int i = n - 1; i >= 0; i--) { /* backward */
            ocplx acc = b[n * i + j];
            for (int k = i + 1; k < n; k++) acc -= a[n * i + k] * b[n * k + j];
            b[n * i + j] = acc / a[n * i + i];
        }
    }
    for (int i = 0; i < n * n; i++) inv[i] = b[i];
    *logabsdet = ld;
    return OR_OK;
}

int or_set_params(oracle *o, double kappa, double csw)
{
    if (!(kappa > 0)) return OR_ERR_ARG;
    o->kappa = kappa;
    o->csw = csw;
    o->m0 = 1.0 / (2.0 * kappa) - 4.0;
    if (!o->A) o->A = malloc(sizeof(ocplx) * 144 * (size_t)o->V);
    if (!o->Ainv) o->Ainv = malloc(sizeof(ocplx) * 144 * (size_t)o->V);
    double *ld = malloc(sizeof(double) * o->V);
    int *st = malloc(sizeof(int) * o->V);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < o->V; x++) {
        clover_site(o, x, o->A + 144 * x);
        st[x] = lu_invert(12, o->A + 144 * x, o->Ainv + 144 * x, &ld[x]);
    }
    int status = OR_OK;
    o->logdet[0] = o->logdet[1] = 0;
    for (long x = 0; x < o->V; x++) { /* serial sum: deterministic */
        if (st[x] != OR_OK) status = st[x];
        o->logdet[o->par[x]] += ld[x];
    }
    free(ld);
    free(st);
    o->have_clover = (status == OR_OK);
    return status;
}

void or_clover_site(const oracle *o, long x, double *A12)
{
    memcpy(A12, o->A + 144 * x, sizeof(ocplx) * 144);
}

void or_clover_inv_site(const oracle *o, long x, double *A12)
{
    memcpy(A12, o->Ainv + 144 * x, sizeof(ocplx) * 144);
}

double or_logdet(const oracle *o, int parity) { return o->logdet[parity]; }

/* ------------------------------------------------------------------------ */
/* hopping term H, Eq. 1 (D_W without the diagonal 4)                       */

/* res += coef * (1 + sgn*gamma_mu) t, t a 12-component spinor */
static void add_proj(ocplx *res, const ocplx *t, int mu, double sgn, ocplx coef)
{
    for (int s = 0; s < 4; s++)
        for (int c = 0; c < 3; c++) {
            ocplx acc = t[3 * s + c];
            for (int r = 0; r < 4; r++) acc += sgn * G[mu][s][r] * t[3 * r + c];
            res[3 * s + c] += coef * acc;
        }
}

/* t = M psi on colour, for each spin; dagger selects M^dag */
static void colour_mul(const ocplx *M, int dagger, const ocplx *psi, ocplx *t)
{
    for (int s = 0; s < 4; s++)
        for (int a = 0; a < 3; a++) {
            ocplx acc = 0;
            for (int b = 0; b < 3; b++)
                acc += (dagger ? conj(M[3 * b + a]) : M[3 * a + b]) * psi[3 * s + b];
            t[3 * s + a] = acc;
        }
}

static void hop_site(const oracle *o, const ocplx *in, long x, ocplx *res)
{
    for (int i = 0; i < 12; i++) res[i] = 0;
    int x0 = o->coord[4 * x];
    for (int mu = 0; mu < 4; mu++) {
        ocplx t[12];
        long y = o->fw[4 * x + mu];
        double sf = (mu == 0 && x0 == o->L[0] - 1) ? o->bc_t : 1.0;
        colour_mul(link(o, x, mu), 0, in + 12 * y, t);
        add_proj(res, t, mu, -1.0, -0.5 * sf);
        long z = o->bw[4 * x + mu];
        double sb = (mu == 0 && x0 == 0) ? o->bc_t : 1.0;
        colour_mul(link(o, z, mu), 1, in + 12 * z, t);
        add_proj(res, t, mu, +1.0, -0.5 * sb);
    }
}

void or_hop(const oracle *o, const double *in_, double *out_)
{
    const ocplx *in = (const ocplx *)in_;
    ocplx *out = (ocplx *)out_;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < o->V; x++) hop_site(o, in, x, out + 12 * x);
}

static void mat12_vec(const ocplx *M, const ocplx *v, ocplx *r)
{
    for (int i = 0; i < 12; i++) {
        ocplx acc = 0;
        for (int j = 0; j < 12; j++) acc += M[12 * i + j] * v[j];
        r[i] = acc;
    }
}

void or_apply_clover(const oracle *o, int inverse, const double *in_, double *out_)
{
    const ocplx *in = (const ocplx *)in_;
    ocplx *out = (ocplx *)out_;
    const ocplx *M = inverse ? o->Ainv : o->A;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < o->V; x++) mat12_vec(M + 144 * x, in + 12 * x, out + 12 * x);
}

void or_apply_D(const oracle *o, const double *in_, double *out_)
{
    const ocplx *in = (const ocplx *)in_;
    ocplx *out = (ocplx *)out_;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < o->V; x++) {
        ocplx h[12], a[12];
        hop_site(o, in, x, h);
        mat12_vec(o->A + 144 * x, in + 12 * x, a);
        for (int i = 0; i < 12; i++) out[12 * x + i] = a[i] + h[i];
    }
}

/* D applied to a full field, evaluated at one site only */
void or_d_site(const oracle *o, const double *in_, long x, double *out12)
{
    const ocplx *in = (const ocplx *)in_;
    ocplx h[12], a[12];
    hop_site(o, in, x, h);
    mat12_vec(o->A + 144 * x, in + 12 * x, a);
    for (int i = 0; i < 12; i++) ((ocplx *)out12)[i] = a[i] + h[i];
}

void or_apply_gamma5(long n, const double *in_, double *out_)
{
    const ocplx *in = (const ocplx *)in_;
    ocplx *out = (ocplx *)out_;
    build_gammas();
    for (long x = 0; x < n; x++)
        for (int s = 0; s < 4; s++)
            for (int c = 0; c < 3; c++) {
                ocplx acc = 0;
                for (int r = 0; r < 4; r++) acc += G[4][s][r] * in[12 * x + 3 * r + c];
                out[12 * x + 3 * s + c] = acc;
            }
}

/* ------------------------------------------------------------------------ */
/* even-odd Schur complement, Eq. 2: Dhat = A_ee - H_eo A_oo^-1 H_oe        */

void or_apply_Dhat(const oracle *o, const double *in_e_, double *out_e_)
{
    const ocplx *in_e = (const ocplx *)in_e_;
    ocplx *out_e = (ocplx *)out_e_;
    size_t n = 12 * (size_t)o->V;
    ocplx *full = calloc(n, sizeof(ocplx));
    ocplx *tmp = calloc(n, sizeof(ocplx));
    /* full = (psi_e, 0) */
    for (long r = 0; r < o->Vh; r++)
        for (int i = 0; i < 12; i++) full[12 * o->site_of[0][r] + i] = in_e[12 * r + i];
    or_hop(o, (double *)full, (double *)tmp); /* tmp_o = H_oe psi_e */
    /* full = (0, A_oo^-1 tmp_o) */
    for (size_t i = 0; i < n; i++) full[i] = 0;
    for (long r = 0; r < o->Vh; r++) {
        long x = o->site_of[1][r];
        mat12_vec(o->Ainv + 144 * x, tmp + 12 * x, full + 12 * x);
    }
    or_hop(o, (double *)full, (double *)tmp); /* tmp_e = H_eo A_oo^-1 H_oe psi_e */
    for (long r = 0; r < o->Vh; r++) {
        long x = o->site_of[0][r];
        ocplx a[12];
        mat12_vec(o->A + 144 * x, in_e + 12 * r, a);
        for (int i = 0; i < 12; i++) out_e[12 * r + i] = a[i] - tmp[12 * x + i];
    }
    free(full);
    free(tmp);
}

/* Hasenbusch's mass-preconditioned operator (Eq. 3): W(dm) = Q_S + dm with
 * Q_S = 1 - Q_ee^-1 Q_eo Q_oo^-1 Q_oe (Eq. 2), Q = gamma5 D.  gamma5 is diagonal
 * on sites, so the gamma5 factors cancel pairwise and
 * Q_S = 1 - A_ee^-1 H_eo A_oo^-1 H_oe, with H the hopping term of D. */
void or_apply_W(const oracle *o, double dm, const double *in_e_, double *out_e_)
{
    const ocplx *in_e = (const ocplx *)in_e_;
    ocplx *out_e = (ocplx *)out_e_;
    size_t n = 12 * (size_t)o->V;
    ocplx *full = calloc(n, sizeof(ocplx));
    ocplx *tmp = calloc(n, sizeof(ocplx));
    for (long r = 0; r < o->Vh; r++)
        for (int i = 0; i < 12; i++) full[12 * o->site_of[0][r] + i] = in_e[12 * r + i];
    or_hop(o, (double *)full, (double *)tmp); /* H_oe psi_e */
    for (size_t i = 0; i < n; i++) full[i] = 0;
    for (long r = 0; r < o->Vh; r++) {
        long x = o->site_of[1][r];
        mat12_vec(o->Ainv + 144 * x, tmp + 12 * x, full + 12 * x); /* A_oo^-1 H_oe psi_e */
    }
    or_hop(o, (double *)full, (double *)tmp); /* H_eo A_oo^-1 H_oe psi_e */
    for (long r = 0; r < o->Vh; r++) {
        long x = o->site_of[0][r];
        ocplx v[12];
        mat12_vec(o->Ainv + 144 * x, tmp + 12 * x, v); /* A_ee^-1 ... */
        for (int i = 0; i < 12; i++) out_e[12 * r + i] = (1.0 + dm) * in_e[12 * r + i] - v[i];
    }
    free(full);
    free(tmp);
}

/* Dhat^dag = gamma5 Dhat gamma5 (gamma5-hermiticity of D carries over to Dhat) */
void or_apply_Dhat_dag(const oracle *o, const double *in_e, double *out_e)
{
    size_t n = 24 * (size_t)o->Vh;
    double *t1 = malloc(sizeof(double) * n), *t2 = malloc(sizeof(double) * n);
    or_apply_gamma5(o->Vh, in_e, t1);
    or_apply_Dhat(o, t1, t2);
    or_apply_gamma5(o->Vh, t2, out_e);
    free(t1);
    free(t2);
}

/* Dhat psi_e evaluated at the single even site of rank re, from the definition
 * (for sampled parity checks on lattices too large for a full oracle sweep). */
void or_dhat_site(const oracle *o, const double *in_e_, long re, double *out12)
{
    const ocplx *in_e = (const ocplx *)in_e_;
    long x = o->site_of[0][re];
    ocplx acc[12];
    mat12_vec(o->A + 144 * x, in_e + 12 * re, acc);
    int x0 = o->coord[4 * x];
    for (int mu = 0; mu < 4; mu++)
        for (int dir = 0; dir < 2; dir++) {
            /* odd neighbour y of x, and chi_o(y) = A^-1(y) (H psi_e)(y) */
            long y = dir == 0 ? o->fw[4 * x + mu] : o->bw[4 * x + mu];
            int y0 = o->coord[4 * y];
            ocplx h[12], chi[12], t[12];
            for (int i = 0; i < 12; i++) h[i] = 0;
            for (int nu = 0; nu < 4; nu++) {
                long z = o->fw[4 * y + nu];
                double sf = (nu == 0 && y0 == o->L[0] - 1) ? o->bc_t : 1.0;
                colour_mul(link(o, y, nu), 0, in_e + 12 * o->rank[z], t);
                add_proj(h, t, nu, -1.0, -0.5 * sf);
                z = o->bw[4 * y + nu];
                double sb = (nu == 0 && y0 == 0) ? o->bc_t : 1.0;
                colour_mul(link(o, z, nu), 1, in_e + 12 * o->rank[z], t);
                add_proj(h, t, nu, +1.0, -0.5 * sb);
            }
            mat12_vec(o->Ainv + 144 * y, h, chi);
            /* subtract the hop from y to x */
            if (dir == 0) {
                double sf = (mu == 0 && x0 == o->L[0] - 1) ? o->bc_t : 1.0;
                colour_mul(link(o, x, mu), 0, chi, t);
                for (int i = 0; i < 12; i++) h[i] = 0;
                add_proj(h, t, mu, -1.0, -0.5 * sf);
            } else {
                double sb = (mu == 0 && x0 == 0) ? o->bc_t : 1.0;
                colour_mul(link(o, y, mu), 1, chi, t);
                for (int i = 0; i < 12; i++) h[i] = 0;
                add_proj(h, t, mu, +1.0, -0.5 * sb);
            }
            for (int i = 0; i < 12; i++) acc[i] -= h[i];
        }
    for (int i = 0; i < 12; i++) ((ocplx *)out12)[i] = acc[i];
}

#ifdef _OPENMP
#include <omp.h>
#endif
/* threads the oracle's site loops use (reported with CPU timings) */
int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Lie derivatives for the molecular-dynamics forces (Sec. 2, Eq. 4: the    */
/* forces F1, F2 of the pseudofermion terms and of the clover log det).     */
/* A link is moved along U_mu(x) -> exp(eps T_a) U_mu(x), T_a = i lambda_a/2 */
/* (Gell-Mann lambda_a); the derivative at eps = 0 replaces the link by     */
/* dU = T_a U_mu(x), and its adjoint by dU^dag = -U^dag T_a.  D is a sum of */
/* products in which a given link occurs at most once per term (every      */
/* clover leaf holds four distinct links when all extents are >= 2), so the */
/* derivative of a term is the term with that one factor replaced.          */

/* T_a = i lambda_a / 2, a = 0..7 for lambda_1..lambda_8 */
static void gen_T(int a, ocplx *T)
{
    for (int i = 0; i < 9; i++) T[i] = 0;
    ocplx h = 0.5 * I;
    switch (a) {
        case 0: T[1] = T[3] = h; break;                          /* lambda_1 */
        case 1: T[1] = -I * h; T[3] = I * h; break;               /* lambda_2 */
        case 2: T[0] = h; T[4] = -h; break;                       /* lambda_3 */
        case 3: T[2] = T[6] = h; break;                           /* lambda_4 */
        case 4: T[2] = -I * h; T[6] = I * h; break;               /* lambda_5 */
        case 5: T[5] = T[7] = h; break;                           /* lambda_6 */
        case 6: T[5] = -I * h; T[7] = I * h; break;               /* lambda_7 */
        default: {                                                /* lambda_8 */
            double r = 1.0 / sqrt(3.0);
            T[0] = T[4] = h * r;
            T[8] = -2.0 * h * r;
        }
    }
}

/* the moved link: (px, pmu) and dU = T_a U_pmu(px) */
typedef struct {
    long px;
    int pmu;
    ocplx dU[9];
} or_pert;

/* derivative of the product f0 f1 f2 f3 of links (site s[i], direction d[i],
 * adjoint if g[i]); returns 0 (and leaves out untouched) if the moved link
 * is not a factor */
static int leaf_deriv(const oracle *o, const long s[4], const int d[4], const int g[4], const or_pert *P,
                      ocplx *out)
{
    int k = -1;
    for (int i = 0; i < 4; i++)
        if (s[i] == P->px && d[i] == P->pmu) k = i;
    if (k < 0) return 0;
    ocplx f[4][9];
    for (int i = 0; i < 4; i++) {
        const ocplx *M = i == k ? P->dU : link(o, s[i], d[i]);
        if (g[i])
            dag(M, f[i]);
        else
            for (int j = 0; j < 9; j++) f[i][j] = M[j];
    }
    mm4(f[0], f[1], f[2], f[3], out);
    return 1;
}

/* d Fhat_{mu nu}(x): the four leaves of or_fhat_site, differentiated */
static int dfhat_site(const oracle *o, long x, int mu, int nu, const or_pert *P, ocplx *dF)
{
    long xpm = o->fw[4 * x + mu], xpn = o->fw[4 * x + nu];
    long xmm = o->bw[4 * x + mu], xmn = o->bw[4 * x + nu];
    long xmm_pn = o->fw[4 * xmm + nu], xmm_mn = o->bw[4 * xmm + nu], xmn_pm = o->fw[4 * xmn + mu];
    const long S[4][4] = {{x, xpm, xpn, x}, {x, xmm_pn, xmm, xmm}, {xmm, xmm_mn, xmm_mn, xmn}, {xmn, xmn, xmn_pm, x}};
    const int Dd[4][4] = {{mu, nu, mu, nu}, {nu, mu, nu, mu}, {mu, nu, mu, nu}, {nu, mu, nu, mu}};
    const int Gd[4][4] = {{0, 0, 1, 1}, {0, 1, 1, 0}, {1, 1, 0, 0}, {1, 0, 0, 1}};
    ocplx q[9] = {0}, t[9];
    int hit = 0;
    for (int l = 0; l < 4; l++)
        if (leaf_deriv(o, S[l], Dd[l], Gd[l], P, t)) {
            hit = 1;
            for (int i = 0; i < 9; i++) q[i] += t[i];
        }
    if (!hit) return 0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) dF[3 * a + b] = (q[3 * a + b] - conj(q[3 * b + a])) / 8.0;
    return 1;
}

/* d A(x) = c_sw sum_{mu != nu} (i/4) sigma_{mu nu} (x) d Fhat_{mu nu}(x); 0 if it vanishes */
static int dclover_site(const oracle *o, long x, const or_pert *P, ocplx *dA)
{
    int hit = 0;
    for (int i = 0; i < 144; i++) dA[i] = 0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = 0; nu < 4; nu++) {
            if (mu == nu) continue;
            ocplx s[4][4], dF[9];
            if (!dfhat_site(o, x, mu, nu, P, dF)) continue;
            hit = 1;
            sigma(mu, nu, s);
            for (int si = 0; si < 4; si++)
                for (int sj = 0; sj < 4; sj++)
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++)
                            dA[12 * (3 * si + a) + 3 * sj + b] += o->csw * 0.25 * I * s[si][sj] * dF[3 * a + b];
        }
    return hit;
}

static void make_pert(const oracle *o, long x, int mu, int a, or_pert *P)
{
    ocplx T[9];
    gen_T(a, T);
    P->px = x;
    P->pmu = mu;
    mm(T, link(o, x, mu), P->dU);
}

/* out = (d D / d eps) in for the link (x, mu) moved along T_a (full fields):
 * the clover term at every site whose leaves hold the link, and the two hops
 * that use it (forward out of x, backward into x + mu) */
static void dD_apply(const oracle *o, const or_pert *P, const ocplx *in, ocplx *out)
{
    for (long i = 0; i < 12 * o->V; i++) out[i] = 0;
    ocplx dA[144];
    for (long y = 0; y < o->V; y++)
        if (dclover_site(o, y, P, dA)) mat12_vec(dA, in + 12 * y, out + 12 * y);
    long x = P->px, y = o->fw[4 * x + P->pmu];
    int mu = P->pmu, x0 = o->coord[4 * x], y0 = o->coord[4 * y];
    ocplx t[12];
    double sf = (mu == 0 && x0 == o->L[0] - 1) ? o->bc_t : 1.0;
    colour_mul(P->dU, 0, in + 12 * y, t);
    add_proj(out + 12 * x, t, mu, -1.0, -0.5 * sf);
    double sb = (mu == 0 && y0 == 0) ? o->bc_t : 1.0;
    colour_mul(P->dU, 1, in + 12 * x, t);
    add_proj(out + 12 * y, t, mu, +1.0, -0.5 * sb);
}

void or_dD_apply(const oracle *o, long x, int mu, int a, const double *in, double *out)
{
    build_gammas();
    or_pert P;
    make_pert(o, x, mu, a, &P);
    dD_apply(o, &P, (const ocplx *)in, (ocplx *)out);
}

/* g[(4 x + mu) 8 + a] = Re <Y, (d D / d eps_{x,mu,a}) X> for every link and
 * generator (X, Y full fields) */
void or_force_dD(const oracle *o, const double *X_, const double *Y_, double *g)
{
    build_gammas();
    const ocplx *X = (const ocplx *)X_, *Y = (const ocplx *)Y_;
#pragma omp parallel for schedule(dynamic)
    for (long l = 0; l < 4 * o->V; l++) {
        ocplx *w = malloc(sizeof(ocplx) * 12 * o->V);
        for (int a = 0; a < 8; a++) {
            or_pert P;
            make_pert(o, l / 4, (int)(l % 4), a, &P);
            dD_apply(o, &P, X, w);
            double acc = 0;
            for (long i = 0; i < 12 * o->V; i++) acc += creal(conj(Y[i]) * w[i]);
            g[8 * l + a] = acc;
        }
        free(w);
    }
}

/* g[(4 x + mu) 8 + a] = d/d eps log|det A| summed over the sites of the given
 * parity = sum_y Re tr(A(y)^-1 dA(y)) */
void or_force_logdet(const oracle *o, int parity, double *g)
{
    build_gammas();
#pragma omp parallel for schedule(dynamic)
    for (long l = 0; l < 4 * o->V; l++)
        for (int a = 0; a < 8; a++) {
            or_pert P;
            make_pert(o, l / 4, (int)(l % 4), a, &P);
            double acc = 0;
            ocplx dA[144];
            for (long y = 0; y < o->V; y++) {
                if (o->par[y] != parity || !dclover_site(o, y, &P, dA)) continue;
                const ocplx *Ai = o->Ainv + 144 * y;
                for (int i = 0; i < 12; i++)
                    for (int k = 0; k < 12; k++) acc += creal(Ai[12 * i + k] * dA[12 * k + i]);
            }
            g[8 * l + a] = acc;
        }
}

/* Wilson gauge action S_g = beta sum_{x, mu < nu} (1 - (1/3) Re tr U_P(x; mu, nu)),
 * U_P(x; mu, nu) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag (the MD step of
 * the HMC, Sec. 2), and its gradient along exp(eps T_a) U link by link. */
static void plaquette_links(const oracle *o, long x, int mu, int nu, long s[4], int d[4], int g[4])
{
    s[0] = x;
    s[1] = o->fw[4 * x + mu];
    s[2] = o->fw[4 * x + nu];
    s[3] = x;
    d[0] = mu;
    d[1] = nu;
    d[2] = mu;
    d[3] = nu;
    g[0] = g[1] = 0;
    g[2] = g[3] = 1;
}

double or_gauge_action(const oracle *o, double beta)
{
    double acc = 0;
    for (long x = 0; x < o->V; x++)
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) {
                long s[4];
                int d[4], g[4];
                plaquette_links(o, x, mu, nu, s, d, g);
                ocplx d1[9], d2[9], P[9];
                dag(link(o, s[2], mu), d1);
                dag(link(o, s[3], nu), d2);
                mm4(link(o, s[0], mu), link(o, s[1], nu), d1, d2, P);
                acc += 1.0 - creal(P[0] + P[4] + P[8]) / 3.0;
            }
    return beta * acc;
}

void or_grad_gauge(const oracle *o, double beta, double *g_out)
{
#pragma omp parallel for schedule(dynamic)
    for (long l = 0; l < 4 * o->V; l++)
        for (int a = 0; a < 8; a++) {
            or_pert P;
            make_pert(o, l / 4, (int)(l % 4), a, &P);
            double acc = 0;
            for (long x = 0; x < o->V; x++)
                for (int mu = 0; mu < 4; mu++)
                    for (int nu = mu + 1; nu < 4; nu++) {
                        long s[4];
                        int d[4], g[4];
                        ocplx dP[9];
                        plaquette_links(o, x, mu, nu, s, d, g);
                        if (leaf_deriv(o, s, d, g, &P, dP)) acc -= creal(dP[0] + dP[4] + dP[8]) / 3.0;
                    }
            g_out[8 * l + a] = beta * acc;
        }
}
