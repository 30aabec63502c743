// Molecular-dynamics forces and the leapfrog step of the two-flavour HMC
// (Sec. 2, Eq. 4), FP64.
//
// A link moves along U_mu(x) -> exp(eps T_a) U_mu(x), T_a = i lambda_a / 2
// (Gell-Mann matrices); a gradient is dS/d eps per link and generator, stored
// g[site][mu][a] (lexicographic sites, the MD force is its negative).  Every
// kernel gathers what one link receives (one thread per link, no atomics):
//
//   hops     D holds U_mu(x) in the forward hop out of x and, as U^dag, in
//            the backward hop into x + mu, so
//              Re <Y, dD X> = Re tr(T_a M),
//              M = -1/2 s U B1 + 1/2 s B2 U^dag,
//            B1 = sum_s [(1 - g_mu) X(x+mu)]_s Y(x)_s^dag,
//            B2 = sum_s [(1 + g_mu) X(x)]_s Y(x+mu)_s^dag (colour outer
//            products), s the antiperiodic time sign of the link;
//   clover   the term c_sw (i/4) sigma_{rho sigma} Fhat_{rho sigma}(y) with
//            Fhat = (Q - Q^dag)/8 and Q the four leaves at y: per site and
//            plane Lam[k][i] = (i/4) sum_ab sigma_ab M_{(b k),(a i)}, with
//            M = X Y^dag (pseudofermion) or M = A(y)^-1 (log det), and
//            Om = Lam - Lam^dag; a leaf f0 f1 f2 f3 whose factor f_j is the
//            link contributes (c_sw / 8) U B Om A for f_j = U and
//            -(c_sw / 8) B Om A U^dag for f_j = U^dag, A = f0..f_{j-1},
//            B = f_{j+1}..f3;
//   gauge    S_g = beta sum_P (1 - Re tr U_P / 3): M = -(beta / 3) U sum
//            (staples).
//
// The leapfrog step (p -= dt/2 g; U <- exp(dt P) U; p -= dt/2 g, with
// P = sum_a p^a T_a) exponentiates with a Taylor series after scaling and
// squaring (Moler & Van Loan, "Nineteen dubious ways to compute the
// exponential of a matrix, twenty-five years later", 2003).
#include <cmath>
#include <vector>

#include "lqcd_internal.cuh"

namespace {

using Cd = cx<double>;

struct M3 {
    Cd m[3][3];
};

__device__ __forceinline__ M3 m3_zero()
{
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) c.m[i][j] = mk(0.0, 0.0);
    return c;
}
__device__ __forceinline__ M3 m3_one()
{
    M3 c = m3_zero();
#pragma unroll
    for (int i = 0; i < 3; i++) c.m[i][i] = mk(1.0, 0.0);
    return c;
}
__device__ __forceinline__ M3 mul(const M3 &a, const M3 &b)
{
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) c.m[i][j] = a.m[i][0] * b.m[0][j] + a.m[i][1] * b.m[1][j] + a.m[i][2] * b.m[2][j];
    return c;
}
__device__ __forceinline__ M3 dag(const M3 &a)
{
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) c.m[i][j] = conjx(a.m[j][i]);
    return c;
}
__device__ __forceinline__ void add_scaled(M3 &acc, double s, const M3 &a)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) acc.m[i][j] = acc.m[i][j] + s * a.m[i][j];
}

// host-built tables: gamma_mu, sigma_{rho sigma} (rho < sigma, planes 01 02 03
// 12 13 23) and the Gell-Mann matrices, complex (re, im)
struct Tabs {
    double2 gam[4][4][4];
    double2 sig[6][4][4];
    double2 lam[8][3][3];
};

__device__ __forceinline__ Cd tc(const double2 &v) { return mk(v.x, v.y); }

// g_a = Re tr(T_a M) = Re tr((i/2) lambda_a M)
__device__ __forceinline__ void project_generators(const Tabs &T, const M3 &M, double g[8])
{
#pragma unroll
    for (int a = 0; a < 8; a++) {
        Cd t = mk(0.0, 0.0);
#pragma unroll
        for (int j = 0; j < 3; j++)
#pragma unroll
            for (int k = 0; k < 3; k++) t = t + tc(T.lam[a][j][k]) * M.m[k][j];
        g[a] = -0.5 * t.im;   // Re(i t / 2)
    }
}

__device__ __forceinline__ void site_coords(const Geom &g, long s, int x[4])
{
    x[3] = (int)(s % g.L[3]);
    long t = s / g.L[3];
    x[2] = (int)(t % g.L[2]);
    t /= g.L[2];
    x[1] = (int)(t % g.L[1]);
    x[0] = (int)(t / g.L[1]);
}
__device__ __forceinline__ long site_index(const Geom &g, const int x[4])
{
    return x[3] + (long)g.L[3] * (x[2] + (long)g.L[2] * (x[1] + (long)g.L[1] * x[0]));
}
__device__ __forceinline__ void shift(const Geom &g, int y[4], int mu, int d)
{
    int v = y[mu] + d;
    y[mu] = v < 0 ? v + g.L[mu] : (v >= g.L[mu] ? v - g.L[mu] : v);
}
// U_mu(x) from the native FP64 copy ([p][mu][9][Vh] at rank site >> 1)
__device__ __forceinline__ M3 link_at(const Geom &g, const double2 *__restrict__ U, const int x[4], int mu)
{
    const long s = site_index(g, x);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const double2 *b = U + (long)((p * 4 + mu) * 9) * g.Vh + (s >> 1);
    M3 u;
#pragma unroll
    for (int e = 0; e < 9; e++) u.m[e / 3][e % 3] = tc(b[e * (long)g.Vh]);
    return u;
}
__device__ __forceinline__ void spinor_at(const double2 *f, long s, Cd v[4][3])
{
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
        for (int c = 0; c < 3; c++) v[sp][c] = tc(f[12 * s + 3 * sp + c]);
}

__device__ __forceinline__ void store_grad(double *gout, long l, const double gv[8], double scale, int accumulate)
{
#pragma unroll
    for (int a = 0; a < 8; a++) gout[8 * l + a] = (accumulate ? gout[8 * l + a] : 0.0) + scale * gv[a];
}

// ------------------------------------------------------------------ hops
__global__ void __launch_bounds__(128) k_force_hop(Geom g, const double2 *__restrict__ U, const double2 *__restrict__ X,
                                                   const double2 *__restrict__ Y, double *gout, double scale,
                                                   int accumulate, Tabs T)
{
    const long l = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (l >= 4L * g.V) return;
    const long s = l >> 2;
    const int mu = (int)(l & 3);
    int x[4], y[4];
    site_coords(g, s, x);
    for (int i = 0; i < 4; i++) y[i] = x[i];
    shift(g, y, mu, +1);
    const long sy = site_index(g, y);
    const double sgn = (mu == 0 && x[0] == g.L[0] - 1) ? double(g.bc_t) : 1.0;
    const M3 u = link_at(g, U, x, mu);
    Cd Xx[4][3], Xy[4][3], Yx[4][3], Yy[4][3];
    spinor_at(X, s, Xx);
    spinor_at(X, sy, Xy);
    spinor_at(Y, s, Yx);
    spinor_at(Y, sy, Yy);
    M3 B1 = m3_zero(), B2 = m3_zero();
#pragma unroll
    for (int sp = 0; sp < 4; sp++) {
        Cd a[3], b[3];   // [(1 - g_mu) X(x+mu)]_sp, [(1 + g_mu) X(x)]_sp
#pragma unroll
        for (int k = 0; k < 3; k++) {
            a[k] = Xy[sp][k];
            b[k] = Xx[sp][k];
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const Cd gm = tc(T.gam[mu][sp][t]);
                a[k] = a[k] - gm * Xy[t][k];
                b[k] = b[k] + gm * Xx[t][k];
            }
        }
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
            for (int i = 0; i < 3; i++) {
                B1.m[k][i] = B1.m[k][i] + a[k] * conjx(Yx[sp][i]);
                B2.m[k][i] = B2.m[k][i] + b[k] * conjx(Yy[sp][i]);
            }
    }
    M3 M = m3_zero();
    add_scaled(M, -0.5 * sgn, mul(u, B1));
    add_scaled(M, 0.5 * sgn, mul(B2, dag(u)));
    double gv[8];
    project_generators(T, M, gv);
    store_grad(gout, l, gv, scale, accumulate);
}

// ------------------------------------------------------------------ clover
// plane index of (rho, sigma), rho < sigma
__device__ __forceinline__ int plane_of(int r, int s) { return r == 0 ? s - 1 : (r == 1 ? s + 1 : 5); }

// Om[site][plane][9]: from X Y^dag (src = 0) or from A^-1 on the sites of
// parity par (src = 1; other sites get zero)
__global__ void __launch_bounds__(128) k_omega(Geom g, int src, const double2 *__restrict__ X,
                                               const double2 *__restrict__ Y, const double2 *__restrict__ Ai,
                                               int par, double2 *Om, Tabs T)
{
    const long s = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int x[4];
    site_coords(g, s, x);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    Cd lam[6][3][3];
#pragma unroll
    for (int pl = 0; pl < 6; pl++)
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
            for (int i = 0; i < 3; i++) lam[pl][k][i] = mk(0.0, 0.0);
    if (src == 0) {
        Cd Xs[4][3], Ys[4][3];
        spinor_at(X, s, Xs);
        spinor_at(Y, s, Ys);
        for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++) {
                Cd m[3][3];   // M_{(b k),(a i)} = X[b][k] conj(Y[a][i])
#pragma unroll
                for (int k = 0; k < 3; k++)
#pragma unroll
                    for (int i = 0; i < 3; i++) m[k][i] = Xs[b][k] * conjx(Ys[a][i]);
#pragma unroll
                for (int pl = 0; pl < 6; pl++) {
                    const Cd sab = tc(T.sig[pl][a][b]);
#pragma unroll
                    for (int k = 0; k < 3; k++)
#pragma unroll
                        for (int i = 0; i < 3; i++) lam[pl][k][i] = lam[pl][k][i] + sab * m[k][i];
                }
            }
    } else if (p == par) {
        const long Vh = g.Vh, r = s >> 1;
        for (int h = 0; h < 2; h++) {   // chirality block: spins 2h, 2h+1
            double d[6];
            Cd o[15];
            const double2 *bp = Ai + (long)(18 * h) * Vh + r;
            for (int q = 0; q < 3; q++) {
                const double2 v = bp[q * Vh];
                d[2 * q] = v.x;
                d[2 * q + 1] = v.y;
            }
            for (int q = 0; q < 15; q++) o[q] = tc(bp[(3 + q) * Vh]);
            Cd blk[6][6];
            int kk = 0;
            for (int i = 0; i < 6; i++) {
                blk[i][i] = mk(d[i], 0.0);
                for (int j = i + 1; j < 6; j++) {
                    blk[i][j] = o[kk];
                    blk[j][i] = conjx(o[kk]);
                    kk++;
                }
            }
            for (int al = 0; al < 2; al++)
                for (int bl = 0; bl < 2; bl++) {
                    const int a = 2 * h + al, b = 2 * h + bl;
                    for (int pl = 0; pl < 6; pl++) {
                        const Cd sab = tc(T.sig[pl][a][b]);
                        for (int k = 0; k < 3; k++)
                            for (int i = 0; i < 3; i++)
                                lam[pl][k][i] = lam[pl][k][i] + sab * blk[3 * bl + k][3 * al + i];
                    }
                }
        }
    }
    // Lam = (i/4) sum, Om = Lam - Lam^dag
#pragma unroll
    for (int pl = 0; pl < 6; pl++)
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const Cd lk = timesI(lam[pl][k][i]), li = timesI(lam[pl][i][k]);
                const Cd om = 0.25 * (lk - conjx(li));
                Om[(s * 6 + pl) * 9 + 3 * k + i] = make_double2(om.re, om.im);
            }
}

// factor q of leaf l in the ordered plane (rho, sigma) at y: offset (in rho,
// sigma steps) of the link's site, its direction (0: rho, 1: sigma) and
// whether it enters as U^dag.  The four leaves run the same way round.
__device__ __forceinline__ void leaf_factor(int l, int q, int &dr, int &ds, int &dir, int &dg)
{
    // [leaf][factor] = (dr, ds, dir, dag)
    const signed char tab[4][4][4] = {
        {{0, 0, 0, 0}, {1, 0, 1, 0}, {0, 1, 0, 1}, {0, 0, 1, 1}},
        {{0, 0, 1, 0}, {-1, 1, 0, 1}, {-1, 0, 1, 1}, {-1, 0, 0, 0}},
        {{-1, 0, 0, 1}, {-1, -1, 1, 1}, {-1, -1, 0, 0}, {0, -1, 1, 0}},
        {{0, -1, 1, 1}, {0, -1, 0, 0}, {1, -1, 1, 0}, {0, 0, 0, 1}},
    };
    dr = tab[l][q][0];
    ds = tab[l][q][1];
    dir = tab[l][q][2];
    dg = tab[l][q][3];
}

__global__ void __launch_bounds__(64) k_force_clover(Geom g, const double2 *__restrict__ U,
                                                     const double2 *__restrict__ Om, double coef, double *gout,
                                                     double scale, int accumulate, Tabs T)
{
    const long l = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (l >= 4L * g.V) return;
    const long s = l >> 2;
    const int mu = (int)(l & 3);
    int x[4];
    site_coords(g, s, x);
    const M3 u = link_at(g, U, x, mu);
    M3 M = m3_zero();
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        for (int ord = 0; ord < 2; ord++) {   // ordered planes (mu, nu) and (nu, mu)
            const int rho = ord == 0 ? mu : nu, sg = ord == 0 ? nu : mu;
            const int dirmu = ord == 0 ? 0 : 1;   // the link's role in the plane
            const int pl = plane_of(min(rho, sg), max(rho, sg));
            const double osign = rho < sg ? 1.0 : -1.0;   // Om_{sigma rho} = -Om_{rho sigma}
            for (int lf = 0; lf < 4; lf++)
                for (int j = 0; j < 4; j++) {
                    int dr, ds, dir, dg;
                    leaf_factor(lf, j, dr, ds, dir, dg);
                    if (dir != dirmu) continue;
                    // the leaf's site: x = y + dr rho + ds sigma
                    int y[4] = {x[0], x[1], x[2], x[3]};
                    shift(g, y, rho, -dr);
                    shift(g, y, sg, -ds);
                    M3 A = m3_one(), B = m3_one();
                    for (int q = 0; q < 4; q++) {
                        if (q == j) continue;
                        int qr, qs, qd, qg;
                        leaf_factor(lf, q, qr, qs, qd, qg);
                        int z[4] = {y[0], y[1], y[2], y[3]};
                        shift(g, z, rho, qr);
                        shift(g, z, sg, qs);
                        M3 f = link_at(g, U, z, qd == 0 ? rho : sg);
                        if (qg) f = dag(f);
                        if (q < j)
                            A = mul(A, f);
                        else
                            B = mul(B, f);
                    }
                    M3 om;
                    const double2 *op = Om + (site_index(g, y) * 6 + pl) * 9;
#pragma unroll
                    for (int e = 0; e < 9; e++) om.m[e / 3][e % 3] = osign * tc(op[e]);
                    const M3 BOA = mul(mul(B, om), A);
                    if (!dg)
                        add_scaled(M, coef / 8.0, mul(u, BOA));
                    else
                        add_scaled(M, -coef / 8.0, mul(BOA, dag(u)));
                }
        }
    }
    double gv[8];
    project_generators(T, M, gv);
    store_grad(gout, l, gv, scale, accumulate);
}

// ------------------------------------------------------------------ gauge
__global__ void __launch_bounds__(128) k_force_gauge(Geom g, const double2 *__restrict__ U, double beta, double *gout,
                                                     double scale, int accumulate, Tabs T)
{
    const long l = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (l >= 4L * g.V) return;
    const long s = l >> 2;
    const int mu = (int)(l & 3);
    int x[4];
    site_coords(g, s, x);
    const M3 u = link_at(g, U, x, mu);
    M3 st = m3_zero();
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        int xm[4] = {x[0], x[1], x[2], x[3]}, xn[4] = {x[0], x[1], x[2], x[3]};
        shift(g, xm, mu, +1);
        shift(g, xn, nu, +1);
        // up: U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
        add_scaled(st, 1.0, mul(mul(link_at(g, U, xm, nu), dag(link_at(g, U, xn, mu))), dag(link_at(g, U, x, nu))));
        // down: U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
        int xmn[4] = {xm[0], xm[1], xm[2], xm[3]}, xd[4] = {x[0], x[1], x[2], x[3]};
        shift(g, xmn, nu, -1);
        shift(g, xd, nu, -1);
        add_scaled(st, 1.0,
                   mul(mul(dag(link_at(g, U, xmn, nu)), dag(link_at(g, U, xd, mu))), link_at(g, U, xd, nu)));
    }
    M3 M = m3_zero();
    add_scaled(M, -beta / 3.0, mul(u, st));
    double gv[8];
    project_generators(T, M, gv);
    store_grad(gout, l, gv, scale, accumulate);
}

// per-site sum over the six planes of 1 - Re tr U_P / 3
__global__ void __launch_bounds__(128) k_plaq_site(Geom g, const double2 *__restrict__ U, double *out)
{
    const long s = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int x[4];
    site_coords(g, s, x);
    double acc = 0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++) {
            int xm[4] = {x[0], x[1], x[2], x[3]}, xn[4] = {x[0], x[1], x[2], x[3]};
            shift(g, xm, mu, +1);
            shift(g, xn, nu, +1);
            const M3 P = mul(mul(link_at(g, U, x, mu), link_at(g, U, xm, nu)),
                             mul(dag(link_at(g, U, xn, mu)), dag(link_at(g, U, x, nu))));
            acc += 1.0 - (P.m[0][0].re + P.m[1][1].re + P.m[2][2].re) / 3.0;
        }
    out[s] = acc;
}

// fixed-order sum of n doubles (one CTA, deterministic)
__global__ void k_sum_md(const double *x, long n, double *out)
{
    __shared__ double sh[256];
    double s = 0;
    for (long i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// ------------------------------------------------------------------ MD step
// U <- exp(dt P) U on canonical links [site][mu][3][3] (complex), P = sum_a p^a T_a
__global__ void __launch_bounds__(128) k_move_links(long nlink, const double *__restrict__ p, double dt, double2 *U,
                                                    Tabs T)
{
    const long l = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (l >= nlink) return;
    M3 P = m3_zero();
    for (int a = 0; a < 8; a++) {
        const double c = dt * p[8 * l + a];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) P.m[i][j] = P.m[i][j] + (0.5 * c) * timesI(tc(T.lam[a][i][j]));
    }
    // scaling: |P| / 2^k <= 1/2 in the max-row-sum norm
    double nrm = 0;
    for (int i = 0; i < 3; i++) {
        double r = 0;
        for (int j = 0; j < 3; j++) r += sqrt(P.m[i][j].re * P.m[i][j].re + P.m[i][j].im * P.m[i][j].im);
        nrm = fmax(nrm, r);
    }
    int k = 0;
    while (nrm > 0.5 && k < 60) {
        nrm *= 0.5;
        k++;
    }
    const double sc = ldexp(1.0, -k);
    M3 A;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) A.m[i][j] = sc * P.m[i][j];
    // Taylor series to order 20: remainder below 0.5^21 / 21! relative
    M3 E = m3_one(), term = m3_one();
    for (int n = 1; n <= 20; n++) {
        term = mul(term, A);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) term.m[i][j] = (1.0 / n) * term.m[i][j];
        add_scaled(E, 1.0, term);
    }
    for (int q = 0; q < k; q++) E = mul(E, E);
    M3 u;
    double2 *up = U + 9 * l;
    for (int e = 0; e < 9; e++) u.m[e / 3][e % 3] = tc(up[e]);
    const M3 v = mul(E, u);
    for (int e = 0; e < 9; e++) up[e] = make_double2(v.m[e / 3][e % 3].re, v.m[e / 3][e % 3].im);
}

__global__ void k_axpy_real(long n, double a, const double *__restrict__ x, double *y)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

// ------------------------------------------------------------------ host
Tabs make_tabs()
{
    Tabs T{};
    auto set = [](double2 &d, double re, double im) { d = make_double2(re, im); };
    // chiral basis: g0 = [[0,-1],[-1,0]], gk = [[0,-i s_k],[i s_k,0]]
    double re[4][4][4] = {}, im[4][4][4] = {};
    re[0][0][2] = re[0][1][3] = re[0][2][0] = re[0][3][1] = -1;
    // s1 = [[0,1],[1,0]]: -i s1 upper right, i s1 lower left
    im[1][0][3] = im[1][1][2] = -1;
    im[1][2][1] = im[1][3][0] = 1;
    // s2 = [[0,-i],[i,0]]: -i s2 = [[0,-1],[1,0]], i s2 = [[0,1],[-1,0]]
    re[2][0][3] = -1;
    re[2][1][2] = 1;
    re[2][2][1] = 1;
    re[2][3][0] = -1;
    // s3 = diag(1,-1): -i s3 = diag(-i, i), i s3 = diag(i, -i)
    im[3][0][2] = -1;
    im[3][1][3] = 1;
    im[3][2][0] = 1;
    im[3][3][1] = -1;
    for (int m = 0; m < 4; m++)
        for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++) set(T.gam[m][a][b], re[m][a][b], im[m][a][b]);
    // sigma_{rs} = (i/2) [g_r, g_s]
    const int pr[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    for (int pl = 0; pl < 6; pl++) {
        const int r = pr[pl][0], s = pr[pl][1];
        for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++) {
                double cr = 0, ci = 0;   // [g_r, g_s]_{ab}
                for (int c = 0; c < 4; c++) {
                    cr += re[r][a][c] * re[s][c][b] - im[r][a][c] * im[s][c][b];
                    ci += re[r][a][c] * im[s][c][b] + im[r][a][c] * re[s][c][b];
                    cr -= re[s][a][c] * re[r][c][b] - im[s][a][c] * im[r][c][b];
                    ci -= re[s][a][c] * im[r][c][b] + im[s][a][c] * re[r][c][b];
                }
                set(T.sig[pl][a][b], -0.5 * ci, 0.5 * cr);   // (i/2)(cr + i ci)
            }
    }
    // Gell-Mann matrices
    const double r3 = 1.0 / std::sqrt(3.0);
    set(T.lam[0][0][1], 1, 0);
    set(T.lam[0][1][0], 1, 0);
    set(T.lam[1][0][1], 0, -1);
    set(T.lam[1][1][0], 0, 1);
    set(T.lam[2][0][0], 1, 0);
    set(T.lam[2][1][1], -1, 0);
    set(T.lam[3][0][2], 1, 0);
    set(T.lam[3][2][0], 1, 0);
    set(T.lam[4][0][2], 0, -1);
    set(T.lam[4][2][0], 0, 1);
    set(T.lam[5][1][2], 1, 0);
    set(T.lam[5][2][1], 1, 0);
    set(T.lam[6][1][2], 0, -1);
    set(T.lam[6][2][1], 0, 1);
    set(T.lam[7][0][0], r3, 0);
    set(T.lam[7][1][1], r3, 0);
    set(T.lam[7][2][2], -2 * r3, 0);
    return T;
}

const Tabs &tabs()
{
    static const Tabs T = make_tabs();
    return T;
}

int grid_links(const lqcd_ctx *c, int tpb) { return div_up(4L * c->g.V, tpb); }

lqcd_status need_state(lqcd_ctx *c)
{
    if (!c->have_gauge) return set_err(c, LQCD_ERR_STATE, "gauge field not set");
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    return LQCD_OK;
}

// g (+)= scale * Re <Y, dD X> (X, Y canonical full FP64 fields on the device)
lqcd_status force_dD(lqcd_ctx *c, const double *X, const double *Y, double *g, double scale, int accumulate)
{
    LQCD_TRY(need_state(c));
    const Tabs &T = tabs();
    k_force_hop<<<grid_links(c, 128), 128, 0, c->stream>>>(c->g, c->U64, (const double2 *)X, (const double2 *)Y, g,
                                                           scale, accumulate, T);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    if (c->csw != 0.0) {
        void *om;
        LQCD_TRY(ws_get(c, WS_MD_OMEGA, (size_t)c->g.V * 6 * 9 * sizeof(double2), &om));
        k_omega<<<div_up(c->g.V, 128), 128, 0, c->stream>>>(c->g, 0, (const double2 *)X, (const double2 *)Y, nullptr, 0,
                                                            (double2 *)om, T);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        k_force_clover<<<grid_links(c, 64), 64, 0, c->stream>>>(c->g, c->U64, (const double2 *)om, c->csw, g, scale, 1,
                                                                T);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
    }
    return LQCD_OK;
}

// g (+)= scale * d log|det A_parity| / d eps = scale * sum_y Re tr(A^-1 dA)
lqcd_status force_logdet(lqcd_ctx *c, int parity, double *g, double scale, int accumulate)
{
    LQCD_TRY(need_state(c));
    if (c->csw == 0.0) {   // A = (4 + m0) 1 does not depend on the links
        if (!accumulate) LQCD_TRY(blas_zero(c, (size_t)c->g.V * 32 * sizeof(double), g));
        return LQCD_OK;
    }
    const Tabs &T = tabs();
    void *om;
    LQCD_TRY(ws_get(c, WS_MD_OMEGA, (size_t)c->g.V * 6 * 9 * sizeof(double2), &om));
    k_omega<<<div_up(c->g.V, 128), 128, 0, c->stream>>>(c->g, 1, nullptr, nullptr, c->Ai64[parity], parity,
                                                        (double2 *)om, T);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    k_force_clover<<<grid_links(c, 64), 64, 0, c->stream>>>(c->g, c->U64, (const double2 *)om, c->csw, g, scale,
                                                            accumulate, T);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

lqcd_status force_gauge(lqcd_ctx *c, double beta, double *g, double scale, int accumulate)
{
    if (!c->have_gauge) return set_err(c, LQCD_ERR_STATE, "gauge field not set");
    k_force_gauge<<<grid_links(c, 128), 128, 0, c->stream>>>(c->g, c->U64, beta, g, scale, accumulate, tabs());
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

lqcd_status gauge_action(lqcd_ctx *c, double beta, double *S)
{
    if (!c->have_gauge) return set_err(c, LQCD_ERR_STATE, "gauge field not set");
    void *w;
    LQCD_TRY(ws_get(c, WS_MD_SCRATCH, (size_t)c->g.V * sizeof(double) + 64, &w));
    double *site = (double *)w;
    k_plaq_site<<<div_up(c->g.V, 128), 128, 0, c->stream>>>(c->g, c->U64, site);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    k_sum_md<<<1, 256, 0, c->stream>>>(site, c->g.V, c->red_out);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    double h = 0;
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(&h, c->red_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    *S = beta * h;
    return LQCD_OK;
}

// The pseudofermion field of S_pf = |Dhat^-1 phi|^2 and its gradient
// -2 Re <Y, dD X>, X = (x_e, -A_oo^-1 H_oe x_e), Y = (y_e, -A_oo^-1 H_eo^dag y_e),
// x_e = Dhat^-1 phi, y_e = Dhat^-dag x_e = gamma5 Dhat^-1 gamma5 x_e; with these
// completions <Y, dD X> = <y_e, dDhat x_e>.  S (optional) = |x_e|^2.
lqcd_status force_pf(lqcd_ctx *c, const lqcd_solver_params *sp, const double *phi_e, double *g, double scale,
                     int accumulate, double *S, lqcd_solve_info *info)
{
    LQCD_TRY(need_state(c));
    const long Vh = c->g.Vh;
    const size_t hb = native_half_bytes(c, LQCD_F64);   // one native half field
    const long ne = 24 * Vh;                              // doubles in an even canonical field
    void *w;
    // canonical: x_e, t_e, y_e (even), X, Y (full); native: three full fields
    LQCD_TRY(ws_get(c, WS_MD_FIELDS, 3 * ne * sizeof(double) + 2 * 2 * ne * sizeof(double) + 6 * hb, &w));
    double *xe = (double *)w, *te = xe + ne, *ye = te + ne, *Xf = ye + ne, *Yf = Xf + 2 * ne;
    double2 *nx = (double2 *)(Yf + 2 * ne), *ny = nx + 24 * Vh, *nt = ny + 24 * Vh;
    lqcd_solve_info inf[2];
    LQCD_TRY(lqcd_solve_dhat(c, sp, phi_e, xe, 1, &inf[0]));
    // gamma5 on a canonical even field: spins 2, 3 change sign
    auto g5 = [&](const double *in, double *out) -> lqcd_status {
        LQCD_TRY(pack_field(c, LQCD_F64, 1, in, nx, 1, false));
        LQCD_TRY(blas_gamma5_native64(c, 1, nx, nx));
        return pack_field(c, LQCD_F64, 1, out, nx, 1, true);
    };
    LQCD_TRY(g5(xe, te));
    LQCD_TRY(lqcd_solve_dhat(c, sp, te, ye, 1, &inf[1]));
    LQCD_TRY(g5(ye, ye));
    if (info) {
        info[0] = inf[0];
        info[1] = inf[1];
    }
    // X = (x_e, -A_oo^-1 H_oe x_e) in native order [even][odd]
    const long hh = 12 * Vh;
    LQCD_TRY(pack_field(c, LQCD_F64, 1, xe, nx, 1, false));
    LQCD_TRY(dirac_hop_parity(c, LQCD_F64, 1, nx, nt, hh, hh, 1));
    LQCD_TRY(clover_apply_native64(c, 1, 1, nt, nx + hh));
    LQCD_TRY(blas_scal(c, 2 * hh, -1.0, 0.0, (double *)(nx + hh)));
    // Y = (y_e, -A_oo^-1 gamma5 H_oe gamma5 y_e)
    LQCD_TRY(pack_field(c, LQCD_F64, 1, ye, ny, 1, false));
    LQCD_TRY(blas_gamma5_native64(c, 1, ny, nt));
    LQCD_TRY(dirac_hop_parity(c, LQCD_F64, 1, nt, nt + hh, hh, hh, 1));
    LQCD_TRY(blas_gamma5_native64(c, 1, nt + hh, nt));
    LQCD_TRY(clover_apply_native64(c, 1, 1, nt, ny + hh));
    LQCD_TRY(blas_scal(c, 2 * hh, -1.0, 0.0, (double *)(ny + hh)));
    LQCD_TRY(pack_field(c, LQCD_F64, 2, Xf, nx, 1, true));
    LQCD_TRY(pack_field(c, LQCD_F64, 2, Yf, ny, 1, true));
    LQCD_TRY(force_dD(c, Xf, Yf, g, -2.0 * scale, accumulate));
    if (S) {
        double n2 = 0;
        LQCD_TRY(blas_norm2(c, ne, xe, &n2));
        *S = n2;
    }
    lqcd_status st = inf[0].status != LQCD_OK ? inf[0].status : inf[1].status;
    if (st != LQCD_OK) return set_err(c, st, "pseudofermion force: solve did not converge");
    return LQCD_OK;
}

// total gradient of S = S_g + |Dhat^-1 phi|^2 - 2 log|det A_oo|
lqcd_status md_gradient(lqcd_ctx *c, const lqcd_md_params *mp, const double *phi_e, double *g, double *S,
                        lqcd_solve_info *info)
{
    LQCD_TRY(force_gauge(c, mp->beta, g, 1.0, 0));
    double spf = 0;
    LQCD_TRY(force_pf(c, &mp->solver, phi_e, g, 1.0, 1, S ? &spf : nullptr, info));
    LQCD_TRY(force_logdet(c, 1, g, -2.0, 1));
    if (S) {
        double sg;
        LQCD_TRY(gauge_action(c, mp->beta, &sg));
        *S = sg + spf - 2.0 * c->logdet_o;
    }
    return LQCD_OK;
}

lqcd_status check_md(lqcd_ctx *c, const lqcd_md_params *mp)
{
    if (!mp) return set_err(c, LQCD_ERR_ARG, "null MD parameters");
    if (mp->nsteps < 0 || !(std::isfinite(mp->dt)) || !(std::isfinite(mp->beta)))
        return set_err(c, LQCD_ERR_ARG, "bad MD parameters");
    return LQCD_OK;
}

}  // namespace

extern "C" {

lqcd_status lqcd_force_dD(lqcd_ctx *c, const double *X, const double *Y, double *g)
{
    if (!c || !X || !Y || !g) return set_err(c, LQCD_ERR_ARG, "null argument");
    return force_dD(c, X, Y, g, 1.0, 0);
}

lqcd_status lqcd_force_logdet(lqcd_ctx *c, int parity, double *g)
{
    if (!c || !g || parity < 0 || parity > 1) return set_err(c, LQCD_ERR_ARG, "bad argument");
    return force_logdet(c, parity, g, 1.0, 0);
}

lqcd_status lqcd_gauge_action(lqcd_ctx *c, double beta, double *S)
{
    if (!c || !S) return set_err(c, LQCD_ERR_ARG, "null argument");
    return gauge_action(c, beta, S);
}

lqcd_status lqcd_force_gauge(lqcd_ctx *c, double beta, double *g)
{
    if (!c || !g) return set_err(c, LQCD_ERR_ARG, "null argument");
    return force_gauge(c, beta, g, 1.0, 0);
}

lqcd_status lqcd_force_pf(lqcd_ctx *c, const lqcd_solver_params *sp, const double *phi_e, double *g,
                          lqcd_solve_info *info)
{
    if (!c || !sp || !phi_e || !g) return set_err(c, LQCD_ERR_ARG, "null argument");
    return force_pf(c, sp, phi_e, g, 1.0, 0, nullptr, info);
}

lqcd_status lqcd_md_gradient(lqcd_ctx *c, const lqcd_md_params *mp, const double *phi_e, double *g, double *S)
{
    if (!c || !phi_e || !g) return set_err(c, LQCD_ERR_ARG, "null argument");
    LQCD_TRY(check_md(c, mp));
    LQCD_TRY(need_state(c));
    return md_gradient(c, mp, phi_e, g, S, nullptr);
}

lqcd_status lqcd_md_leapfrog(lqcd_ctx *c, const lqcd_md_params *mp, double *U, double *p, const double *phi_e)
{
    if (!c || !U || !p || !phi_e) return set_err(c, LQCD_ERR_ARG, "null argument");
    LQCD_TRY(check_md(c, mp));
    LQCD_TRY(need_state(c));
    const double kappa = c->kappa, csw = c->csw;
    const long nl = 4L * c->g.V, np = 8 * nl;
    void *w;
    LQCD_TRY(ws_get(c, WS_MD_GRAD, np * sizeof(double), &w));
    double *g = (double *)w;
    const int gr = (int)std::min<long>(4 * 152, div_up(np, 256));
    // the field in U is the one the context holds: its gradient starts the step
    LQCD_TRY(md_gradient(c, mp, phi_e, g, nullptr, nullptr));
    for (int step = 0; step < mp->nsteps; step++) {
        k_axpy_real<<<gr, 256, 0, c->stream>>>(np, -0.5 * mp->dt, g, p);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        k_move_links<<<div_up(nl, 128), 128, 0, c->stream>>>(nl, p, mp->dt, (double2 *)U, tabs());
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        LQCD_TRY(lqcd_set_gauge(c, U));
        LQCD_TRY(clover_build(c, kappa, csw, nullptr, nullptr));
        LQCD_TRY(md_gradient(c, mp, phi_e, g, nullptr, nullptr));
        k_axpy_real<<<gr, 256, 0, c->stream>>>(np, -0.5 * mp->dt, g, p);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
    }
    LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

}  // extern "C"
