// Clover term of Eq. 1 and its inverse (needed by the Schur complement of
// Eq. 2; its log det enters S_eff in Eq. 4).  Setup work, FP64 throughout.
//
// Fhat_{mu nu}(x) = (Q - Q^dag)/8 with Q the four plaquette leaves at x.  In
// the chiral basis sigma_{mu nu} is block diagonal; with X = F01 - F23,
// Y = F02 + F13, Z = F03 - F12 (upper, spins 0,1) and X = -F01 - F23,
// Y = -F02 + F13, Z = -F03 - F12 (lower, spins 2,3) each 6x6 block is
//     (4 + m0) 1 + (i c_sw / 2) [[Z, X - iY], [X + iY, -Z]].
// One thread per site builds both blocks, inverts each by LU with partial
// pivoting and writes A, A^-1 (FP64 and FP32 native copies) and log|det|.
#include "lqcd_internal.cuh"

namespace {

using C = cx<double>;

struct M3 {
    C m[3][3];
};

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

__device__ M3 link_at(const Geom &g, const double2 *__restrict__ U, const int x[4], int mu)
{
    int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    int r = coords_rank(g, x);
    const double2 *b = U + (long)((p * 4 + mu) * 9) * g.Vh + r;
    M3 u;
#pragma unroll
    for (int e = 0; e < 9; e++) {
        double2 v = b[e * (long)g.Vh];
        u.m[e / 3][e % 3] = mk(v.x, v.y);
    }
    return u;
}

__device__ __forceinline__ void step(const Geom &g, int y[4], int mu, int d)
{
    int v = y[mu] + d;
    y[mu] = v < 0 ? v + g.L[mu] : (v >= g.L[mu] ? v - g.L[mu] : v);
}

// Fhat_{mu nu}(x), mu != nu
__device__ M3 fhat(const Geom &g, const double2 *__restrict__ U, const int x[4], int mu, int nu)
{
    int xpm[4], xpn[4], xmm[4], xmn[4], xmmpn[4], xmmmn[4], xmnpm[4];
    for (int i = 0; i < 4; i++) xpm[i] = xpn[i] = xmm[i] = xmn[i] = x[i];
    step(g, xpm, mu, 1);
    step(g, xpn, nu, 1);
    step(g, xmm, mu, -1);
    step(g, xmn, nu, -1);
    for (int i = 0; i < 4; i++) xmmpn[i] = xmmmn[i] = xmm[i], xmnpm[i] = xmn[i];
    step(g, xmmpn, nu, 1);
    step(g, xmmmn, nu, -1);
    step(g, xmnpm, mu, 1);
    M3 Umx = link_at(g, U, x, mu), Unx = link_at(g, U, x, nu);
    // leaf through x+mu, x+mu+nu, x+nu
    M3 q = mul(mul(Umx, link_at(g, U, xpm, nu)), mul(dag(link_at(g, U, xpn, mu)), dag(Unx)));
    // leaf through x+nu, x-mu+nu, x-mu
    M3 Umxmm = link_at(g, U, xmm, mu);
    M3 l2 = mul(mul(Unx, dag(link_at(g, U, xmmpn, mu))), mul(dag(link_at(g, U, xmm, nu)), Umxmm));
    // leaf through x-mu, x-mu-nu, x-nu
    M3 Unxmn = link_at(g, U, xmn, nu);
    M3 l3 = mul(mul(dag(Umxmm), dag(link_at(g, U, xmmmn, nu))), mul(link_at(g, U, xmmmn, mu), Unxmn));
    // leaf through x-nu, x-nu+mu, x+mu
    M3 l4 = mul(mul(dag(Unxmn), link_at(g, U, xmn, mu)), mul(link_at(g, U, xmnpm, nu), dag(Umx)));
    M3 F;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            C s = q.m[i][j] + l2.m[i][j] + l3.m[i][j] + l4.m[i][j];
            C sd = conjx(q.m[j][i] + l2.m[j][i] + l3.m[j][i] + l4.m[j][i]);
            F.m[i][j] = 0.125 * (s - sd);
        }
    return F;
}

// invert a 6x6 complex matrix in place by LU with partial pivoting
__device__ int lu_inv6(C a[6][6], C inv[6][6], double *logabsdet)
{
    double amax = 0;
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) amax = fmax(amax, hypot(a[i][j].re, a[i][j].im));
    int piv[6];
    double ld = 0;
    for (int k = 0; k < 6; k++) {
        int p = k;
        double best = hypot(a[k][k].re, a[k][k].im);
        for (int i = k + 1; i < 6; i++) {
            double v = hypot(a[i][k].re, a[i][k].im);
            if (v > best) {
                best = v;
                p = i;
            }
        }
        if (!(best >= 1e-12 * amax) || amax == 0) return 1;
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < 6; j++) {
                C t = a[k][j];
                a[k][j] = a[p][j];
                a[p][j] = t;
            }
        ld += log(best);
        C d = a[k][k];
        double dn = d.re * d.re + d.im * d.im;
        C dinv = mk(d.re / dn, -d.im / dn);
        for (int i = k + 1; i < 6; i++) {
            C l = a[i][k] * dinv;
            a[i][k] = l;
            for (int j = k + 1; j < 6; j++) a[i][j] = a[i][j] - l * a[k][j];
        }
    }
    // inverse: solve LU X = P for the identity, column by column
    for (int col = 0; col < 6; col++) {
        C b[6];
        for (int i = 0; i < 6; i++) b[i] = mk(i == col ? 1.0 : 0.0, 0.0);
        for (int k = 0; k < 6; k++)
            if (piv[k] != k) {
                C t = b[k];
                b[k] = b[piv[k]];
                b[piv[k]] = t;
            }
        for (int i = 0; i < 6; i++)
            for (int k = 0; k < i; k++) b[i] = b[i] - a[i][k] * b[k];
        for (int i = 5; i >= 0; i--) {
            for (int k = i + 1; k < 6; k++) b[i] = b[i] - a[i][k] * b[k];
            C d = a[i][i];
            double dn = d.re * d.re + d.im * d.im;
            b[i] = mk((b[i].re * d.re + b[i].im * d.im) / dn, (b[i].im * d.re - b[i].re * d.im) / dn);
        }
        for (int i = 0; i < 6; i++) inv[i][col] = b[i];
    }
    *logabsdet = ld;
    return 0;
}

// write a Hermitian 6x6 (upper triangle taken) to the packed native slots
__device__ void store_herm(const C m[6][6], int blk, int r, long Vh, double2 *A64, float4 *A32, uint2 *A16)
{
    double v[36];
    for (int i = 0; i < 6; i++) v[i] = m[i][i].re;
    int k = 0;
    for (int i = 0; i < 6; i++)
        for (int j = i + 1; j < 6; j++) {
            v[6 + 2 * k] = m[i][j].re;
            v[7 + 2 * k] = m[i][j].im;
            k++;
        }
    for (int q = 0; q < 18; q++) A64[(18 * blk + q) * Vh + r] = make_double2(v[2 * q], v[2 * q + 1]);
    for (int q = 0; q < 9; q++)
        A32[(9 * blk + q) * Vh + r] = make_float4((float)v[4 * q], (float)v[4 * q + 1], (float)v[4 * q + 2],
                                                  (float)v[4 * q + 3]);
    for (int q = 0; q < 9; q++) {
        __half2 a = __floats2half2_rn((float)v[4 * q], (float)v[4 * q + 1]);
        __half2 b = __floats2half2_rn((float)v[4 * q + 2], (float)v[4 * q + 3]);
        A16[(9 * blk + q) * Vh + r] = make_uint2(*reinterpret_cast<unsigned *>(&a), *reinterpret_cast<unsigned *>(&b));
    }
}

struct CloverArgs {
    Geom g;
    const double2 *U;
    double m0, csw;
    double2 *A64[2], *Ai64[2];
    float4 *A32[2], *Ai32[2];
    uint2 *A16[2], *Ai16[2];
    double *logdet;   // [2][Vh]
    int *singular;    // count of singular blocks
    double even_scale;   // A on even sites multiplied by this (1 for D itself)
};

__global__ void __launch_bounds__(128) k_clover(CloverArgs a)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    int p = blockIdx.y;
    if (r >= a.g.Vh) return;
    int x[4];
    rank_coords(a.g, p, r, x);
    M3 F01 = fhat(a.g, a.U, x, 0, 1), F02 = fhat(a.g, a.U, x, 0, 2), F03 = fhat(a.g, a.U, x, 0, 3);
    M3 F12 = fhat(a.g, a.U, x, 1, 2), F13 = fhat(a.g, a.U, x, 1, 3), F23 = fhat(a.g, a.U, x, 2, 3);
    double ldsum = 0;
    for (int blk = 0; blk < 2; blk++) {
        double s = blk == 0 ? 1.0 : -1.0;
        C A[6][6], Ai[6][6];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                C X = s * F01.m[i][j] - F23.m[i][j];
                C Y = s * F02.m[i][j] + F13.m[i][j];
                C Z = s * F03.m[i][j] - F12.m[i][j];
                // (i c_sw / 2) [[Z, X - iY], [X + iY, -Z]]
                C z = timesI(Z), xm = timesI(X - timesI(Y)), xp = timesI(X + timesI(Y));
                double f = 0.5 * a.csw;
                A[i][j] = f * z;
                A[i][3 + j] = f * xm;
                A[3 + i][j] = f * xp;
                A[3 + i][3 + j] = -(f * z);
            }
        for (int i = 0; i < 6; i++) A[i][i].re += 4.0 + a.m0;
        if (p == 0 && a.even_scale != 1.0)
            for (int i = 0; i < 6; i++)
                for (int j = 0; j < 6; j++) A[i][j] = a.even_scale * A[i][j];
        store_herm(A, blk, r, a.g.Vh, a.A64[p], a.A32[p], a.A16[p]);
        double ld = 0;
        if (lu_inv6(A, Ai, &ld)) {
            atomicAdd(a.singular, 1);
            for (int i = 0; i < 6; i++)
                for (int j = 0; j < 6; j++) Ai[i][j] = mk(0.0, 0.0);
        }
        ldsum += ld;
        store_herm(Ai, blk, r, a.g.Vh, a.Ai64[p], a.Ai32[p], a.Ai16[p]);
    }
    a.logdet[p * (long)a.g.Vh + r] = ldsum;
}

// fixed-order sum of n doubles (one CTA, deterministic)
__global__ void k_sum_fixed(const double *x, long n, double *out)
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

// native F64 clover (or inverse) application on one parity
__global__ void k_clover_apply64(Geom g, const double2 *A, const double2 *in, double2 *out)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.Vh) return;
    long Vh = g.Vh;
    C v[12], w[12];
    for (int c = 0; c < 12; c++) {
        double2 t = in[c * Vh + r];
        v[c] = mk(t.x, t.y);
    }
    for (int blk = 0; blk < 2; blk++) {
        double d[6];
        C o[15];
        for (int i = 0; i < 3; i++) {
            double2 t = A[(18 * blk + i) * Vh + r];
            d[2 * i] = t.x;
            d[2 * i + 1] = t.y;
        }
        for (int i = 0; i < 15; i++) {
            double2 t = A[(18 * blk + 3 + i) * Vh + r];
            o[i] = mk(t.x, t.y);
        }
        C *vi = v + 6 * blk, *wi = w + 6 * blk;
        for (int i = 0; i < 6; i++) wi[i] = d[i] * vi[i];
        int k = 0;
        for (int i = 0; i < 6; i++)
            for (int j = i + 1; j < 6; j++) {
                wi[i] = wi[i] + o[k] * vi[j];
                wi[j] = wi[j] + cmulc(o[k], vi[i]);
                k++;
            }
    }
    for (int c = 0; c < 12; c++) out[c * Vh + r] = make_double2(w[c].re, w[c].im);
}

}  // namespace

lqcd_status clover_build(lqcd_ctx *c, double kappa, double csw, double *ld_e, double *ld_o, double even_scale)
{
    if (!c->have_gauge) return set_err(c, LQCD_ERR_STATE, "gauge field not set");
    if (!(kappa > 0)) return set_err(c, LQCD_ERR_ARG, "kappa must be > 0");
    const long Vh = c->g.Vh;
    for (int p = 0; p < 2; p++) {
        if (!c->A64[p]) {
            LQCD_CUDA_CHECK(c, cudaMalloc(&c->A64[p], 36 * Vh * sizeof(double2)));
            LQCD_CUDA_CHECK(c, cudaMalloc(&c->Ai64[p], 36 * Vh * sizeof(double2)));
            LQCD_CUDA_CHECK(c, cudaMalloc(&c->A32[p], 18 * Vh * sizeof(float4)));
            LQCD_CUDA_CHECK(c, cudaMalloc(&c->Ai32[p], 18 * Vh * sizeof(float4)));
            LQCD_CUDA_CHECK(c, cudaMalloc(&c->A16[p], 18 * Vh * sizeof(uint2)));
            LQCD_CUDA_CHECK(c, cudaMalloc(&c->Ai16[p], 18 * Vh * sizeof(uint2)));
        }
    }
    void *scratch;
    LQCD_TRY(ws_get(c, WS_MISC, (2 * Vh + 4) * sizeof(double), &scratch));
    double *logdet = (double *)scratch;
    int *sing = (int *)(logdet + 2 * Vh);
    double *sums = logdet + 2 * Vh + 2;
    LQCD_CUDA_CHECK(c, cudaMemsetAsync(sing, 0, sizeof(int), c->stream));
    CloverArgs a;
    a.g = c->g;
    a.U = c->U64;
    a.m0 = 1.0 / (2.0 * kappa) - 4.0;
    a.csw = csw;
    for (int p = 0; p < 2; p++) {
        a.A64[p] = c->A64[p];
        a.Ai64[p] = c->Ai64[p];
        a.A32[p] = c->A32[p];
        a.Ai32[p] = c->Ai32[p];
        a.A16[p] = c->A16[p];
        a.Ai16[p] = c->Ai16[p];
    }
    a.logdet = logdet;
    a.singular = sing;
    a.even_scale = even_scale;
    k_clover<<<dim3(div_up(Vh, 128), 2), 128, 0, c->stream>>>(a);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    k_sum_fixed<<<1, 256, 0, c->stream>>>(logdet, Vh, sums);
    k_sum_fixed<<<1, 256, 0, c->stream>>>(logdet + Vh, Vh, sums + 1);
    c->n_kernel_launches += 2;
    LQCD_LAUNCH_CHECK(c);
    double h_sums[2];
    int h_sing = 0;
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(h_sums, sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(&h_sing, sing, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    if (ld_e) *ld_e = h_sums[0];
    if (ld_o) *ld_o = h_sums[1];
    c->kappa = kappa;
    c->csw = csw;
    c->logdet_e = h_sums[0];
    c->logdet_o = h_sums[1];
    if (h_sing) {
        c->have_clover = false;
        return set_err(c, LQCD_ERR_SINGULAR_CLOVER, "%d singular 6x6 clover blocks", h_sing);
    }
    c->have_clover = true;
    return LQCD_OK;
}

lqcd_status clover_apply_native64(lqcd_ctx *c, int parity, int inverse, const double2 *in, double2 *out)
{
    const double2 *A = inverse ? c->Ai64[parity] : c->A64[parity];
    k_clover_apply64<<<div_up(c->g.Vh, 128), 128, 0, c->stream>>>(c->g, A, in, out);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}
