// Local deflation: the "locally deflated" Schwarz-preconditioned GCR of
// Sec. 3-4 (Table 1, deflation blocks 6^2 x 4^2 in the paper; 4^4 here).
//
//   subspace  v_l <- M_sap v_l, v_l <- v_l / |v_l| (ninv passes), then
//             Gram-Schmidt of {v_l restricted to Lambda} on every block Lambda
//   little D  A_{(L k),(L' l)} = <phi^L_k, D phi^L'_l>, stored per block row as
//             9 Ns x Ns matrices: entry 0 collects every hop that stays inside
//             the block (and the clover term), entry 1+2mu / 2+2mu the hops
//             through the +mu / -mu face into the neighbour block
//   M_dfl     rho -> M_sap(rho - D Pi A^-1 Pi^dag rho) + Pi A^-1 Pi^dag rho,
//             A^-1 by FP64 GCR to a relative residual coarse_tol
//
// One CTA per block, one thread per block site; block reductions by warp
// shuffles and a fixed-order pass over the warps (deterministic).
#include <algorithm>
#include <cmath>
#include <vector>

#include "lqcd_internal.cuh"
#include "lqcd_stencil.cuh"

namespace {

constexpr int NS_MAX = 32;
constexpr int RCHUNK = 8;

struct DBlk {
    int bs[4], nb[4];
    int vol, nblk;
    int wrap[4];
};

using C = cx<double>;

// native site load / store for F64 (double2 x 12) and F32 (float4 x 6)
__device__ __forceinline__ void ld(const double2 *f, long Vh, long r, C v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) {
        double2 t = f[c * Vh + r];
        v[c] = mk(t.x, t.y);
    }
}
__device__ __forceinline__ void st(double2 *f, long Vh, long r, const C v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) f[c * Vh + r] = make_double2(v[c].re, v[c].im);
}
// block-local site t -> global coordinates, parity, rank
struct BSite {
    int l[4], x[4], p;
    long r;
};
__device__ __forceinline__ void bsite(const Geom &g, const DBlk &B, int b, int t, BSite &s)
{
    int bc[4];
    int u = b;
    bc[3] = u % B.nb[3];
    u /= B.nb[3];
    bc[2] = u % B.nb[2];
    u /= B.nb[2];
    bc[1] = u % B.nb[1];
    bc[0] = u / B.nb[1];
    int v = t;
    s.l[3] = v % B.bs[3];
    v /= B.bs[3];
    s.l[2] = v % B.bs[2];
    v /= B.bs[2];
    s.l[1] = v % B.bs[1];
    s.l[0] = v / B.bs[1];
    for (int i = 0; i < 4; i++) s.x[i] = bc[i] * B.bs[i] + s.l[i];
    s.p = (s.x[0] + s.x[1] + s.x[2] + s.x[3]) & 1;
    s.r = coords_rank(g, s.x);
}

// sum of n values over the CTA; result valid in thread 0..n-1 as out[i] via smem
__device__ void block_sum(double *vals, int n, double *sh, double *res)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < n; i++) {
        double v = vals[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[i * 32 + warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < n) {
        double s = 0;
        for (int w = 0; w < nw; w++) s += sh[threadIdx.x * 32 + w];
        res[threadIdx.x] = s;
    }
    __syncthreads();
}

// as block_sum for float values: the warp sums in float, the sum over warps in
// double (FP64 shuffles and adds are the bound on GB300's FP64 pipe otherwise)
template <int NV>
__device__ void block_sum_f(const float (&vals)[NV], int n, double *sh, double *res)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; i++) {
        if (i >= n) break;
        float v = vals[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[i * 32 + warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < n) {
        double s = 0;
        for (int w = 0; w < nw; w++) s += sh[threadIdx.x * 32 + w];
        res[threadIdx.x] = s;
    }
    __syncthreads();
}

// one projected hop (1 -+ g_mu) acting on psi at the neighbour, times sign
__device__ void hop1(int mu, int sgn, const C psi[12], const C u[3][3], bool dag, double sign, C acc[12])
{
    C h[2][3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        C u0 = psi[c], u1 = psi[3 + c], l0 = psi[6 + c], l1 = psi[9 + c], e0, e1;
        switch (mu) {
            case 0: e0 = -l0; e1 = -l1; break;
            case 1: e0 = timesmI(l1); e1 = timesmI(l0); break;
            case 2: e0 = -l1; e1 = l0; break;
            default: e0 = timesmI(l0); e1 = timesI(l1); break;
        }
        h[0][c] = sgn < 0 ? u0 - e0 : u0 + e0;
        h[1][c] = sgn < 0 ? u1 - e1 : u1 + e1;
    }
    C w[2][3];
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            C t = dag ? (cmulc(u[0][a], h[s][0]) + cmulc(u[1][a], h[s][1]) + cmulc(u[2][a], h[s][2]))
                      : (u[a][0] * h[s][0] + u[a][1] * h[s][1] + u[a][2] * h[s][2]);
            w[s][a] = sign * t;
        }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        acc[a] = acc[a] + w[0][a];
        acc[3 + a] = acc[3 + a] + w[1][a];
        C e0, e1;   // e_mu^dag w
        switch (mu) {
            case 0: e0 = -w[0][a]; e1 = -w[1][a]; break;
            case 1: e0 = timesI(w[1][a]); e1 = timesI(w[0][a]); break;
            case 2: e0 = w[1][a]; e1 = -w[0][a]; break;
            default: e0 = timesI(w[0][a]); e1 = timesmI(w[1][a]); break;
        }
        if (sgn < 0) {
            acc[6 + a] = acc[6 + a] - e0;
            acc[9 + a] = acc[9 + a] - e1;
        } else {
            acc[6 + a] = acc[6 + a] + e0;
            acc[9 + a] = acc[9 + a] + e1;
        }
    }
}

__device__ void link64(const Geom &g, const double2 *U, int p, int mu, long r, C u[3][3])
{
    const double2 *b = U + (long)((p * 4 + mu) * 9) * g.Vh + r;
#pragma unroll
    for (int e = 0; e < 9; e++) {
        double2 t = b[e * (long)g.Vh];
        u[e / 3][e % 3] = mk(t.x, t.y);
    }
}

__device__ void clover64(const double2 *A, long Vh, long r, const C in[12], C out[12])
{
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
        const C *v = in + 6 * blk;
        C *w = out + 6 * blk;
        for (int i = 0; i < 6; i++) w[i] = d[i] * v[i];
        int k = 0;
        for (int i = 0; i < 6; i++)
            for (int j = i + 1; j < 6; j++) {
                w[i] = w[i] + o[k] * v[j];
                w[j] = w[j] + cmulc(o[k], v[i]);
                k++;
            }
    }
}

// ---------------------------------------------------------------- kernels
// block Gram-Schmidt (modified GS, two passes) of Ns native fields in place
template <class T>
__global__ void k_block_gs(Geom g, DBlk B, T *v, int Ns, long fstride, int *bad)
{
    extern __shared__ double sh[];
    double *res = sh + 2 * 32 * 2;
    int b = blockIdx.x, t = threadIdx.x;
    BSite s;
    bsite(g, B, b, t, s);
    const long hs = fstride / 2;   // half-field stride (elements)
    for (int l = 0; l < Ns; l++) {
        T *vl = v + l * fstride + s.p * hs;
        C w[12];
        ld(vl, g.Vh, s.r, w);
        for (int pass = 0; pass < 2; pass++)
            for (int k = 0; k < l; k++) {
                C q[12];
                ld(v + k * fstride + s.p * hs, g.Vh, s.r, q);
                double d[2] = {0, 0};
                for (int c = 0; c < 12; c++) {
                    d[0] += q[c].re * w[c].re + q[c].im * w[c].im;
                    d[1] += q[c].re * w[c].im - q[c].im * w[c].re;
                }
                block_sum(d, 2, sh, res);
                C a = mk(res[0], res[1]);
                for (int c = 0; c < 12; c++) w[c] = w[c] - a * q[c];
            }
        double n2[1] = {0};
        for (int c = 0; c < 12; c++) n2[0] += w[c].re * w[c].re + w[c].im * w[c].im;
        block_sum(n2, 1, sh, res);
        double nn = res[0];
        if (nn <= 0) {
            if (t == 0) atomicAdd(bad, 1);
            nn = 1;
        }
        double inv = 1.0 / sqrt(nn);
        for (int c = 0; c < 12; c++) w[c] = inv * w[c];
        st(vl, g.Vh, s.r, w);
        __syncthreads();
    }
}

// Block Gram-Schmidt of an FP32 subspace: classical Gram-Schmidt applied
// twice per vector (twice is enough for vectors this far from dependent), the
// products and warp sums in float and the sums over warps in double.  Three
// block reductions per vector instead of one per pair, and no FP64
// arithmetic per site (GB300's FP64 pipe bounds the FP64 form).  Like the
// modified form it gives the block-wise QR with a positive diagonal, so the
// two agree up to rounding.
__global__ void k_block_gs32(Geom g, DBlk B, float4 *v, int Ns, long fstride, int *bad)
{
    extern __shared__ double sh[];                // [2 RCHUNK][32] warp sums
    double *coef = sh + 2 * RCHUNK * 32;          // [2 NS_MAX] inner products of one pass
    double *res = coef + 2 * NS_MAX;
    const int b = blockIdx.x, t = threadIdx.x;
    BSite s;
    bsite(g, B, b, t, s);
    const long hs = fstride / 2, Vh = g.Vh;
    for (int l = 0; l < Ns; l++) {
        float4 *vl = v + l * fstride + s.p * hs + s.r;
        float w[24];
#pragma unroll
        for (int q = 0; q < 6; q++) {
            const float4 a = vl[q * Vh];
            w[4 * q] = a.x;
            w[4 * q + 1] = a.y;
            w[4 * q + 2] = a.z;
            w[4 * q + 3] = a.w;
        }
        for (int pass = 0; pass < 2 && l > 0; pass++) {
            // the l inner products, RCHUNK per block reduction, into coef
            for (int k0 = 0; k0 < l; k0 += RCHUNK) {
                const int kn = min(RCHUNK, l - k0);
                float d[2 * RCHUNK];
#pragma unroll
                for (int i = 0; i < RCHUNK; i++) {
                    d[2 * i] = d[2 * i + 1] = 0.f;
                    if (i < kn) {
                        const float4 *vk = v + (k0 + i) * fstride + s.p * hs + s.r;
                        float re = 0.f, im = 0.f;
#pragma unroll
                        for (int q = 0; q < 6; q++) {
                            const float4 a = vk[q * Vh];
                            re = fmx(a.x, w[4 * q], fmx(a.y, w[4 * q + 1], fmx(a.z, w[4 * q + 2], fmx(a.w, w[4 * q + 3], re))));
                            im = fmx(a.x, w[4 * q + 1], fmx(-a.y, w[4 * q], fmx(a.z, w[4 * q + 3], fmx(-a.w, w[4 * q + 2], im))));
                        }
                        d[2 * i] = re;
                        d[2 * i + 1] = im;
                    }
                }
                block_sum_f<2 * RCHUNK>(d, 2 * kn, sh, coef + 2 * k0);
            }
            for (int k = 0; k < l; k++) {
                const float ar = (float)coef[2 * k], ai = (float)coef[2 * k + 1];
                const float4 *vk = v + k * fstride + s.p * hs + s.r;
#pragma unroll
                for (int q = 0; q < 6; q++) {
                    const float4 a = vk[q * Vh];
                    w[4 * q] = fmx(-ar, a.x, fmx(ai, a.y, w[4 * q]));
                    w[4 * q + 1] = fmx(-ar, a.y, fmx(-ai, a.x, w[4 * q + 1]));
                    w[4 * q + 2] = fmx(-ar, a.z, fmx(ai, a.w, w[4 * q + 2]));
                    w[4 * q + 3] = fmx(-ar, a.w, fmx(-ai, a.z, w[4 * q + 3]));
                }
            }
        }
        float n2[1] = {0.f};
#pragma unroll
        for (int i = 0; i < 24; i++) n2[0] = fmx(w[i], w[i], n2[0]);
        block_sum_f<1>(n2, 1, sh, res);
        double nn = res[0];
        if (!(nn > 0)) {
            if (t == 0) atomicAdd(bad, 1);
            nn = 1;
        }
        const float inv = (float)(1.0 / sqrt(nn));
#pragma unroll
        for (int q = 0; q < 6; q++)
            vl[q * Vh] = make_float4(inv * w[4 * q], inv * w[4 * q + 1], inv * w[4 * q + 2], inv * w[4 * q + 3]);
    }
}

// little Dirac build for vector l = blockIdx.y: Aint[b][j][k][l] = <phi_k|_b, W_j>
template <class T>
__global__ void k_little_build(Geom g, DBlk B, const T *phi, int Ns, long fstride, const double2 *U,
                               const double2 *A0, const double2 *A1, double2 *Aint)
{
    extern __shared__ double sh[];
    double *res = sh + 2 * RCHUNK * 32;
    int b = blockIdx.x, l = blockIdx.y, t = threadIdx.x;
    BSite s;
    bsite(g, B, b, t, s);
    const long hs = fstride / 2;
    const T *pl = phi + l * fstride;
    for (int j = 0; j < 9; j++) {
        C w[12];
        for (int c = 0; c < 12; c++) w[c] = mk(0.0, 0.0);
        if (j == 0) {
            C v[12];
            ld(pl + s.p * hs, g.Vh, s.r, v);
            clover64(s.p ? A1 : A0, g.Vh, s.r, v, w);
        }
        for (int mu = 0; mu < 4; mu++)
            for (int d = -1; d <= 1; d += 2) {
                int jj = d > 0 ? 1 + 2 * mu : 2 + 2 * mu;
                int lm = s.l[mu] + d;
                bool inside = (lm >= 0 && lm < B.bs[mu]) || B.wrap[mu];
                if ((j == 0) != inside) continue;
                if (j != 0 && j != jj) continue;
                int y[4] = {s.x[0], s.x[1], s.x[2], s.x[3]};
                y[mu] = (y[mu] + d + g.L[mu]) % g.L[mu];
                long ry = coords_rank(g, y);
                C v[12], u[3][3];
                ld(pl + (1 - s.p) * hs, g.Vh, ry, v);
                double sign;
                if (d > 0) {
                    sign = (mu == 0 && s.x[0] == g.L[0] - 1) ? g.bc_t : 1.0;
                    link64(g, U, s.p, mu, s.r, u);
                    C acc[12];
                    for (int c = 0; c < 12; c++) acc[c] = mk(0.0, 0.0);
                    hop1(mu, -1, v, u, false, sign, acc);
                    for (int c = 0; c < 12; c++) w[c] = w[c] - 0.5 * acc[c];
                } else {
                    sign = (mu == 0 && s.x[0] == 0) ? g.bc_t : 1.0;
                    link64(g, U, 1 - s.p, mu, ry, u);
                    C acc[12];
                    for (int c = 0; c < 12; c++) acc[c] = mk(0.0, 0.0);
                    hop1(mu, +1, v, u, true, sign, acc);
                    for (int c = 0; c < 12; c++) w[c] = w[c] - 0.5 * acc[c];
                }
            }
        for (int k0 = 0; k0 < Ns; k0 += RCHUNK) {
            double d[2 * RCHUNK];
            int kn = min(RCHUNK, Ns - k0);
            for (int i = 0; i < RCHUNK; i++) {
                d[2 * i] = d[2 * i + 1] = 0;
                if (i < kn) {
                    C q[12];
                    ld(phi + (k0 + i) * fstride + s.p * hs, g.Vh, s.r, q);
                    for (int c = 0; c < 12; c++) {
                        d[2 * i] += q[c].re * w[c].re + q[c].im * w[c].im;
                        d[2 * i + 1] += q[c].re * w[c].im - q[c].im * w[c].re;
                    }
                }
            }
            block_sum(d, 2 * kn, sh, res);
            if (t < kn) Aint[(((long)b * 9 + j) * Ns + k0 + t) * Ns + l] = make_double2(res[2 * t], res[2 * t + 1]);
            __syncthreads();
        }
    }
}

// FP32 hop: acc += sign (1 -+ g_mu) U psi (dag: U^dag), runtime direction
__device__ __forceinline__ void hop1f(int mu, int sgn, const stencil::Spinor<float> &psi, const cx<float> u[3][3],
                                      bool dag, float sign, stencil::Spinor<float> &acc)
{
    cx<float> h[2][3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const cx<float> u0 = psi.s[0][c], u1 = psi.s[1][c], l0 = psi.s[2][c], l1 = psi.s[3][c];
        cx<float> e0, e1;
        switch (mu) {
            case 0: e0 = -l0; e1 = -l1; break;
            case 1: e0 = timesmI(l1); e1 = timesmI(l0); break;
            case 2: e0 = -l1; e1 = l0; break;
            default: e0 = timesmI(l0); e1 = timesI(l1); break;
        }
        h[0][c] = sgn < 0 ? u0 - e0 : u0 + e0;
        h[1][c] = sgn < 0 ? u1 - e1 : u1 + e1;
    }
    cx<float> w[2][3];
#pragma unroll
    for (int sp = 0; sp < 2; sp++) {
        if (dag)
            stencil::su3dag_vec(u, h[sp], w[sp]);
        else
            stencil::su3_vec(u, h[sp], w[sp]);
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        cx<float> e0, e1;   // e_mu^dag w
        switch (mu) {
            case 0: e0 = -w[0][a]; e1 = -w[1][a]; break;
            case 1: e0 = timesI(w[1][a]); e1 = timesI(w[0][a]); break;
            case 2: e0 = w[1][a]; e1 = -w[0][a]; break;
            default: e0 = timesI(w[0][a]); e1 = timesmI(w[1][a]); break;
        }
        if (sgn < 0) {
            e0 = -e0;
            e1 = -e1;
        }
        acc.s[0][a].re = fmx(sign, w[0][a].re, acc.s[0][a].re);
        acc.s[0][a].im = fmx(sign, w[0][a].im, acc.s[0][a].im);
        acc.s[1][a].re = fmx(sign, w[1][a].re, acc.s[1][a].re);
        acc.s[1][a].im = fmx(sign, w[1][a].im, acc.s[1][a].im);
        acc.s[2][a].re = fmx(sign, e0.re, acc.s[2][a].re);
        acc.s[2][a].im = fmx(sign, e0.im, acc.s[2][a].im);
        acc.s[3][a].re = fmx(sign, e1.re, acc.s[3][a].re);
        acc.s[3][a].im = fmx(sign, e1.im, acc.s[3][a].im);
    }
}

// The little Dirac build of an FP32 subspace in FP32 arithmetic: the FP32
// operator (2-row links, FP32 clover), FP32 products and per-thread sums,
// warp sums in float and the sum over warps in double.  The subspace itself is
// FP32, so its entries carry FP32 accuracy either way; GB300's FP64 pipe made
// the FP64 form of this kernel the largest single cost of the subspace build.
__global__ void k_little_build32(Geom g, DBlk B, const float4 *phi, int Ns, long fstride, const float4 *U32,
                                 const float4 *A0, const float4 *A1, double2 *Aint)
{
    extern __shared__ double sh[];
    double *res = sh + 2 * RCHUNK * 32;
    const int b = blockIdx.x, l = blockIdx.y, t = threadIdx.x;
    BSite s;
    bsite(g, B, b, t, s);
    const long hs = fstride / 2;
    const float4 *pl = phi + l * fstride;
    for (int j = 0; j < 9; j++) {
        stencil::Spinor<float> w;
#pragma unroll
        for (int sp = 0; sp < 4; sp++)
#pragma unroll
            for (int c = 0; c < 3; c++) w.s[sp][c] = mk(0.f, 0.f);
        if (j == 0) {
            stencil::Spinor<float> v;
            stencil::load_spinor(pl + s.p * hs, g.Vh, (int)s.r, v);
            stencil::clover_apply<float, float4>(s.p ? A1 : A0, g.Vh, (int)s.r, v, w);
        }
        stencil::Spinor<float> acc;
#pragma unroll
        for (int sp = 0; sp < 4; sp++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc.s[sp][c] = mk(0.f, 0.f);
        // W_j (j >= 1) vanishes on the sites that its hop does not reach: they
        // skip the subspace loads below (their products would all be zero)
        bool nz = j == 0;
        for (int mu = 0; mu < 4; mu++)
            for (int d = -1; d <= 1; d += 2) {
                const int jj = d > 0 ? 1 + 2 * mu : 2 + 2 * mu;
                const int lm = s.l[mu] + d;
                const bool inside = (lm >= 0 && lm < B.bs[mu]) || B.wrap[mu];
                if ((j == 0) != inside) continue;
                if (j != 0 && j != jj) continue;
                nz = true;
                int y[4] = {s.x[0], s.x[1], s.x[2], s.x[3]};
                y[mu] = (y[mu] + d + g.L[mu]) % g.L[mu];
                const int ry = coords_rank(g, y);
                stencil::Spinor<float> v;
                cx<float> u[3][3];
                stencil::load_spinor(pl + (1 - s.p) * hs, g.Vh, ry, v);
                if (d > 0) {
                    const float sign = (mu == 0 && s.x[0] == g.L[0] - 1) ? (float)g.bc_t : 1.f;
                    stencil::load_link(U32, g.Vh, s.p, mu, (int)s.r, u);
                    hop1f(mu, -1, v, u, false, sign, acc);
                } else {
                    const float sign = (mu == 0 && s.x[0] == 0) ? (float)g.bc_t : 1.f;
                    stencil::load_link(U32, g.Vh, 1 - s.p, mu, ry, u);
                    hop1f(mu, +1, v, u, true, sign, acc);
                }
            }
#pragma unroll
        for (int sp = 0; sp < 4; sp++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                w.s[sp][c].re = fmx(-0.5f, acc.s[sp][c].re, w.s[sp][c].re);
                w.s[sp][c].im = fmx(-0.5f, acc.s[sp][c].im, w.s[sp][c].im);
            }
        for (int k0 = 0; k0 < Ns; k0 += RCHUNK) {
            float dd[2 * RCHUNK];
            const int kn = min(RCHUNK, Ns - k0);
#pragma unroll
            for (int i = 0; i < RCHUNK; i++) {
                dd[2 * i] = dd[2 * i + 1] = 0.f;
                if (i < kn && nz) {
                    stencil::Spinor<float> q;
                    stencil::load_spinor(phi + (k0 + i) * fstride + s.p * hs, g.Vh, (int)s.r, q);
#pragma unroll
                    for (int sp = 0; sp < 4; sp++)
#pragma unroll
                        for (int c = 0; c < 3; c++) {
                            const cx<float> a = q.s[sp][c], z = w.s[sp][c];
                            dd[2 * i] = fmx(a.re, z.re, fmx(a.im, z.im, dd[2 * i]));
                            dd[2 * i + 1] = fmx(a.re, z.im, fmx(-a.im, z.re, dd[2 * i + 1]));
                        }
                }
            }
            block_sum_f<2 * RCHUNK>(dd, 2 * kn, sh, res);
            if (t < kn) Aint[(((long)b * 9 + j) * Ns + k0 + t) * Ns + l] = make_double2(res[2 * t], res[2 * t + 1]);
            __syncthreads();
        }
    }
}

// c_r[b*Ns + k] = <phi_k|_b, in_r>  (in_r: native F64 full fields, stride in_rs;
// c_r stride c_rs).  The nrhs CTAs of one block are consecutive, so the block's
// subspace vectors are read from DRAM once and from L2 by the other fields.
template <class T>
__global__ void k_project(Geom g, DBlk B, const T *phi, int Ns, long fstride, const double2 *in, double2 *c,
                          int nrhs, long in_rs, long c_rs)
{
    extern __shared__ double sh[];
    double *res = sh + 2 * RCHUNK * 32;
    const int b = blockIdx.x / nrhs, t = threadIdx.x;
    in += (blockIdx.x % nrhs) * in_rs;
    c += (blockIdx.x % nrhs) * c_rs;
    BSite s;
    bsite(g, B, b, t, s);
    C w[12];
    ld(in + s.p * 12 * (long)g.Vh, g.Vh, s.r, w);
    const long hs = fstride / 2;
    // FP32 subspace: the site's products in float (GB300's FP64 pipe is the bound
    // otherwise), the sums over sites in double
    float wf[24];
    if constexpr (sizeof(T) == 16 && !std::is_same<T, double2>::value)
        for (int cc = 0; cc < 12; cc++) {
            wf[2 * cc] = (float)w[cc].re;
            wf[2 * cc + 1] = (float)w[cc].im;
        }
    for (int k0 = 0; k0 < Ns; k0 += RCHUNK) {
        int kn = min(RCHUNK, Ns - k0);
        if constexpr (std::is_same<T, double2>::value) {
            double d[2 * RCHUNK];
            for (int i = 0; i < RCHUNK; i++) {
                d[2 * i] = d[2 * i + 1] = 0;
                if (i < kn) {
                    C q[12];
                    ld(phi + (k0 + i) * fstride + s.p * hs, g.Vh, s.r, q);
                    for (int cc = 0; cc < 12; cc++) {
                        d[2 * i] += q[cc].re * w[cc].re + q[cc].im * w[cc].im;
                        d[2 * i + 1] += q[cc].re * w[cc].im - q[cc].im * w[cc].re;
                    }
                }
            }
            block_sum(d, 2 * kn, sh, res);
        } else {
            float d[2 * RCHUNK];
#pragma unroll
            for (int i = 0; i < RCHUNK; i++) {
                d[2 * i] = d[2 * i + 1] = 0.f;
                if (i < kn) {
                    const float4 *f = (const float4 *)(phi + (k0 + i) * fstride + s.p * hs) + s.r;
                    float re = 0, im = 0;
#pragma unroll
                    for (int q = 0; q < 6; q++) {
                        float4 v = f[q * g.Vh];
                        re += v.x * wf[4 * q] + v.y * wf[4 * q + 1] + v.z * wf[4 * q + 2] + v.w * wf[4 * q + 3];
                        im += v.x * wf[4 * q + 1] - v.y * wf[4 * q] + v.z * wf[4 * q + 3] - v.w * wf[4 * q + 2];
                    }
                    d[2 * i] = re;
                    d[2 * i + 1] = im;
                }
            }
            block_sum_f<2 * RCHUNK>(d, 2 * kn, sh, res);
        }
        if (t < kn) c[(long)b * Ns + k0 + t] = make_double2(res[2 * t], res[2 * t + 1]);
    }
}

// FP32-subspace forms of the two kernels above with a group of PJ_R
// right-hand sides per CTA (the groups of one block in consecutive CTAs), so
// the block's subspace vectors are read once per group instead of once per
// right-hand side.  Two threads per site, one per chirality half (six colour-
// spin components): a thread holds its half of the PJ_R input fields.
constexpr int PJ_R = 4;   // right-hand sides per CTA
constexpr int PJ_K = 4;   // subspace vectors per reduction: PJ_K * PJ_R * 2 = 32 values
static_assert(PJ_K * PJ_R * 2 == 32, "one value per lane in the warp reduction");

// v[0..31] summed over the warp; on return v[0] of lane l holds the sum of
// value l (a halving exchange: 31 shuffles for 32 values)
__device__ __forceinline__ void warp_reduce_scatter32(float v[32])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int i = 0; i < o; i++) {
            const float send = up ? v[i] : v[i + o];
            const float keep = up ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
}

// c_r[b*Ns + k] = <phi_k|_b, in_r> for the PJ_R fields r0 .. r0 + PJ_R - 1;
// blockDim.x = 2 B.vol (a multiple of 32, at most 1024)
__global__ void __launch_bounds__(512, 1) k_project_h(Geom g, DBlk B, const float4 *__restrict__ phi, int Ns,
                                                      long fstride, const double2 *__restrict__ in, double2 *c,
                                                      int nrhs, long in_rs, long c_rs, int ngr)
{
    __shared__ float red[32][32];
    const int b = blockIdx.x / ngr, r0 = (blockIdx.x % ngr) * PJ_R, nr = min(PJ_R, nrhs - r0);
    const int vol = B.vol, hh = threadIdx.x >= vol ? 1 : 0, t = threadIdx.x - hh * vol;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long Vh = g.Vh;
    BSite s;
    bsite(g, B, b, t, s);
    float wf[PJ_R][12];
#pragma unroll
    for (int r = 0; r < PJ_R; r++) {
        const double2 *src = in + (long)(r0 + min(r, nr - 1)) * in_rs + ((long)s.p * 12 + 6 * hh) * Vh + s.r;
#pragma unroll
        for (int cc = 0; cc < 6; cc++) {
            const double2 v = src[cc * Vh];
            wf[r][2 * cc] = r < nr ? (float)v.x : 0.f;
            wf[r][2 * cc + 1] = r < nr ? (float)v.y : 0.f;
        }
    }
    const long hs = fstride / 2;
    for (int k0 = 0; k0 < Ns; k0 += PJ_K) {
        float v[32];
#pragma unroll
        for (int kk = 0; kk < PJ_K; kk++) {
            const int k = min(k0 + kk, Ns - 1);   // past the last vector: computed, never stored
            const float4 *f = phi + k * fstride + s.p * hs + 3 * hh * Vh + s.r;
            float4 q[3];
#pragma unroll
            for (int i = 0; i < 3; i++) q[i] = f[i * Vh];
#pragma unroll
            for (int r = 0; r < PJ_R; r++) {
                float re = 0.f, im = 0.f;
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    const float *w4 = &wf[r][4 * i];
                    re = fmx(q[i].x, w4[0], fmx(q[i].y, w4[1], fmx(q[i].z, w4[2], fmx(q[i].w, w4[3], re))));
                    im = fmx(q[i].x, w4[1], fmx(-q[i].y, w4[0], fmx(q[i].z, w4[3], fmx(-q[i].w, w4[2], im))));
                }
                v[(kk * PJ_R + r) * 2] = re;
                v[(kk * PJ_R + r) * 2 + 1] = im;
            }
        }
        warp_reduce_scatter32(v);
        red[warp][lane] = v[0];
        __syncthreads();
        if (threadIdx.x < 32) {
            double sum = 0;
            for (int w = 0; w < nw; w++) sum += red[w][threadIdx.x];
            const int kk = threadIdx.x / (2 * PJ_R), r = (threadIdx.x >> 1) % PJ_R, comp = threadIdx.x & 1;
            if (k0 + kk < Ns && r < nr)
                reinterpret_cast<double *>(c + (long)(r0 + r) * c_rs + (long)b * Ns + k0 + kk)[comp] = sum;
        }
        __syncthreads();
    }
}

// out_r(x) = sum_k c_r[b(x)*Ns + k] phi_k(x) for PJ_R fields; a CTA covers
// B.vol / nsplit sites of block b (two threads per site)
__global__ void __launch_bounds__(256) k_expand_h(Geom g, DBlk B, const float4 *__restrict__ phi, int Ns, long fstride,
                                                  const double2 *__restrict__ c, double2 *out, int nrhs, long c_rs,
                                                  long out_rs, int ngr, int nsplit)
{
    __shared__ float2 cf[PJ_R][NS_MAX];
    const int gr = blockIdx.x % ngr, bsp = blockIdx.x / ngr, b = bsp / nsplit, sp = bsp % nsplit;
    const int r0 = gr * PJ_R, nr = min(PJ_R, nrhs - r0);
    for (int i = threadIdx.x; i < PJ_R * Ns; i += blockDim.x) {
        const int r = i / Ns, k = i - r * Ns;
        const double2 v = r < nr ? c[(long)(r0 + r) * c_rs + (long)b * Ns + k] : make_double2(0.0, 0.0);
        cf[r][k] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    const int per = B.vol / nsplit, hh = threadIdx.x >= per ? 1 : 0, t = sp * per + threadIdx.x - hh * per;
    const long Vh = g.Vh, hs = fstride / 2;
    BSite s;
    bsite(g, B, b, t, s);
    float acc[PJ_R][12];
#pragma unroll
    for (int r = 0; r < PJ_R; r++)
#pragma unroll
        for (int i = 0; i < 12; i++) acc[r][i] = 0.f;
    for (int k = 0; k < Ns; k++) {
        const float4 *f = phi + k * fstride + s.p * hs + 3 * hh * Vh + s.r;
        float4 q[3];
#pragma unroll
        for (int i = 0; i < 3; i++) q[i] = f[i * Vh];
#pragma unroll
        for (int r = 0; r < PJ_R; r++) {
            const float ar = cf[r][k].x, ai = cf[r][k].y;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                acc[r][4 * i] = fmx(ar, q[i].x, fmx(-ai, q[i].y, acc[r][4 * i]));
                acc[r][4 * i + 1] = fmx(ar, q[i].y, fmx(ai, q[i].x, acc[r][4 * i + 1]));
                acc[r][4 * i + 2] = fmx(ar, q[i].z, fmx(-ai, q[i].w, acc[r][4 * i + 2]));
                acc[r][4 * i + 3] = fmx(ar, q[i].w, fmx(ai, q[i].z, acc[r][4 * i + 3]));
            }
        }
    }
#pragma unroll
    for (int r = 0; r < PJ_R; r++)
        if (r < nr) {
            double2 *dst = out + (long)(r0 + r) * out_rs + ((long)s.p * 12 + 6 * hh) * Vh + s.r;
#pragma unroll
            for (int cc = 0; cc < 6; cc++) dst[cc * Vh] = make_double2(acc[r][2 * cc], acc[r][2 * cc + 1]);
        }
}

// out_r(x) = sum_k c_r[b(x)*Ns + k] phi_k(x)  (out_r: native F64 full fields,
// stride out_rs; c_r stride c_rs; CTA order as in k_project)
template <class T>
__global__ void k_expand(Geom g, DBlk B, const T *phi, int Ns, long fstride, const double2 *c, double2 *out,
                         int nrhs, long c_rs, long out_rs)
{
    const int b = blockIdx.x / nrhs, t = threadIdx.x;
    c += (blockIdx.x % nrhs) * c_rs;
    out += (blockIdx.x % nrhs) * out_rs;
    BSite s;
    bsite(g, B, b, t, s);
    const long hs = fstride / 2;
    C w[12];
    if constexpr (std::is_same<T, double2>::value) {
        for (int cc = 0; cc < 12; cc++) w[cc] = mk(0.0, 0.0);
        for (int k = 0; k < Ns; k++) {
            double2 ck = c[(long)b * Ns + k];
            C a = mk(ck.x, ck.y), q[12];
            ld(phi + k * fstride + s.p * hs, g.Vh, s.r, q);
            for (int cc = 0; cc < 12; cc++) w[cc] = w[cc] + a * q[cc];
        }
    } else {
        // FP32 subspace: products and sums in float; the block's coefficients
        // converted to float once per CTA
        __shared__ float2 cf[NS_MAX];
        if (t < Ns) cf[t] = make_float2((float)c[(long)b * Ns + t].x, (float)c[(long)b * Ns + t].y);
        __syncthreads();
        float acc[24];
#pragma unroll
        for (int i = 0; i < 24; i++) acc[i] = 0.f;
        for (int k = 0; k < Ns; k++) {
            const float ar = cf[k].x, ai = cf[k].y;
            const float4 *f = (const float4 *)(phi + k * fstride + s.p * hs) + s.r;
#pragma unroll
            for (int q = 0; q < 6; q++) {
                float4 v = f[q * g.Vh];
                acc[4 * q] += ar * v.x - ai * v.y;
                acc[4 * q + 1] += ar * v.y + ai * v.x;
                acc[4 * q + 2] += ar * v.z - ai * v.w;
                acc[4 * q + 3] += ar * v.w + ai * v.z;
            }
        }
        for (int cc = 0; cc < 12; cc++) w[cc] = mk((double)acc[2 * cc], (double)acc[2 * cc + 1]);
    }
    st(out + s.p * 12 * (long)g.Vh, g.Vh, s.r, w);
}

// F32 / F64 native field scale and norm helpers
__global__ void k_scale32(long n, float s, float4 *x)
{
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        float4 v = x[j];
        x[j] = make_float4(s * v.x, s * v.y, s * v.z, s * v.w);
    }
}
__global__ void k_norm32_partial(long n, const float4 *x, double *partial)
{
    double s = 0;
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        float4 v = x[j];
        s += (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z + (double)v.w * v.w;
    }
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
        partial[blockIdx.x] = t;
    }
}
__global__ void k_sum_partials(int n, const double *p, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0;
        for (int i = 0; i < n; i++) s += p[i];
        *out = s;
    }
}

// inverse of every diagonal block A_bb of the little operator (block-Jacobi
// preconditioner of the coarse solve): one warp per block, Gauss-Jordan with
// partial pivoting on the Ns x Ns matrix held in shared memory.  Layout as
// Aint: element (row k, column l) at [k*Ns + l].
__global__ void k_block_inverse(int nblk, int Ns, const double2 *Aint, double2 *Dinv, int *bad)
{
    extern __shared__ double2 sm[];
    const int warps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * warps + w;
    if (b >= nblk) return;
    double2 *M = sm + (size_t)w * 2 * Ns * Ns;   // [Ns][2Ns] row-major augmented matrix
    const int n2 = 2 * Ns;
    const double2 *A = Aint + (size_t)b * 9 * Ns * Ns;   // entry j = 0
    for (int e = lane; e < Ns * n2; e += 32) {
        int i = e / n2, j = e % n2;
        M[e] = j < Ns ? A[i * Ns + j] : make_double2(j - Ns == i ? 1.0 : 0.0, 0.0);
    }
    __syncwarp();
    double amax = 0;
    for (int e = 0; e < Ns * Ns; e++) amax = fmax(amax, hypot(M[(e / Ns) * n2 + e % Ns].x, M[(e / Ns) * n2 + e % Ns].y));
    for (int k = 0; k < Ns; k++) {
        int p = k;
        double best = hypot(M[k * n2 + k].x, M[k * n2 + k].y);
        for (int i = k + 1; i < Ns; i++) {
            double v = hypot(M[i * n2 + k].x, M[i * n2 + k].y);
            if (v > best) {
                best = v;
                p = i;
            }
        }
        if (!(best > 1e-14 * amax)) {
            if (lane == 0) atomicAdd(bad, 1);
            return;
        }
        if (p != k)
            for (int j = lane; j < n2; j += 32) {
                double2 t = M[k * n2 + j];
                M[k * n2 + j] = M[p * n2 + j];
                M[p * n2 + j] = t;
            }
        __syncwarp();
        double2 d = M[k * n2 + k];
        double dn = d.x * d.x + d.y * d.y;
        double2 di = make_double2(d.x / dn, -d.y / dn);
        for (int j = lane; j < n2; j += 32) {
            double2 v = M[k * n2 + j];
            M[k * n2 + j] = make_double2(v.x * di.x - v.y * di.y, v.x * di.y + v.y * di.x);
        }
        __syncwarp();
        for (int i = 0; i < Ns; i++) {
            if (i == k) continue;
            double2 f = M[i * n2 + k];
            __syncwarp();
            for (int j = lane; j < n2; j += 32) {
                double2 v = M[k * n2 + j], m = M[i * n2 + j];
                M[i * n2 + j] = make_double2(m.x - (f.x * v.x - f.y * v.y), m.y - (f.x * v.y + f.y * v.x));
            }
            __syncwarp();
        }
    }
    double2 *Di = Dinv + (size_t)b * Ns * Ns;
    for (int e = lane; e < Ns * Ns; e += 32) {
        int k = e / Ns, l = e % Ns;   // row k, column l of the inverse
        Di[k * Ns + l] = M[k * n2 + Ns + l];
    }
}


// Little-operator and block-Jacobi products of nrhs coarse vectors:
// out_r[b*Ns + k] = sum_j sum_l M[b][j][k][l] in_r[n_j(b)*Ns + l] with j over the
// nine couplings of block b (n_j from nbr) or, for the block-Jacobi inverse, the
// block itself (nmat = 1, n_0 = b).  One CTA per (block, chunk of rhs): the
// input segments of the chunk are staged in shared memory as [j][r][l] in the
// matrix's precision with an odd row pitch (conflict-free reads for up to 16
// right-hand sides in a warp), then thread (k, r) forms one output in the
// matrix's precision, summing in (j, l) order.  Matrix rows are read through
// L1, each by all rhs of the chunk.
__device__ __forceinline__ void put2(double2 *p, double re, double im) { *p = make_double2(re, im); }
__device__ __forceinline__ void put2(double2 *p, float re, float im) { *p = make_double2(re, im); }
__device__ __forceinline__ void put2(float2 *p, float re, float im) { *p = make_float2(re, im); }
__device__ __forceinline__ void to_mat(float2 &m, float2 v) { m = v; }
__device__ __forceinline__ void to_mat(float2 &m, double2 v) { m = make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ void to_mat(double2 &m, double2 v) { m = v; }
template <class MT>
struct CAcc;
template <>
struct CAcc<float2> {
    using R = float;
};
template <>
struct CAcc<double2> {
    using R = double;
};
constexpr int COARSE_SMEM = 96 * 1024;

template <class MT, class IT, class OT>
__global__ void __launch_bounds__(256) k_coarse_mul(int Ns, long N, int nrhs, int rc, int nmat, const int *nbr,
                                                    const MT *__restrict__ M, const IT *__restrict__ in, OT *out)
{
    using R = typename CAcc<MT>::R;
    extern __shared__ __align__(16) unsigned char coarse_raw[];
    MT *cs = reinterpret_cast<MT *>(coarse_raw);
    const int b = blockIdx.x, r0 = blockIdx.y * rc, nr = min(rc, nrhs - r0), P = Ns | 1;
    in += r0 * N;
    out += r0 * N;
    for (int e = threadIdx.x; e < nmat * nr * Ns; e += blockDim.x) {
        const int l = e % Ns, jr = e / Ns, r = jr % nr, j = jr / nr;
        const int nb = nbr ? nbr[b * 9 + j] : b;
        to_mat(cs[jr * P + l], in[r * N + (long)nb * Ns + l]);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < Ns * nr; o += blockDim.x) {
        const int k = o / nr, r = o - k * nr;
        R re = 0, im = 0;
        const MT *Mk = M + ((long)b * nmat * Ns + k) * Ns;
        for (int j = 0; j < nmat; j++) {
            const MT *row = Mk + (long)j * Ns * Ns;
            const MT *x = cs + (j * nr + r) * P;
#pragma unroll 2
            for (int l = 0; l < Ns; l++) {
                const MT a = __ldg(row + l), y = x[l];
                re += a.x * y.x - a.y * y.y;
                im += a.x * y.y + a.y * y.x;
            }
        }
        put2(out + r * N + (long)b * Ns + k, re, im);
    }
}

// host side: rhs chunk so that the staged segments fit COARSE_SMEM
template <class MT, class IT, class OT>
lqcd_status coarse_mul(lqcd_ctx *c, int nblk, int Ns, long N, int nrhs, int nmat, const int *nbr, const MT *M,
                       const IT *in, OT *out)
{
    static bool attr = false;
    if (!attr) {
        LQCD_CUDA_CHECK(c, cudaFuncSetAttribute(k_coarse_mul<MT, IT, OT>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, COARSE_SMEM));
        attr = true;
    }
    const int P = Ns | 1;
    const int rc = std::max(1, std::min(nrhs, COARSE_SMEM / (int)(nmat * P * sizeof(MT))));
    const int threads = std::min(256, (Ns * rc + 31) / 32 * 32);
    const size_t smem = (size_t)nmat * rc * P * sizeof(MT);
    k_coarse_mul<MT, IT, OT><<<dim3(nblk, div_up(nrhs, rc)), threads, smem, c->stream>>>(Ns, N, nrhs, rc, nmat, nbr,
                                                                                         M, in, out);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

__global__ void k_to_float2(long n, const double2 *in, float2 *out)
{
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
__global__ void k_to_double2(long n, const float2 *in, double2 *out)
{
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_double2(in[i].x, in[i].y);
}

// FP32 coarse-vector BLAS (the coarse solve with the FP32 operator): per-CTA
// partial dots accumulated in float, partials and their fixed-order sum in
// double.  partial[(r*nb + b)*32 + i] for vector i of rhs r.
constexpr int FDOT_K = 16;
__global__ void __launch_bounds__(256) k_fdot_partial(long n, const float2 *__restrict__ A, long sa, long fa,
                                                      const float2 *__restrict__ B, long fb, int k0, int kn,
                                                      double2 *partial)
{
    const int r = blockIdx.y;
    const float2 *Br = B + r * fb, *Ar = A + r * fa;
    float re[FDOT_K], im[FDOT_K];
#pragma unroll
    for (int i = 0; i < FDOT_K; i++) re[i] = im[i] = 0.f;
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        const float2 bv = Br[j];
#pragma unroll
        for (int i = 0; i < FDOT_K; i++)
            if (i < kn) {
                const float2 a = Ar[(k0 + i) * sa + j];
                re[i] += a.x * bv.x + a.y * bv.y;
                im[i] += a.x * bv.y - a.y * bv.x;
            }
    }
    __shared__ double sh[8][FDOT_K][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < FDOT_K; i++) {
        if (i >= kn) break;   // kn is the same for the whole CTA
        float x = re[i], m = im[i];
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            m += __shfl_down_sync(0xffffffffu, m, o);
        }
        if (lane == 0) {
            sh[warp][i][0] = x;
            sh[warp][i][1] = m;
        }
    }
    __syncthreads();
    if (threadIdx.x < kn) {
        double x = 0, m = 0;
        for (int w = 0; w < 8; w++) {
            x += sh[w][threadIdx.x][0];
            m += sh[w][threadIdx.x][1];
        }
        partial[((long)r * gridDim.x + blockIdx.x) * 32 + k0 + threadIdx.x] = make_double2(x, m);
    }
}
__global__ void k_fdot_final(int nb, int k, const double2 *partial, double2 *out)
{
    const int i = blockIdx.x, r = blockIdx.y;
    __shared__ double sx[128], sm[128];
    double x = 0, m = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const double2 v = partial[((long)r * nb + b) * 32 + i];
        x += v.x;
        m += v.y;
    }
    sx[threadIdx.x] = x;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            sx[threadIdx.x] += sx[threadIdx.x + st];
            sm[threadIdx.x] += sm[threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[r * k + i] = make_double2(sx[0], sm[0]);
}
// y_r += sign * sum_i cf[r*k + i] X_{i,r} (coefficients in device memory, FP64)
__global__ void k_fmulti_axpy(long n, int k, const double2 *__restrict__ cf, const float2 *__restrict__ X, long sa,
                              long fa, float2 *y, long fy, float sign)
{
    const int r = blockIdx.y;
    const float2 *Xr = X + r * fa;
    float2 *yr = y + r * fy;
    // the coefficients converted to float once per CTA (a conversion per element
    // would run on GB300's FP64 pipe)
    __shared__ float2 cs[32];
    for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = make_float2((float)cf[r * k + i].x, (float)cf[r * k + i].y);
    __syncthreads();
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        float2 b = yr[j];
        float sr = 0.f, si = 0.f;
        for (int i = 0; i < k; i++) {
            const float2 a = Xr[i * sa + j];
            const float cx = cs[i].x, cy = cs[i].y;
            sr += cx * a.x - cy * a.y;
            si += cx * a.y + cy * a.x;
        }
        yr[j] = make_float2(b.x + sign * sr, b.y + sign * si);
    }
}
__global__ void k_fsub(long n, const float2 *a, const float2 *b, float2 *out)
{
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2(a[i].x - b[i].x, a[i].y - b[i].y);
}

// Even-odd little operator on block colours.  Coarse vectors of one colour
// are compact: segment i (Ns entries) of a right-hand side belongs to block
// rows[i]; a neighbour block n of the other colour sits at segment pos[n].
//   out_i = xadd_i + sign * P_b sum_{j=1..8} A[b][j] in_{pos[nbr_j(b)]},  b = rows[i],
// with P_b = Dinv[b] (use_dinv) or 1; xadd may be null.
// One CTA per row block, eight warps: warp j takes the hop
// to neighbour j with lane k owning row k of the block (Ns <= 32) and all (up
// to CW_R) right-hand sides of the pass in registers.  Every matrix entry is
// loaded once per launch, coalesced from the column-major copies
// AT [b][j-1][l][k] and DT [b][l][k]; the input segment of neighbour j sits in
// shared memory as [l][r] (one broadcast read per pair of right-hand sides).
// The eight partial sums are added in the order j = 1 .. 8, then Dinv is
// applied by thread (k, r).  Short dependent chains per warp (Ns loads of one
// matrix) and 8 warps per row block keep enough loads in flight.
constexpr int CW_R = 12;   // right-hand sides per pass
__global__ void __launch_bounds__(256) k_coarse_hop_eo_j(int Ns, long Nin, long Nout, int nrhs,
                                                         const int *__restrict__ rows, const int *__restrict__ npos,
                                                         const float2 *__restrict__ AT,
                                                         const float2 *__restrict__ DT, int use_dinv,
                                                         const float2 *__restrict__ in, const float2 *xadd,
                                                         float sign, float2 *out)
{
    extern __shared__ __align__(16) unsigned char eoj_raw[];
    float2 *sm = reinterpret_cast<float2 *>(eoj_raw);
    const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x, b = rows[i], r0 = blockIdx.y * CW_R, nr = min(CW_R, nrhs - r0);
    const int tile = Ns * CW_R;
    float2 *xj = sm + j * tile;     // input segment of neighbour j, then its partial sum
    float2 *hs = sm + 8 * tile;     // hop sum [k][r] for the Dinv stage
    in += r0 * Nin;
    out += r0 * Nout;
    if (xadd) xadd += r0 * Nout;
    const long seg = (long)npos[i * 8 + j] * Ns;
    if (lane < Ns)
#pragma unroll
        for (int r = 0; r < CW_R; r++)
            xj[lane * CW_R + r] = r < nr ? in[r * Nin + seg + lane] : make_float2(0.f, 0.f);
    __syncwarp();
    float re[CW_R], im[CW_R];
#pragma unroll
    for (int r = 0; r < CW_R; r++) re[r] = im[r] = 0.f;
    if (lane < Ns) {
        const float2 *Aj = AT + ((long)b * 8 + j) * Ns * Ns + lane;
        // the matrix column in groups of 8 entries, each group's loads issued together
        for (int l0 = 0; l0 < Ns; l0 += 8) {
            float2 av[8];
#pragma unroll
            for (int u = 0; u < 8; u++) av[u] = l0 + u < Ns ? __ldg(Aj + (l0 + u) * Ns) : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; u++) {
                if (l0 + u >= Ns) break;
                const float2 a = av[u];
                const float4 *y4 = reinterpret_cast<const float4 *>(xj + (l0 + u) * CW_R);
#pragma unroll
                for (int q = 0; q < CW_R / 2; q++) {
                    const float4 y = y4[q];
                    re[2 * q] = fmx(a.x, y.x, fmx(-a.y, y.y, re[2 * q]));
                    im[2 * q] = fmx(a.x, y.y, fmx(a.y, y.x, im[2 * q]));
                    re[2 * q + 1] = fmx(a.x, y.z, fmx(-a.y, y.w, re[2 * q + 1]));
                    im[2 * q + 1] = fmx(a.x, y.w, fmx(a.y, y.z, im[2 * q + 1]));
                }
            }
        }
    }
    __syncwarp();
    if (lane < Ns)
#pragma unroll
        for (int r = 0; r < CW_R; r++) xj[lane * CW_R + r] = make_float2(re[r], im[r]);
    __syncthreads();
    for (int o = threadIdx.x; o < tile; o += blockDim.x) {
        float2 t = sm[o];
#pragma unroll
        for (int jj = 1; jj < 8; jj++) {
            const float2 u = sm[jj * tile + o];
            t.x += u.x;
            t.y += u.y;
        }
        const int k = o / CW_R, r = o - k * CW_R;
        if (use_dinv) {
            hs[o] = t;
        } else if (r < nr) {
            const long oi = r * Nout + (long)i * Ns + k;
            const float2 base = xadd ? xadd[oi] : make_float2(0.f, 0.f);
            out[oi] = make_float2(base.x + sign * t.x, base.y + sign * t.y);
        }
    }
    if (!use_dinv) return;
    __syncthreads();
    for (int o = threadIdx.x; o < tile; o += blockDim.x) {
        const int k = o / CW_R, r = o - k * CW_R;
        if (r >= nr) continue;
        const float2 *D = DT + (long)b * Ns * Ns + k;
        float dre = 0.f, dim = 0.f;
#pragma unroll 4
        for (int l = 0; l < Ns; l++) {
            const float2 a = __ldg(D + l * Ns), y = hs[l * CW_R + r];
            dre = fmx(a.x, y.x, fmx(-a.y, y.y, dre));
            dim = fmx(a.x, y.y, fmx(a.y, y.x, dim));
        }
        const long oi = r * Nout + (long)i * Ns + k;
        const float2 base = xadd ? xadd[oi] : make_float2(0.f, 0.f);
        out[oi] = make_float2(base.x + sign * dre, base.y + sign * dim);
    }
}
// column-major FP32 copies of the eight hopping matrices and of the diagonal
// block inverses: AT[b][j-1][l][k] = A[b][j][k][l], DT[b][l][k] = Dinv[b][k][l]
__global__ void k_coarse_transpose(int nblk, int Ns, const double2 *A, const double2 *Dinv, float2 *AT, float2 *DT)
{
    const long n2 = (long)Ns * Ns, e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= (long)nblk * 9 * n2) return;
    const long b = e / (9 * n2);
    const int j = (int)(e / n2 % 9), l = (int)(e % n2 / Ns), k = (int)(e % Ns);
    if (j == 0) {
        const double2 v = Dinv[(b * Ns + k) * Ns + l];
        DT[b * n2 + (long)l * Ns + k] = make_float2((float)v.x, (float)v.y);
    } else {
        const double2 v = A[((b * 9 + j) * Ns + k) * Ns + l];
        AT[(b * 8 + j - 1) * n2 + (long)l * Ns + k] = make_float2((float)v.x, (float)v.y);
    }
}
// out_i = Dinv[rows[i]] in_i on compact colour vectors
__global__ void __launch_bounds__(256) k_coarse_diag_eo(int Ns, long N, int nrhs, const int *__restrict__ rows,
                                                        const float2 *__restrict__ Dinv, const float2 *__restrict__ in,
                                                        float2 *out)
{
    const int i = blockIdx.x, b = rows[i], r = blockIdx.y;
    const float2 *x = in + r * N + (long)i * Ns;
    for (int k = threadIdx.x; k < Ns; k += blockDim.x) {
        const float2 *row = Dinv + ((long)b * Ns + k) * Ns;
        float re = 0.f, im = 0.f;
        for (int l = 0; l < Ns; l++) {
            const float2 a = __ldg(row + l), y = x[l];
            re = fmx(a.x, y.x, fmx(-a.y, y.y, re));
            im = fmx(a.x, y.y, fmx(a.y, y.x, im));
        }
        out[r * N + (long)i * Ns + k] = make_float2(re, im);
    }
}
// compact colour segments <-> full coarse vectors (FP64 full, FP32 compact)
__global__ void k_gather_col(int Ns, long Nfull, long Nc, int nrows, int nrhs, const int *rows, const double2 *full,
                             float2 *comp)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (e >= (long)nrows * Ns) return;
    const int i = (int)(e / Ns), k = (int)(e % Ns);
    const double2 v = full[r * Nfull + (long)rows[i] * Ns + k];
    comp[r * Nc + e] = make_float2((float)v.x, (float)v.y);
}
__global__ void k_scatter_col(int Ns, long Nfull, long Nc, int nrows, int nrhs, const int *rows, const float2 *comp,
                              double2 *full)
{
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (e >= (long)nrows * Ns) return;
    const int i = (int)(e / Ns), k = (int)(e % Ns);
    const float2 v = comp[r * Nc + e];
    full[r * Nfull + (long)rows[i] * Ns + k] = make_double2(v.x, v.y);
}

}  // namespace

struct DflState {
    DBlk B;
    int Ns;
    lqcd_prec prec;        // storage of the subspace vectors
    void *phi = nullptr;   // Ns native full fields
    int *nbr = nullptr;    // [nblk][9] device
    double2 *Aint = nullptr;
    double2 *Dinv = nullptr;   // [nblk][Ns][Ns] inverses of the diagonal blocks
    float2 *Aint32 = nullptr, *Dinv32 = nullptr;   // FP32 copies (coarse_prec == LQCD_F32)
    float2 *AT32 = nullptr, *DT32 = nullptr;       // column-major FP32 copies (even-odd coarse solve, Ns <= 32)
    lqcd_dfl_params params;
    std::vector<int> nbr_host;
    long coarse_iters = 0, coarse_solves = 0;
    // even-odd form of the little operator on block colours (every block count
    // even, so the +-mu neighbours of a block have the other colour)
    bool eo = false;
    int ncol[2] = {0, 0};
    int *blist = nullptr;   // device [ncol[0] colour-0 block ids, then ncol[1] colour-1 ids]
    int *bpos = nullptr;    // device [nblk]: index of a block within its colour's list
    int *npos = nullptr;    // device [nblk][8]: for list entry i, the list index of its neighbour j + 1
};

void dfl_free(lqcd_ctx *c)
{
    if (!c->dfl) return;
    cudaFree(c->dfl->phi);
    cudaFree(c->dfl->nbr);
    cudaFree(c->dfl->Aint);
    cudaFree(c->dfl->Dinv);
    cudaFree(c->dfl->Aint32);
    cudaFree(c->dfl->AT32);
    cudaFree(c->dfl->DT32);
    cudaFree(c->dfl->Dinv32);
    cudaFree(c->dfl->blist);
    cudaFree(c->dfl->bpos);
    cudaFree(c->dfl->npos);
    delete c->dfl;
    c->dfl = nullptr;
}

namespace {

lqcd_status norm_native(lqcd_ctx *c, lqcd_prec p, const void *x, long nhalf, double *out)
{
    if (p == LQCD_F64) return blas_norm2(c, 24 * c->g.Vh * nhalf, (const double *)x, out);
    long n = 6 * c->g.Vh * nhalf;
    double *partial = c->red;
    k_norm32_partial<<<304, 256, 0, c->stream>>>(n, (const float4 *)x, partial);
    k_sum_partials<<<1, 32, 0, c->stream>>>(304, partial, c->red_out);
    c->n_kernel_launches += 2;
    LQCD_LAUNCH_CHECK(c);
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(c->red_host, c->red_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    *out = c->red_host[0];
    return LQCD_OK;
}

lqcd_status scale_native(lqcd_ctx *c, lqcd_prec p, void *x, long nhalf, double s)
{
    if (p == LQCD_F64) return blas_scal(c, 24 * c->g.Vh * nhalf, s, 0, (double *)x);
    long n = 6 * c->g.Vh * nhalf;
    k_scale32<<<608, 256, 0, c->stream>>>(n, (float)s, (float4 *)x);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

long field_elems(const lqcd_ctx *c, lqcd_prec p) { return 2 * (p == LQCD_F64 ? 12 : 6) * (long)c->g.Vh; }

template <class T>
lqcd_status launch_project(lqcd_ctx *c, const double2 *in, double2 *cv, int nrhs)
{
    DflState *d = c->dfl;
    if (std::is_same<T, float4>::value && (2 * d->B.vol) % 32 == 0 && 2 * d->B.vol <= 1024) {
        const long N = (long)d->B.nblk * d->Ns, nf = 24 * (long)c->g.Vh;
        const int ngr = div_up(nrhs, PJ_R);
        k_project_h<<<d->B.nblk * ngr, 2 * d->B.vol, 0, c->stream>>>(c->g, d->B, (const float4 *)d->phi, d->Ns,
                                                                     field_elems(c, d->prec), in, cv, nrhs, nf, N,
                                                                     ngr);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        return LQCD_OK;
    }
    size_t sm = (2 * RCHUNK * 32 + 2 * RCHUNK) * sizeof(double);
    const long N = (long)d->B.nblk * d->Ns, nf = 24 * (long)c->g.Vh;
    k_project<T><<<d->B.nblk * nrhs, d->B.vol, sm, c->stream>>>(c->g, d->B, (const T *)d->phi, d->Ns,
                                                                field_elems(c, d->prec), in, cv, nrhs, nf, N);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}
template <class T>
lqcd_status launch_expand(lqcd_ctx *c, const double2 *cv, double2 *out, int nrhs)
{
    DflState *d = c->dfl;
    const int nsplit = d->B.vol % 64 == 0 ? std::max(1, d->B.vol / 128) : 0;
    if (std::is_same<T, float4>::value && nsplit > 0 && 2 * (d->B.vol / nsplit) <= 256) {
        const long N = (long)d->B.nblk * d->Ns, nf = 24 * (long)c->g.Vh;
        const int ngr = div_up(nrhs, PJ_R);
        k_expand_h<<<d->B.nblk * nsplit * ngr, 2 * (d->B.vol / nsplit), 0, c->stream>>>(
            c->g, d->B, (const float4 *)d->phi, d->Ns, field_elems(c, d->prec), cv, out, nrhs, N, nf, ngr, nsplit);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        return LQCD_OK;
    }
    const long N = (long)d->B.nblk * d->Ns, nf = 24 * (long)c->g.Vh;
    k_expand<T><<<d->B.nblk * nrhs, d->B.vol, 0, c->stream>>>(c->g, d->B, (const T *)d->phi, d->Ns,
                                                              field_elems(c, d->prec), cv, out, nrhs, N, nf);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

// nrhs fields: in / out native F64 full fields one after the other, coarse
// vectors of nblk*Ns entries one after the other
lqcd_status project(lqcd_ctx *c, const double2 *in, double2 *cv, int nrhs = 1)
{
    return c->dfl->prec == LQCD_F64 ? launch_project<double2>(c, in, cv, nrhs)
                                    : launch_project<float4>(c, in, cv, nrhs);
}
lqcd_status expand(lqcd_ctx *c, const double2 *cv, double2 *out, int nrhs = 1)
{
    return c->dfl->prec == LQCD_F64 ? launch_expand<double2>(c, cv, out, nrhs)
                                    : launch_expand<float4>(c, cv, out, nrhs);
}
lqcd_status little_apply_b(lqcd_ctx *c, const double2 *cv, double2 *out, int nrhs)
{
    DflState *d = c->dfl;
    const long N = (long)d->B.nblk * d->Ns;
    if (d->Aint32) return coarse_mul(c, d->B.nblk, d->Ns, N, nrhs, 9, d->nbr, d->Aint32, cv, out);
    return coarse_mul(c, d->B.nblk, d->Ns, N, nrhs, 9, d->nbr, d->Aint, cv, out);
}
lqcd_status little_apply(lqcd_ctx *c, const double2 *cv, double2 *out) { return little_apply_b(c, cv, out, 1); }

lqcd_status block_jacobi(lqcd_ctx *c, const double2 *in, double2 *out, int nrhs)
{
    DflState *d = c->dfl;
    const long N = (long)d->B.nblk * d->Ns;
    if (d->Dinv32) return coarse_mul(c, d->B.nblk, d->Ns, N, nrhs, 1, (const int *)nullptr, d->Dinv32, in, out);
    return coarse_mul(c, d->B.nblk, d->Ns, N, nrhs, 1, (const int *)nullptr, d->Dinv, in, out);
}

// ---- device-resident scalar bookkeeping of the coarse GCR (one thread per rhs)
constexpr int CG_R = 64, CG_K = 32;
struct CoarseScal {
    double bn2[CG_R], rr[CG_R], tol2;
    int active[CG_R], bad[CG_R];
    double2 a[CG_R][CG_K][CG_K];   // a[r][i][k] = <q_i, q_k>
    double bk[CG_R][CG_K];
    double2 ck[CG_R][CG_K];
    double2 cfR[CG_R], cfS[CG_R];
    double2 alpha[CG_R * CG_K];
    double2 dots[2048];
};

__global__ void k_c_init(int nrhs, double tol2, CoarseScal *s)
{
    int r = threadIdx.x;
    if (r == 0) s->tol2 = tol2;
    if (r >= nrhs) return;
    double b2 = s->dots[r].x;
    s->bn2[r] = b2;
    s->rr[r] = b2;
    s->bad[r] = 0;
    s->active[r] = (b2 > 0 && isfinite(b2)) ? 1 : 0;
}
// store the Gram-Schmidt coefficients <q_i, q_k> (they are applied straight from s->dots)
__global__ void k_c_gs(int nrhs, int k, CoarseScal *s)
{
    int r = blockIdx.x, i = threadIdx.x;
    if (r >= nrhs || i >= k) return;
    s->a[r][i][k] = s->dots[r * k + i];
}
// from |q_k|^2 and <rho, q_k>: b_k, c_k, the coefficients of rho -= c_k q_k / b_k
// and q_k *= 1/b_k, the updated |rho|^2 and the convergence flag
__device__ __forceinline__ void c_norm_body(int r, int k, double q2, double2 rq, CoarseScal *s)
{
    double bk = sqrt(q2);
    bool ok = bk > 0 && isfinite(bk);
    if (s->active[r] && !ok) {
        s->active[r] = 0;
        s->bad[r] = 1;
    }
    double sc = ok ? 1.0 / bk : 0.0;
    double cr = rq.x * sc, ci = -rq.y * sc;   // c_k = <q_k/b_k, rho>
    int act = s->active[r];
    s->bk[r][k] = bk;
    s->ck[r][k] = act ? make_double2(cr, ci) : make_double2(0, 0);
    s->cfR[r] = act ? make_double2(cr * sc, ci * sc) : make_double2(0, 0);
    s->cfS[r] = make_double2(sc - 1.0, 0);
    if (act) {
        double rr = s->rr[r] - (cr * cr + ci * ci);
        s->rr[r] = rr > 0 ? rr : 0;
        if (s->rr[r] <= s->tol2 * s->bn2[r]) s->active[r] = 0;
    }
}
__global__ void k_c_norm(int nrhs, int k, CoarseScal *s)
{
    int r = threadIdx.x;
    if (r >= nrhs) return;
    c_norm_body(r, k, s->dots[2 * r].x, s->dots[2 * r + 1], s);
}
// the same from the per-CTA partial sums of k_fgs_norm (summed in CTA order)
__global__ void k_c_norm_p(int nrhs, int k, int nbp, const double2 *partial, CoarseScal *s)
{
    int r = threadIdx.x;
    if (r >= nrhs) return;
    double q2 = 0, rx = 0, ry = 0;
    for (int b = 0; b < nbp; b++) {
        const double2 *p = partial + ((long)r * nbp + b) * 32;
        q2 += p[0].x;
        rx += p[1].x;
        ry += p[1].y;
    }
    c_norm_body(r, k, q2, make_double2(rx, ry), s);
}
// alpha_j = (c_j - sum_{i>j} a_ji alpha_i) / b_j
__global__ void k_c_backsub(int nrhs, int nk, CoarseScal *s)
{
    int r = threadIdx.x;
    if (r >= nrhs) return;
    double2 *al = s->alpha + r * nk;
    for (int j = nk - 1; j >= 0; j--) {
        double sr = s->ck[r][j].x, si = s->ck[r][j].y;
        for (int i = j + 1; i < nk; i++) {
            double2 a = s->a[r][j][i], x = al[i];
            sr -= a.x * x.x - a.y * x.y;
            si -= a.x * x.y + a.y * x.x;
        }
        double bj = s->bk[r][j];
        al[j] = bj > 0 ? make_double2(sr / bj, si / bj) : make_double2(0, 0);
    }
}
// One Gram-Schmidt step of the FP32 coarse GCR in one pass over q_k:
//   q_k -= sum_{i<k} <q_i, q_k> q_i,
// the coefficients summed by every CTA from the per-CTA partials of
// k_fdot_partial (the same fixed order in every CTA; CTA 0 of each right-hand
// side stores them as a[r][i][k]), then per-CTA partial sums of |q_k|^2 and
// <rho, q_k> of the updated q_k into partial2 [(r*gridDim.x + b)*32 + 0, 1].
__global__ void __launch_bounds__(256) k_fgs_norm(long n, int k, int nbp, const double2 *__restrict__ partial,
                                                  CoarseScal *S, const float2 *__restrict__ Q, long sa, float2 *qk,
                                                  const float2 *__restrict__ rho, double2 *partial2)
{
    const int r = blockIdx.y;
    __shared__ float2 cs[CG_K];
    __shared__ double sh[8][3];
    if (k > 0) {
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            double x = 0, m = 0;
            for (int b = 0; b < nbp; b++) {
                const double2 v = partial[((long)r * nbp + b) * 32 + i];
                x += v.x;
                m += v.y;
            }
            if (blockIdx.x == 0) S->a[r][i][k] = make_double2(x, m);
            cs[i] = make_float2((float)x, (float)m);
        }
        __syncthreads();
    }
    const float2 *Qr = Q + r * n, *pr = rho + r * n;
    float2 *qr = qk + r * n;
    float nq = 0.f, rx = 0.f, ry = 0.f;
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        float2 q = qr[j];
        if (k > 0) {
            float sr = 0.f, si = 0.f;
            for (int i = 0; i < k; i++) {
                const float2 a = Qr[i * sa + j];
                const float cx = cs[i].x, cy = cs[i].y;
                sr += cx * a.x - cy * a.y;
                si += cx * a.y + cy * a.x;
            }
            q.x -= sr;
            q.y -= si;
            qr[j] = q;
        }
        const float2 p = pr[j];
        nq += q.x * q.x + q.y * q.y;
        rx += p.x * q.x + p.y * q.y;   // <rho, q> = sum conj(rho) q
        ry += p.x * q.y - p.y * q.x;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        nq += __shfl_down_sync(0xffffffffu, nq, o);
        rx += __shfl_down_sync(0xffffffffu, rx, o);
        ry += __shfl_down_sync(0xffffffffu, ry, o);
    }
    if (lane == 0) {
        sh[warp][0] = nq;
        sh[warp][1] = rx;
        sh[warp][2] = ry;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, bx = 0, by = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            a += sh[w][0];
            bx += sh[w][1];
            by += sh[w][2];
        }
        double2 *o = partial2 + ((long)r * gridDim.x + blockIdx.x) * 32;
        o[0] = make_double2(a, 0.0);
        o[1] = make_double2(bx, by);
    }
}
// rho -= cfR q_k, q_k *= 1/b_k (q_k += cfS q_k), and the next Krylov start
// vector p_{k+1} = rho (pnext may be null)
__global__ void k_fc_update(long n, const CoarseScal *S, float2 *qk, float2 *rho, float2 *pnext)
{
    const int r = blockIdx.y;
    const float cr = (float)S->cfR[r].x, ci = (float)S->cfR[r].y, cs = (float)S->cfS[r].x;
    float2 *qr = qk + r * n, *pr = rho + r * n, *nr = pnext ? pnext + r * n : nullptr;
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        const float2 q = qr[j];
        float2 p = pr[j];
        p.x = p.x + -1.f * (cr * q.x - ci * q.y);
        p.y = p.y + -1.f * (cr * q.y + ci * q.x);
        pr[j] = p;
        if (nr) nr[j] = p;
        qr[j] = make_float2(q.x + cs * q.x, q.y + cs * q.y);
    }
}
// true residual norm after a restart
__global__ void k_c_restart(int nrhs, CoarseScal *s, int *n_active)
{
    int r = threadIdx.x;
    if (r < nrhs) {
        s->rr[r] = s->dots[r].x;
        if (s->active[r] && s->rr[r] <= s->tol2 * s->bn2[r]) s->active[r] = 0;
        if (!isfinite(s->rr[r])) {
            s->active[r] = 0;
            s->bad[r] = 1;
        }
    }
    __syncthreads();
    if (r == 0) {
        int n = 0;
        for (int i = 0; i < nrhs; i++) n += s->active[i];
        *n_active = n;
    }
}

// FP64 GCR on the little operator for nrhs coarse right-hand sides in
// lockstep, right-preconditioned by the inverse diagonal blocks (block
// Jacobi): x_r ~ A^-1 b_r to a relative residual tol, or nmx steps.  All
// scalars stay on the device: inside a Krylov cycle nothing returns to the
// host; after each cycle the host reads the number of unconverged right-hand
// sides (one synchronisation per cycle).  A right-hand side that converges
// inside a cycle gets zero updates for the rest of it.
lqcd_status coarse_gcr32(lqcd_ctx *c, const double2 *b, double2 *x, int nrhs, double tol, int nkv, int nmx,
                         int *iters);
lqcd_status coarse_gcr32_eo(lqcd_ctx *c, const double2 *b, double2 *x, int nrhs, double tol, int nkv, int nmx,
                            int *iters);

lqcd_status coarse_gcr(lqcd_ctx *c, const double2 *b, double2 *x, int nrhs, double tol, int nkv, int nmx,
                       int *iters)
{
    DflState *d = c->dfl;
    if (d->AT32) return coarse_gcr32_eo(c, b, x, nrhs, tol, nkv, nmx, iters);
    if (d->Aint32) return coarse_gcr32(c, b, x, nrhs, tol, nkv, nmx, iters);
    const long N = (long)d->B.nblk * d->Ns;
    const long n2 = 2 * N;
    if (nkv < 1 || nkv > CG_K || nrhs > CG_R || nrhs * nkv > 2048)
        return set_err(c, LQCD_ERR_ARG, "coarse nkv=%d nrhs=%d", nkv, nrhs);
    const long bN = nrhs * N;
    void *buf;
    const size_t vec_bytes = (size_t)(2 * nkv + 2) * bN * sizeof(double2);
    LQCD_TRY(ws_get(c, WS_COARSE, vec_bytes + sizeof(CoarseScal) + 256, &buf));
    double2 *P = (double2 *)buf, *Q = P + nkv * bN, *rho = Q + nkv * bN, *w = rho + bN;
    CoarseScal *S = (CoarseScal *)((char *)buf + ((vec_bytes + 255) / 256) * 256);
    int *n_active_dev = (int *)c->red_out;
    int *n_active_host = (int *)c->red_host;
    LQCD_TRY(blas_zero(c, bN * sizeof(double2), x));
    LQCD_TRY(blas_copy(c, n2 * nrhs, (const double *)b, (double *)rho));
    LQCD_TRY(bblas_dot_dev(c, n2, nrhs, (const double *)b, 0, n2, (const double *)b, n2, 1, S->dots));
    k_c_init<<<1, CG_R, 0, c->stream>>>(nrhs, tol * tol, S);
    c->n_kernel_launches++;
    int it = 0, active = nrhs;
    while (active > 0 && it < nmx) {
        int nk = 0;
        for (int k = 0; k < nkv && it < nmx; k++) {
            double2 *pk = P + k * bN, *qk = Q + k * bN;
            LQCD_TRY(block_jacobi(c, rho, pk, nrhs));
            LQCD_TRY(little_apply_b(c, pk, qk, nrhs));
            if (k > 0) {
                LQCD_TRY(bblas_dot_dev(c, n2, nrhs, (const double *)Q, 2 * bN, n2, (const double *)qk, n2, k, S->dots));
                k_c_gs<<<nrhs, k, 0, c->stream>>>(nrhs, k, S);
                c->n_kernel_launches++;
                LQCD_TRY(bblas_multi_axpy_dev(c, n2, nrhs, k, S->dots, (const double *)Q, 2 * bN, n2, (double *)qk, n2,
                                              -1.0));
            }
            // |q_k|^2 and <rho, q_k> in one pass
            LQCD_TRY(bblas_dot_dev(c, n2, nrhs, (const double *)qk, 2 * (rho - qk), n2, (const double *)qk, n2, 2,
                                   S->dots));
            k_c_norm<<<1, CG_R, 0, c->stream>>>(nrhs, k, S);
            c->n_kernel_launches++;
            LQCD_TRY(bblas_multi_axpy_dev(c, n2, nrhs, 1, S->cfR, (const double *)qk, 0, n2, (double *)rho, n2, -1.0));
            LQCD_TRY(bblas_multi_axpy_dev(c, n2, nrhs, 1, S->cfS, (const double *)qk, 0, n2, (double *)qk, n2, 1.0));
            it++;
            nk = k + 1;
        }
        k_c_backsub<<<1, CG_R, 0, c->stream>>>(nrhs, nk, S);
        c->n_kernel_launches++;
        LQCD_TRY(bblas_multi_axpy_dev(c, n2, nrhs, nk, S->alpha, (const double *)P, 2 * bN, n2, (double *)x, n2, 1.0));
        LQCD_TRY(little_apply_b(c, x, w, nrhs));
        LQCD_TRY(blas_sub(c, n2 * nrhs, (const double *)b, (const double *)w, (double *)rho));
        LQCD_TRY(bblas_dot_dev(c, n2, nrhs, (const double *)rho, 0, n2, (const double *)rho, n2, 1, S->dots));
        k_c_restart<<<1, CG_R, 0, c->stream>>>(nrhs, S, n_active_dev);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        LQCD_CUDA_CHECK(c, cudaMemcpyAsync(n_active_host, n_active_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
        active = *n_active_host;
    }
    d->coarse_iters += it;
    d->coarse_solves += 1;
    if (iters) *iters = it;
    return active > 0 ? LQCD_ERR_NOT_CONVERGED : LQCD_OK;
}

// The same GCR with the FP32 little operator: coarse vectors, operator
// applications and Gram-Schmidt in float (FP64 scalars and fixed-order FP64
// sums of the per-CTA partial dots).  The coarse solve only needs to reach
// coarse_tol (>= 1e-6 with the FP32 operator); the outer GCR stays FP64.
lqcd_status coarse_gcr32(lqcd_ctx *c, const double2 *b, double2 *x, int nrhs, double tol, int nkv, int nmx,
                         int *iters)
{
    DflState *d = c->dfl;
    const long N = (long)d->B.nblk * d->Ns;
    if (nkv < 1 || nkv > CG_K || nrhs > CG_R || nrhs * nkv > 2048)
        return set_err(c, LQCD_ERR_ARG, "coarse nkv=%d nrhs=%d", nkv, nrhs);
    const long bN = nrhs * N;
    void *buf;
    const size_t vec_bytes = (size_t)(2 * nkv + 4) * bN * sizeof(float2);
    LQCD_TRY(ws_get(c, WS_COARSE, vec_bytes + sizeof(CoarseScal) + 256, &buf));
    float2 *P = (float2 *)buf, *Q = P + nkv * bN, *rho = Q + nkv * bN, *w = rho + bN, *xf = w + bN, *bf = xf + bN;
    CoarseScal *S = (CoarseScal *)((char *)buf + ((vec_bytes + 255) / 256) * 256);
    int *n_active_dev = (int *)c->red_out;
    int *n_active_host = (int *)c->red_host;
    double2 *partial = (double2 *)c->red;
    const int nb = std::max(1, std::min<int>(std::max(8, 4 * 152 / nrhs), (int)((N + 255) / 256)));
    const int ga = std::max(1, std::min<int>(4 * 152 / std::max(1, nrhs), (int)((N + 255) / 256)));
    auto dots = [&](const float2 *A, long sa, const float2 *B, int k, double2 *out) -> lqcd_status {
        for (int k0 = 0; k0 < k; k0 += FDOT_K) {
            const int kn = std::min(FDOT_K, k - k0);
            k_fdot_partial<<<dim3(nb, nrhs), 256, 0, c->stream>>>(N, A, sa, N, B, N, k0, kn, partial);
            c->n_kernel_launches++;
        }
        k_fdot_final<<<dim3(k, nrhs), 128, 0, c->stream>>>(nb, k, partial, out);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        return LQCD_OK;
    };
    auto axpy = [&](int k, const double2 *cf, const float2 *X, long sa, float2 *y, float sign) -> lqcd_status {
        k_fmulti_axpy<<<dim3(ga, nrhs), 256, 0, c->stream>>>(N, k, cf, X, sa, N, y, N, sign);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        return LQCD_OK;
    };
    auto jacobi = [&](const float2 *in, float2 *out) {
        return coarse_mul(c, d->B.nblk, d->Ns, N, nrhs, 1, (const int *)nullptr, d->Dinv32, in, out);
    };
    auto apply = [&](const float2 *in, float2 *out) {
        return coarse_mul(c, d->B.nblk, d->Ns, N, nrhs, 9, d->nbr, d->Aint32, in, out);
    };
    const int gn = div_up(bN, 256);
    k_to_float2<<<gn, 256, 0, c->stream>>>(bN, b, bf);
    c->n_kernel_launches++;
    LQCD_CUDA_CHECK(c, cudaMemsetAsync(xf, 0, bN * sizeof(float2), c->stream));
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(rho, bf, bN * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
    LQCD_TRY(dots(bf, 0, bf, 1, S->dots));
    k_c_init<<<1, CG_R, 0, c->stream>>>(nrhs, tol * tol, S);
    c->n_kernel_launches++;
    int it = 0, active = nrhs;
    while (active > 0 && it < nmx) {
        int nk = 0;
        for (int k = 0; k < nkv && it < nmx; k++) {
            float2 *pk = P + k * bN, *qk = Q + k * bN;
            LQCD_TRY(jacobi(rho, pk));
            LQCD_TRY(apply(pk, qk));
            if (k > 0) {
                LQCD_TRY(dots(Q, bN, qk, k, S->dots));
                k_c_gs<<<nrhs, k, 0, c->stream>>>(nrhs, k, S);
                c->n_kernel_launches++;
                LQCD_TRY(axpy(k, S->dots, Q, bN, qk, -1.f));
            }
            LQCD_TRY(dots(qk, rho - qk, qk, 2, S->dots));   // |q_k|^2 and <rho, q_k>
            k_c_norm<<<1, CG_R, 0, c->stream>>>(nrhs, k, S);
            c->n_kernel_launches++;
            LQCD_TRY(axpy(1, S->cfR, qk, 0, rho, -1.f));
            LQCD_TRY(axpy(1, S->cfS, qk, 0, qk, 1.f));
            it++;
            nk = k + 1;
        }
        k_c_backsub<<<1, CG_R, 0, c->stream>>>(nrhs, nk, S);
        c->n_kernel_launches++;
        LQCD_TRY(axpy(nk, S->alpha, P, bN, xf, 1.f));
        LQCD_TRY(apply(xf, w));
        k_fsub<<<gn, 256, 0, c->stream>>>(bN, bf, w, rho);
        c->n_kernel_launches++;
        LQCD_TRY(dots(rho, 0, rho, 1, S->dots));
        k_c_restart<<<1, CG_R, 0, c->stream>>>(nrhs, S, n_active_dev);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        LQCD_CUDA_CHECK(c, cudaMemcpyAsync(n_active_host, n_active_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
        active = *n_active_host;
    }
    k_to_double2<<<gn, 256, 0, c->stream>>>(bN, xf, x);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    d->coarse_iters += it;
    d->coarse_solves += 1;
    if (iters) *iters = it;
    return active > 0 ? LQCD_ERR_NOT_CONVERGED : LQCD_OK;
}

// The little-Dirac solve in even-odd form (FP32 operator): with the block
// colours e, o and the block-diagonal inverses Dinv,
//   S' x_e = Dinv_e (b_e - A_eo Dinv_o b_o),  S' = 1 - Dinv_e A_eo Dinv_o A_oe,
// solved by the same GCR (no further preconditioner) on the even blocks only,
// then x_o = Dinv_o (b_o - A_oe x_e).  The vectors are half as long and the
// Schur complement is better conditioned than the block-Jacobi preconditioned
// operator; the tolerance applies to the Schur system's residual.
lqcd_status coarse_gcr32_eo(lqcd_ctx *c, const double2 *b, double2 *x, int nrhs, double tol, int nkv, int nmx,
                            int *iters)
{
    DflState *d = c->dfl;
    const int Ns = d->Ns;
    const long N = (long)d->B.nblk * Ns;
    const int ne = d->ncol[0], no = d->ncol[1];
    const long Ne = (long)ne * Ns, No = (long)no * Ns;
    const int *rows_e = d->blist, *rows_o = d->blist + ne;
    if (nkv < 1 || nkv > CG_K || nrhs > CG_R || nrhs * nkv > 2048)
        return set_err(c, LQCD_ERR_ARG, "coarse nkv=%d nrhs=%d", nkv, nrhs);
    const long bE = nrhs * Ne, bO = nrhs * No;
    void *buf;
    const size_t vec_bytes = ((size_t)(2 * nkv + 5) * bE + 3 * bO) * sizeof(float2);
    LQCD_TRY(ws_get(c, WS_COARSE, vec_bytes + sizeof(CoarseScal) + 256, &buf));
    float2 *P = (float2 *)buf, *Q = P + nkv * bE, *rho = Q + nkv * bE, *w = rho + bE, *xf = w + bE, *bf = xf + bE,
           *be = bf + bE, *bo = be + bE, *to = bo + bO, *t2o = to + bO;
    CoarseScal *S = (CoarseScal *)((char *)buf + ((vec_bytes + 255) / 256) * 256);
    int *n_active_dev = (int *)c->red_out;
    int *n_active_host = (int *)c->red_host;
    double2 *partial = (double2 *)c->red;
    double2 *partial2 = partial + 4096 * 32;   // second half of the reduction buffer (4096 * 64 double2)
    const int nb = std::max(1, std::min<int>(std::max(8, 4 * 152 / nrhs), (int)((Ne + 255) / 256)));
    const int ga = std::max(1, std::min<int>(4 * 152 / std::max(1, nrhs), (int)((Ne + 255) / 256)));
    if (!d->AT32) return set_err(c, LQCD_ERR_STATE, "even-odd coarse solve without its FP32 matrix copies");
    const size_t wsm = (size_t)9 * Ns * CW_R * sizeof(float2);
    auto hop = [&](const int *rows, int nrows, long Nin, long Nout, const float2 *in, int dinv, const float2 *xadd,
                   float sign, float2 *out) -> lqcd_status {
        k_coarse_hop_eo_j<<<dim3(nrows, div_up(nrhs, CW_R)), 256, wsm, c->stream>>>(
            Ns, Nin, Nout, nrhs, rows, d->npos + 8 * (rows - d->blist), d->AT32, d->DT32, dinv, in, xadd, sign, out);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        return LQCD_OK;
    };
    auto diag = [&](const int *rows, int nrows, long Nc, const float2 *in, float2 *out) -> lqcd_status {
        k_coarse_diag_eo<<<dim3(nrows, nrhs), 32, 0, c->stream>>>(Ns, Nc, nrhs, rows, d->Dinv32, in, out);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        return LQCD_OK;
    };
    // q = S' v
    auto apply = [&](const float2 *v, float2 *q) -> lqcd_status {
        LQCD_TRY(hop(rows_o, no, Ne, No, v, 1, nullptr, 1.f, t2o));
        return hop(rows_e, ne, No, Ne, t2o, 1, v, -1.f, q);
    };
    auto dots = [&](const float2 *A, long sa, const float2 *B, int k, double2 *out) -> lqcd_status {
        for (int k0 = 0; k0 < k; k0 += FDOT_K) {
            const int kn = std::min(FDOT_K, k - k0);
            k_fdot_partial<<<dim3(nb, nrhs), 256, 0, c->stream>>>(Ne, A, sa, Ne, B, Ne, k0, kn, partial);
            c->n_kernel_launches++;
        }
        k_fdot_final<<<dim3(k, nrhs), 128, 0, c->stream>>>(nb, k, partial, out);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        return LQCD_OK;
    };
    auto axpy = [&](int k, const double2 *cf, const float2 *X, long sa, float2 *y, float sign) -> lqcd_status {
        k_fmulti_axpy<<<dim3(ga, nrhs), 256, 0, c->stream>>>(Ne, k, cf, X, sa, Ne, y, Ne, sign);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        return LQCD_OK;
    };
    // right-hand side of the Schur system
    k_gather_col<<<dim3(div_up(Ne, 256), nrhs), 256, 0, c->stream>>>(Ns, N, Ne, ne, nrhs, rows_e, b, be);
    k_gather_col<<<dim3(div_up(No, 256), nrhs), 256, 0, c->stream>>>(Ns, N, No, no, nrhs, rows_o, b, bo);
    c->n_kernel_launches += 2;
    LQCD_TRY(diag(rows_o, no, No, bo, to));                        // to = Dinv_o b_o
    LQCD_TRY(hop(rows_e, ne, No, Ne, to, 0, be, -1.f, w));         // w = b_e - A_eo to
    LQCD_TRY(diag(rows_e, ne, Ne, w, bf));                         // rhs = Dinv_e w
    const int gn = div_up(bE, 256);
    LQCD_CUDA_CHECK(c, cudaMemsetAsync(xf, 0, bE * sizeof(float2), c->stream));
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(rho, bf, bE * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
    LQCD_TRY(dots(bf, 0, bf, 1, S->dots));
    k_c_init<<<1, CG_R, 0, c->stream>>>(nrhs, tol * tol, S);
    c->n_kernel_launches++;
    int it = 0, active = nrhs;
    while (active > 0 && it < nmx) {
        int nk = 0;
        // a GCR step: the operator (two launches), the dots against the earlier
        // q_i, one fused Gram-Schmidt + norm pass, the scalars, one fused update
        // of rho, q_k and the next start vector
        LQCD_CUDA_CHECK(c, cudaMemcpyAsync(P, rho, bE * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
        for (int k = 0; k < nkv && it < nmx; k++) {
            float2 *pk = P + k * bE, *qk = Q + k * bE;
            LQCD_TRY(apply(pk, qk));
            if (k > 0)
                for (int k0 = 0; k0 < k; k0 += FDOT_K) {
                    const int kn = std::min(FDOT_K, k - k0);
                    k_fdot_partial<<<dim3(nb, nrhs), 256, 0, c->stream>>>(Ne, Q, bE, Ne, qk, Ne, k0, kn, partial);
                    c->n_kernel_launches++;
                }
            k_fgs_norm<<<dim3(nb, nrhs), 256, 0, c->stream>>>(Ne, k, nb, partial, S, Q, bE, qk, rho, partial2);
            k_c_norm_p<<<1, CG_R, 0, c->stream>>>(nrhs, k, nb, partial2, S);
            k_fc_update<<<dim3(ga, nrhs), 256, 0, c->stream>>>(Ne, S, qk, rho, k + 1 < nkv ? pk + bE : nullptr);
            c->n_kernel_launches += 3;
            LQCD_LAUNCH_CHECK(c);
            it++;
            nk = k + 1;
        }
        k_c_backsub<<<1, CG_R, 0, c->stream>>>(nrhs, nk, S);
        c->n_kernel_launches++;
        LQCD_TRY(axpy(nk, S->alpha, P, bE, xf, 1.f));
        LQCD_TRY(apply(xf, w));
        k_fsub<<<gn, 256, 0, c->stream>>>(bE, bf, w, rho);
        c->n_kernel_launches++;
        LQCD_TRY(dots(rho, 0, rho, 1, S->dots));
        k_c_restart<<<1, CG_R, 0, c->stream>>>(nrhs, S, n_active_dev);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        LQCD_CUDA_CHECK(c, cudaMemcpyAsync(n_active_host, n_active_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
        active = *n_active_host;
    }
    // x_o = Dinv_o (b_o - A_oe x_e) = to - Dinv_o A_oe x_e; back to the full FP64 vector
    LQCD_TRY(hop(rows_o, no, Ne, No, xf, 1, to, -1.f, t2o));
    k_scatter_col<<<dim3(div_up(Ne, 256), nrhs), 256, 0, c->stream>>>(Ns, N, Ne, ne, nrhs, rows_e, xf, x);
    k_scatter_col<<<dim3(div_up(No, 256), nrhs), 256, 0, c->stream>>>(Ns, N, No, no, nrhs, rows_o, t2o, x);
    c->n_kernel_launches += 2;
    LQCD_LAUNCH_CHECK(c);
    d->coarse_iters += it;
    d->coarse_solves += 1;
    if (iters) *iters = it;
    return active > 0 ? LQCD_ERR_NOT_CONVERGED : LQCD_OK;
}

lqcd_status precond_sap(lqcd_ctx *c, const lqcd_sap_params *sp, const double2 *rho, double2 *phi, int nrhs)
{
    if (sp->prec == LQCD_F64) return sap_apply(c, sp, rho, phi, nrhs);
    void *a, *b;
    size_t fb = 2 * native_half_bytes(c, sp->prec) * nrhs;
    LQCD_TRY(ws_get(c, WS_SAP_IN, fb, &a));
    LQCD_TRY(ws_get(c, WS_SAP_PSI, fb, &b));
    LQCD_TRY(convert_native(c, LQCD_F64, sp->prec, rho, a, 2 * nrhs));
    LQCD_TRY(sap_apply(c, sp, a, b, nrhs));
    return convert_native(c, sp->prec, LQCD_F64, b, phi, 2 * nrhs);
}

}  // namespace

// phi_r = M_dfl rho_r for nrhs native full FP64 fields
lqcd_status dfl_precond_native(lqcd_ctx *c, const lqcd_sap_params *sp, const double2 *rho, double2 *phi, int nrhs,
                               bool net)
{
    DflState *d = c->dfl;
    if (!d) return set_err(c, LQCD_ERR_STATE, "deflation subspace not built");
    const long N = (long)d->B.nblk * d->Ns;
    const long nf = 24 * (long)c->g.Vh;   // double2 per full F64 field
    void *buf;
    LQCD_TRY(ws_get(c, WS_DFL, (2 * N * nrhs + 2 * nf * nrhs) * sizeof(double2), &buf));
    double2 *cv = (double2 *)buf, *ev = cv + N * nrhs, *u = ev + N * nrhs, *w = u + nf * nrhs;
    ProfClock pc(c);
    // u_r = Pi A^-1 Pi^dag rho_r, the coarse solves of all right-hand sides together
    LQCD_TRY(project(c, rho, cv, nrhs));
    pc.lap(0);
    int it = 0;
    lqcd_status st = coarse_gcr(c, cv, ev, nrhs, d->params.coarse_tol, d->params.coarse_nkv, d->params.coarse_nmx, &it);
    if (st != LQCD_OK && st != LQCD_ERR_NOT_CONVERGED) return set_err(c, st, "coarse solve failed (%d)", (int)st);
    pc.lap(1);
    LQCD_TRY(expand(c, ev, u, nrhs));
    pc.lap(2);
    // w = rho - D u  (D in the SAP precision)
    if (sp->prec == LQCD_F64) {
        LQCD_TRY(dirac_D(c, LQCD_F64, u, w, nrhs));
    } else {
        void *a, *b2;
        size_t fb = 2 * native_half_bytes(c, sp->prec) * nrhs;
        LQCD_TRY(ws_get(c, WS_MISC, fb, &a));
        LQCD_TRY(ws_get(c, WS_MISC2, fb, &b2));
        LQCD_TRY(convert_native(c, LQCD_F64, sp->prec, u, a, 2 * nrhs));
        LQCD_TRY(dirac_D(c, sp->prec, a, b2, nrhs));
        LQCD_TRY(convert_native(c, sp->prec, LQCD_F64, b2, w, 2 * nrhs));
    }
    LQCD_TRY(blas_sub(c, 2 * nf * nrhs, (const double *)rho, (const double *)w, (double *)w));
    pc.lap(3);
    if (net)
        LQCD_TRY(net_apply_native(c, w, phi, nrhs));
    else
        LQCD_TRY(precond_sap(c, sp, w, phi, nrhs));
    pc.lap(4);
    LQCD_TRY(blas_axpy(c, 2 * nf * nrhs, 1.0, 0, (const double *)u, (double *)phi));
    pc.lap(5);
    return LQCD_OK;
}

extern "C" {

lqcd_status lqcd_dfl_build(lqcd_ctx *c, const lqcd_dfl_params *p, const double *v0)
{
    if (!c || !p || !v0) return set_err(c, LQCD_ERR_ARG, "null argument");
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    if (p->Ns < 1 || p->Ns > NS_MAX) return set_err(c, LQCD_ERR_ARG, "Ns=%d (1..%d)", p->Ns, NS_MAX);
    if (p->prec != LQCD_F64 && p->prec != LQCD_F32) return set_err(c, LQCD_ERR_ARG, "subspace precision");
    if (p->coarse_prec == LQCD_F32 && !(p->coarse_tol >= 1e-6))
        return set_err(c, LQCD_ERR_ARG, "coarse_tol %g below 1e-6 with the FP32 little operator", p->coarse_tol);
    DBlk B;
    B.vol = 1;
    B.nblk = 1;
    for (int i = 0; i < 4; i++) {
        if (p->bs[i] <= 0 || p->bs[i] % 2 || c->g.L[i] % p->bs[i])
            return set_err(c, LQCD_ERR_ARG, "deflation block %d does not tile L[%d]", p->bs[i], i);
        B.bs[i] = p->bs[i];
        B.nb[i] = c->g.L[i] / p->bs[i];
        B.wrap[i] = B.nb[i] == 1;
        B.vol *= p->bs[i];
        B.nblk *= B.nb[i];
    }
    if (B.vol > 1024 || B.vol % 32) return set_err(c, LQCD_ERR_ARG, "deflation block volume %d", B.vol);
    dfl_free(c);
    DflState *d = new DflState();
    d->B = B;
    d->Ns = p->Ns;
    d->prec = p->prec;
    d->params = *p;
    if (d->params.coarse_nkv <= 0) d->params.coarse_nkv = 16;
    if (d->params.coarse_nmx <= 0) d->params.coarse_nmx = 4096;
    if (!(d->params.coarse_tol > 0)) d->params.coarse_tol = 1e-8;
    c->dfl = d;
    const long fe = field_elems(c, p->prec);
    const size_t fbytes = 2 * native_half_bytes(c, p->prec);
    if (cudaMalloc(&d->phi, fbytes * p->Ns) != cudaSuccess ||
        cudaMalloc(&d->Aint, (size_t)B.nblk * 9 * p->Ns * p->Ns * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&d->nbr, (size_t)B.nblk * 9 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        dfl_free(c);
        return set_err(c, LQCD_ERR_NOMEM, "deflation subspace allocation");
    }
    // neighbour table: entry 0 self, 1+2mu (+mu), 2+2mu (-mu)
    d->nbr_host.resize(9 * B.nblk);
    for (int b = 0; b < B.nblk; b++) {
        int bc[4], u = b;
        bc[3] = u % B.nb[3];
        u /= B.nb[3];
        bc[2] = u % B.nb[2];
        u /= B.nb[2];
        bc[1] = u % B.nb[1];
        bc[0] = u / B.nb[1];
        d->nbr_host[9 * b] = b;
        for (int mu = 0; mu < 4; mu++)
            for (int s = 0; s < 2; s++) {
                int e[4] = {bc[0], bc[1], bc[2], bc[3]};
                e[mu] = (e[mu] + (s == 0 ? 1 : -1) + B.nb[mu]) % B.nb[mu];
                d->nbr_host[9 * b + 1 + 2 * mu + s] = e[3] + B.nb[3] * (e[2] + B.nb[2] * (e[1] + B.nb[1] * e[0]));
            }
    }
    LQCD_CUDA_CHECK(c, cudaMemcpy(d->nbr, d->nbr_host.data(), 9 * B.nblk * sizeof(int), cudaMemcpyHostToDevice));
    // block colours for the even-odd little-Dirac solve
    d->eo = true;
    for (int mu = 0; mu < 4; mu++)
        if (B.nb[mu] < 2 || B.nb[mu] % 2) d->eo = false;
    if (d->eo) {
        std::vector<int> lst[2], pos(B.nblk);
        for (int b = 0; b < B.nblk; b++) {
            int u = b, sum = 0;
            for (int i = 3; i >= 0; i--) {
                sum += u % B.nb[i];
                u /= B.nb[i];
            }
            pos[b] = (int)lst[sum & 1].size();
            lst[sum & 1].push_back(b);
        }
        d->ncol[0] = (int)lst[0].size();
        d->ncol[1] = (int)lst[1].size();
        std::vector<int> all(lst[0]);
        all.insert(all.end(), lst[1].begin(), lst[1].end());
        std::vector<int> np(8 * (size_t)B.nblk);
        for (int i = 0; i < B.nblk; i++)
            for (int j = 0; j < 8; j++) np[8 * (size_t)i + j] = pos[d->nbr_host[9 * all[i] + 1 + j]];
        if (cudaMalloc(&d->blist, B.nblk * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&d->bpos, B.nblk * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&d->npos, 8 * (size_t)B.nblk * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            dfl_free(c);
            return set_err(c, LQCD_ERR_NOMEM, "deflation colour lists");
        }
        LQCD_CUDA_CHECK(c, cudaMemcpy(d->blist, all.data(), B.nblk * sizeof(int), cudaMemcpyHostToDevice));
        LQCD_CUDA_CHECK(c, cudaMemcpy(d->bpos, pos.data(), B.nblk * sizeof(int), cudaMemcpyHostToDevice));
        LQCD_CUDA_CHECK(c, cudaMemcpy(d->npos, np.data(), 8 * (size_t)B.nblk * sizeof(int), cudaMemcpyHostToDevice));
    }
    // start vectors: canonical FP64 -> native storage precision
    void *t64;
    LQCD_TRY(ws_get(c, WS_PACK_IN, 2 * native_half_bytes(c, LQCD_F64), &t64));
    for (int l = 0; l < p->Ns; l++) {
        LQCD_TRY(pack_field(c, LQCD_F64, 2, v0 + (size_t)l * 48 * c->g.Vh, t64, 1, false));
        LQCD_TRY(convert_native(c, LQCD_F64, p->prec, t64, (char *)d->phi + l * fbytes, 2));
    }
    // inverse iteration with SAP, normalised
    lqcd_sap_params sp;
    for (int i = 0; i < 4; i++) sp.bs[i] = p->bs[i];
    sp.ncy = p->ncy;
    sp.nmr = p->nmr;
    sp.prec = p->prec;
    void *tmp;
    LQCD_TRY(ws_get(c, WS_SAP_PSI, fbytes * p->Ns, &tmp));
    const bool half_sap = p->prec == LQCD_F32 && p->build_sap_prec == LQCD_F16S;
    void *h_in = nullptr, *h_out = tmp;   // an F16S field is smaller than an F32 one
    if (half_sap) {
        sp.prec = LQCD_F16S;
        LQCD_TRY(ws_get(c, WS_SAP_IN, 2 * native_half_bytes(c, LQCD_F16S) * p->Ns, &h_in));
    }
    for (int pass = 0; pass < p->ninv; pass++) {
        // all Ns vectors through one batched SAP application
        if (half_sap) {
            LQCD_TRY(convert_native(c, LQCD_F32, LQCD_F16S, d->phi, h_in, 2L * p->Ns));
            LQCD_TRY(sap_apply(c, &sp, h_in, h_out, p->Ns));
            LQCD_TRY(convert_native(c, LQCD_F16S, LQCD_F32, h_out, d->phi, 2L * p->Ns));
        } else {
            LQCD_TRY(sap_apply(c, &sp, d->phi, tmp, p->Ns));
            LQCD_CUDA_CHECK(c, cudaMemcpyAsync(d->phi, tmp, fbytes * p->Ns, cudaMemcpyDeviceToDevice, c->stream));
        }
        for (int l = 0; l < p->Ns; l++) {
            void *vl = (char *)d->phi + l * fbytes;
            double n2;
            LQCD_TRY(norm_native(c, p->prec, vl, 2, &n2));
            if (!(n2 > 0) || !std::isfinite(n2)) {
                dfl_free(c);
                return set_err(c, LQCD_ERR_BREAKDOWN, "subspace vector %d vanished", l);
            }
            LQCD_TRY(scale_native(c, p->prec, vl, 2, 1.0 / std::sqrt(n2)));
        }
    }
    // block Gram-Schmidt
    int *bad = (int *)c->red_out;
    LQCD_CUDA_CHECK(c, cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    size_t sm = (2 * 32 * 2 + 4) * sizeof(double);
    if (p->prec == LQCD_F64)
        k_block_gs<double2><<<B.nblk, B.vol, sm, c->stream>>>(c->g, B, (double2 *)d->phi, p->Ns, fe, bad);
    else
        k_block_gs32<<<B.nblk, B.vol, (2 * RCHUNK * 32 + 2 * NS_MAX + 2) * sizeof(double), c->stream>>>(
            c->g, B, (float4 *)d->phi, p->Ns, fe, bad);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    int hbad = 0;
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    if (hbad) {
        dfl_free(c);
        return set_err(c, LQCD_ERR_BREAKDOWN, "block Gram-Schmidt: %d dependent block vectors", hbad);
    }
    // little Dirac operator
    size_t sm2 = (2 * RCHUNK * 32 + 2 * RCHUNK) * sizeof(double);
    dim3 grid(B.nblk, p->Ns);
    if (p->prec == LQCD_F64)
        k_little_build<double2><<<grid, B.vol, sm2, c->stream>>>(c->g, B, (const double2 *)d->phi, p->Ns, fe,
                                                                c->U64, c->A64[0], c->A64[1], d->Aint);
    else
        k_little_build32<<<grid, B.vol, sm2, c->stream>>>(c->g, B, (const float4 *)d->phi, p->Ns, fe, c->U32,
                                                          c->A32[0], c->A32[1], d->Aint);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    // block-Jacobi preconditioner of the coarse solve: inverses of the diagonal blocks
    if (cudaMalloc(&d->Dinv, (size_t)B.nblk * p->Ns * p->Ns * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        dfl_free(c);
        return set_err(c, LQCD_ERR_NOMEM, "coarse preconditioner allocation");
    }
    const size_t per_warp = 2 * (size_t)p->Ns * p->Ns * sizeof(double2);
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, (40 * 1024) / per_warp));
    LQCD_CUDA_CHECK(c, cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    k_block_inverse<<<div_up(B.nblk, warps), 32 * warps, warps * per_warp, c->stream>>>(B.nblk, p->Ns, d->Aint,
                                                                                       d->Dinv, bad);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    if (hbad) {
        dfl_free(c);
        return set_err(c, LQCD_ERR_BREAKDOWN, "little Dirac operator: %d singular diagonal blocks", hbad);
    }
    if (p->coarse_prec == LQCD_F32) {
        const long na = (long)B.nblk * 9 * p->Ns * p->Ns, nd = (long)B.nblk * p->Ns * p->Ns;
        if (cudaMalloc(&d->Aint32, na * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&d->Dinv32, nd * sizeof(float2)) != cudaSuccess) {
            cudaGetLastError();
            dfl_free(c);
            return set_err(c, LQCD_ERR_NOMEM, "FP32 little operator allocation");
        }
        k_to_float2<<<div_up(na, 256), 256, 0, c->stream>>>(na, d->Aint, d->Aint32);
        k_to_float2<<<div_up(nd, 256), 256, 0, c->stream>>>(nd, d->Dinv, d->Dinv32);
        c->n_kernel_launches += 2;
        LQCD_LAUNCH_CHECK(c);
        if (d->eo && p->coarse_eo && p->Ns <= 32) {
            if (cudaMalloc(&d->AT32, (na - nd) * sizeof(float2)) != cudaSuccess ||
                cudaMalloc(&d->DT32, nd * sizeof(float2)) != cudaSuccess) {
                cudaGetLastError();
                dfl_free(c);
                return set_err(c, LQCD_ERR_NOMEM, "FP32 little operator allocation");
            }
            k_coarse_transpose<<<div_up(na, 256), 256, 0, c->stream>>>(B.nblk, p->Ns, d->Aint, d->Dinv, d->AT32,
                                                                       d->DT32);
            c->n_kernel_launches++;
            LQCD_LAUNCH_CHECK(c);
        }
    } else if (p->coarse_prec != LQCD_F64) {
        dfl_free(c);
        return set_err(c, LQCD_ERR_ARG, "coarse precision %d", (int)p->coarse_prec);
    }
    return LQCD_OK;
}

lqcd_status lqcd_dfl_export(lqcd_ctx *c, double *phi, double *A)
{
    if (!c) return LQCD_ERR_ARG;
    DflState *d = c->dfl;
    if (!d) return set_err(c, LQCD_ERR_STATE, "no subspace");
    const size_t fb = 2 * native_half_bytes(c, d->prec);
    if (phi) {
        void *t64;
        LQCD_TRY(ws_get(c, WS_PACK_OUT, 2 * native_half_bytes(c, LQCD_F64), &t64));
        for (int l = 0; l < d->Ns; l++) {
            LQCD_TRY(convert_native(c, d->prec, LQCD_F64, (char *)d->phi + l * fb, t64, 2));
            LQCD_TRY(pack_field(c, LQCD_F64, 2, phi + (size_t)l * 48 * c->g.Vh, t64, 1, true));
        }
    }
    if (A) {
        // the internal layout [b][j][k][l] is the exported one
        size_t n = (size_t)d->B.nblk * 9 * d->Ns * d->Ns;
        LQCD_CUDA_CHECK(c, cudaMemcpyAsync(A, d->Aint, n * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    }
    return LQCD_OK;
}

lqcd_status lqcd_dfl_project(lqcd_ctx *c, const double *in, double *cv)
{
    if (!c || !in || !cv) return set_err(c, LQCD_ERR_ARG, "null argument");
    if (!c->dfl) return set_err(c, LQCD_ERR_STATE, "no subspace");
    void *t;
    LQCD_TRY(ws_get(c, WS_PACK_IN, 2 * native_half_bytes(c, LQCD_F64), &t));
    LQCD_TRY(pack_field(c, LQCD_F64, 2, in, t, 1, false));
    return project(c, (const double2 *)t, (double2 *)cv);
}

lqcd_status lqcd_dfl_expand(lqcd_ctx *c, const double *cv, double *out)
{
    if (!c || !cv || !out) return set_err(c, LQCD_ERR_ARG, "null argument");
    if (!c->dfl) return set_err(c, LQCD_ERR_STATE, "no subspace");
    void *t;
    LQCD_TRY(ws_get(c, WS_PACK_OUT, 2 * native_half_bytes(c, LQCD_F64), &t));
    LQCD_TRY(expand(c, (const double2 *)cv, (double2 *)t));
    return pack_field(c, LQCD_F64, 2, out, t, 1, true);
}

lqcd_status lqcd_dfl_little_apply(lqcd_ctx *c, const double *cv, double *out)
{
    if (!c || !cv || !out) return set_err(c, LQCD_ERR_ARG, "null argument");
    if (!c->dfl) return set_err(c, LQCD_ERR_STATE, "no subspace");
    return little_apply(c, (const double2 *)cv, (double2 *)out);
}

lqcd_status lqcd_dfl_coarse_solve(lqcd_ctx *c, const double *b, double *x, int *iters)
{
    if (!c || !b || !x) return set_err(c, LQCD_ERR_ARG, "null argument");
    if (!c->dfl) return set_err(c, LQCD_ERR_STATE, "no subspace");
    DflState *d = c->dfl;
    return coarse_gcr(c, (const double2 *)b, (double2 *)x, 1, d->params.coarse_tol, d->params.coarse_nkv,
                      d->params.coarse_nmx, iters);
}

lqcd_status lqcd_dfl_stats(const lqcd_ctx *c, long *coarse_solves, long *coarse_iters)
{
    if (!c) return LQCD_ERR_ARG;
    if (!c->dfl) return LQCD_ERR_STATE;
    if (coarse_solves) *coarse_solves = c->dfl->coarse_solves;
    if (coarse_iters) *coarse_iters = c->dfl->coarse_iters;
    return LQCD_OK;
}

lqcd_status lqcd_dfl_precond(lqcd_ctx *c, const lqcd_sap_params *sp, const double *rho, double *phi)
{
    if (!c || !sp || !rho || !phi) return set_err(c, LQCD_ERR_ARG, "null argument");
    if (!c->dfl) return set_err(c, LQCD_ERR_STATE, "no subspace");
    size_t fb = 2 * native_half_bytes(c, LQCD_F64);
    void *a, *b;
    LQCD_TRY(ws_get(c, WS_PACK_IN, fb, &a));
    LQCD_TRY(ws_get(c, WS_PACK_OUT, fb, &b));
    LQCD_TRY(pack_field(c, LQCD_F64, 2, rho, a, 1, false));
    LQCD_TRY(dfl_precond_native(c, sp, (const double2 *)a, (double2 *)b, 1));
    return pack_field(c, LQCD_F64, 2, phi, b, 1, true);
}

}  // extern "C"
