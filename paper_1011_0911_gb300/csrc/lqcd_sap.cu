// Schwarz alternating procedure (the Schwarz preconditioner of the GCR solver
// named in Sec. 3-4).  The lattice is tiled by bs0 x bs1 x bs2 x bs3 blocks,
// coloured by the parity of their block coordinates.  One sweep over a colour
// solves D_blk chi = r on every block of that colour approximately and adds
// chi to psi; the residual r = eta - D psi is then recomputed.
//
// Block solve (one CTA per block, all block vectors in shared memory):
//   b_e = r_e - H_eo,blk A_oo^-1 r_o
//   nmr MinRes steps on Dhat_blk = A_ee - H_eo,blk A_oo^-1 H_oe,blk from 0:
//       p = Dhat_blk rho, alpha = <p,rho>/<p,p>, chi_e += alpha rho, rho -= alpha p
//   chi_o = A_oo^-1 (r_o - H_oe,blk chi_e)
// H_blk keeps only hops whose both ends lie in the block (Dirichlet); a block
// that spans a whole lattice direction keeps the wrapped hop of that direction.
#include <algorithm>
#include <list>
#include <type_traits>
#include <vector>

#include "lqcd_f16s.cuh"
#include "lqcd_internal.cuh"
#include "lqcd_stencil.cuh"
#include "lqcd_tune.h"

namespace {

struct BlkGeom {
    int bs[4];
    int nb[4];
    int nh;          // sites of one parity per block
    int bs3h;
    int wrap[4];     // block spans the whole direction
};

// storage per precision tag: arithmetic type, spinor unit, link and clover
// element types, and the length of one native half field in spinor units
template <int P>
struct SapT;
template <>
struct SapT<LQCD_F64> {
    using R = double;
    using SP = double2;
    using LK = double2;
    using CL = double2;
    static __host__ __device__ long half(long Vh) { return 12 * Vh; }
};
template <>
struct SapT<LQCD_F32> {
    using R = float;
    using SP = float4;
    using LK = float4;
    using CL = float4;
    static __host__ __device__ long half(long Vh) { return 6 * Vh; }
};
template <>
struct SapT<LQCD_F16S> {
    using R = float;
    using SP = h16s;
    using LK = uint2;
    using CL = uint2;
    static __host__ __device__ long half(long Vh) { return f16s_half_units(Vh); }
};

// global native accessors (duplicated minimal forms of the stencil loaders)
__device__ __forceinline__ void gload(const double2 *f, long Vh, long r, cx<double> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) {
        double2 t = f[c * Vh + r];
        v[c] = mk(t.x, t.y);
    }
}
__device__ __forceinline__ void gload(const float4 *f, long Vh, long r, cx<float> v[12])
{
#pragma unroll
    for (int q = 0; q < 6; q++) {
        float4 t = f[q * Vh + r];
        v[2 * q] = mk(t.x, t.y);
        v[2 * q + 1] = mk(t.z, t.w);
    }
}
__device__ __forceinline__ void gadd(double2 *f, long Vh, long r, const cx<double> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) {
        double2 t = f[c * Vh + r];
        f[c * Vh + r] = make_double2(t.x + v[c].re, t.y + v[c].im);
    }
}
__device__ __forceinline__ void gadd(float4 *f, long Vh, long r, const cx<float> v[12])
{
#pragma unroll
    for (int q = 0; q < 6; q++) {
        float4 t = f[q * Vh + r];
        f[q * Vh + r] = make_float4(t.x + v[2 * q].re, t.y + v[2 * q].im, t.z + v[2 * q + 1].re,
                                    t.w + v[2 * q + 1].im);
    }
}
__device__ __forceinline__ void glink(const double2 *U, long Vh, int p, int mu, long r, cx<double> u[3][3])
{
    const double2 *b = U + (long)((p * 4 + mu) * 9) * Vh + r;
#pragma unroll
    for (int e = 0; e < 9; e++) {
        double2 t = __ldg(b + e * Vh);
        u[e / 3][e % 3] = mk(t.x, t.y);
    }
}
__device__ __forceinline__ void glink(const float4 *U, long Vh, int p, int mu, long r, cx<float> u[3][3])
{
    const float4 *b = U + (long)((p * 4 + mu) * 3) * Vh + r;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        float4 t = __ldg(b + q * Vh);
        u[(2 * q) / 3][(2 * q) % 3] = mk(t.x, t.y);
        u[(2 * q + 1) / 3][(2 * q + 1) % 3] = mk(t.z, t.w);
    }
    su3_third_row(u);
}
__device__ __forceinline__ void gload(const h16s *f, long Vh, long r, cx<float> v[12]) { f16s_load<false>(f, Vh, r, v); }
__device__ __forceinline__ void gadd(h16s *f, long Vh, long r, const cx<float> v[12])
{
    cx<float> t[12];
    f16s_load<false>(f, Vh, r, t);
#pragma unroll
    for (int c = 0; c < 12; c++) t[c] = t[c] + v[c];
    f16s_store(f, Vh, r, t);
}
__device__ __forceinline__ void glink(const uint2 *U, long Vh, int p, int mu, long r, cx<float> u[3][3])
{
    f16s_link(U, Vh, p, mu, r, u);
}
__device__ __forceinline__ void gclov(const uint2 *A, long Vh, long r, int blk, float d[6], cx<float> o[15])
{
    float v[36];
    f16s_clover(A, Vh, r, blk, v);
#pragma unroll
    for (int i = 0; i < 6; i++) d[i] = v[i];
#pragma unroll
    for (int i = 0; i < 15; i++) o[i] = mk(v[6 + 2 * i], v[7 + 2 * i]);
}
__device__ __forceinline__ void gclov(const double2 *A, long Vh, long r, int blk, double d[6], cx<double> o[15])
{
    const double2 *b = A + (long)(18 * blk) * Vh + r;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        double2 t = __ldg(b + i * Vh);
        d[2 * i] = t.x;
        d[2 * i + 1] = t.y;
    }
#pragma unroll
    for (int i = 0; i < 15; i++) {
        double2 t = __ldg(b + (3 + i) * Vh);
        o[i] = mk(t.x, t.y);
    }
}
__device__ __forceinline__ void gclov(const float4 *A, long Vh, long r, int blk, float d[6], cx<float> o[15])
{
    const float4 *b = A + (long)(9 * blk) * Vh + r;
    float v[36];
#pragma unroll
    for (int q = 0; q < 9; q++) {
        float4 t = __ldg(b + q * Vh);
        v[4 * q] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
#pragma unroll
    for (int i = 0; i < 6; i++) d[i] = v[i];
#pragma unroll
    for (int i = 0; i < 15; i++) o[i] = mk(v[6 + 2 * i], v[7 + 2 * i]);
}

// w = H v for a packed Hermitian 6x6 block (diagonal d, upper entries o),
// every product entering its sum through a fused multiply-add
template <class R>
__device__ __forceinline__ void herm6_apply(const R d[6], const cx<R> o[15], const cx<R> v[6], cx<R> w[6])
{
    stencil::Herm6<R> h;
#pragma unroll
    for (int i = 0; i < 6; i++) h.d[i] = d[i];
#pragma unroll
    for (int i = 0; i < 15; i++) h.o[i] = o[i];
    stencil::herm_apply(h, v, w);
}

template <class R, class CL>
__device__ __forceinline__ void clov_apply(const CL *A, long Vh, long r, const cx<R> in[12], cx<R> out[12])
{
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        R d[6];
        cx<R> o[15];
        gclov(A, Vh, r, blk, d, o);
        herm6_apply(d, o, in + 6 * blk, out + 6 * blk);
    }
}

// shared-memory block field: component-major [12][nh] complex
template <class R>
__device__ __forceinline__ void sload(const cx<R> *s, int nh, int t, cx<R> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) v[c] = s[c * nh + t];
}
template <class R>
__device__ __forceinline__ void sstore(cx<R> *s, int nh, int t, const cx<R> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) s[c * nh + t] = v[c];
}

// projected hop term of direction mu and sense d from the block-local field
// src (opposite parity), accumulated into acc (before the -1/2 factor).
// v = psi[spin][colour] as v[3*spin + colour].
template <class R>
__device__ __forceinline__ void proj_apply(int mu, int sgn, const cx<R> psi[12], const cx<R> u[3][3], bool dag,
                                           R sign, cx<R> acc[12])
{
    cx<R> h[2][3], w[2][3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cx<R> u0 = psi[c], u1 = psi[3 + c], l0 = psi[6 + c], l1 = psi[9 + c];
        cx<R> el0, el1;  // e_mu l
        switch (mu) {
            case 0: el0 = -l0; el1 = -l1; break;
            case 1: el0 = timesmI(l1); el1 = timesmI(l0); break;
            case 2: el0 = -l1; el1 = l0; break;
            default: el0 = timesmI(l0); el1 = timesI(l1); break;
        }
        if (sgn < 0) {
            h[0][c] = u0 - el0;
            h[1][c] = u1 - el1;
        } else {
            h[0][c] = u0 + el0;
            h[1][c] = u1 + el1;
        }
    }
#pragma unroll
    for (int s = 0; s < 2; s++) {
        if (!dag)
            stencil::su3_vec(u, h[s], w[s]);
        else
            stencil::su3dag_vec(u, h[s], w[s]);
    }
    // acc += sign (w ; -+ e_mu^dag w), the boundary sign (+-1) folded into
    // fused multiply-adds
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cx<R> a, b;  // e_mu^dag w
        switch (mu) {
            case 0: a = -w[0][c]; b = -w[1][c]; break;
            case 1: a = timesI(w[1][c]); b = timesI(w[0][c]); break;
            case 2: a = w[1][c]; b = -w[0][c]; break;
            default: a = timesI(w[0][c]); b = timesmI(w[1][c]); break;
        }
        if (sgn < 0) {
            a = -a;
            b = -b;
        }
        acc[c].re = fmx(sign, w[0][c].re, acc[c].re);
        acc[c].im = fmx(sign, w[0][c].im, acc[c].im);
        acc[3 + c].re = fmx(sign, w[1][c].re, acc[3 + c].re);
        acc[3 + c].im = fmx(sign, w[1][c].im, acc[3 + c].im);
        acc[6 + c].re = fmx(sign, a.re, acc[6 + c].re);
        acc[6 + c].im = fmx(sign, a.im, acc[6 + c].im);
        acc[9 + c].re = fmx(sign, b.re, acc[9 + c].re);
        acc[9 + c].im = fmx(sign, b.im, acc[9 + c].im);
    }
}

struct SiteInfo {
    long grank;     // global rank
    int x[4];       // global coordinates
    int l[4];       // block-local coordinates
};

__device__ __forceinline__ void block_site(const Geom &g, const BlkGeom &B, const int org[4], int par, int t,
                                           SiteInfo &s)
{
    int row = t / B.bs3h;
    int x3h = t - row * B.bs3h;
    int tt = row / B.bs[2];
    s.l[2] = row - tt * B.bs[2];
    s.l[0] = tt / B.bs[1];
    s.l[1] = tt - s.l[0] * B.bs[1];
    int b = (par + s.l[0] + s.l[1] + s.l[2]) & 1;   // block origin has even parity
    s.l[3] = 2 * x3h + b;
    for (int i = 0; i < 4; i++) s.x[i] = org[i] + s.l[i];
    s.grank = coords_rank(g, s.x);
}

// local rank of the in-block neighbour l + d mu, or -1 if it leaves the block
__device__ __forceinline__ int blk_nbr(const BlkGeom &B, const int l[4], int mu, int d)
{
    int m[4] = {l[0], l[1], l[2], l[3]};
    int v = m[mu] + d;
    if (v < 0 || v >= B.bs[mu]) {
        if (!B.wrap[mu]) return -1;
        v = v < 0 ? v + B.bs[mu] : v - B.bs[mu];
    }
    m[mu] = v;
    return (m[3] + B.bs[3] * (m[2] + B.bs[2] * (m[1] + B.bs[1] * m[0]))) >> 1;
}

// acc = sum of the 8 in-block projected hops of src (parity 1-par) at site s (parity par)
template <class R, class LK>
__device__ void block_hopsum(const Geom &g, const BlkGeom &B, const LK *U, int par, const SiteInfo &s,
                             const cx<R> *src, cx<R> acc[12])
{
#pragma unroll
    for (int i = 0; i < 12; i++) acc[i] = mk(R(0), R(0));
    cx<R> u[3][3], v[12];
    for (int mu = 0; mu < 4; mu++) {
        int lf = blk_nbr(B, s.l, mu, +1);
        if (lf >= 0) {
            R sg = (mu == 0 && s.x[0] == g.L[0] - 1) ? R(g.bc_t) : R(1);
            glink(U, g.Vh, par, mu, s.grank, u);
            sload(src, B.nh, lf, v);
            proj_apply<R>(mu, -1, v, u, false, sg, acc);
        }
        int lb = blk_nbr(B, s.l, mu, -1);
        if (lb >= 0) {
            R sg = (mu == 0 && s.x[0] == 0) ? R(g.bc_t) : R(1);
            int y[4] = {s.x[0], s.x[1], s.x[2], s.x[3]};
            y[mu] = y[mu] == 0 ? g.L[mu] - 1 : y[mu] - 1;
            glink(U, g.Vh, 1 - par, mu, coords_rank(g, y), u);
            sload(src, B.nh, lb, v);
            proj_apply<R>(mu, +1, v, u, true, sg, acc);
        }
    }
}

template <class R>
__device__ __forceinline__ void block_reduce2(R &a, R &b, R &c, R *red)
{
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) {
        red[3 * warp] = a;
        red[3 * warp + 1] = b;
        red[3 * warp + 2] = c;
    }
    __syncthreads();
    a = b = c = 0;
    for (int w = 0; w < nw; w++) {
        a += red[3 * w];
        b += red[3 * w + 1];
        c += red[3 * w + 2];
    }
}

template <int P>
struct SapArgs {
    Geom g;
    BlkGeom B;
    const int *blocks;   // block ids of this colour
    typename SapT<P>::SP *r;        // native full fields (residual; the block's part is replaced)
    typename SapT<P>::SP *psi;      // native full fields (updated)
    typename SapT<P>::SP *delta;    // native full fields: chi of the blocks of this colour
    long fstride;                    // spinor units between the fields of consecutive right-hand sides
    const typename SapT<P>::LK *U;
    const typename SapT<P>::CL *Ae, *Aio;   // A on even sites, A^-1 on odd sites
    int nmr;
};

__device__ __forceinline__ void gstore(double2 *f, long Vh, long r, const cx<double> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) f[c * Vh + r] = make_double2(v[c].re, v[c].im);
}
__device__ __forceinline__ void gstore(float4 *f, long Vh, long r, const cx<float> v[12])
{
#pragma unroll
    for (int q = 0; q < 6; q++)
        f[q * Vh + r] = make_float4(v[2 * q].re, v[2 * q].im, v[2 * q + 1].re, v[2 * q + 1].im);
}
__device__ __forceinline__ void gstore(h16s *f, long Vh, long r, const cx<float> v[12]) { f16s_store(f, Vh, r, v); }

template <int P>
__global__ void __launch_bounds__(128) k_sap_block(SapArgs<P> a)
{
    using R = typename SapT<P>::R;
    using SP = typename SapT<P>::SP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BlkGeom &B = a.B;
    const int nh = B.nh;
    cx<R> *rho = (cx<R> *)smem_raw;
    cx<R> *chi = rho + 12 * nh;
    cx<R> *pv = chi + 12 * nh;
    cx<R> *to = pv + 12 * nh;
    cx<R> *ro = to + 12 * nh;
    R *red = (R *)(ro + 12 * nh);
    const long Vh = a.g.Vh;
    const long half = SapT<P>::half(Vh);
    const long foff = blockIdx.y * a.fstride;
    SP *r_e = a.r + foff, *r_o = a.r + foff + half;
    SP *psi_e = a.psi + foff, *psi_o = a.psi + foff + half;
    SP *d_e = a.delta + foff, *d_o = a.delta + foff + half;

    int bid = a.blocks[blockIdx.x];
    int org[4];
    {
        int t = bid;
        int c3 = t % B.nb[3];
        t /= B.nb[3];
        int c2 = t % B.nb[2];
        t /= B.nb[2];
        int c1 = t % B.nb[1];
        int c0 = t / B.nb[1];
        org[0] = c0 * B.bs[0];
        org[1] = c1 * B.bs[1];
        org[2] = c2 * B.bs[2];
        org[3] = c3 * B.bs[3];
    }
    cx<R> v[12], w[12];
    // r_o into smem, to = A_oo^-1 r_o
    for (int t = threadIdx.x; t < nh; t += blockDim.x) {
        SiteInfo s;
        block_site(a.g, B, org, 1, t, s);
        gload(r_o, Vh, s.grank, v);
        sstore(ro, nh, t, v);
        clov_apply<R>(a.Aio, Vh, s.grank, v, w);
        sstore(to, nh, t, w);
    }
    __syncthreads();
    // rho = b_e = r_e - H_eo,blk to  (H = -1/2 S)
    for (int t = threadIdx.x; t < nh; t += blockDim.x) {
        SiteInfo s;
        block_site(a.g, B, org, 0, t, s);
        gload(r_e, Vh, s.grank, v);
        block_hopsum<R>(a.g, B, a.U, 0, s, to, w);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            v[c] = v[c] + R(0.5) * w[c];
            chi[c * nh + t] = mk(R(0), R(0));
        }
        sstore(rho, nh, t, v);
    }
    __syncthreads();
    for (int it = 0; it < a.nmr; it++) {
        // to = A_oo^-1 H_oe,blk rho
        for (int t = threadIdx.x; t < nh; t += blockDim.x) {
            SiteInfo s;
            block_site(a.g, B, org, 1, t, s);
            block_hopsum<R>(a.g, B, a.U, 1, s, rho, w);
#pragma unroll
            for (int c = 0; c < 12; c++) w[c] = R(-0.5) * w[c];
            clov_apply<R>(a.Aio, Vh, s.grank, w, v);
            sstore(to, nh, t, v);
        }
        __syncthreads();
        // p = A_ee rho - H_eo,blk to
        R pp = 0, pr_re = 0, pr_im = 0;
        for (int t = threadIdx.x; t < nh; t += blockDim.x) {
            SiteInfo s;
            block_site(a.g, B, org, 0, t, s);
            cx<R> x[12];
            sload(rho, nh, t, x);
            clov_apply<R>(a.Ae, Vh, s.grank, x, v);
            block_hopsum<R>(a.g, B, a.U, 0, s, to, w);
#pragma unroll
            for (int c = 0; c < 12; c++) {
                v[c] = v[c] + R(0.5) * w[c];
                pp += v[c].re * v[c].re + v[c].im * v[c].im;
                pr_re += v[c].re * x[c].re + v[c].im * x[c].im;   // conj(p) rho
                pr_im += v[c].re * x[c].im - v[c].im * x[c].re;
            }
            sstore(pv, nh, t, v);
        }
        block_reduce2<R>(pp, pr_re, pr_im, red);
        if (pp == R(0)) break;   // rho = 0: the block is solved
        R ar = pr_re / pp, ai = pr_im / pp;
        cx<R> alpha = mk(ar, ai);
        for (int t = threadIdx.x; t < nh; t += blockDim.x) {
#pragma unroll
            for (int c = 0; c < 12; c++) {
                cx<R> rv = rho[c * nh + t];
                chi[c * nh + t] = chi[c * nh + t] + alpha * rv;
                rho[c * nh + t] = rv - alpha * pv[c * nh + t];
            }
        }
        __syncthreads();
    }
    // chi_o = A_oo^-1 (r_o - H_oe,blk chi_e); psi += chi; delta = chi.
    // The block's new residual r - D_blk chi is (rho, 0): on odd sites it vanishes
    // by construction of chi_o, on even sites it is the MinRes residual of
    // Dhat_blk chi_e = b_e.  Hops from chi into other blocks are applied by
    // k_sap_face_l afterwards.
    for (int t = threadIdx.x; t < nh; t += blockDim.x) {
        SiteInfo s;
        block_site(a.g, B, org, 1, t, s);
        block_hopsum<R>(a.g, B, a.U, 1, s, chi, w);
        sload(ro, nh, t, v);
#pragma unroll
        for (int c = 0; c < 12; c++) v[c] = v[c] + R(0.5) * w[c];
        clov_apply<R>(a.Aio, Vh, s.grank, v, w);
        gadd(psi_o, Vh, s.grank, w);
        gstore(d_o, Vh, s.grank, w);
#pragma unroll
        for (int c = 0; c < 12; c++) w[c] = mk(R(0), R(0));
        gstore(r_o, Vh, s.grank, w);
        SiteInfo se;
        block_site(a.g, B, org, 0, t, se);
        sload(chi, nh, t, v);
        gadd(psi_e, Vh, se.grank, v);
        gstore(d_e, Vh, se.grank, v);
        sload(rho, nh, t, v);
        gstore(r_e, Vh, se.grank, v);
    }
}

// ------------------------------------------------------------------------
// FP32 block solve with the whole block resident in shared memory.
//
// At the start of a block visit the CTA stages the block's forward links (two
// rows, all sites and directions), A_ee on its even sites, A_oo^-1 on its odd
// sites and r_o into shared memory with coalesced loads; all MinRes phases
// then run from shared memory.  Two threads per site: in a hop phase thread
// h = 0 sums the four forward hops and h = 1 the four backward hops, the pair
// exchanges its partial sums by a lane shuffle, and each thread then applies
// one chirality block (spins 2h, 2h+1) of the clover term.  Same arithmetic
// as k_sap_block, different summation order.
constexpr int SAPS_NH = 128;   // sites of one parity per block (4^4 blocks)

// Shared memory of the resident block kernel.  SA: the clover term of the
// block is staged too (172 KB, one CTA per SM); without it every clover
// application reads its 6x6 block through L1/L2 (same values) and two FP32
// CTAs (98 KB) or three F16S CTAs (74 KB: the links kept in FP16, the
// precision they are stored in) fit on an SM.  The MinRes correction chi stays
// in registers (each thread owns its half-site) and goes through p at the end.
// staging loads: one 4-real word of a link row pair or of the clover term
__device__ __forceinline__ float4 stage4(const float4 *p) { return __ldg(p); }
__device__ __forceinline__ float4 stage4(const uint2 *p)
{
    uint2 t = __ldg(p);
    cx<float> a = f16s_h2c(t.x, 1.f), b = f16s_h2c(t.y, 1.f);
    return make_float4(a.re, a.im, b.re, b.im);
}
__device__ __forceinline__ void stage_link(float4 &d, const float4 *p) { d = __ldg(p); }
__device__ __forceinline__ void stage_link(float4 &d, const uint2 *p) { d = stage4(p); }
__device__ __forceinline__ void stage_link(uint2 &d, const uint2 *p) { d = __ldg(p); }
__device__ __forceinline__ float4 link4(float4 v) { return v; }
__device__ __forceinline__ float4 link4(uint2 t)
{
    cx<float> a = f16s_h2c(t.x, 1.f), b = f16s_h2c(t.y, 1.f);
    return make_float4(a.re, a.im, b.re, b.im);
}
struct SapSmemA {
    float4 U[4][3][2 * SAPS_NH];   // forward links, two rows, site par * SAPS_NH + t
    float4 A[18][2 * SAPS_NH];     // A (even sites) or A^-1 (odd sites), site par * SAPS_NH + t
    float4 rho[6][SAPS_NH], p[6][SAPS_NH], to[6][SAPS_NH], ro[6][SAPS_NH];
    float red[3][8];
};
struct SapSmemL {
    float4 U[4][3][2 * SAPS_NH];
    float4 rho[6][SAPS_NH], p[6][SAPS_NH], to[6][SAPS_NH], ro[6][SAPS_NH];
    float red[3][8];
};
struct SapSmemH {
    uint2 U[4][3][2 * SAPS_NH];    // FP16 link rows
    float4 rho[6][SAPS_NH], p[6][SAPS_NH], to[6][SAPS_NH], ro[6][SAPS_NH];
    float red[3][8];
};
template <int P, bool SA>
using SapSmem = std::conditional_t<SA, SapSmemA, std::conditional_t<P == LQCD_F16S, SapSmemH, SapSmemL>>;
// resident CTAs per SM of each layout (the launch bounds)
template <int P, bool SA>
constexpr int sap_ctas() { return SA ? 1 : (P == LQCD_F16S ? 3 : 2); }

__device__ __forceinline__ int blk_lex(const BlkGeom &B, const int l[4])
{
    return l[3] + B.bs[3] * (l[2] + B.bs[2] * (l[1] + B.bs[1] * l[0]));
}

// local lexicographic index of the in-block neighbour l + d mu, or -1
__device__ __forceinline__ int blk_nbr_lex(const BlkGeom &B, const int l[4], int mu, int d)
{
    int m[4] = {l[0], l[1], l[2], l[3]};
    int v = m[mu] + d;
    if (v < 0 || v >= B.bs[mu]) {
        if (!B.wrap[mu]) return -1;
        v = v < 0 ? v + B.bs[mu] : v - B.bs[mu];
    }
    m[mu] = v;
    return blk_lex(B, m);
}

__device__ __forceinline__ void s_spinor(const float4 (*f)[SAPS_NH], int t, cx<float> v[12])
{
#pragma unroll
    for (int q = 0; q < 6; q++) {
        float4 a = f[q][t];
        v[2 * q] = mk(a.x, a.y);
        v[2 * q + 1] = mk(a.z, a.w);
    }
}
template <class SM>
__device__ __forceinline__ void s_link(const SM &S, int mu, int ls, cx<float> u[3][3])
{
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const float4 a = link4(S.U[mu][q][ls]);
        u[(2 * q) / 3][(2 * q) % 3] = mk(a.x, a.y);
        u[(2 * q + 1) / 3][(2 * q + 1) % 3] = mk(a.z, a.w);
    }
    su3_third_row(u);
}
// one chirality block h of the clover matrix applied to v[6]; the block is
// read from shared memory (local site ls) or from global memory (rank grank)
template <bool SA, class SM, class CL>
__device__ __forceinline__ void s_clover_half(const SM &S, int ls, const CL *A, long Vh, long grank, int h,
                                              const cx<float> v[6], cx<float> w[6])
{
    float a[36];
#pragma unroll
    for (int q = 0; q < 9; q++) {
        float4 t;
        if constexpr (SA)
            t = S.A[9 * h + q][ls];
        else
            t = stage4(A + (9 * h + q) * Vh + grank);
        a[4 * q] = t.x;
        a[4 * q + 1] = t.y;
        a[4 * q + 2] = t.z;
        a[4 * q + 3] = t.w;
    }
    stencil::Herm6<float> hm;
#pragma unroll
    for (int i = 0; i < 6; i++) hm.d[i] = a[i];
#pragma unroll
    for (int i = 0; i < 15; i++) hm.o[i] = mk(a[6 + 2 * i], a[7 + 2 * i]);
    stencil::herm_apply(hm, v, w);
}

// projected hop of direction mu in either sense with the sense a runtime value:
// sgn = -1 (forward, 1 - gamma_mu) or +1 (backward, 1 + gamma_mu), u already
// the matrix to apply (U or U^dag).  The arithmetic of proj_apply with the
// same sense: the signs enter as exact factors of fused multiply-adds, so the
// two threads of a site pair (one per sense) run one instruction stream.
template <int MU>
__device__ __forceinline__ void proj_apply_rt(float sgn, const cx<float> psi[12], const cx<float> u[3][3], float sign,
                                              cx<float> acc[12])
{
    cx<float> h[2][3], w[2][3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const cx<float> u0 = psi[c], u1 = psi[3 + c], l0 = psi[6 + c], l1 = psi[9 + c];
        cx<float> el0, el1;
        switch (MU) {
            case 0: el0 = -l0; el1 = -l1; break;
            case 1: el0 = timesmI(l1); el1 = timesmI(l0); break;
            case 2: el0 = -l1; el1 = l0; break;
            default: el0 = timesmI(l0); el1 = timesI(l1); break;
        }
        h[0][c] = mk(fmx(sgn, el0.re, u0.re), fmx(sgn, el0.im, u0.im));
        h[1][c] = mk(fmx(sgn, el1.re, u1.re), fmx(sgn, el1.im, u1.im));
    }
    stencil::su3_vec(u, h[0], w[0]);
    stencil::su3_vec(u, h[1], w[1]);
    const float ss = sign * sgn;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cx<float> a, b;
        switch (MU) {
            case 0: a = -w[0][c]; b = -w[1][c]; break;
            case 1: a = timesI(w[1][c]); b = timesI(w[0][c]); break;
            case 2: a = w[1][c]; b = -w[0][c]; break;
            default: a = timesI(w[0][c]); b = timesmI(w[1][c]); break;
        }
        acc[c].re = fmx(sign, w[0][c].re, acc[c].re);
        acc[c].im = fmx(sign, w[0][c].im, acc[c].im);
        acc[3 + c].re = fmx(sign, w[1][c].re, acc[3 + c].re);
        acc[3 + c].im = fmx(sign, w[1][c].im, acc[3 + c].im);
        acc[6 + c].re = fmx(ss, a.re, acc[6 + c].re);
        acc[6 + c].im = fmx(ss, a.im, acc[6 + c].im);
        acc[9 + c].re = fmx(ss, b.re, acc[9 + c].re);
        acc[9 + c].im = fmx(ss, b.im, acc[9 + c].im);
    }
}

// half of the in-block hop sum at site (l, x) from the smem field src of the
// other parity: h = 0 forward hops, h = 1 backward hops; then the pair's halves
// are added so both threads hold the full sum S (before the -1/2).  own: the
// site's index par * SAPS_NH + t in the link arrays; the neighbours' links sit
// at (1 - par) * SAPS_NH + their half index.  Both halves run the same
// instructions (the sense, the link slot and U versus U^dag are selected per
// lane), and a hop that leaves the block is computed with weight 0 from an
// in-block slot instead of being skipped, so the warp never diverges here.
template <class SM>
__device__ __forceinline__ void s_hopsum(const Geom &g, const BlkGeom &B, const SM &S, int h, const int l[4],
                                         const int x[4], int own, const float4 (*src)[SAPS_NH], cx<float> acc[12])
{
#pragma unroll
    for (int i = 0; i < 12; i++) acc[i] = mk(0.f, 0.f);
    const float sgn = h ? 1.f : -1.f;
    const int d = h ? -1 : 1;
    const int oth = own < SAPS_NH ? SAPS_NH : 0;
    const int xt = h ? 0 : g.L[0] - 1;
    cx<float> u[3][3], v[12];
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int ln = blk_nbr_lex(B, l, mu, d);
        const int n = ln >= 0 ? ln >> 1 : 0;
        float sg = (mu == 0 && x[0] == xt) ? float(g.bc_t) : 1.f;
        sg = ln >= 0 ? sg : 0.f;
        s_link(S, mu, h ? oth + n : own, u);
        cx<float> m[3][3];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int k = 0; k < 3; k++) m[a][k] = h ? mk(u[k][a].re, -u[k][a].im) : u[a][k];
        s_spinor(src, n, v);
        switch (mu) {
            case 0: proj_apply_rt<0>(sgn, v, m, sg, acc); break;
            case 1: proj_apply_rt<1>(sgn, v, m, sg, acc); break;
            case 2: proj_apply_rt<2>(sgn, v, m, sg, acc); break;
            default: proj_apply_rt<3>(sgn, v, m, sg, acc); break;
        }
    }
#pragma unroll
    for (int i = 0; i < 12; i++) {
        acc[i].re += __shfl_xor_sync(0xffffffffu, acc[i].re, 16);
        acc[i].im += __shfl_xor_sync(0xffffffffu, acc[i].im, 16);
    }
}

// the chirality half h of a 12-component spinor (predicated select, no local memory)
__device__ __forceinline__ void s_half(const cx<float> acc[12], int h, cx<float> out[6])
{
#pragma unroll
    for (int i = 0; i < 6; i++) out[i] = h ? acc[6 + i] : acc[i];
}

__device__ __forceinline__ void stage_site(const float4 *f, long Vh, long r, float4 o[6])
{
#pragma unroll
    for (int q = 0; q < 6; q++) o[q] = f[q * Vh + r];
}
__device__ __forceinline__ void stage_site(const h16s *f, long Vh, long r, float4 o[6])
{
    cx<float> v[12];
    f16s_load<false>(f, Vh, r, v);
#pragma unroll
    for (int q = 0; q < 6; q++) o[q] = make_float4(v[2 * q].re, v[2 * q].im, v[2 * q + 1].re, v[2 * q + 1].im);
}
// chirality half h (components 6h .. 6h+5) of site r.  The F16S forms are
// called by both threads of a site pair (lanes l and l ^ 16) together: the
// pair agrees on the site's scale through a lane shuffle.
__device__ __forceinline__ void half_load(const float4 *f, long Vh, long r, int h, cx<float> v[6])
{
#pragma unroll
    for (int q = 0; q < 3; q++) {
        float4 a = f[(3 * h + q) * Vh + r];
        v[2 * q] = mk(a.x, a.y);
        v[2 * q + 1] = mk(a.z, a.w);
    }
}
__device__ __forceinline__ void half_store(float4 *f, long Vh, long r, int h, const cx<float> v[6])
{
#pragma unroll
    for (int q = 0; q < 3; q++) f[(3 * h + q) * Vh + r] = make_float4(v[2 * q].re, v[2 * q].im, v[2 * q + 1].re, v[2 * q + 1].im);
}
__device__ __forceinline__ void half_load(const h16s *f, long Vh, long r, int h, cx<float> v[6])
{
    // h = 0: components 0..3 (uint4 0) and 4, 5 (low half of uint4 1);
    // h = 1: components 6, 7 (high half of uint4 1) and 8..11 (uint4 2)
    const uint4 *q = reinterpret_cast<const uint4 *>(f);
    const float sc = f16s_scales(f, Vh)[r];
    const uint2 mid = reinterpret_cast<const uint2 *>(q + Vh + r)[h];
    const uint4 end = q[(h ? 2 : 0) * Vh + r];
    const cx<float> a0 = f16s_h2c(end.x, sc), a1 = f16s_h2c(end.y, sc), a2 = f16s_h2c(end.z, sc),
                    a3 = f16s_h2c(end.w, sc), m0 = f16s_h2c(mid.x, sc), m1 = f16s_h2c(mid.y, sc);
    v[0] = h ? m0 : a0;
    v[1] = h ? m1 : a1;
    v[2] = h ? a0 : a2;
    v[3] = h ? a1 : a3;
    v[4] = h ? a2 : m0;
    v[5] = h ? a3 : m1;
}
__device__ __forceinline__ void half_store(h16s *f, long Vh, long r, int h, const cx<float> v[6])
{
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 6; i++) m = fmaxf(m, fmaxf(fabsf(v[i].re), fabsf(v[i].im)));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
    const float inv = m > 0.f ? 1.f / m : 0.f;
    uint4 *q = reinterpret_cast<uint4 *>(f);
    const cx<float> e0 = h ? v[2] : v[0], e1 = h ? v[3] : v[1], e2 = h ? v[4] : v[2], e3 = h ? v[5] : v[3];
    const cx<float> m0 = h ? v[0] : v[4], m1 = h ? v[1] : v[5];
    q[(h ? 2 : 0) * Vh + r] = make_uint4(f16s_c2h(e0, inv), f16s_c2h(e1, inv), f16s_c2h(e2, inv), f16s_c2h(e3, inv));
    reinterpret_cast<uint2 *>(q + Vh + r)[h] = make_uint2(f16s_c2h(m0, inv), f16s_c2h(m1, inv));
    if (h == 0) f16s_scales(f, Vh)[r] = m;
}
template <class SP>
__device__ __forceinline__ void half_add(SP *f, long Vh, long r, int h, const cx<float> v[6])
{
    cx<float> t[6];
    half_load(f, Vh, r, h, t);
#pragma unroll
    for (int i = 0; i < 6; i++) t[i] = t[i] + v[i];
    half_store(f, Vh, r, h, t);
}

// block list entry bi of a.blocks, right-hand side rhs; blockDim.x = 2 nh
template <int P, bool SA>
__device__ __forceinline__ void sap_block_s_body(const SapArgs<P> &a, int bi, int rhs)
{
    using SP = typename SapT<P>::SP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SapSmem<P, SA> &S = *reinterpret_cast<SapSmem<P, SA> *>(smem_raw);
    const BlkGeom &B = a.B;
    const int nh = B.nh;
    const long Vh = a.g.Vh;
    const long half = SapT<P>::half(Vh);
    const long foff = rhs * a.fstride;
    SP *r_e = a.r + foff, *r_o = a.r + foff + half;
    SP *psi_e = a.psi + foff, *psi_o = a.psi + foff + half;
    SP *d_e = a.delta + foff, *d_o = a.delta + foff + half;
    int org[4];
    {
        int t = a.blocks[bi];
        int c3 = t % B.nb[3];
        t /= B.nb[3];
        int c2 = t % B.nb[2];
        t /= B.nb[2];
        int c1 = t % B.nb[1];
        int c0 = t / B.nb[1];
        org[0] = c0 * B.bs[0];
        org[1] = c1 * B.bs[1];
        org[2] = c2 * B.bs[2];
        org[3] = c3 * B.bs[3];
    }
    const int tid = threadIdx.x;
    // ---- stage links, clover and r_o (one thread per block site, both parities)
    for (int i = tid; i < 2 * nh; i += blockDim.x) {
        const int par = i >= nh, t = par ? i - nh : i;
        SiteInfo s;
        block_site(a.g, B, org, par, t, s);
        const int ls = par * SAPS_NH + t;
#pragma unroll
        for (int mu = 0; mu < 4; mu++)
#pragma unroll
            for (int q = 0; q < 3; q++) stage_link(S.U[mu][q][ls], a.U + ((long)(par * 4 + mu) * 3 + q) * Vh + s.grank);
        if constexpr (SA) {
            const typename SapT<P>::CL *A = par ? a.Aio : a.Ae;
#pragma unroll
            for (int q = 0; q < 18; q++) S.A[q][ls] = stage4(A + q * Vh + s.grank);
        }
        float4 site[6];
        stage_site(par ? r_o : r_e, Vh, s.grank, site);
        if (par) {
#pragma unroll
            for (int q = 0; q < 6; q++) S.ro[q][t] = site[q];
        } else {
#pragma unroll
            for (int q = 0; q < 6; q++) S.rho[q][t] = site[q];
        }
    }
    __syncthreads();
    // chirality half / hop direction h and site rank t: lanes 0-15 of a warp
    // take h = 0 of 16 sites, lanes 16-31 h = 1 of the same sites, so the 8
    // lanes of every quarter-warp read consecutive rows of one shared-memory
    // array (no bank conflicts between a site's two halves)
    const int h = (tid >> 4) & 1, t = ((tid >> 5) << 4) | (tid & 15);
    const bool act = t < nh;
    SiteInfo so, se;
    const int lso = SAPS_NH + t, lse = t;   // the sites' slots in the link / clover arrays
    if (act) {
        block_site(a.g, B, org, 1, t, so);
        block_site(a.g, B, org, 0, t, se);
    }
    cx<float> acc[12], v[6], w[6];
    float4 chi4[3];   // this thread's half of chi_e
#pragma unroll
    for (int q = 0; q < 3; q++) chi4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    // to = A_oo^-1 r_o (chirality half h)
    if (act) {
#pragma unroll
        for (int q = 0; q < 3; q++) {
            float4 x = S.ro[3 * h + q][t];
            v[2 * q] = mk(x.x, x.y);
            v[2 * q + 1] = mk(x.z, x.w);
        }
        s_clover_half<SA>(S, lso, a.Aio, Vh, so.grank, h, v, w);
#pragma unroll
        for (int q = 0; q < 3; q++) S.to[3 * h + q][t] = make_float4(w[2 * q].re, w[2 * q].im, w[2 * q + 1].re, w[2 * q + 1].im);
    }
    __syncthreads();
    // rho = r_e - H_eo to = r_e + 1/2 S
    if (act) {
        s_hopsum(a.g, B, S, h, se.l, se.x, lse, S.to, acc);
        cx<float> ah[6];
        s_half(acc, h, ah);
#pragma unroll
        for (int q = 0; q < 3; q++) {
            float4 x = S.rho[3 * h + q][t];
            const cx<float> s0 = ah[2 * q], s1 = ah[2 * q + 1];
            S.rho[3 * h + q][t] = make_float4(x.x + 0.5f * s0.re, x.y + 0.5f * s0.im, x.z + 0.5f * s1.re, x.w + 0.5f * s1.im);
        }
    }
    __syncthreads();
    for (int it = 0; it < a.nmr; it++) {
        // to = A_oo^-1 (-1/2 S(rho))
        if (act) {
            s_hopsum(a.g, B, S, h, so.l, so.x, lso, S.rho, acc);
            s_half(acc, h, v);
#pragma unroll
            for (int i = 0; i < 6; i++) v[i] = -0.5f * v[i];
            s_clover_half<SA>(S, lso, a.Aio, Vh, so.grank, h, v, w);
#pragma unroll
            for (int q = 0; q < 3; q++) S.to[3 * h + q][t] = make_float4(w[2 * q].re, w[2 * q].im, w[2 * q + 1].re, w[2 * q + 1].im);
        }
        __syncthreads();
        // p = A_ee rho + 1/2 S(to); partial <p,p>, <p,rho>
        float pp = 0.f, pr = 0.f, pi = 0.f;
        if (act) {
            s_hopsum(a.g, B, S, h, se.l, se.x, lse, S.to, acc);
            cx<float> x[6];
#pragma unroll
            for (int q = 0; q < 3; q++) {
                float4 y = S.rho[3 * h + q][t];
                x[2 * q] = mk(y.x, y.y);
                x[2 * q + 1] = mk(y.z, y.w);
            }
            s_clover_half<SA>(S, lse, a.Ae, Vh, se.grank, h, x, w);
            cx<float> ah[6];
            s_half(acc, h, ah);
#pragma unroll
            for (int i = 0; i < 6; i++) {
                w[i] = w[i] + 0.5f * ah[i];
                pp += w[i].re * w[i].re + w[i].im * w[i].im;
                pr += w[i].re * x[i].re + w[i].im * x[i].im;
                pi += w[i].re * x[i].im - w[i].im * x[i].re;
            }
#pragma unroll
            for (int q = 0; q < 3; q++) S.p[3 * h + q][t] = make_float4(w[2 * q].re, w[2 * q].im, w[2 * q + 1].re, w[2 * q + 1].im);
        }
        for (int o = 16; o > 0; o >>= 1) {
            pp += __shfl_down_sync(0xffffffffu, pp, o);
            pr += __shfl_down_sync(0xffffffffu, pr, o);
            pi += __shfl_down_sync(0xffffffffu, pi, o);
        }
        if ((tid & 31) == 0) {
            S.red[0][tid >> 5] = pp;
            S.red[1][tid >> 5] = pr;
            S.red[2][tid >> 5] = pi;
        }
        __syncthreads();
        pp = pr = pi = 0.f;
        for (int wv = 0; wv < (int)(blockDim.x >> 5); wv++) {
            pp += S.red[0][wv];
            pr += S.red[1][wv];
            pi += S.red[2][wv];
        }
        __syncthreads();
        if (pp == 0.f) break;   // rho = 0: the block is solved
        const float ar = pr / pp, ai = pi / pp;
        if (act) {
#pragma unroll
            for (int q = 0; q < 3; q++) {
                float4 rv = S.rho[3 * h + q][t], pv = S.p[3 * h + q][t], cv = chi4[q];
                // chi += alpha rho, rho -= alpha p
                cv.x += ar * rv.x - ai * rv.y;
                cv.y += ar * rv.y + ai * rv.x;
                cv.z += ar * rv.z - ai * rv.w;
                cv.w += ar * rv.w + ai * rv.z;
                rv.x -= ar * pv.x - ai * pv.y;
                rv.y -= ar * pv.y + ai * pv.x;
                rv.z -= ar * pv.z - ai * pv.w;
                rv.w -= ar * pv.w + ai * pv.z;
                chi4[q] = cv;
                S.rho[3 * h + q][t] = rv;
            }
        }
        __syncthreads();
    }
    // chi_o = A_oo^-1 (r_o + 1/2 S(chi_e)); psi += chi; delta = chi; r <- (rho, 0)
    // (chi_e goes to the block through p, which is free now)
    if (act)
#pragma unroll
        for (int q = 0; q < 3; q++) S.p[3 * h + q][t] = chi4[q];
    __syncthreads();
    if (act) {
        s_hopsum(a.g, B, S, h, so.l, so.x, lso, S.p, acc);
        cx<float> ah[6];
        s_half(acc, h, ah);
#pragma unroll
        for (int q = 0; q < 3; q++) {
            float4 x = S.ro[3 * h + q][t];
            v[2 * q] = mk(x.x + 0.5f * ah[2 * q].re, x.y + 0.5f * ah[2 * q].im);
            v[2 * q + 1] = mk(x.z + 0.5f * ah[2 * q + 1].re, x.w + 0.5f * ah[2 * q + 1].im);
        }
        s_clover_half<SA>(S, lso, a.Aio, Vh, so.grank, h, v, w);
        cx<float> ce[6], re[6], zero[6];
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const float4 c4 = chi4[q], r4 = S.rho[3 * h + q][t];
            ce[2 * q] = mk(c4.x, c4.y);
            ce[2 * q + 1] = mk(c4.z, c4.w);
            re[2 * q] = mk(r4.x, r4.y);
            re[2 * q + 1] = mk(r4.z, r4.w);
            zero[2 * q] = zero[2 * q + 1] = mk(0.f, 0.f);
        }
        half_add(psi_o, Vh, so.grank, h, w);
        half_store(d_o, Vh, so.grank, h, w);
        half_store(r_o, Vh, so.grank, h, zero);
        half_add(psi_e, Vh, se.grank, h, ce);
        half_store(d_e, Vh, se.grank, h, ce);
        half_store(r_e, Vh, se.grank, h, re);
    }
}

template <int P, bool SA>
__global__ void __launch_bounds__(2 * SAPS_NH, sap_ctas<P, SA>()) k_sap_block_s(SapArgs<P> a)
{
    sap_block_s_body<P, SA>(a, blockIdx.x, blockIdx.y);
}

// LQCD_SAP_STAGE_A = 0 | 1 forces the clover term through L1 or staged in
// shared memory (test instrumentation); otherwise the autotuner chooses.
// Returns -1 when not forced.
int sap_stage_forced()
{
    const char *e = getenv("LQCD_SAP_STAGE_A");
    if (!e || !*e) return -1;
    return e[0] == '1' ? 1 : 0;
}

// r(x) -= sum of the hops into x from neighbours y that lie in another block
// of colour col (delta holds chi there).  One thread per (site, rhs); i is the
// parity-major site index 0 .. V-1.
template <int P>
__device__ __forceinline__ void sap_face_body(const SapArgs<P> &a, int col, long i, int rhs)
{
    using R = typename SapT<P>::R;
    using SP = typename SapT<P>::SP;
    const BlkGeom &B = a.B;
    if (i >= 2L * a.g.Vh) return;
    const long Vh = a.g.Vh;
    const int par = i >= Vh;
    const long rk = par ? i - Vh : i;
    const long half = SapT<P>::half(Vh);
    const long foff = rhs * a.fstride;
    int x[4];
    rank_coords(a.g, par, (int)rk, x);
    int bx[4];
    for (int m = 0; m < 4; m++) bx[m] = x[m] / B.bs[m];
    cx<R> acc[12], u[3][3], v[12];
    bool any = false;
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = mk(R(0), R(0));
    const SP *din = a.delta + foff + (1 - par) * half;
    for (int mu = 0; mu < 4; mu++)
        for (int d = -1; d <= 1; d += 2) {
            int y[4] = {x[0], x[1], x[2], x[3]};
            int vv = y[mu] + d;
            y[mu] = vv < 0 ? vv + a.g.L[mu] : (vv >= a.g.L[mu] ? vv - a.g.L[mu] : vv);
            int by = y[mu] / B.bs[mu];
            if (by == bx[mu]) continue;   // same block (also covers a block spanning the direction)
            int csum = by - bx[mu];
            for (int m = 0; m < 4; m++) csum += bx[m];
            if ((csum & 1) != col) continue;
            long ry = coords_rank(a.g, y);
            gload(din, Vh, ry, v);
            if (d > 0) {
                R sg = (mu == 0 && x[0] == a.g.L[0] - 1) ? R(a.g.bc_t) : R(1);
                glink(a.U, Vh, par, mu, rk, u);
                proj_apply<R>(mu, -1, v, u, false, sg, acc);
            } else {
                R sg = (mu == 0 && x[0] == 0) ? R(a.g.bc_t) : R(1);
                glink(a.U, Vh, 1 - par, mu, ry, u);
                proj_apply<R>(mu, +1, v, u, true, sg, acc);
            }
            any = true;
        }
    if (!any) return;
    // r -= H delta = r + 1/2 S
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = R(0.5) * acc[c];
    gadd(a.r + foff + par * half, Vh, rk, acc);
}

// The update of sap_face_body driven by a precomputed list of the sites that receive hops
// from blocks of colour col: entry (i, mask) with i the parity-major site index
// and bit 2 mu + (d > 0) of mask set for each hop from x + d mu that enters
// from such a block.  The list is sorted by mask, so the threads of a warp
// take the same hops (the site-ordered form branches per site); the hops are
// those of sap_face_body in the same order, so the result is bitwise the same.
template <int P>
__global__ void __launch_bounds__(128) k_sap_face_l(SapArgs<P> a, const int2 *__restrict__ list, int n)
{
    using R = typename SapT<P>::R;
    using SP = typename SapT<P>::SP;
    const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int rhs = blockIdx.y;
    const int2 fs = list[e];
    const long Vh = a.g.Vh;
    const int par = fs.x >= Vh;
    const long rk = par ? fs.x - Vh : fs.x;
    const long half = SapT<P>::half(Vh);
    const long foff = rhs * a.fstride;
    int x[4];
    rank_coords(a.g, par, (int)rk, x);
    cx<R> acc[12], u[3][3], v[12];
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = mk(R(0), R(0));
    const SP *din = a.delta + foff + (1 - par) * half;
    for (int mu = 0; mu < 4; mu++)
        for (int d = -1; d <= 1; d += 2) {
            if (!((fs.y >> (2 * mu + (d > 0))) & 1)) continue;
            const long ry = nbr_rank(a.g, x, mu, d);
            gload(din, Vh, ry, v);
            if (d > 0) {
                R sg = (mu == 0 && x[0] == a.g.L[0] - 1) ? R(a.g.bc_t) : R(1);
                glink(a.U, Vh, par, mu, rk, u);
                proj_apply<R>(mu, -1, v, u, false, sg, acc);
            } else {
                R sg = (mu == 0 && x[0] == 0) ? R(a.g.bc_t) : R(1);
                glink(a.U, Vh, 1 - par, mu, ry, u);
                proj_apply<R>(mu, +1, v, u, true, sg, acc);
            }
        }
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = R(0.5) * acc[c];
    gadd(a.r + foff + par * half, Vh, rk, acc);
}

// ------------------------------------------------------------------ batches
// Several lattices in one launch.  args[2 l + col]: the SAP arguments of
// lattice l for the blocks of colour col.  Persistent CTAs take work items from
// a device counter (*queue, zero before the launch) until the list is empty;
// items of lattices whose active flag is 0 are skipped.
template <int P, bool SA>
__global__ void __launch_bounds__(2 * SAPS_NH, sap_ctas<P, SA>())
    k_sap_block_s_batch(const SapArgs<P> *args, int col, const int2 *items, int nitems, const int *active, int *queue)
{
    __shared__ int s_item;
    __shared__ SapArgs<P> sa;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) return;
        const int2 w = items[it];   // (lattice, index in its list of colour col)
        const bool on = !active || active[w.x];
        if (on && threadIdx.x == 0) sa = args[2 * w.x + col];
        __syncthreads();
        if (on) sap_block_s_body<P, SA>(sa, w.y, 0);
        __syncthreads();
    }
}

// face items: (lattice, first parity-major site of a 128-site tile)
template <int P>
__global__ void __launch_bounds__(128)
    k_sap_face_batch(const SapArgs<P> *args, int col, const int2 *items, int nitems, const int *active)
{
    const int2 w = items[blockIdx.x];
    if (active && !active[w.x]) return;
    __shared__ SapArgs<P> sa;
    if (threadIdx.x == 0) sa = args[2 * w.x + col];
    __syncthreads();
    sap_face_body<P>(sa, col, (long)w.y + threadIdx.x, 0);
}

// LQCD_SAP_GENERIC=1 selects the generic (L1-cached) FP32 block kernel
bool sap_force_generic()
{
    const char *e = getenv("LQCD_SAP_GENERIC");
    return e && e[0] == '1';
}

struct SapPlan {
    int bs[4] = {0, 0, 0, 0};
    int *blocks_dev = nullptr;   // [colour 0 ids..., colour 1 ids...]
    int count[2] = {0, 0};
    BlkGeom B;
    int2 *face_dev[2] = {nullptr, nullptr};   // sites updated after colour col (k_sap_face_l)
    int nface[2] = {0, 0};
};

// one cached plan per context (keyed by block shape)
struct PlanCache {
    lqcd_ctx *ctx;
    SapPlan plan;
};
std::list<PlanCache> g_plans;   // a list: pointers to its plans stay valid as it grows

lqcd_status get_plan(lqcd_ctx *c, const int bs[4], SapPlan **out)
{
    for (auto &pc : g_plans)
        if (pc.ctx == c && pc.plan.bs[0] == bs[0] && pc.plan.bs[1] == bs[1] && pc.plan.bs[2] == bs[2] &&
            pc.plan.bs[3] == bs[3]) {
            *out = &pc.plan;
            return LQCD_OK;
        }
    SapPlan P;
    int vol = 1;
    for (int i = 0; i < 4; i++) {
        if (bs[i] <= 0 || bs[i] % 2 || c->g.L[i] % bs[i])
            return set_err(c, LQCD_ERR_ARG, "block extent %d does not tile L[%d]=%d", bs[i], i, c->g.L[i]);
        P.bs[i] = bs[i];
        P.B.bs[i] = bs[i];
        P.B.nb[i] = c->g.L[i] / bs[i];
        P.B.wrap[i] = P.B.nb[i] == 1;
        vol *= bs[i];
    }
    if (vol / 2 > 1024) return set_err(c, LQCD_ERR_ARG, "SAP block of %d sites too large", vol);
    P.B.nh = vol / 2;
    P.B.bs3h = bs[3] / 2;
    std::vector<int> ids[2];
    for (int c0 = 0; c0 < P.B.nb[0]; c0++)
        for (int c1 = 0; c1 < P.B.nb[1]; c1++)
            for (int c2 = 0; c2 < P.B.nb[2]; c2++)
                for (int c3 = 0; c3 < P.B.nb[3]; c3++) {
                    int id = c3 + P.B.nb[3] * (c2 + P.B.nb[2] * (c1 + P.B.nb[1] * c0));
                    ids[(c0 + c1 + c2 + c3) & 1].push_back(id);
                }
    P.count[0] = (int)ids[0].size();
    P.count[1] = (int)ids[1].size();
    std::vector<int> all(ids[0]);
    all.insert(all.end(), ids[1].begin(), ids[1].end());
    LQCD_CUDA_CHECK(c, cudaMalloc(&P.blocks_dev, all.size() * sizeof(int)));
    LQCD_CUDA_CHECK(c, cudaMemcpy(P.blocks_dev, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice));
    // face lists: for each site, the hops that enter from a block of colour col
    // (a different block; both parities, parity-major index), sorted by hop mask
    {
        const int *L = c->g.L;
        const long Vh = c->g.Vh;
        std::vector<std::pair<int, int>> fl[2];   // (mask, index)
        int x[4];
        for (x[0] = 0; x[0] < L[0]; x[0]++)
            for (x[1] = 0; x[1] < L[1]; x[1]++)
                for (x[2] = 0; x[2] < L[2]; x[2]++)
                    for (x[3] = 0; x[3] < L[3]; x[3]++) {
                        const long lex = x[3] + (long)L[3] * (x[2] + (long)L[2] * (x[1] + (long)L[1] * x[0]));
                        const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
                        const int idx = (int)(par * Vh + (lex >> 1));
                        int bx[4], bsum = 0;
                        for (int m = 0; m < 4; m++) {
                            bx[m] = x[m] / bs[m];
                            bsum += bx[m];
                        }
                        int mask[2] = {0, 0};
                        for (int mu = 0; mu < 4; mu++)
                            for (int d = -1; d <= 1; d += 2) {
                                int y = x[mu] + d;
                                y = y < 0 ? y + L[mu] : (y >= L[mu] ? y - L[mu] : y);
                                const int by = y / bs[mu];
                                if (by == bx[mu]) continue;
                                mask[(bsum - bx[mu] + by) & 1] |= 1 << (2 * mu + (d > 0));
                            }
                        for (int col = 0; col < 2; col++)
                            if (mask[col]) fl[col].push_back({mask[col], idx});
                    }
        for (int col = 0; col < 2; col++) {
            std::sort(fl[col].begin(), fl[col].end());
            std::vector<int2> h(fl[col].size());
            for (size_t k = 0; k < h.size(); k++) h[k] = make_int2(fl[col][k].second, fl[col][k].first);
            P.nface[col] = (int)h.size();
            if (h.empty()) continue;
            LQCD_CUDA_CHECK(c, cudaMalloc(&P.face_dev[col], h.size() * sizeof(int2)));
            LQCD_CUDA_CHECK(c, cudaMemcpy(P.face_dev[col], h.data(), h.size() * sizeof(int2), cudaMemcpyHostToDevice));
        }
    }
    g_plans.push_back({c, P});
    *out = &g_plans.back().plan;
    return LQCD_OK;
}

template <int P>
lqcd_status sap_run(lqcd_ctx *c, const SapPlan &P_, int ncy, int nmr, const void *eta, void *psi, void *r,
                    void *delta, int nrhs)
{
    using T = SapT<P>;
    using R = typename T::R;
    using SP = typename T::SP;
    const SapPlan &Pl = P_;
    const size_t fb = 2 * native_half_bytes(c, (lqcd_prec)P);
    size_t smem = 5 * 12 * Pl.B.nh * sizeof(cx<R>) + 3 * 32 * sizeof(R);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_sap_block<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    if (smem > 200 * 1024) return set_err(c, LQCD_ERR_ARG, "SAP block needs %zu bytes of shared memory", smem);
    if (nrhs < 1 || nrhs > 65535) return set_err(c, LQCD_ERR_ARG, "SAP nrhs=%d", nrhs);
    LQCD_CUDA_CHECK(c, cudaMemsetAsync(psi, 0, fb * nrhs, c->stream));
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(r, eta, fb * nrhs, cudaMemcpyDeviceToDevice, c->stream));
    SapArgs<P> a;
    a.g = c->g;
    a.B = Pl.B;
    a.r = (SP *)r;
    a.psi = (SP *)psi;
    a.delta = (SP *)delta;
    a.fstride = 2 * T::half(c->g.Vh);
    if constexpr (P == LQCD_F64) {
        a.U = c->U64;
        a.Ae = c->A64[0];
        a.Aio = c->Ai64[1];
    } else if constexpr (P == LQCD_F32) {
        a.U = c->U32;
        a.Ae = c->A32[0];
        a.Aio = c->Ai32[1];
    } else {
        a.U = c->U16;
        a.Ae = c->A16[0];
        a.Aio = c->Ai16[1];
    }
    a.nmr = nmr;
    int threads = std::min(128, Pl.B.nh);
    // FP32 / F16S with blocks of <= 128 sites per parity (whole warps of site
    // pairs): the shared-memory resident kernel
    bool resident = false;
    if constexpr (P != LQCD_F64) {
        static bool attr_s = false;
        if (!attr_s) {
            cudaFuncSetAttribute(k_sap_block_s<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(SapSmem<P, true>));
            cudaFuncSetAttribute(k_sap_block_s<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(SapSmem<P, false>));
            attr_s = true;
        }
        resident = Pl.B.nh <= SAPS_NH && (2 * Pl.B.nh) % 32 == 0 && !sap_force_generic();
    }
    // clover term staged in shared memory (stage = 1, one CTA per SM) or read
    // through L1 (stage = 0): identical arithmetic, chosen by timing.  Without
    // a recorded choice the sweeps of this application alternate between the
    // two forms (in-flight tuning: every sweep is part of the result, so the
    // search costs no extra work) and the faster one is recorded.
    int stage = 0;
    bool tuning = false;
    std::string key;
    float best_us[2] = {1e30f, 1e30f};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (P != LQCD_F64 && resident) {
        const int forced = sap_stage_forced();
        if (forced >= 0) {
            stage = forced;
        } else {
            key = tune_key(c, (std::string("k_sap_block_s/b") + std::to_string(Pl.bs[0]) + "x" +
                               std::to_string(Pl.bs[1]) + "x" + std::to_string(Pl.bs[2]) + "x" +
                               std::to_string(Pl.bs[3])).c_str(),
                           0, P, nrhs);
            TuneChoice tc;
            if (tune_lookup(key, &tc)) {
                stage = tc.variant;
            } else if (tune_enabled() && ncy * (Pl.count[1] > 0 ? 2 : 1) >= 4) {
                tuning = true;
                LQCD_CUDA_CHECK(c, cudaEventCreate(&ev[0]));
                LQCD_CUDA_CHECK(c, cudaEventCreate(&ev[1]));
            }
        }
    }
    // the residual is not needed after the last sweep
    int last_col = Pl.count[1] > 0 ? 1 : 0;
    int sweep = 0;
    for (int cyc = 0; cyc < ncy; cyc++)
        for (int col = 0; col < 2; col++) {
            if (Pl.count[col] == 0) continue;
            a.blocks = Pl.blocks_dev + (col == 0 ? 0 : Pl.count[0]);
            if (tuning) {
                stage = (sweep + 1) & 1;   // sweep 0 (cold caches) uses stage 1, then alternate
                cudaEventRecord(ev[0], c->stream);
            }
            if constexpr (P != LQCD_F64) {
                if (resident && stage)
                    k_sap_block_s<P, true>
                        <<<dim3(Pl.count[col], nrhs), 2 * Pl.B.nh, sizeof(SapSmem<P, true>), c->stream>>>(a);
                else if (resident)
                    k_sap_block_s<P, false>
                        <<<dim3(Pl.count[col], nrhs), 2 * Pl.B.nh, sizeof(SapSmem<P, false>), c->stream>>>(a);
                else
                    k_sap_block<P><<<dim3(Pl.count[col], nrhs), threads, smem, c->stream>>>(a);
            } else {
                k_sap_block<P><<<dim3(Pl.count[col], nrhs), threads, smem, c->stream>>>(a);
            }
            c->n_kernel_launches++;
            LQCD_LAUNCH_CHECK(c);
            if (tuning) {
                cudaEventRecord(ev[1], c->stream);
                LQCD_CUDA_CHECK(c, cudaEventSynchronize(ev[1]));
                float ms = 0;
                cudaEventElapsedTime(&ms, ev[0], ev[1]);
                if (sweep > 0) best_us[stage] = std::min(best_us[stage], 1000.f * ms);
                if (tune_verbose())
                    fprintf(stderr, "tune %s: stage=%d sweep %d %.1f us\n", key.c_str(), stage, sweep, 1000.f * ms);
            }
            sweep++;
            if (cyc == ncy - 1 && col == last_col) continue;
            if (Pl.nface[col] > 0)
                k_sap_face_l<P><<<dim3(div_up(Pl.nface[col], 128), nrhs), 128, 0, c->stream>>>(
                    a, Pl.face_dev[col], Pl.nface[col]);
            c->n_kernel_launches++;
            LQCD_LAUNCH_CHECK(c);
        }
    if (tuning) {
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        TuneChoice tc;
        tc.variant = best_us[1] < best_us[0] ? 1 : 0;
        tc.tx = 2 * Pl.B.nh;
        tc.ty = 1;
        tc.us = best_us[tc.variant];
        tune_store(key, tc);
    }
    return LQCD_OK;
}

}  // namespace

// r = eta - r on native full fields
namespace {
template <class T>
__global__ void k_eta_minus(long n, const T *__restrict__ eta, T *r);
template <>
__global__ void k_eta_minus<double2>(long n, const double2 *__restrict__ eta, double2 *r)
{
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        double2 a = eta[j], b = r[j];
        r[j] = make_double2(a.x - b.x, a.y - b.y);
    }
}
template <>
__global__ void k_eta_minus<float4>(long n, const float4 *__restrict__ eta, float4 *r)
{
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        float4 a = eta[j], b = r[j];
        r[j] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
    }
}
}  // namespace

lqcd_status sap_axpby_native(lqcd_ctx *c, lqcd_prec p, const void *eta, void *r)
{
    long n = 2 * (long)c->g.Vh * (p == LQCD_F64 ? 12 : 6);
    int grid = (int)std::min<long>(4 * 152, (n + 255) / 256);
    if (p == LQCD_F64)
        k_eta_minus<double2><<<grid, 256, 0, c->stream>>>(n, (const double2 *)eta, (double2 *)r);
    else
        k_eta_minus<float4><<<grid, 256, 0, c->stream>>>(n, (const float4 *)eta, (float4 *)r);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

lqcd_status sap_apply(lqcd_ctx *c, const lqcd_sap_params *sp, const void *eta, void *psi, int nrhs)
{
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    if (sp->ncy < 1 || sp->nmr < 0) return set_err(c, LQCD_ERR_ARG, "bad SAP cycle counts");
    SapPlan *P;
    LQCD_TRY(get_plan(c, sp->bs, &P));
    void *r;
    const size_t fb = 2 * native_half_bytes(c, sp->prec);
    LQCD_TRY(ws_get(c, WS_SAP_R, 2 * fb * nrhs, &r));
    void *delta = (char *)r + fb * nrhs;
    if (sp->prec == LQCD_F64) return sap_run<LQCD_F64>(c, *P, sp->ncy, sp->nmr, eta, psi, r, delta, nrhs);
    if (sp->prec == LQCD_F32) return sap_run<LQCD_F32>(c, *P, sp->ncy, sp->nmr, eta, psi, r, delta, nrhs);
    if (sp->prec == LQCD_F16S) return sap_run<LQCD_F16S>(c, *P, sp->ncy, sp->nmr, eta, psi, r, delta, nrhs);
    return set_err(c, LQCD_ERR_ARG, "SAP precision %d not supported", (int)sp->prec);
}

// ------------------------------------------------------------------ batches
struct SapBatch {
    lqcd_prec p = LQCD_F16S;
    int ncy = 4, nmr = 5, nh = 0, nsm = 0;
    void *args = nullptr;                  // SapArgs<p>[2 nlat]
    int2 *blk[2] = {nullptr, nullptr};     // (lattice, index in its colour list)
    int nblk[2] = {0, 0};
    int2 *face = nullptr;                  // (lattice, first site of a 128-site tile)
    int nface = 0;
    int *queue = nullptr;                  // one work counter per block launch of an application
    void *r = nullptr, *psi = nullptr, *delta = nullptr;
};

void sap_batch_free(SapBatch *b)
{
    if (!b) return;
    cudaFree(b->args);
    cudaFree(b->blk[0]);
    cudaFree(b->blk[1]);
    cudaFree(b->face);
    cudaFree(b->queue);
    delete b;
}

namespace {
template <int P>
lqcd_status sap_batch_args(lqcd_ctx *hc, lqcd_ctx *const *ctx, int n, const lqcd_sap_params *sp, SapBatch *b,
                           const long *off)
{
    using SP = typename SapT<P>::SP;
    std::vector<SapArgs<P>> v;
    std::vector<int2> it[2], face;
    for (int l = 0; l < n; l++) {
        SapPlan *pl;
        LQCD_TRY(get_plan(ctx[l], sp->bs, &pl));
        if (b->nh == 0) b->nh = pl->B.nh;
        if (pl->B.nh != b->nh || b->nh > SAPS_NH || (2 * b->nh) % 32)
            return set_err(hc, LQCD_ERR_ARG, "batched SAP needs one block shape of <= %d sites per parity", SAPS_NH);
        for (int col = 0; col < 2; col++) {
            SapArgs<P> a;
            a.g = ctx[l]->g;
            a.B = pl->B;
            a.blocks = pl->blocks_dev + (col == 0 ? 0 : pl->count[0]);
            a.r = (SP *)b->r + off[l];
            a.psi = (SP *)b->psi + off[l];
            a.delta = (SP *)b->delta + off[l];
            a.fstride = 0;
            if constexpr (P == LQCD_F32) {
                a.U = ctx[l]->U32;
                a.Ae = ctx[l]->A32[0];
                a.Aio = ctx[l]->Ai32[1];
            } else {
                a.U = ctx[l]->U16;
                a.Ae = ctx[l]->A16[0];
                a.Aio = ctx[l]->Ai16[1];
            }
            a.nmr = sp->nmr;
            v.push_back(a);
            for (int i = 0; i < pl->count[col]; i++) it[col].push_back(make_int2(l, i));
        }
        for (int s0 = 0; s0 < 2 * ctx[l]->g.Vh; s0 += 128) face.push_back(make_int2(l, s0));
    }
    LQCD_CUDA_CHECK(hc, cudaMalloc(&b->args, v.size() * sizeof(v[0])));
    LQCD_CUDA_CHECK(hc, cudaMemcpy(b->args, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice));
    for (int col = 0; col < 2; col++) {
        b->nblk[col] = (int)it[col].size();
        LQCD_CUDA_CHECK(hc, cudaMalloc(&b->blk[col], std::max<size_t>(1, it[col].size()) * sizeof(int2)));
        LQCD_CUDA_CHECK(hc, cudaMemcpy(b->blk[col], it[col].data(), it[col].size() * sizeof(int2), cudaMemcpyHostToDevice));
    }
    b->nface = (int)face.size();
    LQCD_CUDA_CHECK(hc, cudaMalloc(&b->face, face.size() * sizeof(int2)));
    LQCD_CUDA_CHECK(hc, cudaMemcpy(b->face, face.data(), face.size() * sizeof(int2), cudaMemcpyHostToDevice));
    return LQCD_OK;
}

template <int P>
lqcd_status sap_batch_run(lqcd_ctx *hc, SapBatch *b, const int *active)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_sap_block_s_batch<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SapSmem<P, true>));
        cudaFuncSetAttribute(k_sap_block_s_batch<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SapSmem<P, false>));
        attr = true;
    }
    // the batched sweeps are replayed from captured graphs, so no in-flight
    // tuning here: the clover term goes through L1 (two to three CTAs per SM,
    // the work queue's balance) unless the staged form is forced
    const bool sa = sap_stage_forced() == 1;
    const auto *args = (const SapArgs<P> *)b->args;
    const int last_col = b->nblk[1] > 0 ? 1 : 0;
    for (int cyc = 0; cyc < b->ncy; cyc++)
        for (int col = 0; col < 2; col++) {
            if (b->nblk[col] == 0) continue;
            if (sa)
                k_sap_block_s_batch<P, true><<<std::min(b->nblk[col], b->nsm), 2 * b->nh, sizeof(SapSmem<P, true>),
                                               hc->stream>>>(args, col, b->blk[col], b->nblk[col], active,
                                                             b->queue + 2 * cyc + col);
            else
                k_sap_block_s_batch<P, false><<<std::min(b->nblk[col], sap_ctas<P, false>() * b->nsm), 2 * b->nh,
                                                sizeof(SapSmem<P, false>), hc->stream>>>(
                    args, col, b->blk[col], b->nblk[col], active, b->queue + 2 * cyc + col);
            hc->n_kernel_launches++;
            LQCD_LAUNCH_CHECK(hc);
            if (cyc == b->ncy - 1 && col == last_col) continue;
            k_sap_face_batch<P><<<b->nface, 128, 0, hc->stream>>>(args, col, b->face, b->nface, active);
            hc->n_kernel_launches++;
            LQCD_LAUNCH_CHECK(hc);
        }
    return LQCD_OK;
}
}  // namespace

lqcd_status sap_batch_create(lqcd_ctx *hc, lqcd_ctx *const *ctx, int n, const lqcd_sap_params *sp, void *r,
                             void *psi, void *delta, const long *off, SapBatch **out_b)
{
    if (sp->prec != LQCD_F32 && sp->prec != LQCD_F16S)
        return set_err(hc, LQCD_ERR_ARG, "batched SAP runs in F32 or F16S");
    if (sp->ncy < 1 || sp->nmr < 0) return set_err(hc, LQCD_ERR_ARG, "bad SAP cycle counts");
    SapBatch *b = new SapBatch();
    b->p = sp->prec;
    b->ncy = sp->ncy;
    b->nmr = sp->nmr;
    b->r = r;
    b->psi = psi;
    b->delta = delta;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    lqcd_status st = sp->prec == LQCD_F32 ? sap_batch_args<LQCD_F32>(hc, ctx, n, sp, b, off)
                                          : sap_batch_args<LQCD_F16S>(hc, ctx, n, sp, b, off);
    if (st == LQCD_OK && cudaMalloc(&b->queue, 2 * sp->ncy * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        st = set_err(hc, LQCD_ERR_NOMEM, "batched SAP work counters");
    }
    if (st != LQCD_OK) {
        sap_batch_free(b);
        return st;
    }
    *out_b = b;
    return LQCD_OK;
}

// psi = M_sap eta on every lattice whose active flag is set (the arenas given
// at creation; eta: an arena of the same layout, bytes long)
lqcd_status sap_batch_apply(lqcd_ctx *hc, SapBatch *b, const void *eta, size_t bytes, const int *active)
{
    LQCD_CUDA_CHECK(hc, cudaMemsetAsync(b->psi, 0, bytes, hc->stream));
    LQCD_CUDA_CHECK(hc, cudaMemcpyAsync(b->r, eta, bytes, cudaMemcpyDeviceToDevice, hc->stream));
    LQCD_CUDA_CHECK(hc, cudaMemsetAsync(b->queue, 0, 2 * b->ncy * sizeof(int), hc->stream));
    return b->p == LQCD_F32 ? sap_batch_run<LQCD_F32>(hc, b, active) : sap_batch_run<LQCD_F16S>(hc, b, active);
}

void sap_free_plans(lqcd_ctx *c)
{
    for (auto it = g_plans.begin(); it != g_plans.end();) {
        if (it->ctx == c) {
            cudaFree(it->plan.blocks_dev);
            cudaFree(it->plan.face_dev[0]);
            cudaFree(it->plan.face_dev[1]);
            it = g_plans.erase(it);
        } else
            ++it;
    }
}

extern "C" lqcd_status lqcd_sap(lqcd_ctx *c, const lqcd_sap_params *sp, const double *eta, double *psi)
{
    if (!c || !sp || !eta || !psi) return set_err(c, LQCD_ERR_ARG, "null argument");
    lqcd_prec p = sp->prec;
    if (p != LQCD_F64 && p != LQCD_F32 && p != LQCD_F16S) return set_err(c, LQCD_ERR_ARG, "SAP precision %d", (int)p);
    size_t fb = 2 * native_half_bytes(c, p);
    size_t fb64 = 2 * native_half_bytes(c, LQCD_F64);
    void *a, *b, *t;
    LQCD_TRY(ws_get(c, WS_SAP_IN, fb, &a));
    LQCD_TRY(ws_get(c, WS_SAP_PSI, fb, &b));
    LQCD_TRY(ws_get(c, WS_PACK_IN, fb64, &t));
    // canonical FP64 -> native FP64 -> native prec
    LQCD_TRY(pack_field(c, LQCD_F64, 2, eta, t, 1, false));
    LQCD_TRY(convert_native(c, LQCD_F64, p, t, a, 2));
    LQCD_TRY(sap_apply(c, sp, a, b));
    LQCD_TRY(convert_native(c, p, LQCD_F64, b, t, 2));
    return pack_field(c, LQCD_F64, 2, psi, t, 1, true);
}
