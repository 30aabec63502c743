// Device building blocks of the Wilson-clover stencil kernels (native
// site-minor layouts, spin projection in the chiral basis, clover blocks),
// shared by the single-field and register-blocked multi-field kernels.
//
//   H psi(x) = -1/2 sum_mu [(1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^dag psi(x-mu)]
//   D = A + H (Eq. 1),  Dhat = A_ee - H_eo A_oo^-1 H_oe (Eq. 2).
//
// In the chiral basis g_mu = [[0, e_mu], [e_mu^dag, 0]] with e_0 = -1 and
// e_k = -i sigma_k, so (1 -+ g_mu) psi is determined by the half spinor
// h = psi_up -+ e_mu psi_lo: the upper half of the result is h and the lower
// half is -+ e_mu^dag h.  Each hop therefore multiplies only two colour
// vectors by the link (spin projection), 1320 flops per output site.
#pragma once

#include "lqcd_f16s.cuh"
#include "lqcd_internal.cuh"

namespace stencil {

template <lqcd_prec P>
struct PT;
template <>
struct PT<LQCD_F64> {
    using R = double;
};
template <>
struct PT<LQCD_F32> {
    using R = float;
};

// ---------------------------------------------------------------- loads
template <class R>
struct Spinor {
    cx<R> s[4][3];
};

__device__ __forceinline__ void load_spinor(const double2 *__restrict__ f, long Vh, int r,
                                            Spinor<double> &o)
{
#pragma unroll
    for (int c = 0; c < 12; c++) {
        double2 v = __ldg(f + c * Vh + r);
        o.s[c / 3][c % 3] = mk(v.x, v.y);
    }
}
__device__ __forceinline__ void load_spinor(const float4 *__restrict__ f, long Vh, int r,
                                            Spinor<float> &o)
{
#pragma unroll
    for (int q = 0; q < 6; q++) {
        float4 v = __ldg(f + q * Vh + r);
        int c0 = 2 * q, c1 = 2 * q + 1;
        o.s[c0 / 3][c0 % 3] = mk(v.x, v.y);
        o.s[c1 / 3][c1 % 3] = mk(v.z, v.w);
    }
}
__device__ __forceinline__ void store_spinor(double2 *__restrict__ f, long Vh, int r,
                                             const Spinor<double> &o)
{
#pragma unroll
    for (int c = 0; c < 12; c++) f[c * Vh + r] = make_double2(o.s[c / 3][c % 3].re, o.s[c / 3][c % 3].im);
}
__device__ __forceinline__ void store_spinor(float4 *__restrict__ f, long Vh, int r,
                                             const Spinor<float> &o)
{
#pragma unroll
    for (int q = 0; q < 6; q++) {
        int c0 = 2 * q, c1 = 2 * q + 1;
        f[q * Vh + r] = make_float4(o.s[c0 / 3][c0 % 3].re, o.s[c0 / 3][c0 % 3].im,
                                    o.s[c1 / 3][c1 % 3].re, o.s[c1 / 3][c1 % 3].im);
    }
}

// FP16 + per-site scale storage (arithmetic in FP32)
__device__ __forceinline__ void load_spinor(const h16s *__restrict__ f, long Vh, int r, Spinor<float> &o)
{
    cx<float> v[12];
    f16s_load<true>(f, Vh, r, v);
#pragma unroll
    for (int c = 0; c < 12; c++) o.s[c / 3][c % 3] = v[c];
}
__device__ __forceinline__ void store_spinor(h16s *__restrict__ f, long Vh, int r, const Spinor<float> &o)
{
    cx<float> v[12];
#pragma unroll
    for (int c = 0; c < 12; c++) v[c] = o.s[c / 3][c % 3];
    f16s_store(f, Vh, r, v);
}

// SU(3) link of parity p, direction mu, at rank r
__device__ __forceinline__ void load_link(const double2 *__restrict__ U, long Vh, int p, int mu, int r,
                                          cx<double> u[3][3])
{
    const double2 *b = U + (long)((p * 4 + mu) * 9) * Vh + r;
#pragma unroll
    for (int e = 0; e < 9; e++) {
        double2 v = __ldg(b + e * Vh);
        u[e / 3][e % 3] = mk(v.x, v.y);
    }
}
// two stored rows, third = (row0 x row1)^*
__device__ __forceinline__ void load_link(const float4 *__restrict__ U, long Vh, int p, int mu, int r,
                                          cx<float> u[3][3])
{
    const float4 *b = U + (long)((p * 4 + mu) * 3) * Vh + r;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        float4 v = __ldg(b + q * Vh);
        int e0 = 2 * q, e1 = 2 * q + 1;
        u[e0 / 3][e0 % 3] = mk(v.x, v.y);
        u[e1 / 3][e1 % 3] = mk(v.z, v.w);
    }
    su3_third_row(u);
}

__device__ __forceinline__ void load_link(const uint2 *__restrict__ U, long Vh, int p, int mu, int r,
                                          cx<float> u[3][3])
{
    f16s_link(U, Vh, p, mu, r, u);
}

// packed Hermitian 6x6 pair: per block 6 real diagonal entries then the 15
// complex entries above the diagonal in row-major order (36 reals)
template <class R>
struct Herm6 {
    R d[6];
    cx<R> o[15];
};
__device__ __forceinline__ void load_herm(const double2 *__restrict__ A, long Vh, int r, int blk,
                                          Herm6<double> &h)
{
    const double2 *b = A + (long)(18 * blk) * Vh + r;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        double2 v = __ldg(b + i * Vh);
        h.d[2 * i] = v.x;
        h.d[2 * i + 1] = v.y;
    }
#pragma unroll
    for (int i = 0; i < 15; i++) {
        double2 v = __ldg(b + (3 + i) * Vh);
        h.o[i] = mk(v.x, v.y);
    }
}
__device__ __forceinline__ void load_herm(const float4 *__restrict__ A, long Vh, int r, int blk,
                                          Herm6<float> &h)
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
    for (int i = 0; i < 6; i++) h.d[i] = v[i];
#pragma unroll
    for (int i = 0; i < 15; i++) h.o[i] = mk(v[6 + 2 * i], v[7 + 2 * i]);
}

__device__ __forceinline__ void load_herm(const uint2 *__restrict__ A, long Vh, int r, int blk, Herm6<float> &h)
{
    float v[36];
    f16s_clover(A, Vh, r, blk, v);
#pragma unroll
    for (int i = 0; i < 6; i++) h.d[i] = v[i];
#pragma unroll
    for (int i = 0; i < 15; i++) h.o[i] = mk(v[6 + 2 * i], v[7 + 2 * i]);
}

// out[6] = H in[6]; every product enters its sum through a fused multiply-add
template <class R>
__device__ __forceinline__ void herm_apply(const Herm6<R> &h, const cx<R> in[6], cx<R> out[6])
{
#pragma unroll
    for (int i = 0; i < 6; i++) out[i] = h.d[i] * in[i];
    int k = 0;
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
        for (int j = i + 1; j < 6; j++) {
            const cx<R> o = h.o[k++];
            out[i].re = fmx(o.re, in[j].re, out[i].re);   // out_i += o in_j
            out[i].re = fmx(-o.im, in[j].im, out[i].re);
            out[i].im = fmx(o.re, in[j].im, out[i].im);
            out[i].im = fmx(o.im, in[j].re, out[i].im);
            out[j].re = fmx(o.re, in[i].re, out[j].re);   // out_j += conj(o) in_i
            out[j].re = fmx(o.im, in[i].im, out[j].re);
            out[j].im = fmx(o.re, in[i].im, out[j].im);
            out[j].im = fmx(-o.im, in[i].re, out[j].im);
        }
}
// every entry of a packed Hermitian pair times an exact power of two
template <class R>
__device__ __forceinline__ void herm_scale(Herm6<R> &h, R f)
{
#pragma unroll
    for (int i = 0; i < 6; i++) h.d[i] = f * h.d[i];
#pragma unroll
    for (int i = 0; i < 15; i++) h.o[i] = f * h.o[i];
}

template <class R, class CL>
__device__ __forceinline__ void clover_apply(const CL *A, long Vh, int r, const Spinor<R> &in,
                                             Spinor<R> &out)
{
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        Herm6<R> h;
        load_herm(A, Vh, r, blk, h);
        cx<R> v[6], w[6];
#pragma unroll
        for (int s = 0; s < 2; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) v[3 * s + c] = in.s[2 * blk + s][c];
        herm_apply(h, v, w);
#pragma unroll
        for (int s = 0; s < 2; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) out.s[2 * blk + s][c] = w[3 * s + c];
    }
}

// ------------------------------------------------------- spin projection
// h = psi_up + sgn * e_mu psi_lo, sgn = -1 for the forward (1-g) hop, +1 backward
template <class R, int MU, int SGN>
__device__ __forceinline__ void project(const Spinor<R> &p, cx<R> h[2][3])
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cx<R> u0 = p.s[0][c], u1 = p.s[1][c], l0 = p.s[2][c], l1 = p.s[3][c];
        if (MU == 0) {  // e = -1
            h[0][c] = SGN < 0 ? u0 + l0 : u0 - l0;
            h[1][c] = SGN < 0 ? u1 + l1 : u1 - l1;
        } else if (MU == 1) {  // e = -i sigma_x: e l = (-i l1, -i l0)
            h[0][c] = SGN < 0 ? u0 + timesI(l1) : u0 - timesI(l1);
            h[1][c] = SGN < 0 ? u1 + timesI(l0) : u1 - timesI(l0);
        } else if (MU == 2) {  // e = [[0,-1],[1,0]]: e l = (-l1, l0)
            h[0][c] = SGN < 0 ? u0 + l1 : u0 - l1;
            h[1][c] = SGN < 0 ? u1 - l0 : u1 + l0;
        } else {  // e = diag(-i, i): e l = (-i l0, i l1)
            h[0][c] = SGN < 0 ? u0 + timesI(l0) : u0 - timesI(l0);
            h[1][c] = SGN < 0 ? u1 - timesI(l1) : u1 + timesI(l1);
        }
    }
}
// acc += sg (w ; sgn * e_mu^dag w).  SC: sg is the time-boundary sign (+-1),
// folded into fused multiply-adds (exact, the same rounding as adding +-w);
// otherwise sg is ignored and w is added.
template <class R, int MU, int SGN, bool SC = false>
__device__ __forceinline__ void accumulate(Spinor<R> &acc, const cx<R> w[2][3], R sg = R(1))
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cx<R> a, b;  // sgn * e^dag w
        if (MU == 0) {  // e^dag = -1
            a = -w[0][c];
            b = -w[1][c];
        } else if (MU == 1) {  // e^dag = i sigma_x
            a = timesI(w[1][c]);
            b = timesI(w[0][c]);
        } else if (MU == 2) {  // e^dag = [[0,1],[-1,0]]
            a = w[1][c];
            b = -w[0][c];
        } else {  // e^dag = diag(i, -i)
            a = timesI(w[0][c]);
            b = timesmI(w[1][c]);
        }
        if (SGN < 0) {
            a = -a;
            b = -b;
        }
        if (SC) {
            acc.s[0][c].re = fmx(sg, w[0][c].re, acc.s[0][c].re);
            acc.s[0][c].im = fmx(sg, w[0][c].im, acc.s[0][c].im);
            acc.s[1][c].re = fmx(sg, w[1][c].re, acc.s[1][c].re);
            acc.s[1][c].im = fmx(sg, w[1][c].im, acc.s[1][c].im);
            acc.s[2][c].re = fmx(sg, a.re, acc.s[2][c].re);
            acc.s[2][c].im = fmx(sg, a.im, acc.s[2][c].im);
            acc.s[3][c].re = fmx(sg, b.re, acc.s[3][c].re);
            acc.s[3][c].im = fmx(sg, b.im, acc.s[3][c].im);
        } else {
            acc.s[0][c] = acc.s[0][c] + w[0][c];
            acc.s[1][c] = acc.s[1][c] + w[1][c];
            acc.s[2][c] = acc.s[2][c] + a;
            acc.s[3][c] = acc.s[3][c] + b;
        }
    }
}

// w = U h: each real part one product and five fused multiply-adds
template <class R>
__device__ __forceinline__ void su3_vec(const cx<R> u[3][3], const cx<R> h[3], cx<R> w[3])
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        R re = u[a][0].re * h[0].re;
        re = fmx(-u[a][0].im, h[0].im, re);
        re = fmx(u[a][1].re, h[1].re, re);
        re = fmx(-u[a][1].im, h[1].im, re);
        re = fmx(u[a][2].re, h[2].re, re);
        re = fmx(-u[a][2].im, h[2].im, re);
        R im = u[a][0].re * h[0].im;
        im = fmx(u[a][0].im, h[0].re, im);
        im = fmx(u[a][1].re, h[1].im, im);
        im = fmx(u[a][1].im, h[1].re, im);
        im = fmx(u[a][2].re, h[2].im, im);
        im = fmx(u[a][2].im, h[2].re, im);
        w[a] = mk(re, im);
    }
}
// w = U^dag h
template <class R>
__device__ __forceinline__ void su3dag_vec(const cx<R> u[3][3], const cx<R> h[3], cx<R> w[3])
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        R re = u[0][a].re * h[0].re;
        re = fmx(u[0][a].im, h[0].im, re);
        re = fmx(u[1][a].re, h[1].re, re);
        re = fmx(u[1][a].im, h[1].im, re);
        re = fmx(u[2][a].re, h[2].re, re);
        re = fmx(u[2][a].im, h[2].im, re);
        R im = u[0][a].re * h[0].im;
        im = fmx(-u[0][a].im, h[0].re, im);
        im = fmx(u[1][a].re, h[1].im, im);
        im = fmx(-u[1][a].im, h[1].re, im);
        im = fmx(u[2][a].re, h[2].im, im);
        im = fmx(-u[2][a].im, h[2].re, im);
        w[a] = mk(re, im);
    }
}

template <class R, class SP, class LK, int MU>
__device__ __forceinline__ void hop_dir(const Geom &g, int p_out, int r, const int x[4],
                                        const SP *in, long Vh, const LK *U, Spinor<R> &acc)
{
    cx<R> h[2][3], w[2][3];
    cx<R> u[3][3];
    Spinor<R> psi;
    // forward: (1 - g_mu) U_mu(x) psi(x + mu)
    {
        int ry = nbr_rank(g, x, MU, +1);
        R sg = (MU == 0 && x[0] == g.L[0] - 1) ? R(g.bc_t) : R(1);
        load_spinor(in, Vh, ry, psi);
        project<R, MU, -1>(psi, h);
        load_link(U, Vh, p_out, MU, r, u);
        su3_vec(u, h[0], w[0]);
        su3_vec(u, h[1], w[1]);
        accumulate<R, MU, -1, MU == 0>(acc, w, sg);
    }
    // backward: (1 + g_mu) U_mu(x - mu)^dag psi(x - mu)
    {
        int rz = nbr_rank(g, x, MU, -1);
        R sg = (MU == 0 && x[0] == 0) ? R(g.bc_t) : R(1);
        load_spinor(in, Vh, rz, psi);
        project<R, MU, +1>(psi, h);
        load_link(U, Vh, 1 - p_out, MU, rz, u);
        su3dag_vec(u, h[0], w[0]);
        su3dag_vec(u, h[1], w[1]);
        accumulate<R, MU, +1, MU == 0>(acc, w, sg);
    }
}

enum { MODE_HOP = 0, MODE_DHAT1 = 1, MODE_DHAT2 = 2, MODE_D = 3 };

template <class SP, class LK, class CL>
struct HopArgs {
    Geom g;
    int p_out, nrhs;
    const SP *in_other;
    long in_rs;
    const SP *in_same;
    long same_rs;
    SP *out;
    long out_rs;
    const LK *U;
    const CL *clov;   // parity p_out: A^-1 (DHAT1) or A (DHAT2, D)
};

// register-blocked form (lqcd_dirac_mr.cu): nr = 2 fields per thread,
// occupancy variant var (0..2); float arithmetic, modes DHAT1 / DHAT2 / D
template <class R, class SP, class LK, class CL, int MODE>
lqcd_status launch_hop_mr(lqcd_ctx *c, int nr, int var, dim3 b, const HopArgs<SP, LK, CL> &a);
constexpr int NVAR_MR = 3;
inline int var_mr_max_threads(int v) { return v == 1 ? 128 : 256; }
// staged form (lqcd_dirac_sm.cu): tile of b.x = 16 or 32 sites x b.y fields,
// occupancy variant var (0..2); float arithmetic, modes DHAT1 / DHAT2 / D
template <class R, class SP, class LK, class CL, int MODE>
lqcd_status launch_hop_sm(lqcd_ctx *c, int var, dim3 b, const HopArgs<SP, LK, CL> &a);
constexpr int NVAR_SM = 3;
inline int var_sm_max_threads(int v) { return v == 2 ? 256 : 384; }
// kernel forms known to the autotuner
enum { KIND_HOP = 0, KIND_MR = 1, KIND_SM = 2 };

}  // namespace stencil
