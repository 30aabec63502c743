// Wilson-clover stencil kernels on native (site-minor) layouts.
//
//   H psi(x) = -1/2 sum_mu [(1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^dag psi(x-mu)]
//   D = A + H (Eq. 1),  Dhat = A_ee - H_eo A_oo^-1 H_oe (Eq. 2).
//
// One thread per (output site, right-hand side).  A CTA is blockDim.x sites
// by blockDim.y right-hand sides, so a warp reads 32 consecutive sites of one
// field (coalesced 16-byte loads) and the warps of the other right-hand
// sides reuse the same link / clover words from L1: links and clover are
// fetched from HBM once per CTA however many fields it serves.
//
// In the chiral basis g_mu = [[0, e_mu], [e_mu^dag, 0]] with e_0 = -1 and
// e_k = -i sigma_k, so (1 -+ g_mu) psi is determined by the half spinor
// h = psi_up -+ e_mu psi_lo: the upper half of the result is h and the lower
// half is -+ e_mu^dag h.  Each hop therefore multiplies only two colour
// vectors by the link (spin projection), 1320 flops per output site.
#include <type_traits>

#include "lqcd_f16s.cuh"
#include "lqcd_internal.cuh"
#include "lqcd_tune.h"

namespace {

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
    u[2][0] = conjx(u[0][1] * u[1][2] - u[0][2] * u[1][1]);
    u[2][1] = conjx(u[0][2] * u[1][0] - u[0][0] * u[1][2]);
    u[2][2] = conjx(u[0][0] * u[1][1] - u[0][1] * u[1][0]);
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

// out[6] = H in[6]
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
            out[i] = out[i] + h.o[k] * in[j];
            out[j] = out[j] + cmulc(h.o[k], in[i]);
            k++;
        }
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
// acc += (w ; sgn * e_mu^dag w)
template <class R, int MU, int SGN>
__device__ __forceinline__ void accumulate(Spinor<R> &acc, const cx<R> w[2][3])
{
#pragma unroll
    for (int c = 0; c < 3; c++) {
        acc.s[0][c] = acc.s[0][c] + w[0][c];
        acc.s[1][c] = acc.s[1][c] + w[1][c];
        cx<R> a, b;  // e^dag w
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
            acc.s[2][c] = acc.s[2][c] - a;
            acc.s[3][c] = acc.s[3][c] - b;
        } else {
            acc.s[2][c] = acc.s[2][c] + a;
            acc.s[3][c] = acc.s[3][c] + b;
        }
    }
}

template <class R>
__device__ __forceinline__ void su3_vec(const cx<R> u[3][3], const cx<R> h[3], cx<R> w[3], R sign)
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        cx<R> t = u[a][0] * h[0] + u[a][1] * h[1] + u[a][2] * h[2];
        w[a] = sign * t;
    }
}
template <class R>
__device__ __forceinline__ void su3dag_vec(const cx<R> u[3][3], const cx<R> h[3], cx<R> w[3], R sign)
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        cx<R> t = cmulc(u[0][a], h[0]) + cmulc(u[1][a], h[1]) + cmulc(u[2][a], h[2]);
        w[a] = sign * t;
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
        su3_vec(u, h[0], w[0], sg);
        su3_vec(u, h[1], w[1], sg);
        accumulate<R, MU, -1>(acc, w);
    }
    // backward: (1 + g_mu) U_mu(x - mu)^dag psi(x - mu)
    {
        int rz = nbr_rank(g, x, MU, -1);
        R sg = (MU == 0 && x[0] == 0) ? R(g.bc_t) : R(1);
        load_spinor(in, Vh, rz, psi);
        project<R, MU, +1>(psi, h);
        load_link(U, Vh, 1 - p_out, MU, rz, u);
        su3dag_vec(u, h[0], w[0], sg);
        su3dag_vec(u, h[1], w[1], sg);
        accumulate<R, MU, +1>(acc, w);
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

//   MODE_HOP  : out = -1/2 S
//   MODE_DHAT1: out = A^-1 (-1/2 S)            (chi_o = A_oo^-1 H_oe psi_e)
//   MODE_DHAT2: out = A in_same + 1/2 S        (A_ee psi_e - H_eo chi_o)
//   MODE_D    : out = A in_same - 1/2 S        (D psi on one parity)
// with S = sum of the 8 projected hops of in_other.
// occupancy variants: (max threads per CTA, min CTAs per SM)
template <int VAR>
struct Var;
template <>
struct Var<0> {
    static constexpr int T = 384, B = 1;
};
template <>
struct Var<1> {
    static constexpr int T = 384, B = 2;
};
template <>
struct Var<2> {
    static constexpr int T = 256, B = 3;
};
template <>
struct Var<3> {
    static constexpr int T = 256, B = 4;
};
constexpr int NVAR = 4;
inline int var_max_threads(int v) { return v < 2 ? 384 : 256; }

template <class R, class SP, class LK, class CL, int MODE, int VAR>
__global__ void __launch_bounds__(Var<VAR>::T, Var<VAR>::B) k_hop(HopArgs<SP, LK, CL> a)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y * blockDim.y + threadIdx.y;
    const long Vh = a.g.Vh;
    if (r >= a.g.Vh || k >= a.nrhs) return;
    int x[4];
    rank_coords(a.g, a.p_out, r, x);
    const SP *in = a.in_other + k * a.in_rs;
    Spinor<R> acc;
    if (MODE == MODE_HOP || MODE == MODE_DHAT1) {
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc.s[s][c] = mk(R(0), R(0));
    } else {
        // start from (1/f) A in_same, f = +-1/2 (exact power-of-two scaling), so the
        // hops accumulate into the same registers: out = f (A in / f + S)
        Spinor<R> self;
        load_spinor(a.in_same + k * a.same_rs, Vh, r, self);
        clover_apply<R, CL>(a.clov, Vh, r, self, acc);
        const R inv_f = MODE == MODE_DHAT2 ? R(2) : R(-2);
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc.s[s][c] = inv_f * acc.s[s][c];
    }
    hop_dir<R, SP, LK, 0>(a.g, a.p_out, r, x, in, Vh, a.U, acc);
    hop_dir<R, SP, LK, 1>(a.g, a.p_out, r, x, in, Vh, a.U, acc);
    hop_dir<R, SP, LK, 2>(a.g, a.p_out, r, x, in, Vh, a.U, acc);
    hop_dir<R, SP, LK, 3>(a.g, a.p_out, r, x, in, Vh, a.U, acc);
    const R f = MODE == MODE_DHAT2 ? R(0.5) : R(-0.5);
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < 3; c++) acc.s[s][c] = f * acc.s[s][c];
    if (MODE == MODE_DHAT1) {
        Spinor<R> res;
        clover_apply<R, CL>(a.clov, Vh, r, acc, res);
        store_spinor(a.out + k * a.out_rs, Vh, r, res);
    } else {
        store_spinor(a.out + k * a.out_rs, Vh, r, acc);
    }
}

template <class R, class SP, class LK, class CL, int MODE>
lqcd_status launch_var(lqcd_ctx *c, int var, dim3 b, const HopArgs<SP, LK, CL> &a)
{
    dim3 grid(div_up(c->g.Vh, b.x), div_up(a.nrhs, b.y));
    switch (var) {
        case 0: k_hop<R, SP, LK, CL, MODE, 0><<<grid, b, 0, c->stream>>>(a); break;
        case 1: k_hop<R, SP, LK, CL, MODE, 1><<<grid, b, 0, c->stream>>>(a); break;
        case 2: k_hop<R, SP, LK, CL, MODE, 2><<<grid, b, 0, c->stream>>>(a); break;
        default: k_hop<R, SP, LK, CL, MODE, 3><<<grid, b, 0, c->stream>>>(a); break;
    }
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

// candidate launch shapes: tx sites x ty fields per CTA
std::vector<TuneChoice> hop_candidates(int nrhs)
{
    std::vector<TuneChoice> v;
    std::vector<int> tys;
    for (int t : {nrhs, (nrhs + 1) / 2, (nrhs + 2) / 3, 4, 2, 1})
        if (t >= 1 && t <= nrhs && std::find(tys.begin(), tys.end(), t) == tys.end()) tys.push_back(t);
    for (int var = 0; var < NVAR; var++)
        for (int ty : tys)
            for (int tx : {16, 32, 64, 128, 256}) {
                int n = tx * ty;
                if (n > var_max_threads(var) || n < 64) continue;
                TuneChoice t;
                t.variant = var;
                t.tx = tx;
                t.ty = ty;
                v.push_back(t);
            }
    return v;
}

template <class R, class SP, class LK, class CL, int MODE>
lqcd_status launch_hop(lqcd_ctx *c, int p_out, const SP *in_other, long in_rs, const SP *in_same,
                       long same_rs, SP *out, long out_rs, const LK *U, const CL *clov, int nrhs)
{
    HopArgs<SP, LK, CL> a;
    a.g = c->g;
    a.p_out = p_out;
    a.nrhs = nrhs;
    a.in_other = in_other;
    a.in_rs = in_rs;
    a.in_same = in_same;
    a.same_rs = same_rs;
    a.out = out;
    a.out_rs = out_rs;
    a.U = U;
    a.clov = clov;
    const int prec = sizeof(R) == 8 ? 0 : (std::is_same<SP, h16s>::value ? 2 : 1);
    std::string key = tune_key(c, "k_hop", MODE, prec, nrhs);
    TuneChoice tc;
    if (!tune_lookup(key, &tc)) {
        tc = TuneChoice();
        tc.tx = nrhs == 1 ? 128 : 32;
        tc.ty = nrhs == 1 ? 1 : std::min(nrhs, 8);
        if (tune_enabled()) {
            float best = 1e30f;
            for (const TuneChoice &cand : hop_candidates(nrhs)) {
                float us;
                lqcd_status s = tune_time(
                    c, [&]() { return launch_var<R, SP, LK, CL, MODE>(c, cand.variant, dim3(cand.tx, cand.ty), a); },
                    3, &us);
                if (s != LQCD_OK) return s;
                if (us < best) {
                    best = us;
                    tc = cand;
                    tc.us = us;
                }
            }
            tune_store(key, tc);
        }
    }
    return launch_var<R, SP, LK, CL, MODE>(c, tc.variant, dim3(tc.tx, tc.ty), a);
}

}  // namespace

// Dhat on native half fields: in/out even (nrhs fields, rhs stride = one half
// field), tmp_o an odd native half field per rhs.
lqcd_status dirac_dhat(lqcd_ctx *c, lqcd_prec p, const void *in, void *out, void *tmp_o, int nrhs)
{
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    const long Vh = c->g.Vh;
    if (p == LQCD_F64) {
        const long rs = 12 * Vh;
        auto *i = (const double2 *)in;
        auto *o = (double2 *)out;
        auto *t = (double2 *)tmp_o;
        LQCD_TRY((launch_hop<double, double2, double2, double2, MODE_DHAT1>(
            c, 1, i, rs, nullptr, 0, t, rs, c->U64, c->Ai64[1], nrhs)));
        LQCD_TRY((launch_hop<double, double2, double2, double2, MODE_DHAT2>(
            c, 0, t, rs, i, rs, o, rs, c->U64, c->A64[0], nrhs)));
        return LQCD_OK;
    }
    if (p == LQCD_F32) {
        const long rs = 6 * Vh;
        auto *i = (const float4 *)in;
        auto *o = (float4 *)out;
        auto *t = (float4 *)tmp_o;
        LQCD_TRY((launch_hop<float, float4, float4, float4, MODE_DHAT1>(
            c, 1, i, rs, nullptr, 0, t, rs, c->U32, c->Ai32[1], nrhs)));
        LQCD_TRY((launch_hop<float, float4, float4, float4, MODE_DHAT2>(
            c, 0, t, rs, i, rs, o, rs, c->U32, c->A32[0], nrhs)));
        return LQCD_OK;
    }
    if (p == LQCD_F16S) {
        const long rs = f16s_half_units(Vh);
        auto *i = (const h16s *)in;
        auto *o = (h16s *)out;
        auto *t = (h16s *)tmp_o;
        LQCD_TRY((launch_hop<float, h16s, uint2, uint2, MODE_DHAT1>(c, 1, i, rs, nullptr, 0, t, rs, c->U16,
                                                                    c->Ai16[1], nrhs)));
        LQCD_TRY((launch_hop<float, h16s, uint2, uint2, MODE_DHAT2>(c, 0, t, rs, i, rs, o, rs, c->U16, c->A16[0],
                                                                    nrhs)));
        return LQCD_OK;
    }
    return set_err(c, LQCD_ERR_ARG, "precision %d not supported for Dhat", (int)p);
}

// D on native full fields ([rhs][even half][odd half])
lqcd_status dirac_D(lqcd_ctx *c, lqcd_prec p, const void *in, void *out, int nrhs)
{
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    const long Vh = c->g.Vh;
    if (p == LQCD_F64) {
        const long h = 12 * Vh, rs = 2 * h;
        auto *i = (const double2 *)in;
        auto *o = (double2 *)out;
        for (int po = 0; po < 2; po++)
            LQCD_TRY((launch_hop<double, double2, double2, double2, MODE_D>(
                c, po, i + (1 - po) * h, rs, i + po * h, rs, o + po * h, rs, c->U64, c->A64[po], nrhs)));
        return LQCD_OK;
    }
    if (p == LQCD_F32) {
        const long h = 6 * Vh, rs = 2 * h;
        auto *i = (const float4 *)in;
        auto *o = (float4 *)out;
        for (int po = 0; po < 2; po++)
            LQCD_TRY((launch_hop<float, float4, float4, float4, MODE_D>(
                c, po, i + (1 - po) * h, rs, i + po * h, rs, o + po * h, rs, c->U32, c->A32[po], nrhs)));
        return LQCD_OK;
    }
    if (p == LQCD_F16S) {
        const long h = f16s_half_units(Vh), rs = 2 * h;
        auto *i = (const h16s *)in;
        auto *o = (h16s *)out;
        for (int po = 0; po < 2; po++)
            LQCD_TRY((launch_hop<float, h16s, uint2, uint2, MODE_D>(c, po, i + (1 - po) * h, rs, i + po * h, rs,
                                                                    o + po * h, rs, c->U16, c->A16[po], nrhs)));
        return LQCD_OK;
    }
    return set_err(c, LQCD_ERR_ARG, "precision %d not supported for D", (int)p);
}

// out (parity p_out) = H in_other, native half fields with given rhs strides
lqcd_status dirac_hop_parity(lqcd_ctx *c, lqcd_prec p, int p_out, const void *in_other, void *out,
                             long in_rstride, long out_rstride, int nrhs)
{
    if (p == LQCD_F64)
        return launch_hop<double, double2, double2, double2, MODE_HOP>(
            c, p_out, (const double2 *)in_other, in_rstride, nullptr, 0, (double2 *)out, out_rstride,
            c->U64, (const double2 *)nullptr, nrhs);
    if (p == LQCD_F32)
        return launch_hop<float, float4, float4, float4, MODE_HOP>(
            c, p_out, (const float4 *)in_other, in_rstride, nullptr, 0, (float4 *)out, out_rstride,
            c->U32, (const float4 *)nullptr, nrhs);
    return set_err(c, LQCD_ERR_ARG, "precision %d not supported for hop", (int)p);
}
