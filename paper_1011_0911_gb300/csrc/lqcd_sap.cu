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

#include "lqcd_internal.cuh"

namespace {

struct BlkGeom {
    int bs[4];
    int nb[4];
    int nh;          // sites of one parity per block
    int bs3h;
    int wrap[4];     // block spans the whole direction
};

template <class R>
struct SapPT;
template <>
struct SapPT<double> {
    using SP = double2;
    using LK = double2;
    using CL = double2;
};
template <>
struct SapPT<float> {
    using SP = float4;
    using LK = float4;
    using CL = float4;
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
    u[2][0] = conjx(u[0][1] * u[1][2] - u[0][2] * u[1][1]);
    u[2][1] = conjx(u[0][2] * u[1][0] - u[0][0] * u[1][2]);
    u[2][2] = conjx(u[0][0] * u[1][1] - u[0][1] * u[1][0]);
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

template <class R, class CL>
__device__ __forceinline__ void clov_apply(const CL *A, long Vh, long r, const cx<R> in[12], cx<R> out[12])
{
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        R d[6];
        cx<R> o[15];
        gclov(A, Vh, r, blk, d, o);
        const cx<R> *v = in + 6 * blk;
        cx<R> *w = out + 6 * blk;
#pragma unroll
        for (int i = 0; i < 6; i++) w[i] = d[i] * v[i];
        int k = 0;
#pragma unroll
        for (int i = 0; i < 6; i++)
#pragma unroll
            for (int j = i + 1; j < 6; j++) {
                w[i] = w[i] + o[k] * v[j];
                w[j] = w[j] + cmulc(o[k], v[i]);
                k++;
            }
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
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            cx<R> t;
            if (!dag)
                t = u[a][0] * h[s][0] + u[a][1] * h[s][1] + u[a][2] * h[s][2];
            else
                t = cmulc(u[0][a], h[s][0]) + cmulc(u[1][a], h[s][1]) + cmulc(u[2][a], h[s][2]);
            w[s][a] = sign * t;
        }
#pragma unroll
    for (int c = 0; c < 3; c++) {
        acc[c] = acc[c] + w[0][c];
        acc[3 + c] = acc[3 + c] + w[1][c];
        cx<R> a, b;  // e_mu^dag w
        switch (mu) {
            case 0: a = -w[0][c]; b = -w[1][c]; break;
            case 1: a = timesI(w[1][c]); b = timesI(w[0][c]); break;
            case 2: a = w[1][c]; b = -w[0][c]; break;
            default: a = timesI(w[0][c]); b = timesmI(w[1][c]); break;
        }
        if (sgn < 0) {
            acc[6 + c] = acc[6 + c] - a;
            acc[9 + c] = acc[9 + c] - b;
        } else {
            acc[6 + c] = acc[6 + c] + a;
            acc[9 + c] = acc[9 + c] + b;
        }
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

template <class R>
struct SapArgs {
    Geom g;
    BlkGeom B;
    const int *blocks;   // block ids of this colour
    const typename SapPT<R>::SP *r;    // native full field
    typename SapPT<R>::SP *psi;        // native full field (updated)
    const typename SapPT<R>::LK *U;
    const typename SapPT<R>::CL *Ae, *Aio;   // A on even sites, A^-1 on odd sites
    int nmr;
};

template <class R>
__global__ void __launch_bounds__(128) k_sap_block(SapArgs<R> a)
{
    using SP = typename SapPT<R>::SP;
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
    const SP *r_e = a.r, *r_o = a.r + (sizeof(R) == 8 ? 12 : 6) * Vh;
    SP *psi_e = a.psi, *psi_o = a.psi + (sizeof(R) == 8 ? 12 : 6) * Vh;

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
    // chi_o = A_oo^-1 (r_o - H_oe,blk chi_e); psi += chi
    for (int t = threadIdx.x; t < nh; t += blockDim.x) {
        SiteInfo s;
        block_site(a.g, B, org, 1, t, s);
        block_hopsum<R>(a.g, B, a.U, 1, s, chi, w);
        sload(ro, nh, t, v);
#pragma unroll
        for (int c = 0; c < 12; c++) v[c] = v[c] + R(0.5) * w[c];
        clov_apply<R>(a.Aio, Vh, s.grank, v, w);
        gadd(psi_o, Vh, s.grank, w);
        SiteInfo se;
        block_site(a.g, B, org, 0, t, se);
        sload(chi, nh, t, v);
        gadd(psi_e, Vh, se.grank, v);
    }
}

struct SapPlan {
    int bs[4] = {0, 0, 0, 0};
    int *blocks_dev = nullptr;   // [colour 0 ids..., colour 1 ids...]
    int count[2] = {0, 0};
    BlkGeom B;
};

// one cached plan per context (keyed by block shape)
struct PlanCache {
    lqcd_ctx *ctx;
    SapPlan plan;
};
std::vector<PlanCache> g_plans;

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
    g_plans.push_back({c, P});
    *out = &g_plans.back().plan;
    return LQCD_OK;
}

template <class R>
lqcd_status sap_run(lqcd_ctx *c, const SapPlan &P, int ncy, int nmr, const void *eta, void *psi, void *r)
{
    using SP = typename SapPT<R>::SP;
    const lqcd_prec prec = sizeof(R) == 8 ? LQCD_F64 : LQCD_F32;
    const size_t fb = 2 * native_half_bytes(c, prec);
    size_t smem = 5 * 12 * P.B.nh * sizeof(cx<R>) + 3 * 32 * sizeof(R);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_sap_block<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    if (smem > 200 * 1024) return set_err(c, LQCD_ERR_ARG, "SAP block needs %zu bytes of shared memory", smem);
    LQCD_CUDA_CHECK(c, cudaMemsetAsync(psi, 0, fb, c->stream));
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(r, eta, fb, cudaMemcpyDeviceToDevice, c->stream));
    SapArgs<R> a;
    a.g = c->g;
    a.B = P.B;
    a.r = (const SP *)r;
    a.psi = (SP *)psi;
    if (sizeof(R) == 8) {
        a.U = (const typename SapPT<R>::LK *)c->U64;
        a.Ae = (const typename SapPT<R>::CL *)c->A64[0];
        a.Aio = (const typename SapPT<R>::CL *)c->Ai64[1];
    } else {
        a.U = (const typename SapPT<R>::LK *)c->U32;
        a.Ae = (const typename SapPT<R>::CL *)c->A32[0];
        a.Aio = (const typename SapPT<R>::CL *)c->Ai32[1];
    }
    a.nmr = nmr;
    int threads = std::min(128, P.B.nh);
    bool first = true;
    for (int cyc = 0; cyc < ncy; cyc++)
        for (int col = 0; col < 2; col++) {
            if (P.count[col] == 0) continue;
            if (!first) {
                // r = eta - D psi
                LQCD_TRY(dirac_D(c, prec, psi, r, 1));
                LQCD_TRY(sap_axpby_native(c, prec, eta, r));
            }
            first = false;
            a.blocks = P.blocks_dev + (col == 0 ? 0 : P.count[0]);
            k_sap_block<R><<<P.count[col], threads, smem, c->stream>>>(a);
            c->n_kernel_launches++;
            LQCD_LAUNCH_CHECK(c);
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

lqcd_status sap_apply(lqcd_ctx *c, const lqcd_sap_params *sp, const void *eta, void *psi)
{
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    if (sp->ncy < 1 || sp->nmr < 0) return set_err(c, LQCD_ERR_ARG, "bad SAP cycle counts");
    SapPlan *P;
    LQCD_TRY(get_plan(c, sp->bs, &P));
    void *r;
    LQCD_TRY(ws_get(c, WS_SAP_R, 2 * native_half_bytes(c, sp->prec), &r));
    if (sp->prec == LQCD_F64) return sap_run<double>(c, *P, sp->ncy, sp->nmr, eta, psi, r);
    if (sp->prec == LQCD_F32) return sap_run<float>(c, *P, sp->ncy, sp->nmr, eta, psi, r);
    return set_err(c, LQCD_ERR_ARG, "SAP precision %d not supported", (int)sp->prec);
}

void sap_free_plans(lqcd_ctx *c)
{
    for (size_t i = 0; i < g_plans.size();) {
        if (g_plans[i].ctx == c) {
            cudaFree(g_plans[i].plan.blocks_dev);
            g_plans.erase(g_plans.begin() + i);
        } else
            i++;
    }
}

extern "C" lqcd_status lqcd_sap(lqcd_ctx *c, const lqcd_sap_params *sp, const double *eta, double *psi)
{
    if (!c || !sp || !eta || !psi) return set_err(c, LQCD_ERR_ARG, "null argument");
    lqcd_prec p = sp->prec;
    if (p != LQCD_F64 && p != LQCD_F32) return set_err(c, LQCD_ERR_ARG, "SAP precision %d", (int)p);
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
