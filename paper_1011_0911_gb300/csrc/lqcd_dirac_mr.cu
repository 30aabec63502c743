// Register-blocked multi-field stencil: one thread per (output site, group of
// NR = 2 or 3 right-hand sides).  Each link is loaded and its third row rebuilt once per
// NR fields, each clover block is loaded once and applied to all NR fields,
// and the coordinate / neighbour arithmetic is shared; the NR independent
// accumulation chains also give the scheduler more independent work per
// thread.  The arithmetic of every field is that of the single-field kernel
// in the same order, so results are bitwise identical to it.
#include "lqcd_stencil.cuh"

namespace stencil {

namespace {

// chirality half blk (spins 2 blk, 2 blk + 1) of a read-only native spinor
__device__ __forceinline__ void load_half(const float4 *__restrict__ f, long Vh, int r, int blk, cx<float> v[6])
{
#pragma unroll
    for (int q = 0; q < 3; q++) {
        float4 t = __ldg(f + (3 * blk + q) * Vh + r);
        v[2 * q] = mk(t.x, t.y);
        v[2 * q + 1] = mk(t.z, t.w);
    }
}
__device__ __forceinline__ void load_half(const h16s *__restrict__ f, long Vh, int r, int blk, cx<float> v[6])
{
    const uint4 *q = reinterpret_cast<const uint4 *>(f);
    const float s = __ldg(f16s_scales(f, Vh) + r);
    const uint2 mid = __ldg(reinterpret_cast<const uint2 *>(q + Vh + r) + blk);
    const uint4 end = __ldg(q + (blk ? 2 : 0) * Vh + r);
    const cx<float> a0 = f16s_h2c(end.x, s), a1 = f16s_h2c(end.y, s), a2 = f16s_h2c(end.z, s),
                    a3 = f16s_h2c(end.w, s), m0 = f16s_h2c(mid.x, s), m1 = f16s_h2c(mid.y, s);
    if (blk == 0) {
        v[0] = a0, v[1] = a1, v[2] = a2, v[3] = a3, v[4] = m0, v[5] = m1;
    } else {
        v[0] = m0, v[1] = m1, v[2] = a0, v[3] = a1, v[4] = a2, v[5] = a3;
    }
}

// The loads of all NR fields of a direction are issued before any of their
// arithmetic; a field index past the last valid one reads the last valid field
// again (its result is never stored), so no load is conditional and the loads
// can all be in flight together.
template <class R, class SP, class LK, int MU, int NR>
__device__ __forceinline__ void hop_dir_mr(const Geom &g, int p_out, int r, const int x[4], const SP *const (&fin)[NR],
                                           long Vh, const LK *U, Spinor<R> (&acc)[NR])
{
    cx<R> u[3][3];
    Spinor<R> psi[NR];
    {   // forward: (1 - g_mu) U_mu(x) psi(x + mu)
        const int ry = nbr_rank(g, x, MU, +1);
        const R sg = (MU == 0 && x[0] == g.L[0] - 1) ? R(g.bc_t) : R(1);
#pragma unroll
        for (int j = 0; j < NR; j++) load_spinor(fin[j], Vh, ry, psi[j]);
        load_link(U, Vh, p_out, MU, r, u);
#pragma unroll
        for (int j = 0; j < NR; j++) {
            cx<R> h[2][3], w[2][3];
            project<R, MU, -1>(psi[j], h);
            su3_vec(u, h[0], w[0]);
            su3_vec(u, h[1], w[1]);
            accumulate<R, MU, -1, MU == 0>(acc[j], w, sg);
        }
    }
    {   // backward: (1 + g_mu) U_mu(x - mu)^dag psi(x - mu)
        const int rz = nbr_rank(g, x, MU, -1);
        const R sg = (MU == 0 && x[0] == 0) ? R(g.bc_t) : R(1);
#pragma unroll
        for (int j = 0; j < NR; j++) load_spinor(fin[j], Vh, rz, psi[j]);
        load_link(U, Vh, 1 - p_out, MU, rz, u);
#pragma unroll
        for (int j = 0; j < NR; j++) {
            cx<R> h[2][3], w[2][3];
            project<R, MU, +1>(psi[j], h);
            su3dag_vec(u, h[0], w[0]);
            su3dag_vec(u, h[1], w[1]);
            accumulate<R, MU, +1, MU == 0>(acc[j], w, sg);
        }
    }
}

// occupancy variants of the blocked kernel: (max threads per CTA, min CTAs per SM)
template <int VAR>
struct VarMR;
template <>
struct VarMR<0> {
    static constexpr int T = 256, B = 1;
};
template <>
struct VarMR<1> {
    static constexpr int T = 128, B = 3;
};
template <>
struct VarMR<2> {
    static constexpr int T = 256, B = 2;
};

// modes as in k_hop (MODE_DHAT1 / MODE_DHAT2 / MODE_D).  One-dimensional grid:
// CTA b covers site tile b / ngy and field-group block b % ngy, so the CTAs of
// all field groups of a site tile run next to each other and share its links
// and clover term through L1/L2.
template <class R, class SP, class LK, class CL, int MODE, int NR, int VAR>
__global__ void __launch_bounds__(VarMR<VAR>::T, VarMR<VAR>::B) k_hop_mr(HopArgs<SP, LK, CL> a, int ngy)
{
    const int gy = blockIdx.x % ngy, tile = blockIdx.x / ngy;
    const int r = tile * blockDim.x + threadIdx.x;
    const int k0 = (gy * blockDim.y + threadIdx.y) * NR;
    const long Vh = a.g.Vh;
    if (r >= a.g.Vh || k0 >= a.nrhs) return;
    const int nk = min(NR, a.nrhs - k0);
    int x[4];
    rank_coords(a.g, a.p_out, r, x);
    const SP *fin[NR];
#pragma unroll
    for (int j = 0; j < NR; j++) fin[j] = a.in_other + (k0 + min(j, nk - 1)) * a.in_rs;
    Spinor<R> acc[NR];
    if (MODE == MODE_DHAT1) {
#pragma unroll
        for (int j = 0; j < NR; j++)
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int c = 0; c < 3; c++) acc[j].s[s][c] = mk(R(0), R(0));
    } else {
        // (1/f) A in_same with f = +-1/2: the exact factor 1/f is folded into the
        // clover entries (the same rounding as scaling the product)
        const R inv_f = MODE == MODE_DHAT2 ? R(2) : R(-2);
#pragma unroll
        for (int blk = 0; blk < 2; blk++) {
            Herm6<R> hm;
            load_herm(a.clov, Vh, r, blk, hm);
            herm_scale(hm, inv_f);
#pragma unroll
            for (int j = 0; j < NR; j++) {
                cx<R> v[6], w[6];
                load_half(a.in_same + (k0 + min(j, nk - 1)) * a.same_rs, Vh, r, blk, v);
                herm_apply(hm, v, w);
#pragma unroll
                for (int s = 0; s < 2; s++)
#pragma unroll
                    for (int c = 0; c < 3; c++) acc[j].s[2 * blk + s][c] = w[3 * s + c];
            }
        }
    }
    hop_dir_mr<R, SP, LK, 0, NR>(a.g, a.p_out, r, x, fin, Vh, a.U, acc);
    hop_dir_mr<R, SP, LK, 1, NR>(a.g, a.p_out, r, x, fin, Vh, a.U, acc);
    hop_dir_mr<R, SP, LK, 2, NR>(a.g, a.p_out, r, x, fin, Vh, a.U, acc);
    hop_dir_mr<R, SP, LK, 3, NR>(a.g, a.p_out, r, x, fin, Vh, a.U, acc);
    if (MODE == MODE_DHAT1) {
        // A^-1 (-1/2 S): the exact factor -1/2 is folded into the entries of A^-1
#pragma unroll
        for (int blk = 0; blk < 2; blk++) {
            Herm6<R> hm;
            load_herm(a.clov, Vh, r, blk, hm);
            herm_scale(hm, R(-0.5));
#pragma unroll
            for (int j = 0; j < NR; j++) {
                cx<R> v[6], w[6];
#pragma unroll
                for (int s = 0; s < 2; s++)
#pragma unroll
                    for (int c = 0; c < 3; c++) v[3 * s + c] = acc[j].s[2 * blk + s][c];
                herm_apply(hm, v, w);
#pragma unroll
                for (int s = 0; s < 2; s++)
#pragma unroll
                    for (int c = 0; c < 3; c++) acc[j].s[2 * blk + s][c] = w[3 * s + c];
            }
        }
    } else {
        const R f = MODE == MODE_DHAT2 ? R(0.5) : R(-0.5);
#pragma unroll
        for (int j = 0; j < NR; j++)
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int c = 0; c < 3; c++) acc[j].s[s][c] = f * acc[j].s[s][c];
    }
#pragma unroll
    for (int j = 0; j < NR; j++)
        if (j < nk) store_spinor(a.out + (k0 + j) * a.out_rs, Vh, r, acc[j]);
}

template <class R, class SP, class LK, class CL, int MODE, int NR>
void launch_nr(int var, int grid, dim3 b, int ngy, cudaStream_t st, const HopArgs<SP, LK, CL> &a)
{
    switch (var) {
        case 0: k_hop_mr<R, SP, LK, CL, MODE, NR, 0><<<grid, b, 0, st>>>(a, ngy); break;
        case 1: k_hop_mr<R, SP, LK, CL, MODE, NR, 1><<<grid, b, 0, st>>>(a, ngy); break;
        default: k_hop_mr<R, SP, LK, CL, MODE, NR, 2><<<grid, b, 0, st>>>(a, ngy); break;
    }
}

}  // namespace

template <class R, class SP, class LK, class CL, int MODE>
lqcd_status launch_hop_mr(lqcd_ctx *c, int nr, int var, dim3 b, const HopArgs<SP, LK, CL> &a)
{
    const int groups = (a.nrhs + nr - 1) / nr;
    const int ngy = div_up(groups, b.y);
    const long grid = (long)div_up(c->g.Vh, b.x) * ngy;
    if (grid > 0x7fffffffL) return set_err(c, LQCD_ERR_ARG, "blocked stencil: grid of %ld CTAs", grid);
    if (nr == 2)
        launch_nr<R, SP, LK, CL, MODE, 2>(var, (int)grid, b, ngy, c->stream, a);
    else if (nr == 3)
        launch_nr<R, SP, LK, CL, MODE, 3>(var, (int)grid, b, ngy, c->stream, a);
    else
        return set_err(c, LQCD_ERR_ARG, "no blocked stencil for %d fields per thread", nr);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

#define LQCD_MR_INST(R, SP, LK, CL, MODE) \
    template lqcd_status launch_hop_mr<R, SP, LK, CL, MODE>(lqcd_ctx *, int, int, dim3, const HopArgs<SP, LK, CL> &);
LQCD_MR_INST(float, float4, float4, float4, MODE_DHAT1)
LQCD_MR_INST(float, float4, float4, float4, MODE_DHAT2)
LQCD_MR_INST(float, float4, float4, float4, MODE_D)
LQCD_MR_INST(float, h16s, uint2, uint2, MODE_DHAT1)
LQCD_MR_INST(float, h16s, uint2, uint2, MODE_DHAT2)
LQCD_MR_INST(float, h16s, uint2, uint2, MODE_D)
#undef LQCD_MR_INST

}  // namespace stencil
