// Multi-field stencil with the per-site operator staged in shared memory.
//
// A CTA covers TS consecutive output sites and blockDim.y right-hand sides.
// First its threads stage, once per site of the tile, the eight links of the
// site's hops with their third rows rebuilt (forward U_mu(x) and backward
// U_mu(x - mu)), the eight neighbour ranks, the time-boundary signs and the
// clover pair of the output parity.  Then one thread per (site, field)
// applies the hops and the clover term reading the operator from shared
// memory and only the spinors from global memory, so the link and clover
// loads, the third-row rebuild and the coordinate arithmetic are done once per
// site instead of once per (site, field).  The arithmetic of every field is
// that of k_hop in the same order: results are bitwise identical.
#include "lqcd_stencil.cuh"

namespace stencil {

namespace {

__device__ __forceinline__ float4 stage_cl(const float4 *p) { return __ldg(p); }
__device__ __forceinline__ float4 stage_cl(const uint2 *p)
{
    const uint2 t = __ldg(p);
    const cx<float> a = f16s_h2c(t.x, 1.f), b = f16s_h2c(t.y, 1.f);
    return make_float4(a.re, a.im, b.re, b.im);
}

template <int TS>
struct SmStage {
    cx<float> U[8][9][TS];   // link l: 0..3 forward U_mu(x), 4..7 backward U_mu(x - mu)
    float4 A[18][TS];        // clover pair of the output site
    int nbr[8][TS];          // neighbour ranks, in the order of U
    float sg[2][TS];         // boundary sign of the forward / backward time hop
};

template <int TS>
__device__ __forceinline__ void sm_herm(const SmStage<TS> &S, int s, int blk, Herm6<float> &h)
{
    float v[36];
#pragma unroll
    for (int q = 0; q < 9; q++) {
        const float4 t = S.A[9 * blk + q][s];
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

template <int TS>
__device__ __forceinline__ void sm_clover(const SmStage<TS> &S, int s, const Spinor<float> &in, Spinor<float> &out)
{
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        Herm6<float> h;
        sm_herm<TS>(S, s, blk, h);
        cx<float> v[6], w[6];
#pragma unroll
        for (int sp = 0; sp < 2; sp++)
#pragma unroll
            for (int c = 0; c < 3; c++) v[3 * sp + c] = in.s[2 * blk + sp][c];
        herm_apply(h, v, w);
#pragma unroll
        for (int sp = 0; sp < 2; sp++)
#pragma unroll
            for (int c = 0; c < 3; c++) out.s[2 * blk + sp][c] = w[3 * sp + c];
    }
}

template <int TS>
__device__ __forceinline__ void sm_link(const SmStage<TS> &S, int l, int s, cx<float> u[3][3])
{
#pragma unroll
    for (int e = 0; e < 9; e++) u[e / 3][e % 3] = S.U[l][e][s];
}

template <class SP, int MU, int TS>
__device__ __forceinline__ void sm_hop_dir(const SmStage<TS> &S, int s, const SP *in, long Vh, Spinor<float> &acc)
{
    cx<float> h[2][3], w[2][3], u[3][3];
    Spinor<float> psi;
    {
        const float sg = MU == 0 ? S.sg[0][s] : 1.f;
        load_spinor(in, Vh, S.nbr[MU][s], psi);
        project<float, MU, -1>(psi, h);
        sm_link<TS>(S, MU, s, u);
        su3_vec(u, h[0], w[0]);
        su3_vec(u, h[1], w[1]);
        accumulate<float, MU, -1, MU == 0>(acc, w, sg);
    }
    {
        const float sg = MU == 0 ? S.sg[1][s] : 1.f;
        load_spinor(in, Vh, S.nbr[4 + MU][s], psi);
        project<float, MU, +1>(psi, h);
        sm_link<TS>(S, 4 + MU, s, u);
        su3dag_vec(u, h[0], w[0]);
        su3dag_vec(u, h[1], w[1]);
        accumulate<float, MU, +1, MU == 0>(acc, w, sg);
    }
}

// occupancy variants: (max threads per CTA, min CTAs per SM)
template <int VAR>
struct VarSM;
template <>
struct VarSM<0> {
    static constexpr int T = 384, B = 1;
};
template <>
struct VarSM<1> {
    static constexpr int T = 384, B = 2;
};
template <>
struct VarSM<2> {
    static constexpr int T = 256, B = 3;
};

template <class SP, class LK, class CL, int MODE, int TS, int VAR>
__global__ void __launch_bounds__(VarSM<VAR>::T, VarSM<VAR>::B) k_hop_sm(HopArgs<SP, LK, CL> a, int ngy)
{
    __shared__ SmStage<TS> S;
    const long Vh = a.g.Vh;
    // one-dimensional grid, the field blocks of a site tile next to each other
    const int gy = blockIdx.x % ngy;
    const int r0 = (blockIdx.x / ngy) * TS;
    const int tid = threadIdx.y * TS + threadIdx.x, nthr = TS * blockDim.y;
    // ---- stage the operator of the tile's sites
    for (int w = tid; w < 8 * TS; w += nthr) {
        const int s = w % TS, l = w / TS, r = r0 + s;
        if (r >= Vh) continue;
        int x[4];
        rank_coords(a.g, a.p_out, r, x);
        const int mu = l & 3;
        const bool fwd = l < 4;
        const int nr = nbr_rank(a.g, x, mu, fwd ? +1 : -1);
        cx<float> u[3][3];
        load_link(a.U, Vh, fwd ? a.p_out : 1 - a.p_out, mu, fwd ? r : nr, u);
#pragma unroll
        for (int e = 0; e < 9; e++) S.U[l][e][s] = u[e / 3][e % 3];
        S.nbr[l][s] = nr;
        if (mu == 0)
            S.sg[fwd ? 0 : 1][s] =
                (fwd ? x[0] == a.g.L[0] - 1 : x[0] == 0) ? float(a.g.bc_t) : 1.f;
    }
    for (int w = tid; w < 18 * TS; w += nthr) {
        const int s = w % TS, q = w / TS, r = r0 + s;
        if (r < Vh) S.A[q][s] = stage_cl(a.clov + q * Vh + r);
    }
    __syncthreads();
    // ---- one thread per (site, field)
    const int s = threadIdx.x, r = r0 + s;
    const int k = gy * blockDim.y + threadIdx.y;
    if (r >= Vh || k >= a.nrhs) return;
    const SP *in = a.in_other + k * a.in_rs;
    Spinor<float> acc;
    if (MODE == MODE_DHAT1) {
#pragma unroll
        for (int sp = 0; sp < 4; sp++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc.s[sp][c] = mk(0.f, 0.f);
    } else {
        Spinor<float> self;
        load_spinor(a.in_same + k * a.same_rs, Vh, r, self);
        sm_clover<TS>(S, s, self, acc);
        const float inv_f = MODE == MODE_DHAT2 ? 2.f : -2.f;
#pragma unroll
        for (int sp = 0; sp < 4; sp++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc.s[sp][c] = inv_f * acc.s[sp][c];
    }
    sm_hop_dir<SP, 0, TS>(S, s, in, Vh, acc);
    sm_hop_dir<SP, 1, TS>(S, s, in, Vh, acc);
    sm_hop_dir<SP, 2, TS>(S, s, in, Vh, acc);
    sm_hop_dir<SP, 3, TS>(S, s, in, Vh, acc);
    const float f = MODE == MODE_DHAT2 ? 0.5f : -0.5f;
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
        for (int c = 0; c < 3; c++) acc.s[sp][c] = f * acc.s[sp][c];
    if (MODE == MODE_DHAT1) {
        Spinor<float> res;
        sm_clover<TS>(S, s, acc, res);
        store_spinor(a.out + k * a.out_rs, Vh, r, res);
    } else {
        store_spinor(a.out + k * a.out_rs, Vh, r, acc);
    }
}

template <class SP, class LK, class CL, int MODE, int TS>
void launch_ts(int var, int grid, dim3 b, int ngy, cudaStream_t st, const HopArgs<SP, LK, CL> &a)
{
    switch (var) {
        case 0: k_hop_sm<SP, LK, CL, MODE, TS, 0><<<grid, b, 0, st>>>(a, ngy); break;
        case 1: k_hop_sm<SP, LK, CL, MODE, TS, 1><<<grid, b, 0, st>>>(a, ngy); break;
        default: k_hop_sm<SP, LK, CL, MODE, TS, 2><<<grid, b, 0, st>>>(a, ngy); break;
    }
}

}  // namespace

template <class R, class SP, class LK, class CL, int MODE>
lqcd_status launch_hop_sm(lqcd_ctx *c, int var, dim3 b, const HopArgs<SP, LK, CL> &a)
{
    const int ngy = div_up(a.nrhs, b.y);
    const long nb = (long)div_up(c->g.Vh, b.x) * ngy;
    if (nb > 0x7fffffffL) return set_err(c, LQCD_ERR_ARG, "staged stencil: grid of %ld CTAs", nb);
    if (b.x == 16)
        launch_ts<SP, LK, CL, MODE, 16>(var, (int)nb, b, ngy, c->stream, a);
    else if (b.x == 32)
        launch_ts<SP, LK, CL, MODE, 32>(var, (int)nb, b, ngy, c->stream, a);
    else
        return set_err(c, LQCD_ERR_ARG, "staged stencil: tile of %d sites", (int)b.x);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

#define LQCD_SM_INST(SP, LK, CL, MODE) \
    template lqcd_status launch_hop_sm<float, SP, LK, CL, MODE>(lqcd_ctx *, int, dim3, const HopArgs<SP, LK, CL> &);
LQCD_SM_INST(float4, float4, float4, MODE_DHAT1)
LQCD_SM_INST(float4, float4, float4, MODE_DHAT2)
LQCD_SM_INST(float4, float4, float4, MODE_D)
LQCD_SM_INST(h16s, uint2, uint2, MODE_DHAT1)
LQCD_SM_INST(h16s, uint2, uint2, MODE_DHAT2)
LQCD_SM_INST(h16s, uint2, uint2, MODE_D)
#undef LQCD_SM_INST

}  // namespace stencil
