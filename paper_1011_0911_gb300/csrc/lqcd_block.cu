// DD-HMC block solves (Sec. 3: the inversions on the blocks needed for the
// block force use BiCGstab).  Every Dirichlet block's Schur operator
//   Dhat_blk = A_ee - H_eo,blk A_oo^-1 H_oe,blk
// (hops whose other end lies in another block are dropped; a block that spans
// a whole direction keeps the wrapped hop) is an independent system.  All
// blocks run BiCGstab (van der Vorst) in lockstep from psi = 0 with
// rhat = r_0 = eta|_blk:
//   rho = <rhat, r>, beta = (rho / rho_prev)(alpha / omega),
//   p = r + beta (p - omega v), v = Dhat_blk p, alpha = rho / <rhat, v>,
//   s = r - alpha v, (|s| <= tol |eta|: x += alpha p, done), t = Dhat_blk s,
//   omega = <t, s> / <t, t>, x += alpha p + omega s, r = s - omega t.
// The operator is one pair of lattice-wide launches; inner products are
// per-block reductions over a block-major list of the even sites (fixed order:
// per-CTA partials, then a per-block sum); the scalars and the activity flags
// live per block in device memory, and a block that has converged (or broken
// down) takes no further updates.  FP64 throughout.
#include <cmath>
#include <vector>

#include "lqcd_stencil.cuh"

namespace {

using namespace stencil;

struct BlkG {
    int bs[4], nb[4];
    int nblk, hb;   // blocks, even sites per block
};

__device__ __forceinline__ int blk_id(const BlkG &B, const int x[4])
{
    return x[3] / B.bs[3] + B.nb[3] * (x[2] / B.bs[2] + B.nb[2] * (x[1] / B.bs[1] + B.nb[1] * (x[0] / B.bs[0])));
}
// does the hop from x by d along mu stay in x's block (after the periodic wrap)?
__device__ __forceinline__ bool in_blk(const Geom &g, const BlkG &B, const int x[4], int mu, int d)
{
    int v = x[mu] + d;
    v = v < 0 ? v + g.L[mu] : (v >= g.L[mu] ? v - g.L[mu] : v);
    return v / B.bs[mu] == x[mu] / B.bs[mu];
}

// the hops of direction MU into x, each kept only inside x's block (same
// arithmetic as the lattice-wide stencil)
template <int MU>
__device__ __forceinline__ void bhop_dir(const Geom &g, const BlkG &B, int p_out, int r, const int x[4],
                                         const double2 *in, long Vh, const double2 *U, Spinor<double> &acc)
{
    cx<double> h[2][3], w[2][3], u[3][3];
    Spinor<double> psi;
    if (in_blk(g, B, x, MU, +1)) {
        const int ry = nbr_rank(g, x, MU, +1);
        const double sg = (MU == 0 && x[0] == g.L[0] - 1) ? double(g.bc_t) : 1.0;
        load_spinor(in, Vh, ry, psi);
        project<double, MU, -1>(psi, h);
        load_link(U, Vh, p_out, MU, r, u);
        su3_vec(u, h[0], w[0]);
        su3_vec(u, h[1], w[1]);
        accumulate<double, MU, -1, MU == 0>(acc, w, sg);
    }
    if (in_blk(g, B, x, MU, -1)) {
        const int rz = nbr_rank(g, x, MU, -1);
        const double sg = (MU == 0 && x[0] == 0) ? double(g.bc_t) : 1.0;
        load_spinor(in, Vh, rz, psi);
        project<double, MU, +1>(psi, h);
        load_link(U, Vh, 1 - p_out, MU, rz, u);
        su3dag_vec(u, h[0], w[0]);
        su3dag_vec(u, h[1], w[1]);
        accumulate<double, MU, +1, MU == 0>(acc, w, sg);
    }
}

// MODE_DHAT1: out_o = A_oo^-1 (-1/2 S_blk in_e);  MODE_DHAT2: out_e = A_ee same_e + 1/2 S_blk in_o
template <int MODE>
__global__ void __launch_bounds__(128) k_bhop(Geom g, BlkG B, const double2 *in, const double2 *same, double2 *out,
                                              const double2 *U, const double2 *cl)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.Vh) return;
    const long Vh = g.Vh;
    const int p_out = MODE == MODE_DHAT1 ? 1 : 0;
    int x[4];
    rank_coords(g, p_out, r, x);
    Spinor<double> acc;
    if (MODE == MODE_DHAT1) {
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc.s[s][c] = mk(0.0, 0.0);
    } else {
        Spinor<double> self;
        load_spinor(same, Vh, r, self);
        clover_apply<double, double2>(cl, Vh, r, self, acc);
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc.s[s][c] = 2.0 * acc.s[s][c];
    }
    bhop_dir<0>(g, B, p_out, r, x, in, Vh, U, acc);
    bhop_dir<1>(g, B, p_out, r, x, in, Vh, U, acc);
    bhop_dir<2>(g, B, p_out, r, x, in, Vh, U, acc);
    bhop_dir<3>(g, B, p_out, r, x, in, Vh, U, acc);
    const double f = MODE == MODE_DHAT2 ? 0.5 : -0.5;
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < 3; c++) acc.s[s][c] = f * acc.s[s][c];
    if (MODE == MODE_DHAT1) {
        Spinor<double> res;
        clover_apply<double, double2>(cl, Vh, r, acc, res);
        store_spinor(out, Vh, r, res);
    } else {
        store_spinor(out, Vh, r, acc);
    }
}

// list[b*hb + k] = rank of the k-th even site of block b (local lexicographic
// order; the block origin has even parity, so k = local lex / 2), blk[r] = b
__global__ void k_blist(Geom g, BlkG B, int *list, int *blk)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.Vh) return;
    int x[4];
    rank_coords(g, 0, r, x);
    const int b = blk_id(B, x);
    int l[4];
#pragma unroll
    for (int m = 0; m < 4; m++) l[m] = x[m] % B.bs[m];
    const int lex = l[3] + B.bs[3] * (l[2] + B.bs[2] * (l[1] + B.bs[1] * l[0]));
    list[(long)b * B.hb + (lex >> 1)] = r;
    blk[r] = b;
}

// per-block inner products <a_j, b_j> (j < ND) over the block's even sites:
// partial[(b*nch + c)*ND + j] for chunk c of the block's list
template <int ND>
struct DotSet {
    const double2 *a[ND], *b[ND];
};
template <int ND>
__global__ void __launch_bounds__(256) k_bdot(long Vh, int hb, int nch, const int *list, DotSet<ND> d,
                                              double2 *partial)
{
    const int b = blockIdx.x, c = blockIdx.y;   // blocks on x (no 65535 limit), chunks on y
    const int per = (hb + nch - 1) / nch, k0 = c * per, k1 = min(hb, k0 + per);
    double re[ND], im[ND];
#pragma unroll
    for (int j = 0; j < ND; j++) re[j] = im[j] = 0;
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const long r = list[(long)b * hb + k];
#pragma unroll
        for (int j = 0; j < ND; j++)
#pragma unroll
            for (int q = 0; q < 12; q++) {
                const double2 u = d.a[j][q * Vh + r], v = d.b[j][q * Vh + r];
                re[j] += u.x * v.x + u.y * v.y;
                im[j] += u.x * v.y - u.y * v.x;
            }
    }
    __shared__ double sh[8][ND][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < ND; j++) {
        double x = re[j], m = im[j];
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            m += __shfl_down_sync(0xffffffffu, m, o);
        }
        if (lane == 0) {
            sh[warp][j][0] = x;
            sh[warp][j][1] = m;
        }
    }
    __syncthreads();
    if (threadIdx.x < ND) {
        double x = 0, m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            x += sh[w][threadIdx.x][0];
            m += sh[w][threadIdx.x][1];
        }
        partial[((long)b * nch + c) * ND + threadIdx.x] = make_double2(x, m);
    }
}
// dots[b*ND + j] = sum over the block's chunks, in order
template <int ND>
__global__ void k_bdot_fin(int nblk, int nch, const double2 *partial, double2 *dots)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nblk * ND) return;
    const int b = i / ND, j = i - b * ND;
    double x = 0, m = 0;
    for (int c = 0; c < nch; c++) {
        const double2 v = partial[((long)b * nch + c) * ND + j];
        x += v.x;
        m += v.y;
    }
    dots[i] = make_double2(x, m);
}

// ---- per-block BiCGstab state and scalar steps (one thread per block)
struct BState {
    double2 rho, rho_prev, alpha, omega, beta;
    double e2;
    int active, half, iters, status;
};
__device__ __forceinline__ double2 cmul2(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv2(double2 a, double2 b)
{
    const double n = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / n, (a.y * b.x - a.x * b.y) / n);
}
__global__ void k_bs_init(int nblk, const double2 *dots, BState *S)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    BState s;
    s.e2 = dots[b].x;
    s.rho = s.beta = make_double2(0, 0);
    s.rho_prev = s.alpha = s.omega = make_double2(1, 0);
    s.active = s.e2 > 0 && isfinite(s.e2);
    s.half = 0;
    s.iters = 0;
    s.status = s.active ? LQCD_ERR_NOT_CONVERGED : (s.e2 == 0 ? LQCD_OK : LQCD_ERR_NAN);
    S[b] = s;
}
// from <rhat, r> and |r|^2: the convergence test of the previous step, the
// iteration limit, then beta; *nact = blocks still iterating
__global__ void k_bs_beta(int nblk, double tol2, int nmx, const double2 *dots, BState *S, int *nact)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nblk) {
        BState &s = S[b];
        if (s.active) {
            const double r2 = dots[2 * b + 1].x;
            if (s.iters > 0 && r2 <= tol2 * s.e2) {
                s.status = LQCD_OK;
                s.active = 0;
            } else if (!isfinite(r2)) {
                s.status = LQCD_ERR_NAN;
                s.active = 0;
            } else if (s.iters >= nmx) {
                s.active = 0;
            } else {
                const double2 rho = dots[2 * b];
                if (rho.x == 0 && rho.y == 0) {
                    s.status = LQCD_ERR_BREAKDOWN;
                    s.active = 0;
                } else {
                    s.rho = rho;
                    s.beta = cmul2(cdiv2(rho, s.rho_prev), cdiv2(s.alpha, s.omega));
                }
            }
        }
        if (s.active) atomicAdd(nact, 1);
    }
}
__global__ void k_bs_alpha(int nblk, const double2 *dots, BState *S)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk || !S[b].active) return;
    const double2 rv = dots[b];
    if (rv.x == 0 && rv.y == 0) {
        S[b].status = LQCD_ERR_BREAKDOWN;
        S[b].active = 0;
        return;
    }
    S[b].alpha = cdiv2(S[b].rho, rv);
}
// |s|^2: the step is counted; a block whose s is already small finishes with x += alpha p
__global__ void k_bs_s(int nblk, double tol2, const double2 *dots, BState *S)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk || !S[b].active) return;
    S[b].iters++;
    if (dots[b].x <= tol2 * S[b].e2) {
        S[b].half = 1;
        S[b].status = LQCD_OK;
    }
}
// <t, s> and |t|^2: omega
__global__ void k_bs_omega(int nblk, const double2 *dots, BState *S)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk || !S[b].active || S[b].half) return;
    const double tt = dots[2 * b + 1].x;
    if (tt == 0) {
        S[b].status = LQCD_ERR_BREAKDOWN;
        S[b].active = 0;
        return;
    }
    const double2 ts = dots[2 * b];
    S[b].omega = make_double2(ts.x / tt, ts.y / tt);
}
__global__ void k_bs_end(int nblk, BState *S)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk || !S[b].active) return;
    if (S[b].half)
        S[b].active = 0;
    else
        S[b].rho_prev = S[b].rho;
}

// ---- elementwise updates on the even sites of active blocks
__device__ __forceinline__ double2 cfma(double2 a, double2 x, double2 y)   // y + a x
{
    return make_double2(y.x + a.x * x.x - a.y * x.y, y.y + a.x * x.y + a.y * x.x);
}
// p = r + beta (p - omega v)
__global__ void k_bu_p(long Vh, const int *blk, const BState *S, const double2 *r, const double2 *v, double2 *p)
{
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= 12 * Vh) return;
    const BState &s = S[blk[i % Vh]];
    if (!s.active) return;
    const double2 w = cfma(make_double2(-s.omega.x, -s.omega.y), v[i], p[i]);
    p[i] = cfma(s.beta, w, r[i]);
}
// s = r - alpha v
__global__ void k_bu_s(long Vh, const int *blk, const BState *S, const double2 *r, const double2 *v, double2 *sv)
{
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= 12 * Vh) return;
    const BState &s = S[blk[i % Vh]];
    if (!s.active) return;
    sv[i] = cfma(make_double2(-s.alpha.x, -s.alpha.y), v[i], r[i]);
}
// x += alpha p (+ omega s); r = s - omega t
__global__ void k_bu_xr(long Vh, const int *blk, const BState *S, const double2 *p, const double2 *sv,
                        const double2 *t, double2 *x, double2 *r)
{
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= 12 * Vh) return;
    const BState &s = S[blk[i % Vh]];
    if (!s.active) return;
    if (s.half) {
        x[i] = cfma(s.alpha, p[i], x[i]);
        return;
    }
    x[i] = cfma(s.omega, sv[i], cfma(s.alpha, p[i], x[i]));
    r[i] = cfma(make_double2(-s.omega.x, -s.omega.y), t[i], sv[i]);
}
__global__ void k_bsub(long n, const double2 *a, const double2 *b, double2 *out)
{
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_double2(a[i].x - b[i].x, a[i].y - b[i].y);
}

// ---- host side
struct BlockRun {
    lqcd_ctx *c;
    BlkG B;
    int nch;
    int *list = nullptr, *blk = nullptr;
    double2 *partial = nullptr, *dots = nullptr;
    BState *S = nullptr;
    int *nact = nullptr;
    ~BlockRun()
    {
        cudaFree(list);
        cudaFree(blk);
        cudaFree(partial);
        cudaFree(dots);
        cudaFree(S);
        cudaFree(nact);
    }
    lqcd_status init()
    {
        const long Vh = c->g.Vh;
        // about 4 CTAs per SM over all blocks, at least 64 sites per chunk
        nch = std::max(1, std::min(B.hb / 64, (4 * 152 + B.nblk - 1) / B.nblk));
        if (cudaMalloc(&list, sizeof(int) * (size_t)B.nblk * B.hb) != cudaSuccess ||
            cudaMalloc(&blk, sizeof(int) * Vh) != cudaSuccess ||
            cudaMalloc(&partial, sizeof(double2) * (size_t)B.nblk * nch * 2) != cudaSuccess ||
            cudaMalloc(&dots, sizeof(double2) * (size_t)B.nblk * 2) != cudaSuccess ||
            cudaMalloc(&S, sizeof(BState) * B.nblk) != cudaSuccess || cudaMalloc(&nact, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, LQCD_ERR_NOMEM, "block solver buffers");
        }
        k_blist<<<div_up(Vh, 256), 256, 0, c->stream>>>(c->g, B, list, blk);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        return LQCD_OK;
    }
    // out_e = Dhat_blk in_e (tmp_o: one odd FP64 half field)
    lqcd_status dhat(const double2 *in, double2 *out, double2 *tmp)
    {
        const int grid = div_up(c->g.Vh, 128);
        k_bhop<MODE_DHAT1><<<grid, 128, 0, c->stream>>>(c->g, B, in, nullptr, tmp, c->U64, c->Ai64[1]);
        k_bhop<MODE_DHAT2><<<grid, 128, 0, c->stream>>>(c->g, B, tmp, in, out, c->U64, c->A64[0]);
        c->n_kernel_launches += 2;
        LQCD_LAUNCH_CHECK(c);
        return LQCD_OK;
    }
    template <int ND>
    lqcd_status bdots(DotSet<ND> d)
    {
        k_bdot<ND><<<dim3(B.nblk, nch), 256, 0, c->stream>>>(c->g.Vh, B.hb, nch, list, d, partial);
        k_bdot_fin<ND><<<div_up(B.nblk * ND, 128), 128, 0, c->stream>>>(B.nblk, nch, partial, dots);
        c->n_kernel_launches += 2;
        LQCD_LAUNCH_CHECK(c);
        return LQCD_OK;
    }
};

lqcd_status make_blocking(lqcd_ctx *c, const int bs[4], BlkG &B)
{
    B.nblk = 1;
    int vol = 1;
    for (int m = 0; m < 4; m++) {
        if (bs[m] <= 0 || bs[m] % 2 || c->g.L[m] % bs[m])
            return set_err(c, LQCD_ERR_ARG, "block extent %d does not tile L[%d] = %d evenly", bs[m], m, c->g.L[m]);
        B.bs[m] = bs[m];
        B.nb[m] = c->g.L[m] / bs[m];
        B.nblk *= B.nb[m];
        vol *= bs[m];
    }
    B.hb = vol / 2;
    return LQCD_OK;
}

}  // namespace

extern "C" {

long lqcd_block_count(const lqcd_ctx *c, const int bs[4])
{
    if (!c || !bs) return -1;
    long n = 1;
    for (int m = 0; m < 4; m++) {
        if (bs[m] <= 0 || bs[m] % 2 || c->g.L[m] % bs[m]) return -1;
        n *= c->g.L[m] / bs[m];
    }
    return n;
}

lqcd_status lqcd_apply_Dhat_block(lqcd_ctx *c, const int bs[4], const double *in_e, double *out_e)
{
    if (!c || !bs || !in_e || !out_e) return set_err(c, LQCD_ERR_ARG, "null argument");
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    BlockRun R{c};
    LQCD_TRY(make_blocking(c, bs, R.B));
    const size_t hb = native_half_bytes(c, LQCD_F64);
    void *a, *o, *t;
    LQCD_TRY(ws_get(c, WS_PACK_IN, hb, &a));
    LQCD_TRY(ws_get(c, WS_PACK_OUT, hb, &o));
    LQCD_TRY(ws_get(c, WS_TMP_O, hb, &t));
    LQCD_TRY(pack_field(c, LQCD_F64, 1, in_e, a, 1, false));
    LQCD_TRY(R.dhat((const double2 *)a, (double2 *)o, (double2 *)t));
    return pack_field(c, LQCD_F64, 1, out_e, o, 1, true);
}

lqcd_status lqcd_block_solve(lqcd_ctx *c, const lqcd_block_params *p, const double *eta_e, double *psi_e, int *iters,
                             double *relres, int *status)
{
    if (!c || !p || !eta_e || !psi_e) return set_err(c, LQCD_ERR_ARG, "null argument");
    if (!(p->tol > 0) || p->nmx < 0) return set_err(c, LQCD_ERR_ARG, "tol must be > 0 and nmx >= 0");
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    BlockRun R{c};
    LQCD_TRY(make_blocking(c, p->bs, R.B));
    LQCD_TRY(R.init());
    const long Vh = c->g.Vh, nh = 12 * Vh;
    void *buf;
    LQCD_TRY(ws_get(c, WS_SOLVER, 9 * nh * sizeof(double2), &buf));
    double2 *eta = (double2 *)buf, *x = eta + nh, *r = x + nh, *rh = r + nh, *pv = rh + nh, *v = pv + nh,
            *sv = v + nh, *t = sv + nh, *tmp = t + nh;
    LQCD_TRY(pack_field(c, LQCD_F64, 1, eta_e, eta, 1, false));
    LQCD_CUDA_CHECK(c, cudaMemsetAsync(x, 0, nh * sizeof(double2), c->stream));
    LQCD_CUDA_CHECK(c, cudaMemsetAsync(pv, 0, nh * sizeof(double2), c->stream));
    LQCD_CUDA_CHECK(c, cudaMemsetAsync(v, 0, nh * sizeof(double2), c->stream));
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(r, eta, nh * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(rh, eta, nh * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    const int nb = R.B.nblk, gb = div_up(nb, 128), ge = (int)div_up(nh, 256);
    const double tol2 = p->tol * p->tol;
    LQCD_TRY(R.bdots<1>(DotSet<1>{{eta}, {eta}}));
    k_bs_init<<<gb, 128, 0, c->stream>>>(nb, R.dots, R.S);
    c->n_kernel_launches++;
    int *nact_host = (int *)c->red_host;
    for (;;) {
        // <rhat, r>, |r|^2: convergence of the last step, iteration limit, beta
        LQCD_TRY(R.bdots<2>(DotSet<2>{{rh, r}, {r, r}}));
        LQCD_CUDA_CHECK(c, cudaMemsetAsync(R.nact, 0, sizeof(int), c->stream));
        k_bs_beta<<<gb, 128, 0, c->stream>>>(nb, tol2, p->nmx, R.dots, R.S, R.nact);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
        LQCD_CUDA_CHECK(c, cudaMemcpyAsync(nact_host, R.nact, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
        if (*nact_host == 0) break;
        k_bu_p<<<ge, 256, 0, c->stream>>>(Vh, R.blk, R.S, r, v, pv);
        c->n_kernel_launches++;
        LQCD_TRY(R.dhat(pv, v, tmp));
        LQCD_TRY(R.bdots<1>(DotSet<1>{{rh}, {v}}));
        k_bs_alpha<<<gb, 128, 0, c->stream>>>(nb, R.dots, R.S);
        k_bu_s<<<ge, 256, 0, c->stream>>>(Vh, R.blk, R.S, r, v, sv);
        c->n_kernel_launches += 2;
        LQCD_TRY(R.bdots<1>(DotSet<1>{{sv}, {sv}}));
        k_bs_s<<<gb, 128, 0, c->stream>>>(nb, tol2, R.dots, R.S);
        c->n_kernel_launches++;
        LQCD_TRY(R.dhat(sv, t, tmp));
        LQCD_TRY(R.bdots<2>(DotSet<2>{{t, t}, {sv, t}}));
        k_bs_omega<<<gb, 128, 0, c->stream>>>(nb, R.dots, R.S);
        k_bu_xr<<<ge, 256, 0, c->stream>>>(Vh, R.blk, R.S, pv, sv, t, x, r);
        k_bs_end<<<gb, 128, 0, c->stream>>>(nb, R.S);
        c->n_kernel_launches += 3;
        LQCD_LAUNCH_CHECK(c);
    }
    // recomputed residual of every block
    LQCD_TRY(R.dhat(x, t, tmp));
    k_bsub<<<ge, 256, 0, c->stream>>>(nh, eta, t, t);
    c->n_kernel_launches++;
    LQCD_TRY(R.bdots<1>(DotSet<1>{{t}, {t}}));
    std::vector<BState> hs(nb);
    std::vector<double2> hd(nb);
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(hs.data(), R.S, nb * sizeof(BState), cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(hd.data(), R.dots, nb * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    lqcd_status worst = LQCD_OK;
    for (int b = 0; b < nb; b++) {
        if (iters) iters[b] = hs[b].iters;
        if (relres) relres[b] = hs[b].e2 > 0 ? std::sqrt(hd[b].x / hs[b].e2) : 0.0;
        if (status) status[b] = hs[b].status;
        if (hs[b].status != LQCD_OK && worst == LQCD_OK) worst = (lqcd_status)hs[b].status;
    }
    LQCD_TRY(pack_field(c, LQCD_F64, 1, psi_e, x, 1, true));
    if (worst != LQCD_OK) set_err(c, worst, "block solve: a block did not converge (status %d)", (int)worst);
    return worst;
}

}  // extern "C"
