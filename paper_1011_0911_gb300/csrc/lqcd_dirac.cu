// Wilson-clover stencil kernels on native (site-minor) layouts: the
// single-field form and the dispatch of D, Dhat (Eq. 1, Eq. 2) over it and
// the register-blocked multi-field form (lqcd_dirac_mr.cu).
//
// One thread per (output site, right-hand side).  A CTA is blockDim.x sites
// by blockDim.y right-hand sides, so a warp reads 32 consecutive sites of one
// field (coalesced 16-byte loads) and the warps of the other right-hand
// sides reuse the same link / clover words from L1.
#include <type_traits>

#include "lqcd_stencil.cuh"
#include "lqcd_tune.h"

namespace {

using namespace stencil;

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

// output site r (rank of parity p_out), right-hand side k
template <class R, class SP, class LK, class CL, int MODE>
__device__ __forceinline__ void hop_site(const HopArgs<SP, LK, CL> &a, int r, int k)
{
    const long Vh = a.g.Vh;
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

// one-dimensional grid: CTA b covers site tile b / ngy and field block b % ngy,
// so the CTAs of all fields of a site tile run next to each other and share
// its links and clover term through L1/L2
template <class R, class SP, class LK, class CL, int MODE, int VAR>
__global__ void __launch_bounds__(Var<VAR>::T, Var<VAR>::B) k_hop(HopArgs<SP, LK, CL> a, int ngy)
{
    const int gy = blockIdx.x % ngy, tile = blockIdx.x / ngy;
    const int r = tile * blockDim.x + threadIdx.x;
    const int k = gy * blockDim.y + threadIdx.y;
    if (r >= a.g.Vh || k >= a.nrhs) return;
    hop_site<R, SP, LK, CL, MODE>(a, r, k);
}

// D on the full fields of several lattices in one launch.  items: (index of
// the HopArgs of a lattice and output parity, first rank of the tile, sites in
// the tile, lattice); tiles of lattices whose active flag is 0 are skipped.
template <class R, class SP, class LK, class CL>
__global__ void __launch_bounds__(256) k_hop_batch(const HopArgs<SP, LK, CL> *args, const int4 *items, const int *active)
{
    __shared__ HopArgs<SP, LK, CL> sa;
    const int4 w = items[blockIdx.x];
    if (active && !active[w.w]) return;
    if (threadIdx.x == 0) sa = args[w.x];
    __syncthreads();
    if ((int)threadIdx.x < w.z) hop_site<R, SP, LK, CL, MODE_D>(sa, w.y + threadIdx.x, 0);
}

template <class R, class SP, class LK, class CL, int MODE>
lqcd_status launch_var(lqcd_ctx *c, int var, dim3 b, const HopArgs<SP, LK, CL> &a)
{
    const int ngy = div_up(a.nrhs, b.y);
    const long nb = (long)div_up(c->g.Vh, b.x) * ngy;
    if (nb > 0x7fffffffL) return set_err(c, LQCD_ERR_ARG, "stencil: grid of %ld CTAs", nb);
    const int grid = (int)nb;
    switch (var) {
        case 0: k_hop<R, SP, LK, CL, MODE, 0><<<grid, b, 0, c->stream>>>(a, ngy); break;
        case 1: k_hop<R, SP, LK, CL, MODE, 1><<<grid, b, 0, c->stream>>>(a, ngy); break;
        case 2: k_hop<R, SP, LK, CL, MODE, 2><<<grid, b, 0, c->stream>>>(a, ngy); break;
        default: k_hop<R, SP, LK, CL, MODE, 3><<<grid, b, 0, c->stream>>>(a, ngy); break;
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

// LQCD_HOP_KIND = hop | mr | sm restricts the search to one kernel form
// (test instrumentation; ignored where that form does not exist)
int hop_force_kind(bool has_alt, int nrhs)
{
    const char *e = getenv("LQCD_HOP_KIND");
    if (!e || !*e) return -1;
    const std::string k(e);
    if (k == "hop") return KIND_HOP;
    if (k == "mr" && has_alt && nrhs >= 2) return KIND_MR;
    if (k == "sm" && has_alt) return KIND_SM;
    return -1;
}

// staged shapes: tx sites (16 or 32) x ty fields per CTA
std::vector<TuneChoice> hop_sm_candidates(int nrhs)
{
    std::vector<TuneChoice> v;
    std::vector<int> tys;
    for (int t : {nrhs, (nrhs + 1) / 2, (nrhs + 2) / 3, 4, 2, 1})
        if (t >= 1 && t <= nrhs && std::find(tys.begin(), tys.end(), t) == tys.end()) tys.push_back(t);
    for (int var = 0; var < NVAR_SM; var++)
        for (int ty : tys)
            for (int tx : {16, 32}) {
                const int n = tx * ty;
                if (n > var_sm_max_threads(var) || n < 32) continue;
                TuneChoice t;
                t.kind = KIND_SM;
                t.variant = var;
                t.tx = tx;
                t.ty = ty;
                v.push_back(t);
            }
    return v;
}

// register-blocked shapes: nr fields per thread, tx sites x ty field groups
std::vector<TuneChoice> hop_mr_candidates(int nrhs)
{
    std::vector<TuneChoice> v;
    for (int nr : {2, 3}) {
        if (nr > nrhs) continue;
        const int groups = (nrhs + nr - 1) / nr;
        std::vector<int> tys;
        for (int t : {1, 2, (groups + 1) / 2, groups})
            if (t >= 1 && t <= groups && std::find(tys.begin(), tys.end(), t) == tys.end()) tys.push_back(t);
        for (int var = 0; var < NVAR_MR; var++)
            for (int ty : tys)
                for (int tx : {32, 64, 128, 256}) {
                    const int n = tx * ty;
                    if (n > var_mr_max_threads(var) || n < 64) continue;
                    TuneChoice t;
                    t.variant = var;
                    t.tx = tx;
                    t.ty = ty;
                    t.nr = nr;
                    t.kind = KIND_MR;
                    v.push_back(t);
                }
    }
    return v;
}

template <class R, class SP, class LK, class CL, int MODE>
lqcd_status launch_choice(lqcd_ctx *c, const TuneChoice &t, const HopArgs<SP, LK, CL> &a)
{
    if constexpr (std::is_same<R, float>::value && MODE != MODE_HOP) {
        if (t.kind == KIND_MR) return launch_hop_mr<R, SP, LK, CL, MODE>(c, t.nr, t.variant, dim3(t.tx, t.ty), a);
        if (t.kind == KIND_SM) return launch_hop_sm<R, SP, LK, CL, MODE>(c, t.variant, dim3(t.tx, t.ty), a);
    }
    return launch_var<R, SP, LK, CL, MODE>(c, t.variant, dim3(t.tx, t.ty), a);
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
    constexpr bool has_alt = std::is_same<R, float>::value && MODE != MODE_HOP;
    const int force = hop_force_kind(has_alt, nrhs);
    static const char *kname[3] = {"k_hop4_hop", "k_hop4_mr", "k_hop4_sm"};
    std::string key = tune_key(c, force >= 0 ? kname[force] : "k_hop4", MODE, prec, nrhs);
    TuneChoice tc;
    if (!tune_lookup(key, &tc)) {
        tc = TuneChoice();
        tc.tx = nrhs == 1 ? 128 : 32;
        tc.ty = nrhs == 1 ? 1 : std::min(nrhs, 8);
        if (force == KIND_MR) {
            tc.kind = KIND_MR;
            tc.nr = 2;
            tc.tx = 64;
            tc.ty = 1;
        } else if (force == KIND_SM) {
            tc.kind = KIND_SM;
            tc.tx = 32;
            tc.ty = std::min(nrhs, 8);
        }
        if (tune_enabled()) {
            float best = 1e30f;
            std::vector<TuneChoice> cands;
            if (force < 0 || force == KIND_HOP) cands = hop_candidates(nrhs);
            if (has_alt && (force < 0 || force == KIND_MR))
                for (const TuneChoice &m : hop_mr_candidates(nrhs)) cands.push_back(m);
            if (has_alt && (force < 0 || force == KIND_SM))
                for (const TuneChoice &m : hop_sm_candidates(nrhs)) cands.push_back(m);
            for (const TuneChoice &cand : cands) {
                float us;
                lqcd_status s = tune_time(c, [&]() { return launch_choice<R, SP, LK, CL, MODE>(c, cand, a); }, 3, &us);
                if (s != LQCD_OK) return s;
                if (tune_verbose())
                    fprintf(stderr, "tune %s: kind=%d nr=%d var=%d %dx%d %.1f us\n", key.c_str(), cand.kind, cand.nr,
                            cand.variant, cand.tx, cand.ty, us);
                if (us < best) {
                    best = us;
                    tc = cand;
                    tc.us = us;
                }
            }
            tune_store(key, tc);
        }
    }
    return launch_choice<R, SP, LK, CL, MODE>(c, tc, a);
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

// ------------------------------------------------------------------ batches
struct DBatch {
    lqcd_prec p = LQCD_F32;
    int nlat = 0;
    long sites = 0;
    void *args = nullptr;                       // HopArgs[2 nlat]: (lattice, output parity)
    int4 *items[3] = {nullptr, nullptr, nullptr};   // tiles of 64 / 128 / 256 sites
    int nitems[3] = {0, 0, 0};
    int choice = -1;                            // tuned tile size index
};
static const int kBatchTile[3] = {64, 128, 256};

namespace {
template <class SP, class LK, class CL>
std::vector<HopArgs<SP, LK, CL>> batch_args(lqcd_ctx *const *ctx, int n, const SP *in, SP *out, const long *off,
                                            long units_per_site, const LK *const *U, const CL *const *A0,
                                            const CL *const *A1)
{
    std::vector<HopArgs<SP, LK, CL>> v;
    for (int l = 0; l < n; l++)
        for (int p = 0; p < 2; p++) {
            HopArgs<SP, LK, CL> a;
            const long half = units_per_site * ctx[l]->g.Vh;
            a.g = ctx[l]->g;
            a.p_out = p;
            a.nrhs = 1;
            a.in_other = in + off[l] + (1 - p) * half;
            a.in_rs = 0;
            a.in_same = in + off[l] + p * half;
            a.same_rs = 0;
            a.out = out + off[l] + p * half;
            a.out_rs = 0;
            a.U = U[l];
            a.clov = p ? A1[l] : A0[l];
            v.push_back(a);
        }
    return v;
}
}  // namespace

lqcd_status dirac_batch_create(lqcd_ctx *hc, lqcd_ctx *const *ctx, int n, lqcd_prec p, const void *in, void *out,
                               const long *off, DBatch **out_b)
{
    if (p != LQCD_F32 && p != LQCD_F64) return set_err(hc, LQCD_ERR_ARG, "batched D: precision %d", (int)p);
    DBatch *b = new DBatch();
    b->p = p;
    b->nlat = n;
    size_t argbytes;
    std::vector<unsigned char> host;
    if (p == LQCD_F32) {
        std::vector<const float4 *> U(n), A0(n), A1(n);
        for (int l = 0; l < n; l++) {
            U[l] = ctx[l]->U32;
            A0[l] = ctx[l]->A32[0];
            A1[l] = ctx[l]->A32[1];
        }
        auto v = batch_args<float4, float4, float4>(ctx, n, (const float4 *)in, (float4 *)out, off, 6, U.data(),
                                                    A0.data(), A1.data());
        argbytes = v.size() * sizeof(v[0]);
        host.assign((unsigned char *)v.data(), (unsigned char *)v.data() + argbytes);
    } else {
        std::vector<const double2 *> U(n), A0(n), A1(n);
        for (int l = 0; l < n; l++) {
            U[l] = ctx[l]->U64;
            A0[l] = ctx[l]->A64[0];
            A1[l] = ctx[l]->A64[1];
        }
        auto v = batch_args<double2, double2, double2>(ctx, n, (const double2 *)in, (double2 *)out, off, 12,
                                                       U.data(), A0.data(), A1.data());
        argbytes = v.size() * sizeof(v[0]);
        host.assign((unsigned char *)v.data(), (unsigned char *)v.data() + argbytes);
    }
    if (cudaMalloc(&b->args, argbytes) != cudaSuccess) {
        delete b;
        cudaGetLastError();
        return set_err(hc, LQCD_ERR_NOMEM, "batched D arguments");
    }
    cudaMemcpy(b->args, host.data(), argbytes, cudaMemcpyHostToDevice);
    for (int t = 0; t < 3; t++) {
        std::vector<int4> it;
        for (int l = 0; l < n; l++)
            for (int par = 0; par < 2; par++)
                for (int r0 = 0; r0 < ctx[l]->g.Vh; r0 += kBatchTile[t])
                    it.push_back(make_int4(2 * l + par, r0, std::min(kBatchTile[t], ctx[l]->g.Vh - r0), l));
        b->nitems[t] = (int)it.size();
        if (cudaMalloc(&b->items[t], it.size() * sizeof(int4)) != cudaSuccess) {
            cudaGetLastError();
            dirac_batch_free(b);
            return set_err(hc, LQCD_ERR_NOMEM, "batched D work list");
        }
        cudaMemcpy(b->items[t], it.data(), it.size() * sizeof(int4), cudaMemcpyHostToDevice);
    }
    for (int l = 0; l < n; l++) b->sites += ctx[l]->g.V;
    *out_b = b;
    return LQCD_OK;
}

void dirac_batch_free(DBatch *b)
{
    if (!b) return;
    cudaFree(b->args);
    for (int t = 0; t < 3; t++) cudaFree(b->items[t]);
    delete b;
}

namespace {
lqcd_status batch_launch(lqcd_ctx *hc, DBatch *b, int t, const int *active)
{
    if (b->p == LQCD_F32)
        k_hop_batch<float, float4, float4, float4><<<b->nitems[t], kBatchTile[t], 0, hc->stream>>>(
            (const HopArgs<float4, float4, float4> *)b->args, b->items[t], active);
    else
        k_hop_batch<double, double2, double2, double2><<<b->nitems[t], kBatchTile[t], 0, hc->stream>>>(
            (const HopArgs<double2, double2, double2> *)b->args, b->items[t], active);
    hc->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(hc);
    return LQCD_OK;
}
}  // namespace

// out = D in on every lattice of the batch (tile size chosen by the autotuner
// on the first call, which must not be inside a stream capture)
lqcd_status dirac_batch_D(lqcd_ctx *hc, DBatch *b, const int *active)
{
    if (b->choice < 0) {
        std::string key = "k_hop_batch/p" + std::to_string((int)b->p) + "/n" + std::to_string(b->nlat) + "/s" +
                          std::to_string(b->sites);
        TuneChoice tc;
        if (tune_lookup(key, &tc)) {
            b->choice = tc.variant;
        } else {
            b->choice = 1;
            if (tune_enabled()) {
                float best = 1e30f;
                for (int t = 0; t < 3; t++) {
                    float us;
                    LQCD_TRY(tune_time(hc, [&]() { return batch_launch(hc, b, t, active); }, 3, &us));
                    if (tune_verbose()) fprintf(stderr, "tune %s: tile %d %.1f us\n", key.c_str(), kBatchTile[t], us);
                    if (us < best) {
                        best = us;
                        b->choice = t;
                    }
                }
                tc.variant = b->choice;
                tc.tx = kBatchTile[b->choice];
                tc.us = best;
                tune_store(key, tc);
            }
        }
    }
    return batch_launch(hc, b, b->choice, active);
}
