// Batched solve of several independent lattices with the SAP-preconditioned
// flexible GCR (Sec. 3-4; Dhat systems through Eq. 5), one right-hand side per
// lattice.  All lattices' fields live in shared arenas (lattice l at a fixed
// offset); every phase of a GCR step is one launch over a flat work list of
// (lattice, item) pairs of all lattices, so small and large lattices fill the
// GPU together:
//
//   phi_k = M_sap rho      FP64 -> sap precision, batched SAP, -> FP64
//   chi_k = D phi_k        FP64 -> F32, batched D, -> FP64
//   Gram-Schmidt           one cooperative persistent kernel (k_gs): dot
//                          products, per-lattice coefficients, updates, the new
//                          residual and its norm, separated by grid barriers
//                          whose waits are bounded (LQCD_ERR_TIMEOUT)
//
// Per-lattice scalars and flags stay on the device: a lattice that has
// converged in the cycle stops taking steps (its work items are skipped) and
// the cycle ends with the solution update; the next cycle starts from the FP64
// true residual.  The host waits once per cycle, after the restart, to see
// which lattices are still running.  A cycle's steps and update can be
// captured once as a CUDA graph and replayed.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "lqcd_f16s.cuh"
#include "lqcd_internal.cuh"

namespace {

constexpr int BNKV = 32;           // largest Krylov space of a cycle
constexpr int CHUNK = 2048;        // complex entries per BLAS work item
constexpr int PS = BNKV + 2;       // partial-sum slots per work item
constexpr int GS_THREADS = 256;
constexpr int TILE = 128;          // sites per conversion work item

struct BLat {            // layout of lattice l in the arenas
    long Vh;
    long off64;          // double2 units (FP64 arena, 24 Vh per full field)
    long off32;          // float4 units (F32 arena, 12 Vh)
    long offs;           // units of the SAP arena (F32: float4, 12 Vh; F16S: h16s, 13 Vh / 2)
    int it0, it1;        // its BLAS work items
};

struct BItem {           // complex entries [s0, s0 + n) of a full FP64 field of lattice lat
    int lat, n;
    long s0;
};

struct BScal {           // per-lattice GCR state (device)
    int done;            // converged: FP64 true residual below tolerance
    int nk;              // steps of the current cycle
    int iters;           // steps in total
    int restarts;
    int status;
    int pass2;           // second Gram-Schmidt pass in this step
    double eta2, tol2, rn2, cyc_tol2, true_rn2;
};

struct BMat {            // per-lattice Krylov coefficients (device)
    double b[BNKV];
    double2 c[BNKV], coef[BNKV], alpha[BNKV];
    double2 a[BNKV][BNKV];   // a[i][k], i < k
};

struct GridBar {
    unsigned int count, gen;
};

__device__ __forceinline__ double2 ld2(const double2 *p) { return __ldcg(p); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
// conj(a) b
__device__ __forceinline__ double2 cdot(double2 a, double2 b)
{
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Grid-wide barrier of a cooperative launch.  Every wait is bounded: after
// `limit` clock cycles the CTA records LQCD_ERR_TIMEOUT in *status and the
// barrier returns false (the caller then leaves the kernel).
__device__ bool grid_wait(GridBar *bar, unsigned int expected, long long limit, int *status)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int *vg = &bar->gen;
        const unsigned int g = *vg;
        __threadfence();
        const unsigned int arrived = atomicAdd(&bar->count, 1u) + 1u;
        if (arrived == expected) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vg == g) {
                if (clock64() - t0 > limit) {
                    ok = 0;
                    atomicExch(status, (int)LQCD_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// block sum of one double2 (fixed order); valid in thread 0
__device__ double2 block_sum(double2 v, double2 *sm)
{
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm[w] = v;
    __syncthreads();
    double2 s = make_double2(0, 0);
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s = cadd(s, sm[i]);
    return s;
}

// fixed-order sum of slot j of the partials of lattice items [i0, i1), by one warp
__device__ double2 warp_items_sum(const double2 *part, int i0, int i1, int j)
{
    double2 s = make_double2(0, 0);
    for (int it = i0 + (threadIdx.x & 31); it < i1; it += 32) s = cadd(s, ld2(part + (long)it * PS + j));
    for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_down_sync(0xffffffffu, s.x, o);
        s.y += __shfl_down_sync(0xffffffffu, s.y, o);
    }
    return s;   // lane 0
}

struct GsArgs {
    const BLat *lat;
    const BItem *items;
    int nitems, nlat, k;
    long N;              // complex entries of one FP64 arena vector
    double2 *chi;        // chi_0 .. chi_{nkv-1}, N apart
    double2 *rho;
    BScal *sc;
    BMat *mat;
    int *act;
    double2 *part;
    GridBar *bar;
    long long limit;
    int stall;           // test aid: the first barrier waits for one CTA too many
    int *status;         // LQCD_ERR_TIMEOUT when a wait ran out
    int nmx;
};

// One GCR step k for every active lattice: classical Gram-Schmidt of chi_k
// against chi_0..chi_{k-1} (a second pass where the first removed more than
// half of |chi_k|^2), b_k = |chi_k|, c_k = <chi_k, rho> / b_k, chi_k /= b_k,
// rho -= c_k chi_k, |rho|^2, and the per-lattice stopping tests.
__global__ void __launch_bounds__(GS_THREADS) k_gs(GsArgs a)
{
    __shared__ double2 sm[GS_THREADS / 32];
    const int k = a.k, G = gridDim.x;
    const unsigned int nb = gridDim.x;
    double2 *chik = a.chi + (long)k * a.N;
    constexpr int PER = CHUNK / GS_THREADS;
    for (int pass = 0; pass < 2; pass++) {
        // ---- A: partial <chi_i, chi_k>, i < k (pass 0 also i = k)
        for (int it = blockIdx.x; it < a.nitems; it += G) {
            const BItem w = a.items[it];
            if (!a.act[w.lat]) continue;
            if (pass == 1 && !__ldcg(&a.sc[w.lat].pass2)) continue;
            const long base = a.lat[w.lat].off64 + w.s0;
            double2 xk[PER];
#pragma unroll
            for (int e = 0; e < PER; e++) {
                const int j = threadIdx.x + e * GS_THREADS;
                xk[e] = j < w.n ? chik[base + j] : make_double2(0, 0);
            }
            const int m = pass == 0 ? k + 1 : k;
            for (int i = 0; i < m; i++) {
                const double2 *ci = a.chi + (long)i * a.N + base;
                double2 s = make_double2(0, 0);
#pragma unroll
                for (int e = 0; e < PER; e++) {
                    const int j = threadIdx.x + e * GS_THREADS;
                    if (j < w.n) s = cadd(s, cdot(ci[j], xk[e]));
                }
                s = block_sum(s, sm);
                if (threadIdx.x == 0) a.part[(long)it * PS + i] = s;
            }
        }
        if (!grid_wait(a.bar, nb + (a.stall && pass == 0 ? 1u : 0u), a.limit, a.status)) return;
        // ---- B: per-lattice coefficients
        if (threadIdx.x < 32)
            for (int l = blockIdx.x; l < a.nlat; l += G) {
                if (!a.act[l]) continue;
                if (pass == 1 && !__ldcg(&a.sc[l].pass2)) continue;
                const int m = pass == 0 ? k + 1 : k;
                double removed = 0, dkk = 0;
                for (int i = 0; i < m; i++) {
                    const double2 d = warp_items_sum(a.part, a.lat[l].it0, a.lat[l].it1, i);
                    if (threadIdx.x == 0) {
                        if (i == k) {
                            dkk = d.x;
                        } else {
                            double2 &ai = a.mat[l].a[i][k];
                            ai = pass == 0 ? d : cadd(ai, d);
                            a.mat[l].coef[i] = d;
                            removed += d.x * d.x + d.y * d.y;
                        }
                    }
                }
                if (threadIdx.x == 0) {
                    if (pass == 0) a.sc[l].pass2 = (k > 0 && removed > 0.5 * dkk) ? 1 : 0;
                    __threadfence();
                }
            }
        if (!grid_wait(a.bar, nb, a.limit, a.status)) return;
        // ---- C: chi_k -= sum_i coef_i chi_i; final |chi_k|^2, <chi_k, rho> where done
        for (int it = blockIdx.x; it < a.nitems; it += G) {
            const BItem w = a.items[it];
            if (!a.act[w.lat]) continue;
            const int p2 = __ldcg(&a.sc[w.lat].pass2);
            if (pass == 1 && !p2) continue;
            const long base = a.lat[w.lat].off64 + w.s0;
            double2 xk[PER];
#pragma unroll
            for (int e = 0; e < PER; e++) {
                const int j = threadIdx.x + e * GS_THREADS;
                xk[e] = j < w.n ? chik[base + j] : make_double2(0, 0);
            }
            for (int i = 0; i < k; i++) {
                const double2 cf = ld2(&a.mat[w.lat].coef[i]);
                const double2 *ci = a.chi + (long)i * a.N + base;
#pragma unroll
                for (int e = 0; e < PER; e++) {
                    const int j = threadIdx.x + e * GS_THREADS;
                    if (j < w.n) {
                        const double2 t = cmul(cf, ci[j]);
                        xk[e].x -= t.x;
                        xk[e].y -= t.y;
                    }
                }
            }
            double2 q = make_double2(0, 0), cr = make_double2(0, 0);
#pragma unroll
            for (int e = 0; e < PER; e++) {
                const int j = threadIdx.x + e * GS_THREADS;
                if (j < w.n) {
                    if (k > 0) chik[base + j] = xk[e];
                    q.x += xk[e].x * xk[e].x + xk[e].y * xk[e].y;
                    cr = cadd(cr, cdot(xk[e], a.rho[base + j]));
                }
            }
            if (pass == 1 || !p2) {
                q = block_sum(q, sm);
                cr = block_sum(cr, sm);
                if (threadIdx.x == 0) {
                    a.part[(long)it * PS + 0] = q;
                    a.part[(long)it * PS + 1] = cr;
                }
            }
        }
        if (!grid_wait(a.bar, nb, a.limit, a.status)) return;
    }
    // ---- D: b_k, c_k per lattice
    if (threadIdx.x < 32)
        for (int l = blockIdx.x; l < a.nlat; l += G) {
            if (!a.act[l]) continue;
            const double2 q = warp_items_sum(a.part, a.lat[l].it0, a.lat[l].it1, 0);
            const double2 cr = warp_items_sum(a.part, a.lat[l].it0, a.lat[l].it1, 1);
            if (threadIdx.x == 0) {
                const double b = sqrt(q.x);
                if (!(b > 0) || !isfinite(b) || !isfinite(cr.x) || !isfinite(cr.y)) {
                    a.sc[l].status = isfinite(b) ? LQCD_ERR_BREAKDOWN : LQCD_ERR_NAN;
                    a.sc[l].done = 1;
                    a.act[l] = 0;
                } else {
                    a.mat[l].b[k] = b;
                    a.mat[l].c[k] = make_double2(cr.x / b, cr.y / b);
                }
                __threadfence();
            }
        }
    if (!grid_wait(a.bar, nb, a.limit, a.status)) return;
    // ---- E: chi_k /= b_k; rho -= c_k chi_k; partial |rho|^2
    for (int it = blockIdx.x; it < a.nitems; it += G) {
        const BItem w = a.items[it];
        if (!__ldcg(&a.act[w.lat])) continue;
        const long base = a.lat[w.lat].off64 + w.s0;
        const double inv = 1.0 / __ldcg(&a.mat[w.lat].b[k]);
        const double2 c = ld2(&a.mat[w.lat].c[k]);
        double2 s = make_double2(0, 0);
        for (int j = threadIdx.x; j < w.n; j += GS_THREADS) {
            double2 x = chik[base + j];
            x.x *= inv;
            x.y *= inv;
            chik[base + j] = x;
            const double2 t = cmul(c, x);
            double2 r = a.rho[base + j];
            r.x -= t.x;
            r.y -= t.y;
            a.rho[base + j] = r;
            s.x += r.x * r.x + r.y * r.y;
        }
        s = block_sum(s, sm);
        if (threadIdx.x == 0) a.part[(long)it * PS + 0] = s;
    }
    if (!grid_wait(a.bar, nb, a.limit, a.status)) return;
    // ---- F: |rho|^2 and the stopping tests of the cycle
    if (threadIdx.x < 32)
        for (int l = blockIdx.x; l < a.nlat; l += G) {
            if (!__ldcg(&a.act[l])) continue;
            const double2 s = warp_items_sum(a.part, a.lat[l].it0, a.lat[l].it1, 0);
            if (threadIdx.x == 0) {
                BScal &S = a.sc[l];
                S.rn2 = s.x;
                S.nk = k + 1;
                S.iters++;
                if (!(s.x > S.cyc_tol2) || S.iters >= a.nmx) a.act[l] = 0;
            }
        }
}

// ---- cycle start: rho = eta - D psi (FP64), |rho|^2, activity of the cycle
__global__ void k_b_resid(const BLat *lat, const BItem *items, const int *act, const double2 *eta, const double2 *t,
                          double2 *rho, double2 *part)
{
    __shared__ double2 sm[GS_THREADS / 32];
    const BItem w = items[blockIdx.x];
    if (!act[w.lat]) return;
    const long base = lat[w.lat].off64 + w.s0;
    double2 s = make_double2(0, 0);
    for (int j = threadIdx.x; j < w.n; j += blockDim.x) {
        const double2 e = eta[base + j], d = t[base + j];
        const double2 r = make_double2(e.x - d.x, e.y - d.y);
        rho[base + j] = r;
        s.x += r.x * r.x + r.y * r.y;
    }
    s = block_sum(s, sm);
    if (threadIdx.x == 0) part[(long)blockIdx.x * PS] = s;
}
// one warp per lattice; gain2: the cycle stops once |rho|^2 fell by this factor
__global__ void k_b_restart(const BLat *lat, const double2 *part, int *act, BScal *sc, int nlat, double gain2)
{
    const int l = blockIdx.x;
    if (l >= nlat || !act[l]) return;
    const double2 s = warp_items_sum(part, lat[l].it0, lat[l].it1, 0);
    if (threadIdx.x != 0) return;
    BScal &S = sc[l];
    S.true_rn2 = s.x;
    S.rn2 = s.x;
    S.nk = 0;
    if (S.iters > 0) S.restarts++;
    if (!(s.x > S.tol2)) {
        S.done = 1;
        S.status = LQCD_OK;
        act[l] = 0;
    } else if (!isfinite(s.x)) {
        S.done = 1;
        S.status = LQCD_ERR_NAN;
        act[l] = 0;
    } else {
        S.cyc_tol2 = fmax(S.tol2, s.x * gain2);
    }
}
// cycle start: every lattice not done and below the step limit runs; no
// lattice carries steps (and so a solution update) over from the last cycle
__global__ void k_b_activate(int *act, BScal *sc, int nlat, int nmx)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlat) return;
    sc[l].nk = 0;
    act[l] = (!sc[l].done && sc[l].iters < nmx) ? 1 : 0;
}

// ---- cycle end: R alpha = c (R upper triangular: a[i][j], b[j]), psi += sum alpha_j phi_j
__global__ void k_b_backsub(BScal *sc, BMat *mat, int nlat)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlat) return;
    const int nk = sc[l].nk;
    BMat &M = mat[l];
    for (int i = nk - 1; i >= 0; i--) {
        double2 t = M.c[i];
        for (int j = i + 1; j < nk; j++) {
            const double2 u = cmul(M.a[i][j], M.alpha[j]);
            t.x -= u.x;
            t.y -= u.y;
        }
        M.alpha[i] = make_double2(t.x / M.b[i], t.y / M.b[i]);
    }
}
__global__ void k_b_update(const BLat *lat, const BItem *items, const BScal *sc, const BMat *mat, const double2 *phi,
                           long N, double2 *psi)
{
    const BItem w = items[blockIdx.x];
    const int nk = sc[w.lat].nk;
    if (nk == 0) return;
    const long base = lat[w.lat].off64 + w.s0;
    for (int j = threadIdx.x; j < w.n; j += blockDim.x) {
        double2 x = psi[base + j];
        for (int i = 0; i < nk; i++) x = cadd(x, cmul(mat[w.lat].alpha[i], phi[(long)i * N + base + j]));
        psi[base + j] = x;
    }
}

// ---- arena conversions over (lattice, half, first rank, count) tiles
enum { CV_64_TO_S = 0, CV_S_TO_64 = 1, CV_64_TO_32 = 2, CV_32_TO_64 = 3 };
__device__ __forceinline__ void ld64(const double2 *f, long Vh, long r, cx<float> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) {
        const double2 t = f[c * Vh + r];
        v[c] = mk((float)t.x, (float)t.y);
    }
}
__device__ __forceinline__ void st64(double2 *f, long Vh, long r, const cx<float> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) f[c * Vh + r] = make_double2(v[c].re, v[c].im);
}
__device__ __forceinline__ void ld32(const float4 *f, long Vh, long r, cx<float> v[12])
{
#pragma unroll
    for (int q = 0; q < 6; q++) {
        const float4 t = f[q * Vh + r];
        v[2 * q] = mk(t.x, t.y);
        v[2 * q + 1] = mk(t.z, t.w);
    }
}
__device__ __forceinline__ void st32(float4 *f, long Vh, long r, const cx<float> v[12])
{
#pragma unroll
    for (int q = 0; q < 6; q++) f[q * Vh + r] = make_float4(v[2 * q].re, v[2 * q].im, v[2 * q + 1].re, v[2 * q + 1].im);
}
// sprec: precision of the SAP arena (LQCD_F32 / LQCD_F16S) for CV_64_TO_S, CV_S_TO_64
template <int MODE, int SPREC>
__global__ void __launch_bounds__(TILE) k_b_conv(const BLat *lat, const int4 *items, const int *act, const void *in,
                                                 void *out)
{
    const int4 w = items[blockIdx.x];   // (lattice, half, first rank, count)
    if (act && !act[w.x]) return;
    if ((int)threadIdx.x >= w.w) return;
    const BLat L = lat[w.x];
    const long r = w.z + threadIdx.x, Vh = L.Vh;
    const long h64 = L.off64 + w.y * 12 * Vh, h32 = L.off32 + w.y * 6 * Vh;
    const long hs = L.offs + (SPREC == LQCD_F16S ? w.y * f16s_half_units(Vh) : w.y * 6 * Vh);
    cx<float> v[12];
    if (MODE == CV_64_TO_S || MODE == CV_64_TO_32) ld64((const double2 *)in + h64, Vh, r, v);
    else if (MODE == CV_32_TO_64) ld32((const float4 *)in + h32, Vh, r, v);
    else if (SPREC == LQCD_F16S) f16s_load<false>((const h16s *)in + hs, Vh, r, v);
    else ld32((const float4 *)in + hs, Vh, r, v);
    if (MODE == CV_S_TO_64 || MODE == CV_32_TO_64) st64((double2 *)out + h64, Vh, r, v);
    else if (MODE == CV_64_TO_32) st32((float4 *)out + h32, Vh, r, v);
    else if (SPREC == LQCD_F16S) f16s_store((h16s *)out + hs, Vh, r, v);
    else st32((float4 *)out + hs, Vh, r, v);
}

}  // namespace

// ====================================================================== batch
struct lqcd_batch {
    int n = 0;
    std::vector<lqcd_ctx *> ctx;
    lqcd_batch_params p;
    cudaStream_t user = nullptr, st = nullptr;
    lqcd_ctx *hc = nullptr;          // the batch's own stream / error text / launch counter
    std::vector<BLat> lat_h;
    BLat *lat = nullptr;
    BItem *items = nullptr;
    int nitems = 0;
    int4 *tiles = nullptr;
    int ntiles = 0;
    long N = 0;                      // complex entries of one FP64 arena vector
    long N32 = 0, NS = 0;            // F32 / SAP arena units
    size_t sap_bytes = 0;
    double2 *eta = nullptr, *psi = nullptr, *rho = nullptr, *tmp = nullptr, *phi = nullptr, *chi = nullptr;
    float4 *x32 = nullptr, *y32 = nullptr;
    void *s_eta = nullptr, *s_r = nullptr, *s_psi = nullptr, *s_delta = nullptr;
    BScal *sc = nullptr;
    BMat *mat = nullptr;
    int *act = nullptr;
    double2 *part = nullptr;
    GridBar *bar = nullptr;
    int *status = nullptr;
    DBatch *d32 = nullptr, *d64 = nullptr;
    SapBatch *sap = nullptr;
    int gs_grid = 0;
    long long limit = 0;
    cudaGraphExec_t graph = nullptr;
    bool graph_failed = false;
    int cycles = 0, replays = 0;
    long launches0 = 0;
    long graph_launches = 0;         // kernels of one replayed cycle
};

namespace {

void batch_free_all(lqcd_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    dirac_batch_free(b->d32);
    dirac_batch_free(b->d64);
    sap_batch_free(b->sap);
    for (void *q : {(void *)b->lat, (void *)b->items, (void *)b->tiles, (void *)b->eta, (void *)b->psi, (void *)b->rho,
                    (void *)b->tmp, (void *)b->phi, (void *)b->chi, (void *)b->x32, (void *)b->y32, b->s_eta, b->s_r,
                    b->s_psi, b->s_delta, (void *)b->sc, (void *)b->mat, (void *)b->act, (void *)b->part,
                    (void *)b->bar, (void *)b->status})
        cudaFree(q);
    if (b->st) cudaStreamDestroy(b->st);
    delete b->hc;
}

template <class T>
lqcd_status dalloc(lqcd_batch *b, T **p, size_t bytes, const char *what)
{
    if (cudaMalloc((void **)p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        return set_err(b->hc, LQCD_ERR_NOMEM, "batch: cannot allocate %zu bytes (%s)", bytes, what);
    }
    return LQCD_OK;
}

lqcd_status conv(lqcd_batch *b, int mode, const void *in, void *out, const int *act)
{
    const bool s16 = b->p.sap.prec == LQCD_F16S;
    switch (mode) {
        case CV_64_TO_S:
            if (s16) k_b_conv<CV_64_TO_S, LQCD_F16S><<<b->ntiles, TILE, 0, b->st>>>(b->lat, b->tiles, act, in, out);
            else k_b_conv<CV_64_TO_S, LQCD_F32><<<b->ntiles, TILE, 0, b->st>>>(b->lat, b->tiles, act, in, out);
            break;
        case CV_S_TO_64:
            if (s16) k_b_conv<CV_S_TO_64, LQCD_F16S><<<b->ntiles, TILE, 0, b->st>>>(b->lat, b->tiles, act, in, out);
            else k_b_conv<CV_S_TO_64, LQCD_F32><<<b->ntiles, TILE, 0, b->st>>>(b->lat, b->tiles, act, in, out);
            break;
        case CV_64_TO_32:
            k_b_conv<CV_64_TO_32, LQCD_F32><<<b->ntiles, TILE, 0, b->st>>>(b->lat, b->tiles, act, in, out);
            break;
        default:
            k_b_conv<CV_32_TO_64, LQCD_F32><<<b->ntiles, TILE, 0, b->st>>>(b->lat, b->tiles, act, in, out);
            break;
    }
    b->hc->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(b->hc);
    return LQCD_OK;
}

lqcd_status gs_step(lqcd_batch *b, int k, int stall)
{
    GsArgs a;
    a.lat = b->lat;
    a.items = b->items;
    a.nitems = b->nitems;
    a.nlat = b->n;
    a.k = k;
    a.N = b->N;
    a.chi = b->chi;
    a.rho = b->rho;
    a.sc = b->sc;
    a.mat = b->mat;
    a.act = b->act;
    a.part = b->part;
    a.bar = b->bar;
    a.limit = b->limit;
    a.stall = stall;
    a.status = b->status;
    a.nmx = b->p.nmx;
    void *args[] = {&a};
    // a barrier left behind by a wait that ran out must not reach this launch
    LQCD_CUDA_CHECK(b->hc, cudaMemsetAsync(b->bar, 0, sizeof(GridBar), b->st));
    LQCD_CUDA_CHECK(b->hc, cudaLaunchCooperativeKernel((const void *)k_gs, dim3(b->gs_grid), dim3(GS_THREADS), args,
                                                       0, b->st));
    b->hc->n_kernel_launches++;
    return LQCD_OK;
}

// the steps of one cycle and the solution update (no host synchronisation)
lqcd_status cycle_steps(lqcd_batch *b, int stall)
{
    for (int k = 0; k < b->p.nkv; k++) {
        double2 *phk = b->phi + (long)k * b->N, *chk = b->chi + (long)k * b->N;
        LQCD_TRY(conv(b, CV_64_TO_S, b->rho, b->s_eta, b->act));
        LQCD_TRY(sap_batch_apply(b->hc, b->sap, b->s_eta, b->sap_bytes, b->act));
        LQCD_TRY(conv(b, CV_S_TO_64, b->s_psi, phk, b->act));
        LQCD_TRY(conv(b, CV_64_TO_32, phk, b->x32, b->act));
        LQCD_TRY(dirac_batch_D(b->hc, b->d32, b->act));
        LQCD_TRY(conv(b, CV_32_TO_64, b->y32, chk, b->act));
        LQCD_TRY(gs_step(b, k, stall && k == 0));
    }
    k_b_backsub<<<(b->n + 63) / 64, 64, 0, b->st>>>(b->sc, b->mat, b->n);
    k_b_update<<<b->nitems, GS_THREADS, 0, b->st>>>(b->lat, b->items, b->sc, b->mat, b->phi, b->N, b->psi);
    b->hc->n_kernel_launches += 2;
    LQCD_LAUNCH_CHECK(b->hc);
    return LQCD_OK;
}

// rho = eta - D psi on every lattice still running; flags of the new cycle
lqcd_status cycle_restart(lqcd_batch *b)
{
    k_b_activate<<<(b->n + 63) / 64, 64, 0, b->st>>>(b->act, b->sc, b->n, b->p.nmx);
    b->hc->n_kernel_launches++;
    LQCD_TRY(dirac_batch_D(b->hc, b->d64, b->act));
    k_b_resid<<<b->nitems, GS_THREADS, 0, b->st>>>(b->lat, b->items, b->act, b->eta, b->tmp, b->rho, b->part);
    // a cycle in which D phi is FP32 gains at most 1e-5 before the FP64 restart
    k_b_restart<<<b->n, 32, 0, b->st>>>(b->lat, b->part, b->act, b->sc, b->n, 1e-10);
    b->hc->n_kernel_launches += 2;
    LQCD_LAUNCH_CHECK(b->hc);
    return LQCD_OK;
}

}  // namespace

extern "C" {

lqcd_status lqcd_batch_create(lqcd_ctx *const *ctxs, int n, const lqcd_batch_params *p, void *stream,
                              lqcd_batch **out)
{
    if (!ctxs || !p || !out || n < 1) return LQCD_ERR_ARG;
    *out = nullptr;
    lqcd_batch *b = new lqcd_batch();
    b->hc = new lqcd_ctx();
    b->n = n;
    b->p = *p;
    b->user = (cudaStream_t)stream;
    auto fail = [&](lqcd_status s) {
        // keep the message: the caller reads it through a batch that is not returned
        for (int l = 0; l < n; l++)
            if (ctxs[l]) set_err(ctxs[l], s, "%s", b->hc->err);
        batch_free_all(b);
        delete b;
        return s;
    };
    if (p->nkv < 1 || p->nkv > BNKV || p->nmx < 1 || !(p->tol > 0))
        return fail(set_err(b->hc, LQCD_ERR_ARG, "batch: nkv %d (1..%d), nmx %d, tol %g", p->nkv, BNKV, p->nmx, p->tol));
    if (p->sap.prec != LQCD_F16S && p->sap.prec != LQCD_F32)
        return fail(set_err(b->hc, LQCD_ERR_ARG, "batch: SAP precision must be F16S or F32"));
    if (!(p->wait_timeout_s > 0)) return fail(set_err(b->hc, LQCD_ERR_ARG, "batch: wait_timeout_s must be > 0"));
    for (int l = 0; l < n; l++) {
        if (!ctxs[l] || !ctxs[l]->have_clover)
            return fail(set_err(b->hc, LQCD_ERR_STATE, "batch: context %d has no clover term", l));
        b->ctx.push_back(ctxs[l]);
    }
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess)
        return fail(set_err(b->hc, LQCD_ERR_CUDA, "batch: stream creation failed"));
    b->hc->stream = b->st;
    // arena layout and work lists
    const bool s16 = p->sap.prec == LQCD_F16S;
    std::vector<BItem> items;
    std::vector<int4> tiles;
    std::vector<long> off64(n), off32(n), offs(n);
    for (int l = 0; l < n; l++) {
        BLat L;
        L.Vh = b->ctx[l]->g.Vh;
        L.off64 = b->N;
        L.off32 = b->N32;
        L.offs = b->NS;
        off64[l] = L.off64;
        off32[l] = L.off32;
        offs[l] = L.offs;
        const long nc = 24 * L.Vh;   // complex entries of a full field
        L.it0 = (int)items.size();
        for (long s0 = 0; s0 < nc; s0 += CHUNK) items.push_back(BItem{l, (int)std::min<long>(CHUNK, nc - s0), s0});
        L.it1 = (int)items.size();
        for (int h = 0; h < 2; h++)
            for (long r0 = 0; r0 < L.Vh; r0 += TILE)
                tiles.push_back(make_int4(l, h, (int)r0, (int)std::min<long>(TILE, L.Vh - r0)));
        b->lat_h.push_back(L);
        b->N += nc;
        b->N32 += 12 * L.Vh;
        b->NS += s16 ? 2 * f16s_half_units(L.Vh) : 12 * L.Vh;
    }
    b->nitems = (int)items.size();
    b->ntiles = (int)tiles.size();
    b->sap_bytes = (size_t)b->NS * 16;
    const size_t f64b = (size_t)b->N * sizeof(double2);
    lqcd_status st = LQCD_OK;
#define BALLOC(ptr, bytes, what)                         \
    if ((st = dalloc(b, &(ptr), (bytes), (what))) != LQCD_OK) return fail(st);
    BALLOC(b->lat, n * sizeof(BLat), "layout");
    BALLOC(b->items, items.size() * sizeof(BItem), "work list");
    BALLOC(b->tiles, tiles.size() * sizeof(int4), "tiles");
    BALLOC(b->eta, f64b, "eta");
    BALLOC(b->psi, f64b, "psi");
    BALLOC(b->rho, f64b, "rho");
    BALLOC(b->tmp, f64b, "D psi");
    BALLOC(b->phi, f64b * p->nkv, "phi");
    BALLOC(b->chi, f64b * p->nkv, "chi");
    BALLOC(b->x32, (size_t)b->N32 * 16, "F32 input");
    BALLOC(b->y32, (size_t)b->N32 * 16, "F32 output");
    BALLOC(b->s_eta, b->sap_bytes, "SAP input");
    BALLOC(b->s_r, b->sap_bytes, "SAP residual");
    BALLOC(b->s_psi, b->sap_bytes, "SAP output");
    BALLOC(b->s_delta, b->sap_bytes, "SAP block corrections");
    BALLOC(b->sc, n * sizeof(BScal), "scalars");
    BALLOC(b->mat, n * sizeof(BMat), "coefficients");
    BALLOC(b->act, n * sizeof(int), "flags");
    BALLOC(b->part, (size_t)b->nitems * PS * sizeof(double2), "partial sums");
    BALLOC(b->bar, sizeof(GridBar), "barrier");
    BALLOC(b->status, sizeof(int), "status");
#undef BALLOC
    cudaMemcpy(b->lat, b->lat_h.data(), n * sizeof(BLat), cudaMemcpyHostToDevice);
    cudaMemcpy(b->items, items.data(), items.size() * sizeof(BItem), cudaMemcpyHostToDevice);
    cudaMemcpy(b->tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if ((st = dirac_batch_create(b->hc, b->ctx.data(), n, LQCD_F32, b->x32, b->y32, off32.data(), &b->d32)) != LQCD_OK)
        return fail(st);
    if ((st = dirac_batch_create(b->hc, b->ctx.data(), n, LQCD_F64, b->psi, b->tmp, off64.data(), &b->d64)) != LQCD_OK)
        return fail(st);
    if ((st = sap_batch_create(b->hc, b->ctx.data(), n, &p->sap, b->s_r, b->s_psi, b->s_delta, offs.data(), &b->sap)) !=
        LQCD_OK)
        return fail(st);
    // cooperative grid: every CTA resident at once
    int dev = 0, nsm = 0, occ = 0, coop = 0, khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gs, GS_THREADS, 0);
    if (!coop || occ < 1) return fail(set_err(b->hc, LQCD_ERR_CUDA, "batch: cooperative launch unavailable"));
    b->gs_grid = std::max(1, std::min(nsm * std::min(occ, 2), std::max(b->nitems, n)));
    b->limit = (long long)(p->wait_timeout_s * (double)khz * 1e3);
    *out = b;
    return LQCD_OK;
}

lqcd_status lqcd_batch_destroy(lqcd_batch *b)
{
    if (!b) return LQCD_ERR_ARG;
    batch_free_all(b);
    delete b;
    return LQCD_OK;
}

const char *lqcd_batch_last_error(const lqcd_batch *b) { return b ? b->hc->err : "null batch"; }

lqcd_status lqcd_batch_stats(const lqcd_batch *b, int *cycles, int *graph_replays, long *launches)
{
    if (!b) return LQCD_ERR_ARG;
    if (cycles) *cycles = b->cycles;
    if (graph_replays) *graph_replays = b->replays;
    if (launches) *launches = b->hc->n_kernel_launches - b->launches0;
    return LQCD_OK;
}

lqcd_status lqcd_batch_solve_dhat(lqcd_batch *b, const double *const *eta_dev, double *const *psi_dev,
                                  lqcd_solve_info *info)
{
    if (!b || !eta_dev || !psi_dev) return LQCD_ERR_ARG;
    const int n = b->n;
    lqcd_ctx *hc = b->hc;
    const auto t0 = std::chrono::steady_clock::now();
    b->cycles = b->replays = 0;
    b->launches0 = hc->n_kernel_launches;
    // order after the caller's stream
    cudaEvent_t ev;
    LQCD_CUDA_CHECK(hc, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    LQCD_CUDA_CHECK(hc, cudaEventRecord(ev, b->user));
    LQCD_CUDA_CHECK(hc, cudaStreamWaitEvent(b->st, ev, 0));
    // eta: even half from the caller's field, odd half zero (Eq. 5); psi = 0
    const size_t f64b = (size_t)b->N * sizeof(double2);
    LQCD_CUDA_CHECK(hc, cudaMemsetAsync(b->eta, 0, f64b, b->st));
    LQCD_CUDA_CHECK(hc, cudaMemsetAsync(b->psi, 0, f64b, b->st));
    LQCD_CUDA_CHECK(hc, cudaMemsetAsync(b->status, 0, sizeof(int), b->st));
    LQCD_CUDA_CHECK(hc, cudaMemsetAsync(b->bar, 0, sizeof(GridBar), b->st));
    LQCD_CUDA_CHECK(hc, cudaStreamSynchronize(b->st));
    std::vector<BScal> S(n);
    std::vector<cudaStream_t> saved(n);
    for (int l = 0; l < n; l++) {
        lqcd_ctx *c = b->ctx[l];
        saved[l] = c->stream;
        c->stream = b->st;
        LQCD_TRY(pack_field(c, LQCD_F64, 1, eta_dev[l], b->eta + b->lat_h[l].off64, 1, false));
        double e2 = 0;
        LQCD_TRY(blas_norm2(c, 24 * b->lat_h[l].Vh, (const double *)(b->eta + b->lat_h[l].off64), &e2));
        std::memset(&S[l], 0, sizeof(BScal));
        S[l].status = LQCD_ERR_NOT_CONVERGED;
        S[l].eta2 = e2;
        S[l].tol2 = b->p.tol * b->p.tol * e2;
        if (e2 == 0) {
            S[l].done = 1;
            S[l].status = LQCD_OK;
        }
    }
    LQCD_CUDA_CHECK(hc, cudaMemcpyAsync(b->sc, S.data(), n * sizeof(BScal), cudaMemcpyHostToDevice, b->st));
    std::vector<int> act(n);
    std::vector<double> dhat_rel(n, 0.0);
    lqcd_status st = LQCD_OK;
    for (int attempt = 0; attempt < 4 && st == LQCD_OK; attempt++) {
        for (;;) {
            if ((st = cycle_restart(b)) != LQCD_OK) break;
            if (cudaMemcpyAsync(act.data(), b->act, n * sizeof(int), cudaMemcpyDeviceToHost, b->st) != cudaSuccess ||
                cudaStreamSynchronize(b->st) != cudaSuccess) {
                st = set_err(hc, LQCD_ERR_CUDA, "batch: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            if (std::none_of(act.begin(), act.end(), [](int a) { return a != 0; })) break;
            b->cycles++;
            // the first cycle runs eagerly (it also settles the autotuned launch
            // shapes); later cycles replay its captured graph when asked to
            if (b->p.use_graph && b->cycles > 1 && !b->graph && !b->graph_failed) {
                cudaGraph_t g = nullptr;
                const long before = hc->n_kernel_launches;
                bool ok = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                lqcd_status cs = ok ? cycle_steps(b, 0) : LQCD_OK;
                b->graph_launches = hc->n_kernel_launches - before;   // recorded, not run
                hc->n_kernel_launches = before;
                const bool ended = ok && cudaStreamEndCapture(b->st, &g) == cudaSuccess;
                ok = ok && ended && cs == LQCD_OK && g && cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess;
                if (g) cudaGraphDestroy(g);
                if (!ok) {
                    cudaGetLastError();
                    b->graph = nullptr;
                    b->graph_failed = true;
                }
            }
            if (b->graph) {
                if (cudaGraphLaunch(b->graph, b->st) != cudaSuccess) {
                    st = set_err(hc, LQCD_ERR_CUDA, "batch: graph launch: %s", cudaGetErrorString(cudaGetLastError()));
                    break;
                }
                b->replays++;
                hc->n_kernel_launches += b->graph_launches;
            } else if ((st = cycle_steps(b, b->p.stall_test && b->cycles == 1)) != LQCD_OK) {
                break;
            }
            int dstat = 0;
            if (b->p.stall_test) {
                cudaMemcpyAsync(&dstat, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->st);
                cudaStreamSynchronize(b->st);
            }
            if (dstat != 0) {
                st = set_err(hc, (lqcd_status)dstat, "batch: a device-side wait ran out of time");
                break;
            }
        }
        if (st != LQCD_OK) break;
        int dstat = 0;
        LQCD_CUDA_CHECK(hc, cudaMemcpyAsync(&dstat, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->st));
        LQCD_CUDA_CHECK(hc, cudaMemcpyAsync(S.data(), b->sc, n * sizeof(BScal), cudaMemcpyDeviceToHost, b->st));
        LQCD_CUDA_CHECK(hc, cudaStreamSynchronize(b->st));
        if (dstat != 0) {
            st = set_err(hc, (lqcd_status)dstat, "batch: a device-side wait ran out of time");
            break;
        }
        // the Dhat residual of every converged lattice, in FP64 (Eq. 5 only bounds it by the full one)
        bool again = false;
        for (int l = 0; l < n && st == LQCD_OK; l++) {
            lqcd_ctx *c = b->ctx[l];
            const long Vh = b->lat_h[l].Vh;
            if (S[l].status != LQCD_OK || S[l].eta2 == 0) continue;
            void *o, *t;
            if ((st = ws_get(c, WS_MISC, 12 * Vh * sizeof(double2), &o)) != LQCD_OK) break;
            if ((st = ws_get(c, WS_TMP_O, 12 * Vh * sizeof(double2), &t)) != LQCD_OK) break;
            const double2 *pe = b->psi + b->lat_h[l].off64, *ee = b->eta + b->lat_h[l].off64;
            double r2 = 0;
            if ((st = dirac_dhat(c, LQCD_F64, pe, o, t, 1)) != LQCD_OK) break;
            if ((st = blas_sub(c, 24 * Vh, (const double *)ee, (const double *)o, (double *)o)) != LQCD_OK) break;
            if ((st = blas_norm2(c, 24 * Vh, (const double *)o, &r2)) != LQCD_OK) break;
            dhat_rel[l] = std::sqrt(r2 / S[l].eta2);
            if (dhat_rel[l] > b->p.tol && attempt < 3) {
                const double f = b->p.tol / dhat_rel[l];
                S[l].tol2 *= 0.25 * f * f;
                S[l].done = 0;
                S[l].status = LQCD_ERR_NOT_CONVERGED;
                again = true;
            }
        }
        if (!again || st != LQCD_OK) break;
        LQCD_CUDA_CHECK(hc, cudaMemcpyAsync(b->sc, S.data(), n * sizeof(BScal), cudaMemcpyHostToDevice, b->st));
    }
    // results
    lqcd_status worst = st;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int l = 0; l < n; l++) {
        lqcd_ctx *c = b->ctx[l];
        if (st == LQCD_OK) st = pack_field(c, LQCD_F64, 1, psi_dev[l], b->psi + b->lat_h[l].off64, 1, true);
        if (info) {
            info[l].iters = S[l].iters;
            info[l].restarts = S[l].restarts;
            info[l].true_relres = S[l].eta2 > 0 ? std::sqrt(S[l].true_rn2 / S[l].eta2) : 0;
            info[l].relres_dhat = dhat_rel[l];
            info[l].seconds = secs;
            info[l].status = (lqcd_status)S[l].status;
            info[l].net_fallbacks = 0;
        }
        if (worst == LQCD_OK && S[l].status != LQCD_OK) worst = (lqcd_status)S[l].status;
        c->stream = saved[l];
    }
    cudaEventRecord(ev, b->st);
    cudaStreamWaitEvent(b->user, ev, 0);
    cudaEventDestroy(ev);
    if (st != LQCD_OK) return st;
    return worst;
}

}  // extern "C"
