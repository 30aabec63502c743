// Gauge-equivariant parallel-transport network: the learned preconditioner
// that sits next to SAP in the flexible GCR (lqcd.h, "learned preconditioner").
//
//   y_o(x) = sum_i sum_d W_{o,i,d} (T_d y_i)(x)
//
// A layer is a transport (gather of the nine parallel-transported neighbour
// fields, FP32 SU(3) products, bandwidth bound) followed by a small dense
// contraction per (site, colour) row: K = 36 cin complex inputs against
// N = 4 cout complex outputs.  In the real block form
//   [Re z, Im z] x [[Re W^T, Im W^T], [-Im W^T, Re W^T]]
// it is a (rows x 72 cin) x (72 cin x 8 cout) real GEMM, which the BF16 path
// runs on the tensor cores with mma.sync m16n8k16 (bf16 in, fp32 accumulate):
// one warp per 16 rows, the whole K and N of the layer per warp.  The
// contraction is too narrow (N = 16) to fill a 128-row tcgen05 tile with TMEM
// round trips, and the layer is bound by its transports, so the warp-level
// tensor-core form is the better fit.  The FP32 path contracts with FMAs.
//
// Backward (data): T_d^dag = T_{-d} and W commutes with T, so the backward pass
// of a layer is the same kernel with weights W^b_{i,o,d}[s'][s] =
// conj(W_{o,i,-d}[s][s']) and the channel roles swapped.  Weight gradients are
// reduced per CTA and then across CTAs in a fixed order (deterministic).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "lqcd_internal.cuh"

namespace {

constexpr int PT_SITES = 64;
constexpr int PT_ROWS = 3 * PT_SITES;   // (site, colour) rows per CTA
constexpr int PT_THREADS = 192;         // 6 warps x 32 rows (two m16 tiles each)
constexpr int PT_CMAX = 2;

using bf16 = __nv_bfloat16;
using bf162 = __nv_bfloat162;

// ------------------------------------------------------------ activations
__device__ __forceinline__ void act_load(const bf162 *f, long x, cx<float> v[12])
{
    const uint4 *p = reinterpret_cast<const uint4 *>(f + 12 * x);
#pragma unroll
    for (int q = 0; q < 3; q++) {
        uint4 w = p[q];
        unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            bf162 h = *reinterpret_cast<bf162 *>(&u[j]);
            float2 fl = __bfloat1622float2(h);
            v[4 * q + j] = mk(fl.x, fl.y);
        }
    }
}
__device__ __forceinline__ void act_load(const float2 *f, long x, cx<float> v[12])
{
    const float4 *p = reinterpret_cast<const float4 *>(f + 12 * x);
#pragma unroll
    for (int q = 0; q < 6; q++) {
        float4 w = p[q];
        v[2 * q] = mk(w.x, w.y);
        v[2 * q + 1] = mk(w.z, w.w);
    }
}
__device__ __forceinline__ void act_store1(bf162 *f, long i, float re, float im)
{
    f[i] = __floats2bfloat162_rn(re, im);
}
__device__ __forceinline__ void act_store1(float2 *f, long i, float re, float im) { f[i] = make_float2(re, im); }

// ------------------------------------------------------------ geometry
__device__ __forceinline__ void lex_coords(const Geom &g, long x, int c[4])
{
    c[3] = x % g.L[3];
    long t = x / g.L[3];
    c[2] = t % g.L[2];
    t /= g.L[2];
    c[1] = t % g.L[1];
    c[0] = t / g.L[1];
}
__device__ __forceinline__ long lex_index(const Geom &g, const int c[4])
{
    return c[3] + (long)g.L[3] * (c[2] + (long)g.L[2] * (c[1] + (long)g.L[1] * c[0]));
}
// ------------------------------------------------------------ gather
// Per CTA, once per site of its tile and path d: the neighbour site, the
// first float4 of the path's link (two stored rows) and the hop's boundary sign.
struct PtStage {
    long lnk[9][PT_SITES];
    int nbr[9][PT_SITES];
    float sg[9][PT_SITES];
};

__device__ void pt_stage_sites(const Geom &g, long x0, PtStage &S)
{
    for (int it = threadIdx.x; it < 9 * PT_SITES; it += blockDim.x) {
        const int s = it % PT_SITES, d = it / PT_SITES;
        const long x = x0 + s;
        if (x >= g.V) continue;
        int c[4];
        lex_coords(g, x, c);
        if (d == 0) {
            S.nbr[0][s] = (int)x;
            S.lnk[0][s] = -1;
            S.sg[0][s] = 1.f;
            continue;
        }
        const int mu = (d - 1) >> 1;
        const bool fwd = d & 1;
        int yc[4] = {c[0], c[1], c[2], c[3]};
        const int v = yc[mu] + (fwd ? 1 : -1);
        yc[mu] = v < 0 ? v + g.L[mu] : (v >= g.L[mu] ? v - g.L[mu] : v);
        const long y = lex_index(g, yc);
        float sgn = 1.f;
        if (mu == 0 && ((fwd && c[0] == g.L[0] - 1) || (!fwd && c[0] == 0))) sgn = (float)g.bc_t;
        // forward: U_mu(x) (parity of x); backward: U_mu(y) (parity of y), daggered
        const int *lc = fwd ? c : yc;
        const long ls = fwd ? x : y;
        const int p = (lc[0] + lc[1] + lc[2] + lc[3]) & 1;
        S.nbr[d][s] = (int)y;
        S.lnk[d][s] = (long)((p * 4 + mu) * 3) * g.Vh + (ls >> 1);
        S.sg[d][s] = sgn;
    }
}

// w = u h and w = u^dag h for colour vectors: each real part one product and
// five fused multiply-adds
__device__ __forceinline__ void su3_mul_fma(const cx<float> u[3][3], const cx<float> *h, cx<float> *w)
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float re = u[a][0].re * h[0].re;
        re = fmx(-u[a][0].im, h[0].im, re);
        re = fmx(u[a][1].re, h[1].re, re);
        re = fmx(-u[a][1].im, h[1].im, re);
        re = fmx(u[a][2].re, h[2].re, re);
        re = fmx(-u[a][2].im, h[2].im, re);
        float im = u[a][0].re * h[0].im;
        im = fmx(u[a][0].im, h[0].re, im);
        im = fmx(u[a][1].re, h[1].im, im);
        im = fmx(u[a][1].im, h[1].re, im);
        im = fmx(u[a][2].re, h[2].im, im);
        im = fmx(u[a][2].im, h[2].re, im);
        w[a] = mk(re, im);
    }
}
__device__ __forceinline__ void su3dag_mul_fma(const cx<float> u[3][3], const cx<float> *h, cx<float> *w)
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float re = u[0][a].re * h[0].re;
        re = fmx(u[0][a].im, h[0].im, re);
        re = fmx(u[1][a].re, h[1].re, re);
        re = fmx(u[1][a].im, h[1].im, re);
        re = fmx(u[2][a].re, h[2].re, re);
        re = fmx(u[2][a].im, h[2].im, re);
        float im = u[0][a].re * h[0].im;
        im = fmx(-u[0][a].im, h[0].re, im);
        im = fmx(u[1][a].re, h[1].im, im);
        im = fmx(-u[1][a].im, h[1].re, im);
        im = fmx(u[2][a].re, h[2].im, im);
        im = fmx(-u[2][a].im, h[2].re, im);
        w[a] = mk(re, im);
    }
}

// The transported inputs (T_d y_i)(x) of the tile: one item per (site, path);
// the path's link is loaded and its third row rebuilt once and applied to every
// input channel.  sink(s, i, d, z) receives the 12 spin-colour components.
template <class ACT, class SINK>
__device__ __forceinline__ void pt_gather(const Geom &g, const float4 *U, const ACT *in, int cin, long x0,
                                          const PtStage &S, SINK sink)
{
    const long V = g.V;
    for (int it = threadIdx.x; it < 9 * PT_SITES; it += blockDim.x) {
        const int s = it % PT_SITES, d = it / PT_SITES;
        const bool ok = x0 + s < V;
        cx<float> u[3][3];
        if (ok && d > 0) {
            const float4 *b = U + S.lnk[d][s];
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const float4 t = __ldg(b + q * (long)g.Vh);
                u[(2 * q) / 3][(2 * q) % 3] = mk(t.x, t.y);
                u[(2 * q + 1) / 3][(2 * q + 1) % 3] = mk(t.z, t.w);
            }
            su3_third_row(u);
        }
        const bool fwd = d & 1;
        const int y = ok ? S.nbr[d][s] : 0;
        const float sgn = ok ? S.sg[d][s] : 1.f;
        for (int i = 0; i < cin; i++) {
            cx<float> z[12];
            if (!ok) {
#pragma unroll
                for (int k = 0; k < 12; k++) z[k] = mk(0.f, 0.f);
            } else {
                cx<float> v[12];
                act_load(in + (long)i * 12 * V, y, v);
                if (d == 0) {
#pragma unroll
                    for (int k = 0; k < 12; k++) z[k] = v[k];
                } else {
                    // U v or U^dag v per spin, as fused multiply-add chains with the
                    // boundary sign (+-1, exact) folded into the link
                    cx<float> us[3][3];
#pragma unroll
                    for (int a = 0; a < 3; a++)
#pragma unroll
                        for (int b = 0; b < 3; b++) us[a][b] = sgn * u[a][b];
#pragma unroll
                    for (int sp = 0; sp < 4; sp++) {
                        if (fwd)
                            su3_mul_fma(us, v + 3 * sp, z + 3 * sp);
                        else
                            su3dag_mul_fma(us, v + 3 * sp, z + 3 * sp);
                    }
                }
            }
            sink(s, i, d, z);
        }
    }
}

// ------------------------------------------------------------ layer
struct LayerArgs {
    Geom g;
    const float4 *U;
    const void *in;
    void *out;
    int cin, cout;
    long in_ss, out_ss;     // elements (complex) between samples
    const bf16 *Bt;         // [8 cout][Kp] real block weights (BF16 path)
    const float2 *Wc;       // [cout][cin][9][4][4] complex weights (FP32 path)
};

__device__ __forceinline__ unsigned ld_b32(const bf16 *p) { return *reinterpret_cast<const unsigned *>(p); }

// row pitch (bf16) of the A tile: room for Kp columns, even, and an odd
// number of 4-byte words per 3 rows, so that the stride-3-row stores of the
// gather and the fragment loads of the MMA both spread over the banks
__host__ __device__ inline int pt_ld(int Kp)
{
    int ld = Kp + 8;
    if (((3 * ld / 2) & 1) == 0) ld += 2;
    return ld;
}

template <class ACT>
__global__ void __launch_bounds__(PT_THREADS) k_ptc_layer(LayerArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const ACT *in = (const ACT *)a.in + blockIdx.y * a.in_ss;
    ACT *out = (ACT *)a.out + blockIdx.y * a.out_ss;
    const long x0 = (long)blockIdx.x * PT_SITES;
    const long V = a.g.V;
    const int cin = a.cin, cout = a.cout, tid = threadIdx.x;
    const int K = 72 * cin, Kp = (K + 15) / 16 * 16, ld = pt_ld(Kp);
    constexpr bool BF = sizeof(ACT) == 4;
    PtStage &S = *reinterpret_cast<PtStage *>(smraw);
    unsigned char *tile = smraw + sizeof(PtStage);
    bf16 *A = (bf16 *)tile;                                    // [rows][ld]
    bf16 *Bs = A + PT_ROWS * ld;                               // [8 cout][ld]
    cx<float> *Z = (cx<float> *)tile;                          // [rows][36 cin]
    cx<float> *Ws = Z + PT_ROWS * 36 * cin;                    // [cout*cin*144]
    if (BF) {
        for (int e = tid; e < 8 * cout * Kp; e += blockDim.x) Bs[(e / Kp) * ld + e % Kp] = a.Bt[e];
        for (int e = tid; e < PT_ROWS * (Kp - K); e += blockDim.x)
            A[(e / (Kp - K)) * ld + K + e % (Kp - K)] = __float2bfloat16(0.f);
    } else {
        for (int e = tid; e < cout * cin * 144; e += blockDim.x) {
            float2 w = a.Wc[e];
            Ws[e] = mk(w.x, w.y);
        }
    }
    pt_stage_sites(a.g, x0, S);
    __syncthreads();
    if (BF) {
        pt_gather(a.g, a.U, in, cin, x0, S, [&](int s, int i, int d, const cx<float> z[12]) {
#pragma unroll
            for (int sp = 0; sp < 4; sp++)
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
                    const int kk = (i * 9 + d) * 4 + sp, row = 3 * s + cc;
                    *reinterpret_cast<bf162 *>(A + row * ld + 2 * kk) =
                        __floats2bfloat162_rn(z[3 * sp + cc].re, z[3 * sp + cc].im);
                }
        });
    } else {
        pt_gather(a.g, a.U, in, cin, x0, S, [&](int s, int i, int d, const cx<float> z[12]) {
#pragma unroll
            for (int sp = 0; sp < 4; sp++)
#pragma unroll
                for (int cc = 0; cc < 3; cc++) Z[(3 * s + cc) * 36 * cin + (i * 9 + d) * 4 + sp] = z[3 * sp + cc];
        });
    }
    __syncthreads();
    if (BF) {
        // tensor-core contraction: warp w owns rows 32w .. 32w+31 (two m16 tiles)
        const int w = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
        for (int nt = 0; nt < cout; nt++) {
            const bf16 *Br = Bs + (8 * nt + gq) * ld;
#pragma unroll
            for (int mi = 0; mi < 2; mi++) {
                const bf16 *Ar = A + (32 * w + 16 * mi) * ld;
                float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
                for (int k0 = 0; k0 < Kp; k0 += 16) {
                    unsigned a0 = ld_b32(Ar + gq * ld + k0 + 2 * tq);
                    unsigned a1 = ld_b32(Ar + (gq + 8) * ld + k0 + 2 * tq);
                    unsigned a2 = ld_b32(Ar + gq * ld + k0 + 8 + 2 * tq);
                    unsigned a3 = ld_b32(Ar + (gq + 8) * ld + k0 + 8 + 2 * tq);
                    unsigned b0 = ld_b32(Br + k0 + 2 * tq);
                    unsigned b1 = ld_b32(Br + k0 + 8 + 2 * tq);
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                        "{%0,%1,%2,%3};\n"
                        : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
                }
                // columns 2tq, 2tq+1 of n-tile nt are (re, im) of output channel nt, spin tq
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int row = 32 * w + 16 * mi + gq + 8 * h;
                    const int sl = row / 3, cc = row % 3;
                    const long x = x0 + sl;
                    if (x < V) act_store1(out, (long)nt * 12 * V + 12 * x + 3 * tq + cc, h ? d2 : d0, h ? d3 : d1);
                }
            }
        }
    } else {
        for (int e = tid; e < PT_ROWS * cout * 4; e += blockDim.x) {
            const int row = e / (cout * 4), o = (e / 4) % cout, s = e % 4;
            const long x = x0 + row / 3;
            cx<float> acc = mk(0.f, 0.f);
            for (int i = 0; i < cin; i++)
                for (int d = 0; d < 9; d++) {
                    const cx<float> *w = Ws + ((o * cin + i) * 9 + d) * 16 + 4 * s;
                    const cx<float> *zr = Z + row * 36 * cin + (i * 9 + d) * 4;
#pragma unroll
                    for (int sp = 0; sp < 4; sp++) acc = acc + w[sp] * zr[sp];
                }
            if (x < V) act_store1(out, (long)o * 12 * V + 12 * x + 3 * s + row % 3, acc.re, acc.im);
        }
    }
}

// per-CTA partial weight gradient: G[o][s][kk] = sum_rows delta_o[s][c] conj(Z[kk][c])
struct WgradArgs {
    Geom g;
    const float4 *U;
    const void *y;        // layer input (cin channels)
    const void *delta;    // gradient at the layer output (cout channels)
    int cin, cout;
    long y_ss, d_ss;
    float2 *partial;      // [sample][cta][cout*4*36*cin]
};

template <class ACT>
__global__ void __launch_bounds__(PT_THREADS) k_ptc_wgrad(WgradArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const ACT *y = (const ACT *)a.y + blockIdx.y * a.y_ss;
    const ACT *dl = (const ACT *)a.delta + blockIdx.y * a.d_ss;
    const long x0 = (long)blockIdx.x * PT_SITES;
    const long V = a.g.V;
    const int cin = a.cin, cout = a.cout, tid = threadIdx.x;
    PtStage &S = *reinterpret_cast<PtStage *>(smraw);
    cx<float> *Z = (cx<float> *)(smraw + sizeof(PtStage));   // [rows][36 cin]
    cx<float> *Dt = Z + PT_ROWS * 36 * cin;                   // [rows][4 cout]
    pt_stage_sites(a.g, x0, S);
    __syncthreads();
    pt_gather(a.g, a.U, y, cin, x0, S, [&](int s, int i, int d, const cx<float> z[12]) {
#pragma unroll
        for (int sp = 0; sp < 4; sp++)
#pragma unroll
            for (int cc = 0; cc < 3; cc++) Z[(3 * s + cc) * 36 * cin + (i * 9 + d) * 4 + sp] = z[3 * sp + cc];
    });
    for (int it = tid; it < PT_SITES * cout; it += blockDim.x) {
        const int sl = it % PT_SITES, o = it / PT_SITES;
        const long x = x0 + sl;
        cx<float> v[12];
        if (x < V)
            act_load(dl + (long)o * 12 * V, x, v);
        else
            for (int k = 0; k < 12; k++) v[k] = mk(0.f, 0.f);
        for (int s = 0; s < 4; s++)
            for (int cc = 0; cc < 3; cc++) Dt[(3 * sl + cc) * 4 * cout + 4 * o + s] = v[3 * s + cc];
    }
    __syncthreads();
    const int nout = cout * 4 * 36 * cin;
    float2 *part = a.partial + ((long)blockIdx.y * gridDim.x + blockIdx.x) * nout;
    for (int e = tid; e < nout; e += blockDim.x) {
        const int os = e / (36 * cin), kk = e % (36 * cin);
        cx<float> acc = mk(0.f, 0.f);
        for (int row = 0; row < PT_ROWS; row++) acc = acc + cmulc(Z[row * 36 * cin + kk], Dt[row * 4 * cout + os]);
        part[e] = make_float2(acc.re, acc.im);
    }
}

// sum the partials (fixed order) into G[o][i][d][s][s'] (complex float)
__global__ void k_ptc_wgrad_reduce(int nparts, int cin, int cout, const float2 *partial, float2 *G)
{
    const int e = blockIdx.x;   // output (o*4 + s)*36 cin + kk
    const int nout = cout * 4 * 36 * cin;
    __shared__ double sr[256], si[256];
    double r = 0, m = 0;
    for (int p = threadIdx.x; p < nparts; p += blockDim.x) {
        float2 v = partial[(long)p * nout + e];
        r += v.x;
        m += v.y;
    }
    sr[threadIdx.x] = r;
    si[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sr[threadIdx.x] += sr[threadIdx.x + s];
            si[threadIdx.x] += si[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int os = e / (36 * cin), kk = e % (36 * cin);
        const int o = os / 4, s = os % 4, i = kk / 36, d = (kk / 4) % 9, sp = kk % 4;
        G[((o * cin + i) * 9 + d) * 16 + 4 * s + sp] = make_float2((float)sr[0], (float)si[0]);
    }
}

// real block weights for the tensor-core path: Bt[n'][k'], n' = (o*4+s)*2 + op,
// k' = ((i*9+d)*4+s')*2 + kp; zero in the padding columns
__global__ void k_ptc_build_B(int cin, int cout, int Kp, const float2 *W, bf16 *Bt)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 8 * cout * Kp) return;
    const int n = e / Kp, k = e % Kp;
    float v = 0.f;
    if (k < 72 * cin) {
        const int op = n & 1, os = n >> 1, o = os >> 2, s = os & 3;
        const int kp = k & 1, kk = k >> 1, i = kk / 36, d = (kk / 4) % 9, sp = kk & 3;
        const float2 w = W[((o * cin + i) * 9 + d) * 16 + 4 * s + sp];
        v = op == 0 ? (kp == 0 ? w.x : -w.y) : (kp == 0 ? w.y : w.x);
    }
    Bt[e] = __float2bfloat16(v);
}

// backward weights W^b[i][o][d][s'][s] = conj(W[o][i][-d][s][s'])
__global__ void k_ptc_build_Wb(int cin, int cout, const float2 *W, float2 *Wb)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cin * cout * 144) return;
    const int i = e / (cout * 144), o = (e / 144) % cout, d = (e / 16) % 9, sp = (e / 4) % 4, s = e % 4;
    const int dr = d == 0 ? 0 : ((d & 1) ? d + 1 : d - 1);
    const float2 w = W[((o * cin + i) * 9 + dr) * 16 + 4 * s + sp];
    Wb[e] = make_float2(w.x, -w.y);
}

// ------------------------------------------------------------ conversions
template <class ACT>
__global__ void k_canon_to_act(long n, const double2 *in, ACT *out)
{
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x)
        act_store1(out, j, (float)in[j].x, (float)in[j].y);
}
__device__ __forceinline__ float2 act_get(const bf162 *f, long j) { return __bfloat1622float2(f[j]); }
__device__ __forceinline__ float2 act_get(const float2 *f, long j) { return f[j]; }
template <class ACT>
__global__ void k_act_to_canon(long n, const ACT *in, double2 *out)
{
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        float2 v = act_get(in, j);
        out[j] = make_double2(v.x, v.y);
    }
}
// native full FP64 field(s) <-> AoS activations (lexicographic sites)
template <class ACT>
__global__ void k_native_to_act(Geom g, int nrhs, const double2 *in, ACT *out)
{
    long x = blockIdx.x * (long)blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (x >= g.V || r >= nrhs) return;
    int c[4];
    lex_coords(g, x, c);
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
    const double2 *src = in + (long)r * 24 * g.Vh + (long)p * 12 * g.Vh + (x >> 1);
    for (int k = 0; k < 12; k++) {
        double2 v = src[k * (long)g.Vh];
        act_store1(out, (long)r * 12 * g.V + 12 * x + k, (float)v.x, (float)v.y);
    }
}
template <class ACT>
__global__ void k_act_to_native(Geom g, int nrhs, const ACT *in, double2 *out)
{
    long x = blockIdx.x * (long)blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (x >= g.V || r >= nrhs) return;
    int c[4];
    lex_coords(g, x, c);
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
    double2 *dst = out + (long)r * 24 * g.Vh + (long)p * 12 * g.Vh + (x >> 1);
    for (int k = 0; k < 12; k++) {
        float2 v = act_get(in, (long)r * 12 * g.V + 12 * x + k);
        dst[k * (long)g.Vh] = make_double2(v.x, v.y);
    }
}
// native full FP32 fields -> AoS float2 (targets)
__global__ void k_native32_to_f2(Geom g, int nrhs, const float4 *in, float2 *out)
{
    long x = blockIdx.x * (long)blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (x >= g.V || r >= nrhs) return;
    int c[4];
    lex_coords(g, x, c);
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
    const float4 *src = in + (long)r * 12 * g.Vh + (long)p * 6 * g.Vh + (x >> 1);
    for (int q = 0; q < 6; q++) {
        float4 v = src[q * (long)g.Vh];
        out[(long)r * 12 * g.V + 12 * x + 2 * q] = make_float2(v.x, v.y);
        out[(long)r * 12 * g.V + 12 * x + 2 * q + 1] = make_float2(v.z, v.w);
    }
}

// ------------------------------------------------------------ loss
// partial[(b*nblk + blk)*2 + {0,1}] = block sums of |t|^2 and |n - t|^2
template <class ACT>
__global__ void k_loss_partial(long n, const ACT *net, const float2 *t, double *partial)
{
    const int b = blockIdx.y;
    const ACT *nb = net + b * n;
    const float2 *tb = t + b * n;
    double tt = 0, ee = 0;
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        float2 v = act_get(nb, j), w = tb[j];
        double dx = (double)v.x - w.x, dy = (double)v.y - w.y;
        tt += (double)w.x * w.x + (double)w.y * w.y;
        ee += dx * dx + dy * dy;
    }
    __shared__ double s1[256], s2[256];
    s1[threadIdx.x] = tt;
    s2[threadIdx.x] = ee;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            s1[threadIdx.x] += s1[threadIdx.x + s];
            s2[threadIdx.x] += s2[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[((long)b * gridDim.x + blockIdx.x) * 2] = s1[0];
        partial[((long)b * gridDim.x + blockIdx.x) * 2 + 1] = s2[0];
    }
}
// norms[b] = (|t_b|^2, |n_b - t_b|^2); loss = mean_b |n_b - t_b|^2 / |t_b|^2
__global__ void k_loss_final(int nb, int nblk, const double *partial, double *norms, double *loss)
{
    if (threadIdx.x != 0) return;
    double L = 0;
    for (int b = 0; b < nb; b++) {
        double tt = 0, ee = 0;
        for (int k = 0; k < nblk; k++) {
            tt += partial[((long)b * nblk + k) * 2];
            ee += partial[((long)b * nblk + k) * 2 + 1];
        }
        norms[2 * b] = tt;
        norms[2 * b + 1] = ee;
        L += tt > 0 ? ee / tt : 0;
    }
    *loss = L / nb;
}
// delta_b = 2 (n_b - t_b) / (|t_b|^2 nb), the conjugate gradient of the loss
template <class ACT>
__global__ void k_loss_delta(long n, int nb, const ACT *net, const float2 *t, const double *norms, ACT *delta)
{
    const int b = blockIdx.y;
    const double tt = norms[2 * b];
    const float f = tt > 0 ? (float)(2.0 / (tt * nb)) : 0.f;
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        float2 v = act_get(net + b * n, j), w = t[b * n + j];
        act_store1(delta + b * n, j, f * (v.x - w.x), f * (v.y - w.y));
    }
}

// ------------------------------------------------------------ Adam
__global__ void k_adam(long nw, float2 *W, const float2 *G, float2 *m, float2 *v, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (e >= nw) return;
    float2 g = G[e], mm = m[e], vv = v[e], w = W[e];
    mm.x = b1 * mm.x + (1 - b1) * g.x;
    mm.y = b1 * mm.y + (1 - b1) * g.y;
    vv.x = b2 * vv.x + (1 - b2) * g.x * g.x;
    vv.y = b2 * vv.y + (1 - b2) * g.y * g.y;
    w.x -= lr * (mm.x / c1) / (sqrtf(vv.x / c2) + eps);
    w.y -= lr * (mm.y / c1) / (sqrtf(vv.y / c2) + eps);
    m[e] = mm;
    v[e] = vv;
    W[e] = w;
}

inline int gs_grid(long n) { return (int)std::min<long>(1216, (n + 255) / 256); }

}  // namespace

// ====================================================================== state
struct NetState {
    int nl = 0;
    int chans[5] = {0, 0, 0, 0, 0};
    lqcd_prec act = LQCD_BF16;
    long nw = 0;
    long woff[5] = {0, 0, 0, 0, 0};
    float2 *W = nullptr, *m = nullptr, *v = nullptr, *G = nullptr;
    float2 *Wb = nullptr;     // backward weights, per layer at woff[l]
    bf16 *Bf = nullptr, *Bb = nullptr;   // real block weights per layer, offsets boff[l]
    long boff[5] = {0, 0, 0, 0, 0}, bboff[5] = {0, 0, 0, 0, 0};
    int adam_t = 0;
    // training set of the current gauge field
    void *X = nullptr;        // inputs (AoS act)
    float2 *Tg = nullptr;     // targets (AoS float2)
    int ntrain = 0;
    size_t X_bytes = 0, T_bytes = 0;
};

void net_free(lqcd_ctx *c)
{
    NetState *n = c->net;
    if (!n) return;
    cudaFree(n->W);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->G);
    cudaFree(n->Wb);
    cudaFree(n->Bf);
    cudaFree(n->Bb);
    cudaFree(n->X);
    cudaFree(n->Tg);
    delete n;
    c->net = nullptr;
}

namespace {

inline int kpad(int cin) { return (72 * cin + 15) / 16 * 16; }
inline size_t act_elem(lqcd_prec a) { return a == LQCD_BF16 ? sizeof(bf162) : sizeof(float2); }

lqcd_status net_rebuild(lqcd_ctx *c)
{
    NetState *n = c->net;
    for (int l = 0; l < n->nl; l++) {
        int ci = n->chans[l], co = n->chans[l + 1];
        k_ptc_build_Wb<<<div_up((long)ci * co * 144, 256), 256, 0, c->stream>>>(ci, co, n->W + n->woff[l],
                                                                                n->Wb + n->woff[l]);
        k_ptc_build_B<<<div_up(8L * co * kpad(ci), 256), 256, 0, c->stream>>>(ci, co, kpad(ci), n->W + n->woff[l],
                                                                               n->Bf + n->boff[l]);
        k_ptc_build_B<<<div_up(8L * ci * kpad(co), 256), 256, 0, c->stream>>>(co, ci, kpad(co), n->Wb + n->woff[l],
                                                                               n->Bb + n->bboff[l]);
        c->n_kernel_launches += 3;
    }
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

size_t layer_smem(lqcd_prec act, int cin, int cout)
{
    if (act == LQCD_BF16) return sizeof(PtStage) + (size_t)(PT_ROWS + 8 * cout) * pt_ld(kpad(cin)) * sizeof(bf16);
    return sizeof(PtStage) + (size_t)PT_ROWS * 36 * cin * sizeof(cx<float>) +
           (size_t)cout * cin * 144 * sizeof(cx<float>);
}
size_t wgrad_smem(int cin, int cout)
{
    return sizeof(PtStage) + (size_t)PT_ROWS * 36 * cin * sizeof(cx<float>) +
           (size_t)PT_ROWS * 4 * cout * sizeof(cx<float>);
}

template <class ACT>
lqcd_status launch_layer(lqcd_ctx *c, const void *in, void *out, int cin, int cout, int nb, const bf16 *Bt,
                         const float2 *Wc)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_ptc_layer<ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    LayerArgs a;
    a.g = c->g;
    a.U = c->U32;
    a.in = in;
    a.out = out;
    a.cin = cin;
    a.cout = cout;
    a.in_ss = (long)cin * 12 * c->g.V;
    a.out_ss = (long)cout * 12 * c->g.V;
    a.Bt = Bt;
    a.Wc = Wc;
    lqcd_prec act = sizeof(ACT) == 4 ? LQCD_BF16 : LQCD_F32;
    k_ptc_layer<ACT><<<dim3(div_up(c->g.V, PT_SITES), nb), PT_THREADS, layer_smem(act, cin, cout), c->stream>>>(a);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

lqcd_status layer_fwd(lqcd_ctx *c, int l, const void *in, void *out, int nb)
{
    NetState *n = c->net;
    int ci = n->chans[l], co = n->chans[l + 1];
    if (n->act == LQCD_BF16) return launch_layer<bf162>(c, in, out, ci, co, nb, n->Bf + n->boff[l], nullptr);
    return launch_layer<float2>(c, in, out, ci, co, nb, nullptr, n->W + n->woff[l]);
}
lqcd_status layer_bwd(lqcd_ctx *c, int l, const void *dout, void *din, int nb)
{
    NetState *n = c->net;
    int ci = n->chans[l], co = n->chans[l + 1];
    if (n->act == LQCD_BF16) return launch_layer<bf162>(c, dout, din, co, ci, nb, n->Bb + n->bboff[l], nullptr);
    return launch_layer<float2>(c, dout, din, co, ci, nb, nullptr, n->Wb + n->woff[l]);
}

template <class ACT>
lqcd_status wgrad_t(lqcd_ctx *c, int l, const void *y, const void *delta, int nb, float2 *G)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_ptc_wgrad<ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    NetState *n = c->net;
    const int ci = n->chans[l], co = n->chans[l + 1];
    const int ncta = div_up(c->g.V, PT_SITES);
    const int nout = co * 4 * 36 * ci;
    void *part;
    LQCD_TRY(ws_get(c, WS_NET_PART, (size_t)ncta * nb * nout * sizeof(float2), &part));
    WgradArgs a;
    a.g = c->g;
    a.U = c->U32;
    a.y = y;
    a.delta = delta;
    a.cin = ci;
    a.cout = co;
    a.y_ss = (long)ci * 12 * c->g.V;
    a.d_ss = (long)co * 12 * c->g.V;
    a.partial = (float2 *)part;
    k_ptc_wgrad<ACT><<<dim3(ncta, nb), PT_THREADS, wgrad_smem(ci, co), c->stream>>>(a);
    k_ptc_wgrad_reduce<<<nout, 256, 0, c->stream>>>(ncta * nb, ci, co, (const float2 *)part, G + n->woff[l]);
    c->n_kernel_launches += 2;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}
lqcd_status wgrad(lqcd_ctx *c, int l, const void *y, const void *delta, int nb, float2 *G)
{
    return c->net->act == LQCD_BF16 ? wgrad_t<bf162>(c, l, y, delta, nb, G) : wgrad_t<float2>(c, l, y, delta, nb, G);
}

// activation buffers for nb samples: acts[l] for l = 0..nl (acts[0] = input)
struct ActBufs {
    void *a[5];
    void *d[5];
};
lqcd_status net_buffers(lqcd_ctx *c, int nb, ActBufs &B)
{
    NetState *n = c->net;
    size_t per = 12 * (size_t)c->g.V * act_elem(n->act) * nb;
    size_t total = 0;
    for (int l = 0; l <= n->nl; l++) total += 2 * per * n->chans[l];
    void *buf;
    LQCD_TRY(ws_get(c, WS_NET_ACT, total, &buf));
    char *p = (char *)buf;
    for (int l = 0; l <= n->nl; l++) {
        B.a[l] = p;
        p += per * n->chans[l];
        B.d[l] = p;
        p += per * n->chans[l];
    }
    return LQCD_OK;
}

lqcd_status net_forward(lqcd_ctx *c, ActBufs &B, int nb)
{
    for (int l = 0; l < c->net->nl; l++) LQCD_TRY(layer_fwd(c, l, B.a[l], B.a[l + 1], nb));
    return LQCD_OK;
}

// loss on B.a[nl] against targets T (float2 AoS, nb samples); delta into B.d[nl]
lqcd_status net_loss(lqcd_ctx *c, ActBufs &B, const float2 *T, int nb, double *loss_dev)
{
    NetState *n = c->net;
    const long ns = 12 * (long)c->g.V;
    const int nblk = std::max(1, std::min(64, div_up(ns, 4096)));
    double *partial = c->red, *norms = c->red + 2 * 64 * nb;
    if (n->act == LQCD_BF16) {
        k_loss_partial<bf162><<<dim3(nblk, nb), 256, 0, c->stream>>>(ns, (const bf162 *)B.a[n->nl], T, partial);
        k_loss_final<<<1, 32, 0, c->stream>>>(nb, nblk, partial, norms, loss_dev);
        k_loss_delta<bf162><<<dim3(gs_grid(ns) / 4 + 1, nb), 256, 0, c->stream>>>(ns, nb, (const bf162 *)B.a[n->nl], T,
                                                                                 norms, (bf162 *)B.d[n->nl]);
    } else {
        k_loss_partial<float2><<<dim3(nblk, nb), 256, 0, c->stream>>>(ns, (const float2 *)B.a[n->nl], T, partial);
        k_loss_final<<<1, 32, 0, c->stream>>>(nb, nblk, partial, norms, loss_dev);
        k_loss_delta<float2><<<dim3(gs_grid(ns) / 4 + 1, nb), 256, 0, c->stream>>>(
            ns, nb, (const float2 *)B.a[n->nl], T, norms, (float2 *)B.d[n->nl]);
    }
    c->n_kernel_launches += 3;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

// GCR residual loss: L = (1/nb) sum_b |x_b - D N(x_b)|^2 / |x_b|^2 on the
// batch in B.a[0] with N(x) in B.a[nl]; the gradient at the network output,
// -2 D^dag r_b / (nb |x_b|^2) with r = x - D N(x) and D^dag = gamma5 D gamma5,
// goes to B.d[nl] (all in FP64 between the activation conversions)
template <class ACT>
lqcd_status residual_loss_t(lqcd_ctx *c, ActBufs &B, int nb, double *loss_dev)
{
    NetState *n = c->net;
    const long Vh = c->g.Vh, nf = 24 * Vh;   // double2 per native full field
    void *w;
    LQCD_TRY(ws_get(c, WS_NET_FALLBACK, 3 * (size_t)nb * nf * sizeof(double2), &w));
    double2 *xn = (double2 *)w, *yn = xn + nb * nf, *tn = yn + nb * nf;
    const dim3 grid(div_up(c->g.V, 256), nb);
    k_act_to_native<ACT><<<grid, 256, 0, c->stream>>>(c->g, nb, (const ACT *)B.a[0], xn);
    k_act_to_native<ACT><<<grid, 256, 0, c->stream>>>(c->g, nb, (const ACT *)B.a[n->nl], yn);
    c->n_kernel_launches += 2;
    LQCD_LAUNCH_CHECK(c);
    LQCD_TRY(dirac_D(c, LQCD_F64, yn, tn, nb));                          // t = D N(x)
    LQCD_TRY(blas_sub(c, 2 * nb * nf, (const double *)xn, (const double *)tn, (double *)tn));   // r
    double L = 0;
    std::vector<double> sc(nb);
    for (int b = 0; b < nb; b++) {
        double xx, rr;
        LQCD_TRY(blas_norm2(c, 2 * nf, (const double *)(xn + b * nf), &xx));
        LQCD_TRY(blas_norm2(c, 2 * nf, (const double *)(tn + b * nf), &rr));
        L += xx > 0 ? rr / xx / nb : 0.0;
        sc[b] = xx > 0 ? -2.0 / (nb * xx) : 0.0;
    }
    LQCD_TRY(blas_gamma5_native64(c, 2L * nb, tn, tn));
    LQCD_TRY(dirac_D(c, LQCD_F64, tn, yn, nb));
    LQCD_TRY(blas_gamma5_native64(c, 2L * nb, yn, yn));                   // D^dag r
    for (int b = 0; b < nb; b++) LQCD_TRY(blas_scal(c, 2 * nf, sc[b], 0.0, (double *)(yn + b * nf)));
    k_native_to_act<ACT><<<grid, 256, 0, c->stream>>>(c->g, nb, yn, (ACT *)B.d[n->nl]);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(loss_dev, &L, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}
lqcd_status net_residual_loss(lqcd_ctx *c, ActBufs &B, int nb, double *loss_dev)
{
    return c->net->act == LQCD_BF16 ? residual_loss_t<bf162>(c, B, nb, loss_dev)
                                    : residual_loss_t<float2>(c, B, nb, loss_dev);
}

lqcd_status net_backward(lqcd_ctx *c, ActBufs &B, int nb)
{
    NetState *n = c->net;
    for (int l = n->nl - 1; l >= 0; l--) {
        LQCD_TRY(wgrad(c, l, B.a[l], B.d[l + 1], nb, n->G));
        if (l > 0) LQCD_TRY(layer_bwd(c, l, B.d[l + 1], B.d[l], nb));
    }
    return LQCD_OK;
}

lqcd_status canon_to_act(lqcd_ctx *c, const double *in, void *out, long ncomplex)
{
    if (c->net->act == LQCD_BF16)
        k_canon_to_act<bf162><<<gs_grid(ncomplex), 256, 0, c->stream>>>(ncomplex, (const double2 *)in, (bf162 *)out);
    else
        k_canon_to_act<float2><<<gs_grid(ncomplex), 256, 0, c->stream>>>(ncomplex, (const double2 *)in, (float2 *)out);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

}  // namespace

// phi = N(rho) for nrhs native full FP64 fields (GCR preconditioner)
lqcd_status net_apply_native(lqcd_ctx *c, const double2 *rho, double2 *phi, int nrhs)
{
    NetState *n = c->net;
    if (!n) return set_err(c, LQCD_ERR_STATE, "network not set");
    ActBufs B;
    LQCD_TRY(net_buffers(c, nrhs, B));
    dim3 grid(div_up(c->g.V, 256), nrhs);
    if (n->act == LQCD_BF16)
        k_native_to_act<bf162><<<grid, 256, 0, c->stream>>>(c->g, nrhs, rho, (bf162 *)B.a[0]);
    else
        k_native_to_act<float2><<<grid, 256, 0, c->stream>>>(c->g, nrhs, rho, (float2 *)B.a[0]);
    c->n_kernel_launches++;
    LQCD_TRY(net_forward(c, B, nrhs));
    if (n->act == LQCD_BF16)
        k_act_to_native<bf162><<<grid, 256, 0, c->stream>>>(c->g, nrhs, (const bf162 *)B.a[n->nl], phi);
    else
        k_act_to_native<float2><<<grid, 256, 0, c->stream>>>(c->g, nrhs, (const float2 *)B.a[n->nl], phi);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

extern "C" {

lqcd_status lqcd_net_set(lqcd_ctx *c, const lqcd_net_desc *desc, const float *W_host)
{
    if (!c || !desc || !W_host) return set_err(c, LQCD_ERR_ARG, "null argument");
    if (desc->nlayers < 1 || desc->nlayers > 4) return set_err(c, LQCD_ERR_ARG, "nlayers=%d", desc->nlayers);
    if (desc->act != LQCD_BF16 && desc->act != LQCD_F32) return set_err(c, LQCD_ERR_ARG, "activation precision");
    if (desc->chans[0] != 1 || desc->chans[desc->nlayers] != 1)
        return set_err(c, LQCD_ERR_ARG, "the network maps one field to one field");
    for (int l = 0; l <= desc->nlayers; l++)
        if (desc->chans[l] < 1 || desc->chans[l] > PT_CMAX)
            return set_err(c, LQCD_ERR_ARG, "channel count %d (1..%d)", desc->chans[l], PT_CMAX);
    net_free(c);
    NetState *n = new NetState();
    c->net = n;
    n->nl = desc->nlayers;
    n->act = desc->act;
    long nw = 0, nbf = 0, nbb = 0;
    for (int l = 0; l <= n->nl; l++) n->chans[l] = desc->chans[l];
    for (int l = 0; l < n->nl; l++) {
        int ci = n->chans[l], co = n->chans[l + 1];
        n->woff[l] = nw;
        n->boff[l] = nbf;
        n->bboff[l] = nbb;
        nw += (long)ci * co * 144;
        nbf += 8L * co * kpad(ci);
        nbb += 8L * ci * kpad(co);
    }
    n->nw = nw;
    if (cudaMalloc(&n->W, nw * sizeof(float2)) != cudaSuccess || cudaMalloc(&n->m, nw * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&n->v, nw * sizeof(float2)) != cudaSuccess || cudaMalloc(&n->G, nw * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&n->Wb, nw * sizeof(float2)) != cudaSuccess || cudaMalloc(&n->Bf, nbf * sizeof(bf16)) != cudaSuccess ||
        cudaMalloc(&n->Bb, nbb * sizeof(bf16)) != cudaSuccess) {
        cudaGetLastError();
        net_free(c);
        return set_err(c, LQCD_ERR_NOMEM, "network allocation");
    }
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(n->W, W_host, nw * sizeof(float2), cudaMemcpyHostToDevice, c->stream));
    LQCD_CUDA_CHECK(c, cudaMemsetAsync(n->m, 0, nw * sizeof(float2), c->stream));
    LQCD_CUDA_CHECK(c, cudaMemsetAsync(n->v, 0, nw * sizeof(float2), c->stream));
    LQCD_TRY(net_rebuild(c));
    LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

lqcd_status lqcd_net_get(lqcd_ctx *c, float *W_host)
{
    if (!c || !W_host) return set_err(c, LQCD_ERR_ARG, "null argument");
    if (!c->net) return set_err(c, LQCD_ERR_STATE, "network not set");
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(W_host, c->net->W, c->net->nw * sizeof(float2), cudaMemcpyDeviceToHost,
                                       c->stream));
    LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

lqcd_status lqcd_net_apply(lqcd_ctx *c, const double *in, double *out, int nrhs)
{
    if (!c || !in || !out || nrhs < 1) return set_err(c, LQCD_ERR_ARG, "bad argument");
    if (!c->net) return set_err(c, LQCD_ERR_STATE, "network not set");
    if (!c->have_gauge) return set_err(c, LQCD_ERR_STATE, "gauge field not set");
    NetState *n = c->net;
    ActBufs B;
    LQCD_TRY(net_buffers(c, nrhs, B));
    const long ns = 12 * (long)c->g.V;
    LQCD_TRY(canon_to_act(c, in, B.a[0], ns * nrhs));
    LQCD_TRY(net_forward(c, B, nrhs));
    if (n->act == LQCD_BF16)
        k_act_to_canon<bf162><<<gs_grid(ns * nrhs), 256, 0, c->stream>>>(ns * nrhs, (const bf162 *)B.a[n->nl],
                                                                          (double2 *)out);
    else
        k_act_to_canon<float2><<<gs_grid(ns * nrhs), 256, 0, c->stream>>>(ns * nrhs, (const float2 *)B.a[n->nl],
                                                                           (double2 *)out);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

lqcd_status lqcd_net_loss_grad(lqcd_ctx *c, const double *in, const double *target, int nb, double *loss,
                               float *grad_host)
{
    if (!c || !in || !target || nb < 1) return set_err(c, LQCD_ERR_ARG, "bad argument");
    if (!c->net) return set_err(c, LQCD_ERR_STATE, "network not set");
    if (!c->have_gauge) return set_err(c, LQCD_ERR_STATE, "gauge field not set");
    if (nb > 64) return set_err(c, LQCD_ERR_ARG, "nb=%d (<= 64)", nb);
    NetState *n = c->net;
    ActBufs B;
    LQCD_TRY(net_buffers(c, nb, B));
    const long ns = 12 * (long)c->g.V;
    LQCD_TRY(canon_to_act(c, in, B.a[0], ns * nb));
    void *tb;
    LQCD_TRY(ws_get(c, WS_NET_TGT, ns * nb * sizeof(float2), &tb));
    k_canon_to_act<float2><<<gs_grid(ns * nb), 256, 0, c->stream>>>(ns * nb, (const double2 *)target, (float2 *)tb);
    c->n_kernel_launches++;
    LQCD_TRY(net_forward(c, B, nb));
    double *loss_dev = c->red_out;
    LQCD_TRY(net_loss(c, B, (const float2 *)tb, nb, loss_dev));
    LQCD_TRY(net_backward(c, B, nb));
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(c->red_host, loss_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (grad_host)
        LQCD_CUDA_CHECK(c, cudaMemcpyAsync(grad_host, n->G, n->nw * sizeof(float2), cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    if (loss) *loss = c->red_host[0];
    return LQCD_OK;
}

lqcd_status lqcd_net_train(lqcd_ctx *c, const lqcd_net_train_params *p, const double *sources, int nsrc,
                           double *loss_history)
{
    if (!c || !p || !sources || nsrc < 1) return set_err(c, LQCD_ERR_ARG, "bad argument");
    if (!c->net) return set_err(c, LQCD_ERR_STATE, "network not set");
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    if (p->batch < 1 || p->batch > 64 || p->batch > nsrc || p->steps < 0)
        return set_err(c, LQCD_ERR_ARG, "batch %d / steps %d", p->batch, p->steps);
    if (p->loss != 0 && p->loss != 1) return set_err(c, LQCD_ERR_ARG, "loss %d", p->loss);
    if (p->loss == 0 && p->sap.prec != LQCD_F32 && p->sap.prec != LQCD_F64)
        return set_err(c, LQCD_ERR_ARG, "SAP precision");
    NetState *n = c->net;
    const long ns = 12 * (long)c->g.V;
    const size_t xb = ns * nsrc * act_elem(n->act), tbytes = ns * nsrc * sizeof(float2);
    if (n->X_bytes < xb) {
        cudaFree(n->X);
        n->X = nullptr;
        n->X_bytes = 0;
        LQCD_CUDA_CHECK(c, cudaMalloc(&n->X, xb));
        n->X_bytes = xb;
    }
    if (n->T_bytes < tbytes) {
        cudaFree(n->Tg);
        n->Tg = nullptr;
        n->T_bytes = 0;
        LQCD_CUDA_CHECK(c, cudaMalloc(&n->Tg, tbytes));
        n->T_bytes = tbytes;
    }
    // inputs and SAP targets of every source, in chunks of up to 16 sources
    LQCD_TRY(canon_to_act(c, sources, n->X, ns * nsrc));
    const size_t f64b = 2 * native_half_bytes(c, LQCD_F64), fpb = 2 * native_half_bytes(c, p->sap.prec);
    const int chunk = 16;
    void *a64, *ain, *aout, *a32;
    LQCD_TRY(ws_get(c, WS_NET_TGT, f64b * chunk, &a64));
    LQCD_TRY(ws_get(c, WS_SAP_IN, fpb * chunk, &ain));
    LQCD_TRY(ws_get(c, WS_SAP_PSI, fpb * chunk, &aout));
    LQCD_TRY(ws_get(c, WS_MISC, 2 * native_half_bytes(c, LQCD_F32) * chunk, &a32));
    for (int s0 = 0; s0 < nsrc && p->loss == 0; s0 += chunk) {
        const int cnt = std::min(chunk, nsrc - s0);
        LQCD_TRY(pack_field(c, LQCD_F64, 2, sources + (size_t)s0 * 2 * ns, a64, cnt, false));
        LQCD_TRY(convert_native(c, LQCD_F64, p->sap.prec, a64, ain, 2L * cnt));
        LQCD_TRY(sap_apply(c, &p->sap, ain, aout, cnt));
        LQCD_TRY(convert_native(c, p->sap.prec, LQCD_F32, aout, a32, 2L * cnt));
        k_native32_to_f2<<<dim3(div_up(c->g.V, 256), cnt), 256, 0, c->stream>>>(c->g, cnt, (const float4 *)a32,
                                                                                 n->Tg + (size_t)s0 * ns);
        c->n_kernel_launches++;
        LQCD_LAUNCH_CHECK(c);
    }
    ActBufs B;
    LQCD_TRY(net_buffers(c, p->batch, B));
    const size_t ae = act_elem(n->act);
    std::vector<double> hist;
    double *loss_dev = c->red_out + 8;
    for (int step = 0; step < p->steps; step++) {
        // batch: sources (step*batch + j) mod nsrc, copied into the input slot
        void *tslot;
        LQCD_TRY(ws_get(c, WS_NET_BATCH_T, ns * p->batch * sizeof(float2), &tslot));
        for (int j = 0; j < p->batch; j++) {
            const int s = (int)(((long)step * p->batch + j) % nsrc);
            LQCD_CUDA_CHECK(c, cudaMemcpyAsync((char *)B.a[0] + (size_t)j * ns * ae, (char *)n->X + (size_t)s * ns * ae,
                                               ns * ae, cudaMemcpyDeviceToDevice, c->stream));
            if (p->loss == 0)
                LQCD_CUDA_CHECK(c, cudaMemcpyAsync((float2 *)tslot + (size_t)j * ns, n->Tg + (size_t)s * ns,
                                                   ns * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
        }
        LQCD_TRY(net_forward(c, B, p->batch));
        if (p->loss == 0)
            LQCD_TRY(net_loss(c, B, (const float2 *)tslot, p->batch, loss_dev));
        else
            LQCD_TRY(net_residual_loss(c, B, p->batch, loss_dev));
        LQCD_TRY(net_backward(c, B, p->batch));
        n->adam_t++;
        const float c1 = 1.f - powf((float)p->beta1, (float)n->adam_t), c2 = 1.f - powf((float)p->beta2, (float)n->adam_t);
        k_adam<<<div_up(n->nw, 256), 256, 0, c->stream>>>(n->nw, n->W, n->G, n->m, n->v, (float)p->lr, (float)p->beta1,
                                                          (float)p->beta2, (float)p->eps, c1, c2);
        c->n_kernel_launches++;
        LQCD_TRY(net_rebuild(c));
        if (loss_history) {
            double l;
            LQCD_CUDA_CHECK(c, cudaMemcpyAsync(&c->red_host[8], loss_dev, sizeof(double), cudaMemcpyDeviceToHost,
                                               c->stream));
            LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
            l = c->red_host[8];
            loss_history[step] = l;
        }
    }
    LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

}  // extern "C"
