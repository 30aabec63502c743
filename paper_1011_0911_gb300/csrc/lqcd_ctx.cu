// Context management, layout conversion and the operator entry points of the
// C ABI (include/lqcd.h).
#include <cstdarg>
#include <cstring>

#include <type_traits>

#include "lqcd_f16s.cuh"
#include <cstdlib>

#include "lqcd_internal.cuh"

lqcd_status set_err(lqcd_ctx *c, lqcd_status s, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

lqcd_status ws_get(lqcd_ctx *c, int slot, size_t bytes, void **out)
{
    Workspace &w = c->ws[slot];
    if (w.bytes < bytes) {
        if (w.p) cudaFree(w.p);
        w.p = nullptr;
        w.bytes = 0;
        if (cudaMalloc(&w.p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, LQCD_ERR_NOMEM, "workspace %d: cannot allocate %zu bytes", slot, bytes);
        }
        w.bytes = bytes;
    }
    *out = w.p;
    return LQCD_OK;
}

void geom_init(Geom &g, const int L[4], int bc_t)
{
    long V = 1;
    for (int i = 0; i < 4; i++) {
        g.L[i] = L[i];
        V *= L[i];
    }
    g.V = (int)V;
    g.Vh = (int)(V / 2);
    g.L3h = L[3] / 2;
    g.bc_t = bc_t;
    g.dL3h = make_fastdiv(g.L3h);
    g.dL2 = make_fastdiv(L[2]);
    g.dL1 = make_fastdiv(L[1]);
}

size_t native_half_bytes(const lqcd_ctx *c, lqcd_prec p)
{
    long Vh = c->g.Vh;
    if (p == LQCD_F64) return (size_t)12 * Vh * sizeof(double2);
    if (p == LQCD_F32) return (size_t)6 * Vh * sizeof(float4);
    return (size_t)3 * Vh * sizeof(uint4) + (size_t)Vh * sizeof(float);
}

namespace {

// canonical full-lattice links [site][mu][3][3] (FP64) -> native F64 (all 9
// entries) and F32 / F16 (first two rows)
__global__ void k_pack_links(Geom g, const double2 *__restrict__ U, double2 *U64, float4 *U32, uint2 *U16)
{
    long site = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (site >= g.V) return;
    int x3 = site % g.L[3];
    long t = site / g.L[3];
    int x2 = t % g.L[2];
    t /= g.L[2];
    int x1 = t % g.L[1];
    int x0 = t / g.L[1];
    int p = (x0 + x1 + x2 + x3) & 1;
    long r = site >> 1;
    long Vh = g.Vh;
    for (int mu = 0; mu < 4; mu++) {
        const double2 *src = U + (site * 4 + mu) * 9;
        double2 e[9];
        for (int i = 0; i < 9; i++) e[i] = src[i];
        for (int i = 0; i < 9; i++) U64[((long)(p * 4 + mu) * 9 + i) * Vh + r] = e[i];
        for (int q = 0; q < 3; q++) {
            U32[((long)(p * 4 + mu) * 3 + q) * Vh + r] =
                make_float4((float)e[2 * q].x, (float)e[2 * q].y, (float)e[2 * q + 1].x, (float)e[2 * q + 1].y);
            __half2 a = __floats2half2_rn((float)e[2 * q].x, (float)e[2 * q].y);
            __half2 b = __floats2half2_rn((float)e[2 * q + 1].x, (float)e[2 * q + 1].y);
            uint2 w;
            w.x = *reinterpret_cast<unsigned *>(&a);
            w.y = *reinterpret_cast<unsigned *>(&b);
            U16[((long)(p * 4 + mu) * 3 + q) * Vh + r] = w;
        }
    }
}

// canonical spinor fields <-> native.  nsub = 1: canonical half field, site
// index = rank; nsub = 2: canonical full field, lexicographic sites.
template <class CT>
__device__ __forceinline__ void site_of(const Geom &g, int nsub, long i, int &p, long &r)
{
    if (nsub == 1) {
        p = 0;
        r = i;
    } else {
        int x3 = i % g.L[3];
        long t = i / g.L[3];
        int x2 = t % g.L[2];
        t /= g.L[2];
        int x1 = t % g.L[1];
        int x0 = t / g.L[1];
        p = (x0 + x1 + x2 + x3) & 1;
        r = i >> 1;
    }
}

template <class CT, int PREC>
__global__ void k_pack(Geom g, int nsub, int nrhs, const CT *__restrict__ canon, void *native, int unpack)
{
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    int k = blockIdx.y;
    long nsite = (long)nsub * g.Vh;
    if (i >= nsite || k >= nrhs) return;
    int p;
    long r;
    site_of<CT>(g, nsub, i, p, r);
    long Vh = g.Vh;
    long half = (long)k * nsub + (nsub == 2 ? p : 0);
    CT *cs = (CT *)canon + ((long)k * nsite + i) * 24;
    if (PREC == LQCD_F64) {
        double2 *n = (double2 *)native + half * 12 * Vh + r;
        for (int c = 0; c < 12; c++) {
            if (unpack) {
                double2 v = n[c * Vh];
                cs[2 * c] = (CT)v.x;
                cs[2 * c + 1] = (CT)v.y;
            } else {
                n[c * Vh] = make_double2((double)cs[2 * c], (double)cs[2 * c + 1]);
            }
        }
    } else if (PREC == LQCD_F16S) {
        h16s *n = (h16s *)native + half * f16s_half_units(Vh);
        cx<float> v[12];
        if (unpack) {
            f16s_load<false>(n, Vh, r, v);
            for (int c = 0; c < 12; c++) {
                cs[2 * c] = (CT)v[c].re;
                cs[2 * c + 1] = (CT)v[c].im;
            }
        } else {
            for (int c = 0; c < 12; c++) v[c] = mk((float)cs[2 * c], (float)cs[2 * c + 1]);
            f16s_store(n, Vh, r, v);
        }
    } else if (PREC == LQCD_F32) {
        float4 *n = (float4 *)native + half * 6 * Vh + r;
        for (int q = 0; q < 6; q++) {
            if (unpack) {
                float4 v = n[q * Vh];
                cs[4 * q] = (CT)v.x;
                cs[4 * q + 1] = (CT)v.y;
                cs[4 * q + 2] = (CT)v.z;
                cs[4 * q + 3] = (CT)v.w;
            } else {
                n[q * Vh] = make_float4((float)cs[4 * q], (float)cs[4 * q + 1], (float)cs[4 * q + 2],
                                        (float)cs[4 * q + 3]);
            }
        }
    }
}

// native F64 <-> native F32 (same site/chunk structure), nhalf half fields
__global__ void k_conv64to32(long Vh, long nhalf, const double2 *__restrict__ in, float4 *out)
{
    long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
    long h = blockIdx.y;
    if (r >= Vh || h >= nhalf) return;
    const double2 *i = in + h * 12 * Vh + r;
    float4 *o = out + h * 6 * Vh + r;
    for (int q = 0; q < 6; q++) {
        double2 a = i[(2 * q) * Vh], b = i[(2 * q + 1) * Vh];
        o[q * Vh] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    }
}
__global__ void k_conv32to64(long Vh, long nhalf, const float4 *__restrict__ in, double2 *out)
{
    long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
    long h = blockIdx.y;
    if (r >= Vh || h >= nhalf) return;
    const float4 *i = in + h * 6 * Vh + r;
    double2 *o = out + h * 12 * Vh + r;
    for (int q = 0; q < 6; q++) {
        float4 a = i[q * Vh];
        o[(2 * q) * Vh] = make_double2(a.x, a.y);
        o[(2 * q + 1) * Vh] = make_double2(a.z, a.w);
    }
}

// native F64 / F32 <-> native F16S, nhalf half fields
__device__ __forceinline__ void nat_load(const double2 *f, long Vh, long r, cx<float> v[12])
{
    for (int c = 0; c < 12; c++) {
        double2 a = f[c * Vh + r];
        v[c] = mk((float)a.x, (float)a.y);
    }
}
__device__ __forceinline__ void nat_load(const float4 *f, long Vh, long r, cx<float> v[12])
{
    for (int q = 0; q < 6; q++) {
        float4 a = f[q * Vh + r];
        v[2 * q] = mk(a.x, a.y);
        v[2 * q + 1] = mk(a.z, a.w);
    }
}
__device__ __forceinline__ void nat_store(double2 *f, long Vh, long r, const cx<float> v[12])
{
    for (int c = 0; c < 12; c++) f[c * Vh + r] = make_double2(v[c].re, v[c].im);
}
__device__ __forceinline__ void nat_store(float4 *f, long Vh, long r, const cx<float> v[12])
{
    for (int q = 0; q < 6; q++) f[q * Vh + r] = make_float4(v[2 * q].re, v[2 * q].im, v[2 * q + 1].re, v[2 * q + 1].im);
}
template <class T>
__global__ void k_conv_to16s(long Vh, long nhalf, const T *__restrict__ in, h16s *out)
{
    long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
    long h = blockIdx.y;
    if (r >= Vh || h >= nhalf) return;
    cx<float> v[12];
    nat_load(in + h * (std::is_same<T, double2>::value ? 12 : 6) * Vh, Vh, r, v);
    f16s_store(out + h * f16s_half_units(Vh), Vh, r, v);
}
template <class T>
__global__ void k_conv_from16s(long Vh, long nhalf, const h16s *__restrict__ in, T *out)
{
    long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
    long h = blockIdx.y;
    if (r >= Vh || h >= nhalf) return;
    cx<float> v[12];
    f16s_load<true>(in + h * f16s_half_units(Vh), Vh, r, v);
    nat_store(out + h * (std::is_same<T, double2>::value ? 12 : 6) * Vh, Vh, r, v);
}

}  // namespace

lqcd_status convert_native(lqcd_ctx *c, lqcd_prec from, lqcd_prec to, const void *in, void *out, long nhalf)
{
    dim3 grid(div_up(c->g.Vh, 256), (unsigned)nhalf);
    if (from == LQCD_F64 && to == LQCD_F32)
        k_conv64to32<<<grid, 256, 0, c->stream>>>(c->g.Vh, nhalf, (const double2 *)in, (float4 *)out);
    else if (from == LQCD_F32 && to == LQCD_F64)
        k_conv32to64<<<grid, 256, 0, c->stream>>>(c->g.Vh, nhalf, (const float4 *)in, (double2 *)out);
    else if (from == LQCD_F64 && to == LQCD_F16S)
        k_conv_to16s<double2><<<grid, 256, 0, c->stream>>>(c->g.Vh, nhalf, (const double2 *)in, (h16s *)out);
    else if (from == LQCD_F32 && to == LQCD_F16S)
        k_conv_to16s<float4><<<grid, 256, 0, c->stream>>>(c->g.Vh, nhalf, (const float4 *)in, (h16s *)out);
    else if (from == LQCD_F16S && to == LQCD_F64)
        k_conv_from16s<double2><<<grid, 256, 0, c->stream>>>(c->g.Vh, nhalf, (const h16s *)in, (double2 *)out);
    else if (from == LQCD_F16S && to == LQCD_F32)
        k_conv_from16s<float4><<<grid, 256, 0, c->stream>>>(c->g.Vh, nhalf, (const h16s *)in, (float4 *)out);
    else if (from == to) {
        LQCD_CUDA_CHECK(c, cudaMemcpyAsync(out, in, nhalf * native_half_bytes(c, from),
                                           cudaMemcpyDeviceToDevice, c->stream));
        return LQCD_OK;
    } else
        return set_err(c, LQCD_ERR_ARG, "conversion %d -> %d not supported", (int)from, (int)to);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

lqcd_status pack_field(lqcd_ctx *c, lqcd_prec p, int nsub, const void *canon, void *native, int nrhs,
                       bool unpack)
{
    if (nsub != 1 && nsub != 2) return set_err(c, LQCD_ERR_ARG, "nsub must be 1 or 2");
    if (nrhs < 1 || nrhs > 65535) return set_err(c, LQCD_ERR_ARG, "bad nrhs %d", nrhs);
    dim3 grid(div_up((long)nsub * c->g.Vh, 256), nrhs);
    if (p == LQCD_F64)
        k_pack<double, LQCD_F64><<<grid, 256, 0, c->stream>>>(c->g, nsub, nrhs, (const double *)canon, native,
                                                               unpack);
    else if (p == LQCD_F32)
        k_pack<float, LQCD_F32><<<grid, 256, 0, c->stream>>>(c->g, nsub, nrhs, (const float *)canon, native,
                                                             unpack);
    else if (p == LQCD_F16S)
        k_pack<float, LQCD_F16S><<<grid, 256, 0, c->stream>>>(c->g, nsub, nrhs, (const float *)canon, native,
                                                               unpack);
    else
        return set_err(c, LQCD_ERR_ARG, "pack: precision %d has no canonical form", (int)p);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

// ======================================================================== ABI
extern "C" {

lqcd_status lqcd_create(const lqcd_geom *geom, void *stream, lqcd_ctx **out)
{
    if (!geom || !out) return LQCD_ERR_ARG;
    *out = nullptr;
    int L[4] = {geom->T, geom->L1, geom->L2, geom->L3};
    long V = 1;
    for (int i = 0; i < 4; i++) {
        if (L[i] <= 0 || L[i] % 2) return LQCD_ERR_ARG;
        V *= L[i];
    }
    if (V > (1L << 29)) return LQCD_ERR_ARG;
    lqcd_ctx *c = new lqcd_ctx();
    c->geom = *geom;
    geom_init(c->g, L, geom->antiperiodic_t ? -1 : 1);
    c->stream = (cudaStream_t)stream;
    c->prof_on = getenv("LQCD_PROFILE") && getenv("LQCD_PROFILE")[0] == '1';
    if (cudaMalloc(&c->red, 4096 * 2 * 64 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->red_out, 4 * 2048 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->red_host, 4 * 2048 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        lqcd_destroy(c);
        return LQCD_ERR_NOMEM;
    }
    *out = c;
    return LQCD_OK;
}

lqcd_status lqcd_destroy(lqcd_ctx *c)
{
    if (!c) return LQCD_OK;
    dfl_free(c);
    net_free(c);
    chrono_free(c);
    sap_free_plans(c);
    cudaFree(c->U64);
    cudaFree(c->U32);
    cudaFree(c->U16);
    for (int p = 0; p < 2; p++) {
        cudaFree(c->A64[p]);
        cudaFree(c->Ai64[p]);
        cudaFree(c->A32[p]);
        cudaFree(c->Ai32[p]);
        cudaFree(c->A16[p]);
        cudaFree(c->Ai16[p]);
    }
    cudaFree(c->red);
    cudaFree(c->red_out);
    if (c->red_host) cudaFreeHost(c->red_host);
    for (auto &w : c->ws)
        if (w.p) cudaFree(w.p);
    delete c;
    return LQCD_OK;
}

const char *lqcd_last_error(const lqcd_ctx *c) { return c ? c->err : "no context"; }

long lqcd_kernel_launches(const lqcd_ctx *c) { return c ? c->n_kernel_launches : 0; }

lqcd_status lqcd_set_stream(lqcd_ctx *c, void *stream)
{
    if (!c) return LQCD_ERR_ARG;
    c->stream = (cudaStream_t)stream;
    return LQCD_OK;
}

lqcd_status lqcd_set_gauge(lqcd_ctx *c, const double *U_dev)
{
    if (!c || !U_dev) return set_err(c, LQCD_ERR_ARG, "null argument");
    long Vh = c->g.Vh;
    if (!c->U64) {
        LQCD_CUDA_CHECK(c, cudaMalloc(&c->U64, 2 * 4 * 9 * Vh * sizeof(double2)));
        LQCD_CUDA_CHECK(c, cudaMalloc(&c->U32, 2 * 4 * 3 * Vh * sizeof(float4)));
        LQCD_CUDA_CHECK(c, cudaMalloc(&c->U16, 2 * 4 * 3 * Vh * sizeof(uint2)));
    }
    k_pack_links<<<div_up(c->g.V, 128), 128, 0, c->stream>>>(c->g, (const double2 *)U_dev, c->U64, c->U32,
                                                             c->U16);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    c->have_gauge = true;
    c->have_clover = false;
    dfl_free(c);
    return LQCD_OK;
}

lqcd_status lqcd_clover_invert(lqcd_ctx *c, double kappa, double csw, double *ld_e, double *ld_o)
{
    if (!c) return LQCD_ERR_ARG;
    dfl_free(c);
    return clover_build(c, kappa, csw, ld_e, ld_o);
}

lqcd_status lqcd_apply_clover(lqcd_ctx *c, int parity, int inverse, const double *in, double *out)
{
    if (!c || !in || !out || parity < 0 || parity > 1) return set_err(c, LQCD_ERR_ARG, "bad argument");
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    size_t hb = native_half_bytes(c, LQCD_F64);
    void *a, *b;
    LQCD_TRY(ws_get(c, WS_PACK_IN, hb, &a));
    LQCD_TRY(ws_get(c, WS_PACK_OUT, hb, &b));
    LQCD_TRY(pack_field(c, LQCD_F64, 1, in, a, 1, false));
    LQCD_TRY(clover_apply_native64(c, parity, inverse, (const double2 *)a, (double2 *)b));
    LQCD_TRY(pack_field(c, LQCD_F64, 1, out, b, 1, true));
    return LQCD_OK;
}

size_t lqcd_native_bytes(const lqcd_ctx *c, lqcd_prec p, int nsub, int nrhs)
{
    if (!c || nsub < 1 || nsub > 2 || nrhs < 1) return 0;
    return native_half_bytes(c, p) * nsub * nrhs;
}

lqcd_status lqcd_pack(lqcd_ctx *c, lqcd_prec p, int nsub, const void *canon, void *native, int nrhs)
{
    if (!c || !canon || !native) return set_err(c, LQCD_ERR_ARG, "null argument");
    return pack_field(c, p, nsub, canon, native, nrhs, false);
}

lqcd_status lqcd_unpack(lqcd_ctx *c, lqcd_prec p, int nsub, const void *native, void *canon, int nrhs)
{
    if (!c || !canon || !native) return set_err(c, LQCD_ERR_ARG, "null argument");
    return pack_field(c, p, nsub, canon, (void *)native, nrhs, true);
}

lqcd_status lqcd_apply_Dhat_native(lqcd_ctx *c, lqcd_prec p, const void *in, void *out, int nrhs)
{
    if (!c || !in || !out || nrhs < 1) return set_err(c, LQCD_ERR_ARG, "bad argument");
    if (p != LQCD_F64 && p != LQCD_F32 && p != LQCD_F16S) return set_err(c, LQCD_ERR_ARG, "precision %d", (int)p);
    void *tmp;
    LQCD_TRY(ws_get(c, WS_TMP_O, native_half_bytes(c, p) * nrhs, &tmp));
    return dirac_dhat(c, p, in, out, tmp, nrhs);
}

lqcd_status lqcd_apply_D_native(lqcd_ctx *c, lqcd_prec p, const void *in, void *out, int nrhs)
{
    if (!c || !in || !out || nrhs < 1) return set_err(c, LQCD_ERR_ARG, "bad argument");
    if (p != LQCD_F64 && p != LQCD_F32 && p != LQCD_F16S) return set_err(c, LQCD_ERR_ARG, "precision %d", (int)p);
    return dirac_D(c, p, in, out, nrhs);
}

lqcd_status lqcd_apply_Dhat(lqcd_ctx *c, lqcd_prec p, const void *in, void *out, int nrhs)
{
    if (!c || !in || !out || nrhs < 1) return set_err(c, LQCD_ERR_ARG, "bad argument");
    if (p != LQCD_F64 && p != LQCD_F32 && p != LQCD_F16S) return set_err(c, LQCD_ERR_ARG, "precision %d", (int)p);
    size_t hb = native_half_bytes(c, p) * nrhs;
    void *a, *b;
    LQCD_TRY(ws_get(c, WS_PACK_IN, hb, &a));
    LQCD_TRY(ws_get(c, WS_PACK_OUT, hb, &b));
    LQCD_TRY(pack_field(c, p, 1, in, a, nrhs, false));
    LQCD_TRY(lqcd_apply_Dhat_native(c, p, a, b, nrhs));
    return pack_field(c, p, 1, out, b, nrhs, true);
}

lqcd_status lqcd_apply_D(lqcd_ctx *c, lqcd_prec p, const void *in, void *out, int nrhs)
{
    if (!c || !in || !out || nrhs < 1) return set_err(c, LQCD_ERR_ARG, "bad argument");
    if (p != LQCD_F64 && p != LQCD_F32 && p != LQCD_F16S) return set_err(c, LQCD_ERR_ARG, "precision %d", (int)p);
    size_t fb = native_half_bytes(c, p) * 2 * nrhs;
    void *a, *b;
    LQCD_TRY(ws_get(c, WS_PACK_IN, fb, &a));
    LQCD_TRY(ws_get(c, WS_PACK_OUT, fb, &b));
    LQCD_TRY(pack_field(c, p, 2, in, a, nrhs, false));
    LQCD_TRY(dirac_D(c, p, a, b, nrhs));
    return pack_field(c, p, 2, out, b, nrhs, true);
}

}  // extern "C"
