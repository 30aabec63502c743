// FP64 BLAS-1 on complex vectors (arrays of re,im doubles) for the outer
// solvers: batched dot products with a fixed reduction order (results are
// bitwise reproducible run to run), axpy forms, gamma5.
#include <algorithm>

#include "lqcd_internal.cuh"

namespace {

constexpr int RED_THREADS = 256;
constexpr int DOT_CHUNK = 8;

__global__ void k_axpy(long n, double ar, double ai, const double2 *__restrict__ x, double2 *y)
{
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        double2 a = x[j], b = y[j];
        b.x += ar * a.x - ai * a.y;
        b.y += ar * a.y + ai * a.x;
        y[j] = b;
    }
}
__global__ void k_xpay(long n, const double2 *__restrict__ x, double ar, double2 *y)
{
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        double2 a = x[j], b = y[j];
        y[j] = make_double2(a.x + ar * b.x, a.y + ar * b.y);
    }
}
__global__ void k_scal(long n, double ar, double ai, double2 *y)
{
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        double2 b = y[j];
        y[j] = make_double2(ar * b.x - ai * b.y, ar * b.y + ai * b.x);
    }
}
__global__ void k_sub(long n, const double2 *__restrict__ x, const double2 *__restrict__ y, double2 *z)
{
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        double2 a = x[j], b = y[j];
        z[j] = make_double2(a.x - b.x, a.y - b.y);
    }
}
// y += sign * sum_i c_i X_i  (c complex, up to 64 terms)
struct Coefs {
    double c[2 * 64];
};
__global__ void k_multi_axpy(long n, int k, Coefs cf, const double2 *__restrict__ X, long stride, double2 *y,
                             double sign)
{
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        double2 b = y[j];
        double sr = 0, si = 0;
        for (int i = 0; i < k; i++) {
            double2 a = X[i * stride + j];
            sr += cf.c[2 * i] * a.x - cf.c[2 * i + 1] * a.y;
            si += cf.c[2 * i] * a.y + cf.c[2 * i + 1] * a.x;
        }
        y[j] = make_double2(b.x + sign * sr, b.y + sign * si);
    }
}
// gamma5 = diag(1,1,-1,-1): negate spins 2,3 = complex components 6..11
__global__ void k_gamma5_64(long Vh, long nhalf, const double2 *__restrict__ in, double2 *out)
{
    long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
    long h = blockIdx.y;
    if (r >= Vh || h >= nhalf) return;
    const double2 *i = in + h * 12 * Vh + r;
    double2 *o = out + h * 12 * Vh + r;
    for (int c = 0; c < 12; c++) {
        double2 v = i[c * Vh];
        o[c * Vh] = c < 6 ? v : make_double2(-v.x, -v.y);
    }
}

inline int grid_for(long n) { return (int)std::min<long>(4 * 152, (n + 255) / 256); }

// ---------------------------------------------------------------- batched
// partial[(r*nb + b)*64 + i] = block b's share of <A_{i,r}, B_r>
__global__ void __launch_bounds__(RED_THREADS) k_bdot_partial(long n, const double2 *__restrict__ A, long sa,
                                                              long fa, const double2 *__restrict__ B, long fb,
                                                              int k0, int kn, double2 *partial)
{
    const int r = blockIdx.y;
    const double2 *Br = B + r * fb;
    const double2 *Ar = A + r * fa;
    double re[DOT_CHUNK], im[DOT_CHUNK];
#pragma unroll
    for (int i = 0; i < DOT_CHUNK; i++) re[i] = im[i] = 0;
    const long st = (long)gridDim.x * blockDim.x;
    long j = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (kn <= 2) {
        // few vectors: four grid-strided elements per pass, their loads issued
        // together (one element per pass leaves too few loads in flight to
        // cover the memory latency)
        for (; j + 3 * st < n; j += 4 * st) {
            double2 b[4], a0[4], a1[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                b[u] = Br[j + u * st];
                a0[u] = Ar[k0 * sa + j + u * st];
                if (kn == 2) a1[u] = Ar[(k0 + 1) * sa + j + u * st];
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                re[0] += a0[u].x * b[u].x + a0[u].y * b[u].y;
                im[0] += a0[u].x * b[u].y - a0[u].y * b[u].x;
                if (kn == 2) {
                    re[1] += a1[u].x * b[u].x + a1[u].y * b[u].y;
                    im[1] += a1[u].x * b[u].y - a1[u].y * b[u].x;
                }
            }
        }
    }
    for (; j < n; j += st) {
        double2 b = Br[j];
#pragma unroll
        for (int i = 0; i < DOT_CHUNK; i++)
            if (i < kn) {
                double2 a = Ar[(k0 + i) * sa + j];
                re[i] += a.x * b.x + a.y * b.y;
                im[i] += a.x * b.y - a.y * b.x;
            }
    }
    __shared__ double sh[RED_THREADS / 32][DOT_CHUNK][2];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < DOT_CHUNK; i++) {
        double x = re[i], m = im[i];
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            m += __shfl_down_sync(0xffffffffu, m, o);
        }
        if (lane == 0) {
            sh[warp][i][0] = x;
            sh[warp][i][1] = m;
        }
    }
    __syncthreads();
    if (threadIdx.x < kn) {
        double x = 0, m = 0;
        for (int w = 0; w < RED_THREADS / 32; w++) {
            x += sh[w][threadIdx.x][0];
            m += sh[w][threadIdx.x][1];
        }
        partial[((long)r * gridDim.x + blockIdx.x) * 64 + k0 + threadIdx.x] = make_double2(x, m);
    }
}
// one CTA per (vector i, rhs r): fixed-order tree over the nb partial sums
__global__ void k_bdot_final(int nb, int k, const double2 *partial, double2 *out)
{
    const int i = blockIdx.x, r = blockIdx.y;
    __shared__ double sx[256], sm[256];
    double x = 0, m = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        double2 v = partial[((long)r * nb + b) * 64 + i];
        x += v.x;
        m += v.y;
    }
    sx[threadIdx.x] = x;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sx[threadIdx.x] += sx[threadIdx.x + s];
            sm[threadIdx.x] += sm[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[r * k + i] = make_double2(sx[0], sm[0]);
}
// coefficients passed by value (16 KB of launch parameters)
struct CoefParam {
    static constexpr int N = 1024;
    double2 c[N];
};

// y_r += sign * sum_i c[r*k + i] X_{i,r}
__global__ void k_bmulti_axpy(long n, int k, const __grid_constant__ CoefParam cf, const double2 *__restrict__ X,
                              long sa, long fa, double2 *y, long fy, double sign)
{
    const int r = blockIdx.y;
    const double2 *c = cf.c + r * k;
    const double2 *Xr = X + r * fa;
    double2 *yr = y + r * fy;
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        double2 b = yr[j];
        double sr = 0, si = 0;
        for (int i = 0; i < k; i++) {
            double2 a = Xr[i * sa + j], ci = c[i];
            sr += ci.x * a.x - ci.y * a.y;
            si += ci.x * a.y + ci.y * a.x;
        }
        yr[j] = make_double2(b.x + sign * sr, b.y + sign * si);
    }
}

// y_r += sign * sum_i cf[r*k + i] X_{i,r} with the coefficients in device memory
__global__ void k_bmulti_axpy_dev(long n, int k, const double2 *__restrict__ cf, const double2 *__restrict__ X,
                                  long sa, long fa, double2 *y, long fy, double sign)
{
    const int r = blockIdx.y;
    const double2 *c = cf + r * k;
    const double2 *Xr = X + r * fa;
    double2 *yr = y + r * fy;
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        double2 b = yr[j];
        double sr = 0, si = 0;
        for (int i = 0; i < k; i++) {
            double2 a = Xr[i * sa + j], ci = c[i];
            sr += ci.x * a.x - ci.y * a.y;
            si += ci.x * a.y + ci.y * a.x;
        }
        yr[j] = make_double2(b.x + sign * sr, b.y + sign * si);
    }
}

// ---------------------------------------------------------------- FP32 Krylov
// Batched kernels of the GCR with FP32 Krylov vectors (native F32 full fields,
// float4 = two complex components).  Products are formed in float; each
// thread folds its float sums into double every FOLD elements, and the
// per-CTA and final sums are double in a fixed order.
constexpr int FOLD = 16;
constexpr int DOT32_K = 9;

// partial[(r*nb + b)*64 + k0 + i] = block b's share of <A_{k0+i,r}, B_r>
__global__ void __launch_bounds__(RED_THREADS) k_bdot32_partial(long n, const float4 *__restrict__ A, long sa,
                                                                long fa, const float4 *__restrict__ B, long fb,
                                                                int k0, int kn, double2 *partial)
{
    const int r = blockIdx.y;
    const float4 *Br = B + r * fb;
    const float4 *Ar = A + r * fa + k0 * sa;
    double dre[DOT32_K], dim[DOT32_K];
    float re[DOT32_K], im[DOT32_K];
#pragma unroll
    for (int i = 0; i < DOT32_K; i++) dre[i] = dim[i] = re[i] = im[i] = 0;
    int cnt = 0;
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        const float4 b = Br[j];
#pragma unroll
        for (int i = 0; i < DOT32_K; i++)
            if (i < kn) {
                const float4 a = Ar[i * sa + j];
                re[i] += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
                im[i] += a.x * b.y - a.y * b.x + a.z * b.w - a.w * b.z;
            }
        if (++cnt == FOLD) {
            cnt = 0;
#pragma unroll
            for (int i = 0; i < DOT32_K; i++) {
                dre[i] += re[i];
                dim[i] += im[i];
                re[i] = im[i] = 0;
            }
        }
    }
    __shared__ double sh[RED_THREADS / 32][DOT32_K][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < DOT32_K; i++) {
        double x = dre[i] + re[i], m = dim[i] + im[i];
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            m += __shfl_down_sync(0xffffffffu, m, o);
        }
        if (lane == 0) {
            sh[warp][i][0] = x;
            sh[warp][i][1] = m;
        }
    }
    __syncthreads();
    if (threadIdx.x < kn) {
        double x = 0, m = 0;
        for (int w = 0; w < RED_THREADS / 32; w++) {
            x += sh[w][threadIdx.x][0];
            m += sh[w][threadIdx.x][1];
        }
        partial[((long)r * gridDim.x + blockIdx.x) * 64 + k0 + threadIdx.x] = make_double2(x, m);
    }
}

// |x_r|^2 and <rho_r, x_r> (x: F32 full fields, rho: F64 full fields) as the two
// partial sums partial[(r*nb + b)*64 + {0, 1}]; site r of half h, float4 q of x
// holds the complex components 2q, 2q+1 of rho
__global__ void __launch_bounds__(RED_THREADS) k_norm_rdot32_partial(long Vh, const float4 *__restrict__ X, long fx,
                                                                     const double2 *__restrict__ R, long fr,
                                                                     double2 *partial)
{
    const int rh = blockIdx.y;
    const float4 *Xr = X + rh * fx;
    const double2 *Rr = R + rh * fr;
    double nn = 0, dre = 0, dim = 0;
    for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < Vh; s += (long)gridDim.x * blockDim.x) {
        float fn = 0, fre = 0, fim = 0;
#pragma unroll
        for (int p = 0; p < 12; p++) {
            const float4 a = Xr[p * Vh + s];
            const double2 u = Rr[(2 * p) * Vh + s], v = Rr[(2 * p + 1) * Vh + s];
            fn += a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
            const float ux = (float)u.x, uy = (float)u.y, vx = (float)v.x, vy = (float)v.y;
            fre += ux * a.x + uy * a.y + vx * a.z + vy * a.w;
            fim += ux * a.y - uy * a.x + vx * a.w - vy * a.z;
        }
        nn += fn;
        dre += fre;
        dim += fim;
    }
    __shared__ double sh[RED_THREADS / 32][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        nn += __shfl_down_sync(0xffffffffu, nn, o);
        dre += __shfl_down_sync(0xffffffffu, dre, o);
        dim += __shfl_down_sync(0xffffffffu, dim, o);
    }
    if (lane == 0) {
        sh[warp][0] = nn;
        sh[warp][1] = dre;
        sh[warp][2] = dim;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int w = 0; w < RED_THREADS / 32; w++) {
            a += sh[w][0];
            b += sh[w][1];
            c += sh[w][2];
        }
        double2 *o = partial + ((long)rh * gridDim.x + blockIdx.x) * 64;
        o[0] = make_double2(a, 0);
        o[1] = make_double2(b, c);
    }
}

// y_r += sign * sum_i c[r*k + i] X_{i,r}, all F32 (coefficients by value)
__global__ void k_bmulti_axpy32(long n, int k, const __grid_constant__ CoefParam cf, const float4 *__restrict__ X,
                                long sa, long fa, float4 *y, long fy, float sign)
{
    const int r = blockIdx.y;
    const float4 *Xr = X + r * fa;
    float4 *yr = y + r * fy;
    // coefficients converted to float once per CTA (not per element on the FP64 pipe)
    __shared__ float2 c[64];
    for (int i = threadIdx.x; i < k; i += blockDim.x)
        c[i] = make_float2((float)cf.c[r * k + i].x, (float)cf.c[r * k + i].y);
    __syncthreads();
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        float4 b = yr[j];
        float s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        int i = 0;
        for (; i + 4 <= k; i += 4) {
            float4 a[4];
#pragma unroll
            for (int u = 0; u < 4; u++) a[u] = Xr[(i + u) * sa + j];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const float cr = c[i + u].x, ci = c[i + u].y;
                s0 += cr * a[u].x - ci * a[u].y;
                s1 += cr * a[u].y + ci * a[u].x;
                s2 += cr * a[u].z - ci * a[u].w;
                s3 += cr * a[u].w + ci * a[u].z;
            }
        }
        for (; i < k; i++) {
            const float4 a = Xr[i * sa + j];
            const float cr = c[i].x, ci = c[i].y;
            s0 += cr * a.x - ci * a.y;
            s1 += cr * a.y + ci * a.x;
            s2 += cr * a.z - ci * a.w;
            s3 += cr * a.w + ci * a.z;
        }
        yr[j] = make_float4(b.x + sign * s0, b.y + sign * s1, b.z + sign * s2, b.w + sign * s3);
    }
}

// rho_r -= cR_r x_r (rho F64, x F32; the product in float), then x_r *= sx_r
struct RhoScale {
    double2 cR[64];
    float sx[64];
};
__global__ void k_rho_update32(long Vh, const __grid_constant__ RhoScale cf, float4 *X, long fx, double2 *R, long fr)
{
    const int rh = blockIdx.y;
    float4 *Xr = X + rh * fx;
    double2 *Rr = R + rh * fr;
    const float cr = (float)cf.cR[rh].x, ci = (float)cf.cR[rh].y, sx = cf.sx[rh];
    for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < Vh; s += (long)gridDim.x * blockDim.x) {
#pragma unroll 4
        for (int p = 0; p < 12; p++) {
            const float4 a = Xr[p * Vh + s];
            double2 u = Rr[(2 * p) * Vh + s], v = Rr[(2 * p + 1) * Vh + s];
            u.x -= (double)(cr * a.x - ci * a.y);
            u.y -= (double)(cr * a.y + ci * a.x);
            v.x -= (double)(cr * a.z - ci * a.w);
            v.y -= (double)(cr * a.w + ci * a.z);
            Rr[(2 * p) * Vh + s] = u;
            Rr[(2 * p + 1) * Vh + s] = v;
            Xr[p * Vh + s] = make_float4(sx * a.x, sx * a.y, sx * a.z, sx * a.w);
        }
    }
}

// psi_r += sum_i c[r*k + i] X_{i,r} (X F32 full fields, psi F64; the sum in float)
__global__ void k_bmulti_axpy_mixed(long Vh, int k, const __grid_constant__ CoefParam cf,
                                    const float4 *__restrict__ X, long sa, long fa, double2 *y, long fy)
{
    const int rh = blockIdx.y;
    const float4 *Xr = X + rh * fa;
    double2 *yr = y + rh * fy;
    __shared__ float2 c[64];
    for (int i = threadIdx.x; i < k; i += blockDim.x)
        c[i] = make_float2((float)cf.c[rh * k + i].x, (float)cf.c[rh * k + i].y);
    __syncthreads();
    for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < Vh; s += (long)gridDim.x * blockDim.x) {
        for (int p = 0; p < 12; p++) {
            float s0 = 0, s1 = 0, s2 = 0, s3 = 0;
            for (int i = 0; i < k; i++) {
                const float4 a = Xr[i * sa + p * Vh + s];
                const float cr = c[i].x, ci = c[i].y;
                s0 += cr * a.x - ci * a.y;
                s1 += cr * a.y + ci * a.x;
                s2 += cr * a.z - ci * a.w;
                s3 += cr * a.w + ci * a.z;
            }
            double2 u = yr[(2 * p) * Vh + s], v = yr[(2 * p + 1) * Vh + s];
            yr[(2 * p) * Vh + s] = make_double2(u.x + s0, u.y + s1);
            yr[(2 * p + 1) * Vh + s] = make_double2(v.x + s2, v.y + s3);
        }
    }
}

}  // namespace

// as bblas_dot, results left in device memory: out_dev[r*k + i] (complex)
lqcd_status bblas_dot_dev(lqcd_ctx *c, long n2, int nrhs, const double *A, long sa, long fa, const double *B, long fb,
                          int k, double2 *out_dev)
{
    if (k < 1 || k > 64 || nrhs < 1 || nrhs * k > 2048) return set_err(c, LQCD_ERR_ARG, "bblas_dot_dev k=%d", k);
    long n = n2 / 2;
    // about 4 CTAs per SM over the batch, but no more than one CTA per 256 elements
    int nb = std::max(1, (int)std::min<long>(std::max(8, 4 * 152 / nrhs), (n + 255) / 256));
    nb = std::min(nb, 4096 / nrhs);
    double2 *partial = (double2 *)c->red;
    for (int k0 = 0; k0 < k; k0 += DOT_CHUNK) {
        int kn = std::min(DOT_CHUNK, k - k0);
        k_bdot_partial<<<dim3(nb, nrhs), RED_THREADS, 0, c->stream>>>(n, (const double2 *)A, sa / 2, fa / 2,
                                                                      (const double2 *)B, fb / 2, k0, kn, partial);
        c->n_kernel_launches++;
    }
    k_bdot_final<<<dim3(k, nrhs), 256, 0, c->stream>>>(nb, k, partial, out_dev);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

lqcd_status bblas_multi_axpy_dev(lqcd_ctx *c, long n2, int nrhs, int k, const double2 *coef_dev, const double *X,
                                 long sa, long fa, double *y, long fy, double sign)
{
    if (k < 1) return LQCD_OK;
    long n = n2 / 2;
    dim3 grid(std::max(1, grid_for(n) / std::max(1, nrhs / 2)), nrhs);
    k_bmulti_axpy_dev<<<grid, 256, 0, c->stream>>>(n, k, coef_dev, (const double2 *)X, sa / 2, fa / 2, (double2 *)y,
                                                   fy / 2, sign);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

// dots[r][i] = <A + i*sa + r*fa, B + r*fb> for i < k, r < nrhs (lengths and strides in doubles)
lqcd_status bblas_dot(lqcd_ctx *c, long n2, int nrhs, const double *A, long sa, long fa, const double *B, long fb,
                      int k, double *host_out)
{
    if (k < 1 || k > 64 || nrhs < 1 || nrhs * k > 2048) return set_err(c, LQCD_ERR_ARG, "bblas_dot k=%d", k);
    long n = n2 / 2;
    // about 4 CTAs per SM over the batch, but no more than one CTA per 256 elements
    int nb = std::max(1, (int)std::min<long>(std::max(8, 4 * 152 / nrhs), (n + 255) / 256));
    nb = std::min(nb, 4096 / nrhs);
    double2 *partial = (double2 *)c->red;   // nrhs * nb * 64 double2 <= 4096 * 64 (sized at create)
    for (int k0 = 0; k0 < k; k0 += DOT_CHUNK) {
        int kn = std::min(DOT_CHUNK, k - k0);
        k_bdot_partial<<<dim3(nb, nrhs), RED_THREADS, 0, c->stream>>>(n, (const double2 *)A, sa / 2, fa / 2,
                                                                      (const double2 *)B, fb / 2, k0, kn, partial);
        c->n_kernel_launches++;
    }
    k_bdot_final<<<dim3(k, nrhs), 256, 0, c->stream>>>(nb, k, partial, (double2 *)c->red_out);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(c->red_host, c->red_out, 2 * (size_t)k * nrhs * sizeof(double),
                                       cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 2 * k * nrhs; i++) host_out[i] = c->red_host[i];
    return LQCD_OK;
}

// y_r += sign * sum_i coef[r][i] X_{i,r}; coef: host, nrhs*k complex
lqcd_status bblas_multi_axpy(lqcd_ctx *c, long n2, int nrhs, int k, const double *coef_host, const double *X,
                             long sa, long fa, double *y, long fy, double sign)
{
    if (k < 1) return LQCD_OK;
    if (k > 64 || nrhs * k > CoefParam::N) return set_err(c, LQCD_ERR_ARG, "bblas_multi_axpy k=%d", k);
    // the coefficients travel by value in the launch parameters: no staging
    // buffer, no host synchronisation
    CoefParam cp;
    for (int i = 0; i < k * nrhs; i++) cp.c[i] = make_double2(coef_host[2 * i], coef_host[2 * i + 1]);
    long n = n2 / 2;
    dim3 grid(std::max(1, grid_for(n) / std::max(1, nrhs / 2)), nrhs);
    k_bmulti_axpy<<<grid, 256, 0, c->stream>>>(n, k, cp, (const double2 *)X, sa / 2, fa / 2, (double2 *)y, fy / 2,
                                               sign);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

lqcd_status blas_dot(lqcd_ctx *c, long n2, const double *A, const double *B, int k, long stride_a,
                     double *host_out)
{
    if (k < 1 || k > 64) return set_err(c, LQCD_ERR_ARG, "blas_dot: k=%d", k);
    return bblas_dot(c, n2, 1, A, stride_a, 0, B, 0, k, host_out);
}

lqcd_status blas_norm2(lqcd_ctx *c, long n2, const double *a, double *host_out)
{
    double t[2];
    LQCD_TRY(blas_dot(c, n2, a, a, 1, 0, t));
    *host_out = t[0];
    return LQCD_OK;
}

lqcd_status blas_axpy(lqcd_ctx *c, long n2, double ar, double ai, const double *x, double *y)
{
    long n = n2 / 2;
    k_axpy<<<grid_for(n), 256, 0, c->stream>>>(n, ar, ai, (const double2 *)x, (double2 *)y);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}
lqcd_status blas_xpay(lqcd_ctx *c, long n2, const double *x, double ar, double *y)
{
    long n = n2 / 2;
    k_xpay<<<grid_for(n), 256, 0, c->stream>>>(n, (const double2 *)x, ar, (double2 *)y);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}
lqcd_status blas_scal(lqcd_ctx *c, long n2, double ar, double ai, double *y)
{
    long n = n2 / 2;
    k_scal<<<grid_for(n), 256, 0, c->stream>>>(n, ar, ai, (double2 *)y);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}
lqcd_status blas_sub(lqcd_ctx *c, long n2, const double *x, const double *y, double *z)
{
    long n = n2 / 2;
    k_sub<<<grid_for(n), 256, 0, c->stream>>>(n, (const double2 *)x, (const double2 *)y, (double2 *)z);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}
lqcd_status blas_copy(lqcd_ctx *c, long n2, const double *x, double *y)
{
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(y, x, n2 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    return LQCD_OK;
}
lqcd_status blas_zero(lqcd_ctx *c, size_t bytes, void *p)
{
    LQCD_CUDA_CHECK(c, cudaMemsetAsync(p, 0, bytes, c->stream));
    return LQCD_OK;
}
lqcd_status blas_multi_axpy(lqcd_ctx *c, long n2, int k, const double *coef_host, const double *X, long stride,
                            double *y, double sign)
{
    if (k < 1) return LQCD_OK;
    if (k > 64) return set_err(c, LQCD_ERR_ARG, "multi_axpy: k=%d", k);
    Coefs cf;
    for (int i = 0; i < 2 * k; i++) cf.c[i] = coef_host[i];
    long n = n2 / 2;
    k_multi_axpy<<<grid_for(n), 256, 0, c->stream>>>(n, k, cf, (const double2 *)X, stride / 2, (double2 *)y,
                                                     sign);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}
lqcd_status blas_gamma5_native64(lqcd_ctx *c, long nhalf, const double2 *in, double2 *out)
{
    dim3 grid(div_up(c->g.Vh, 256), (unsigned)nhalf);
    k_gamma5_64<<<grid, 256, 0, c->stream>>>(c->g.Vh, nhalf, in, out);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

// ---------------------------------------------------------------- FP32 Krylov
namespace {
int red_blocks(long n, int nrhs)
{
    int nb = std::max(1, (int)std::min<long>(std::max(8, 4 * 152 / nrhs), (n + 255) / 256));
    return std::min(nb, 4096 / nrhs);
}
lqcd_status finish_dots(lqcd_ctx *c, int nb, int nrhs, int k, double *host_out)
{
    k_bdot_final<<<dim3(k, nrhs), 256, 0, c->stream>>>(nb, k, (const double2 *)c->red, (double2 *)c->red_out);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    LQCD_CUDA_CHECK(c, cudaMemcpyAsync(c->red_host, c->red_out, 2 * (size_t)k * nrhs * sizeof(double),
                                       cudaMemcpyDeviceToHost, c->stream));
    LQCD_CUDA_CHECK(c, cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 2 * k * nrhs; i++) host_out[i] = c->red_host[i];
    return LQCD_OK;
}
}  // namespace

lqcd_status bdot32(lqcd_ctx *c, long n4, int nrhs, const float4 *A, long sa, long fa, const float4 *B, long fb, int k,
                   double *host_out)
{
    if (k < 1 || k > 64 || nrhs < 1 || nrhs * k > 2048) return set_err(c, LQCD_ERR_ARG, "bdot32 k=%d", k);
    const int nb = red_blocks(n4, nrhs);
    for (int k0 = 0; k0 < k; k0 += DOT32_K) {
        const int kn = std::min(DOT32_K, k - k0);
        k_bdot32_partial<<<dim3(nb, nrhs), RED_THREADS, 0, c->stream>>>(n4, A, sa, fa, B, fb, k0, kn,
                                                                        (double2 *)c->red);
        c->n_kernel_launches++;
    }
    return finish_dots(c, nb, nrhs, k, host_out);
}

lqcd_status bnorm_rdot32(lqcd_ctx *c, int nrhs, const float4 *x, long fx, const double2 *rho, long fr,
                         double *host_out)
{
    if (nrhs < 1 || nrhs > 1024) return set_err(c, LQCD_ERR_ARG, "bnorm_rdot32 nrhs=%d", nrhs);
    const long Vh = c->g.Vh;
    const int nb = red_blocks(Vh, nrhs);
    k_norm_rdot32_partial<<<dim3(nb, nrhs), RED_THREADS, 0, c->stream>>>(Vh, x, fx, rho, fr, (double2 *)c->red);
    c->n_kernel_launches++;
    return finish_dots(c, nb, nrhs, 2, host_out);
}

lqcd_status bmulti_axpy32(lqcd_ctx *c, long n4, int nrhs, int k, const double *coef_host, const float4 *X, long sa,
                          long fa, float4 *y, long fy, double sign)
{
    if (k < 1) return LQCD_OK;
    if (k > 64 || nrhs * k > CoefParam::N) return set_err(c, LQCD_ERR_ARG, "bmulti_axpy32 k=%d", k);
    CoefParam cp;
    for (int i = 0; i < k * nrhs; i++) cp.c[i] = make_double2(coef_host[2 * i], coef_host[2 * i + 1]);
    dim3 grid(std::max(1, grid_for(n4) / std::max(1, nrhs / 2)), nrhs);
    k_bmulti_axpy32<<<grid, 256, 0, c->stream>>>(n4, k, cp, X, sa, fa, y, fy, (float)sign);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

lqcd_status brho_update32(lqcd_ctx *c, int nrhs, const double *cR_host, const double *sx_host, float4 *x, long fx,
                          double2 *rho, long fr)
{
    if (nrhs < 1 || nrhs > 64) return set_err(c, LQCD_ERR_ARG, "brho_update32 nrhs=%d", nrhs);
    RhoScale cp;
    for (int r = 0; r < nrhs; r++) {
        cp.cR[r] = make_double2(cR_host[2 * r], cR_host[2 * r + 1]);
        cp.sx[r] = (float)sx_host[r];
    }
    const long Vh = c->g.Vh;
    dim3 grid(std::max(1, grid_for(Vh) / std::max(1, nrhs / 2)), nrhs);
    k_rho_update32<<<grid, 256, 0, c->stream>>>(Vh, cp, x, fx, rho, fr);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}

lqcd_status bmulti_axpy_mixed(lqcd_ctx *c, int nrhs, int k, const double *coef_host, const float4 *X, long sa,
                              long fa, double2 *y, long fy)
{
    if (k < 1) return LQCD_OK;
    if (k > 64 || nrhs * k > CoefParam::N) return set_err(c, LQCD_ERR_ARG, "bmulti_axpy_mixed k=%d", k);
    CoefParam cp;
    for (int i = 0; i < k * nrhs; i++) cp.c[i] = make_double2(coef_host[2 * i], coef_host[2 * i + 1]);
    const long Vh = c->g.Vh;
    dim3 grid(std::max(1, grid_for(Vh) / std::max(1, nrhs / 2)), nrhs);
    k_bmulti_axpy_mixed<<<grid, 256, 0, c->stream>>>(Vh, k, cp, X, sa, fa, y, fy);
    c->n_kernel_launches++;
    LQCD_LAUNCH_CHECK(c);
    return LQCD_OK;
}
