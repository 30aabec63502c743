// Internal declarations of the sm_103a Wilson-clover library: context,
// device-private ("native") layouts, geometry and the chiral-basis spin
// algebra of the hopping term (Eq. 1).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <ctime>
#include <string>
#include <vector>

#include "lqcd.h"

// ------------------------------------------------------------------ complex
template <class R>
struct cx {
    R re, im;
};
template <class R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <class R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R>
__device__ __forceinline__ cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
template <class R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <class R>
__device__ __forceinline__ cx<R> conjx(cx<R> a) { return {a.re, -a.im}; }
template <class R>
__device__ __forceinline__ cx<R> timesI(cx<R> a) { return {-a.im, a.re}; }   // i a
template <class R>
__device__ __forceinline__ cx<R> timesmI(cx<R> a) { return {a.im, -a.re}; }  // -i a
// a * b with a conjugated
template <class R>
__device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> b)
{
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}

// a * b + c with a single rounding
__device__ __forceinline__ float fmx(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return __fma_rn(a, b, c); }

// third row of an SU(3) matrix from the first two, u2 = (u0 x u1)^*, each real
// part one product and three fused multiply-adds
template <class R>
__device__ __forceinline__ void su3_third_row(cx<R> u[3][3])
{
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int k = (j + 1) % 3, l = (j + 2) % 3;
        const cx<R> a = u[0][k], b = u[1][l], c = u[0][l], d = u[1][k];
        // conj(a b - c d)
        R re = a.re * b.re;
        re = fmx(-a.im, b.im, re);
        re = fmx(-c.re, d.re, re);
        re = fmx(c.im, d.im, re);
        R im = -a.re * b.im;
        im = fmx(-a.im, b.re, im);
        im = fmx(c.re, d.im, im);
        im = fmx(c.im, d.re, im);
        u[2][j] = mk(re, im);
    }
}

// ------------------------------------------------------------------ geometry
// Division of a non-negative 31-bit n by an invariant d >= 1 as a multiply-high,
// an add and a shift (Granlund & Montgomery, "Division by invariant integers
// using multiplication", 1994, round-up method): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (mulhi(m, n) + n) >> l exactly for
// 0 <= n < 2^31 (mulhi(m, n) < n, so the sum does not overflow 32 bits).
struct FastDiv {
    unsigned m;
    int l;
};
inline FastDiv make_fastdiv(int d)
{
    int l = 0;
    while ((1u << l) < (unsigned)d) l++;
    const unsigned long long m =
        ((1ull << 32) * ((1ull << l) - (unsigned long long)d)) / (unsigned long long)d + 1;
    return FastDiv{(unsigned)m, l};
}
__device__ __forceinline__ int fast_div(const FastDiv &f, int n)
{
    return (int)((__umulhi(f.m, (unsigned)n) + (unsigned)n) >> f.l);
}

struct Geom {
    int L[4];      // L[0] = T
    int V, Vh;
    int L3h;       // L3 / 2
    int bc_t;      // -1 antiperiodic fermion field in time, +1 periodic
    FastDiv dL3h, dL2, dL1;   // divisions by L3h, L[2], L[1]
};
// fills the derived fields of a geometry from its extents
void geom_init(Geom &g, const int L[4], int bc_t);

// coordinates of the site of parity p and rank r (site = 2r + b)
__device__ __forceinline__ void rank_coords(const Geom &g, int p, int r, int x[4])
{
    const int row = fast_div(g.dL3h, r);
    const int x3h = r - row * g.L3h;
    const int t = fast_div(g.dL2, row);
    x[2] = row - t * g.L[2];
    x[0] = fast_div(g.dL1, t);
    x[1] = t - x[0] * g.L[1];
    const int b = (p + x[0] + x[1] + x[2]) & 1;
    x[3] = 2 * x3h + b;
}
__device__ __forceinline__ int coords_rank(const Geom &g, const int x[4])
{
    return (x[3] + g.L[3] * (x[2] + g.L[2] * (x[1] + g.L[1] * x[0]))) >> 1;
}
// rank of the neighbour x + d*mu (d = +-1), periodic wrap
__device__ __forceinline__ int nbr_rank(const Geom &g, const int x[4], int mu, int d)
{
    int y[4] = {x[0], x[1], x[2], x[3]};
    int v = y[mu] + d;
    y[mu] = v < 0 ? v + g.L[mu] : (v >= g.L[mu] ? v - g.L[mu] : v);
    return coords_rank(g, y);
}

// ------------------------------------------------------------------ context
struct Workspace {
    void *p = nullptr;
    size_t bytes = 0;
};

struct DflState;   // deflation subspace (lqcd_dfl.cu)
struct NetState;   // learned preconditioner (lqcd_ptc.cu)
struct ChronoState;   // stored solutions for initial guesses (lqcd_chrono.cu)

struct lqcd_ctx {
    lqcd_geom geom;
    Geom g;
    cudaStream_t stream = nullptr;
    char err[512] = {0};
    // gauge field, native layouts
    double2 *U64 = nullptr;   // [p][mu][9][Vh]      full SU(3), FP64
    float4 *U32 = nullptr;    // [p][mu][3][Vh]      two rows, FP32
    uint2 *U16 = nullptr;     // [p][mu][3][Vh]      two rows, FP16 (4 halves per uint2)
    bool have_gauge = false;
    // clover term: A and A^-1 for both parities, packed Hermitian 6x6 pairs
    double2 *A64[2] = {nullptr, nullptr}, *Ai64[2] = {nullptr, nullptr};  // [36][Vh]
    float4 *A32[2] = {nullptr, nullptr}, *Ai32[2] = {nullptr, nullptr};   // [18][Vh]
    uint2 *A16[2] = {nullptr, nullptr}, *Ai16[2] = {nullptr, nullptr};    // [18][Vh], FP16
    bool have_clover = false;
    double kappa = 0, csw = 0;
    double logdet_e = 0, logdet_o = 0;   // log|det A| of each parity, from the last clover build
    // device scratch for reductions
    double *red = nullptr;        // partial sums
    double *red_out = nullptr;    // final reduction results (device)
    double *red_host = nullptr;   // pinned host mirror
    // named temporary buffers, grown on demand
    Workspace ws[24];   // indexed by the WS_ slots below
    DflState *dfl = nullptr;
    NetState *net = nullptr;
    ChronoState *chrono = nullptr;
    long n_kernel_launches = 0;
    // LQCD_PROFILE=1: synchronised wall time of solver phases, reported on
    // stderr by the GCR (developer instrumentation; off by default)
    bool prof_on = false;
    double prof_t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double prof_gs_bytes = 0;   // algorithmic bytes of the outer Gram-Schmidt
    long prof_gs_second = 0;    // second Gram-Schmidt passes taken
};

// laps of the LQCD_PROFILE clock: lap(i) adds the time since the previous lap
// (or construction) to c->prof_t[i]; nothing happens when profiling is off
struct ProfClock {
    lqcd_ctx *c;
    double t0 = 0;
    static double wall()
    {
        timespec ts;
        clock_gettime(CLOCK_MONOTONIC, &ts);
        return ts.tv_sec + 1e-9 * ts.tv_nsec;
    }
    explicit ProfClock(lqcd_ctx *ctx) : c(ctx)
    {
        if (!c->prof_on) return;
        cudaStreamSynchronize(c->stream);
        t0 = wall();
    }
    void lap(int i)
    {
        if (!c->prof_on) return;
        cudaStreamSynchronize(c->stream);
        const double t = wall();
        c->prof_t[i] += t - t0;
        t0 = t;
    }
};

// error helpers
lqcd_status set_err(lqcd_ctx *c, lqcd_status s, const char *fmt, ...);
#define LQCD_CUDA_CHECK(ctx, call)                                                          \
    do {                                                                                    \
        cudaError_t e__ = (call);                                                           \
        if (e__ != cudaSuccess)                                                             \
            return set_err(ctx, LQCD_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,   \
                           cudaGetErrorString(e__));                                        \
    } while (0)
#define LQCD_LAUNCH_CHECK(ctx) LQCD_CUDA_CHECK(ctx, cudaGetLastError())
#define LQCD_TRY(expr)                         \
    do {                                       \
        lqcd_status s__ = (expr);              \
        if (s__ != LQCD_OK) return s__;        \
    } while (0)

// workspace slots
enum {
    WS_PACK_IN = 0,
    WS_PACK_OUT,
    WS_TMP_O,       // odd temporaries of Dhat
    WS_SAP_R,
    WS_SAP_PSI,
    WS_SAP_IN,
    WS_SOLVER,      // solver vectors
    WS_DFL,
    WS_CGNR,
    WS_MISC,
    WS_MISC2,
    WS_COARSE,
    WS_SOLVE_IO,
    WS_NET_PART,
    WS_NET_ACT,
    WS_NET_TGT,
    WS_NET_BATCH_T,
    WS_NET_FALLBACK,
    WS_HASEN,
    WS_PHI64,       // F64 preconditioner output converted into FP32 Krylov vectors
    WS_MD_OMEGA,    // per-site clover force weights (MD forces)
    WS_MD_SCRATCH,  // per-site partial sums (gauge action)
    WS_MD_FIELDS,   // pseudofermion force fields
    WS_MD_GRAD,     // MD gradient of the leapfrog step
};
lqcd_status ws_get(lqcd_ctx *c, int slot, size_t bytes, void **out);

// native element counts per site
inline int native_chunks(lqcd_prec p) { return p == LQCD_F64 ? 12 : (p == LQCD_F32 ? 6 : 3); }
inline size_t native_chunk_bytes(lqcd_prec p) { return p == LQCD_F64 ? 16 : (p == LQCD_F32 ? 16 : 16); }
size_t native_half_bytes(const lqcd_ctx *c, lqcd_prec p);   // one rhs, one parity

// launch helpers
inline int div_up(long a, long b) { return (int)((a + b - 1) / b); }

// --------------------------------------------------------------- internals
// dirac
lqcd_status dirac_dhat(lqcd_ctx *c, lqcd_prec p, const void *in, void *out, void *tmp_o, int nrhs);
lqcd_status dirac_D(lqcd_ctx *c, lqcd_prec p, const void *in, void *out, int nrhs);
lqcd_status dirac_hop_parity(lqcd_ctx *c, lqcd_prec p, int p_out, const void *in_other,
                             void *out, long in_rstride, long out_rstride, int nrhs);
lqcd_status convert_native(lqcd_ctx *c, lqcd_prec from, lqcd_prec to, const void *in, void *out,
                           long nhalf);
lqcd_status pack_field(lqcd_ctx *c, lqcd_prec p, int nsub, const void *canon, void *native,
                       int nrhs, bool unpack);
// even_scale != 1: the even-site blocks of A (and so of A^-1) belong to
// even_scale * A_ee (the shifted operator of the Hasenbusch solve)
lqcd_status clover_build(lqcd_ctx *c, double kappa, double csw, double *ld_e, double *ld_o, double even_scale = 1.0);
lqcd_status clover_apply_native64(lqcd_ctx *c, int parity, int inverse, const double2 *in,
                                  double2 *out);

// blas (FP64 native vectors viewed as arrays of double; complex pairs)
lqcd_status blas_dot(lqcd_ctx *c, long n2, const double *a, const double *b, int k, long stride_a,
                     double *host_out);  // k dots <a_i, b>, host_out: 2k doubles
lqcd_status blas_norm2(lqcd_ctx *c, long n2, const double *a, double *host_out);
lqcd_status blas_axpy(lqcd_ctx *c, long n2, double ar, double ai, const double *x, double *y);
lqcd_status blas_xpay(lqcd_ctx *c, long n2, const double *x, double ar, double *y);  // y = x + a y
lqcd_status blas_scal(lqcd_ctx *c, long n2, double ar, double ai, double *y);
lqcd_status blas_copy(lqcd_ctx *c, long n2, const double *x, double *y);
lqcd_status blas_sub(lqcd_ctx *c, long n2, const double *x, const double *y, double *z);  // z = x - y
lqcd_status blas_multi_axpy(lqcd_ctx *c, long n2, int k, const double *coef_host, const double *X,
                            long stride, double *y, double sign);
lqcd_status bblas_dot(lqcd_ctx *c, long n2, int nrhs, const double *A, long sa, long fa, const double *B, long fb,
                      int k, double *host_out);
lqcd_status bblas_multi_axpy(lqcd_ctx *c, long n2, int nrhs, int k, const double *coef_host, const double *X,
                             long sa, long fa, double *y, long fy, double sign);
lqcd_status bblas_dot_dev(lqcd_ctx *c, long n2, int nrhs, const double *A, long sa, long fa, const double *B, long fb,
                          int k, double2 *out_dev);
lqcd_status bblas_multi_axpy_dev(lqcd_ctx *c, long n2, int nrhs, int k, const double2 *coef_dev, const double *X,
                                 long sa, long fa, double *y, long fy, double sign);
// GCR with FP32 Krylov vectors: x, A, B, X, y are native F32 full fields
// (float4, strides in float4), rho and psi native F64 full fields (double2,
// strides in double2); dots land on the host as (re, im) pairs [r][i]
lqcd_status bdot32(lqcd_ctx *c, long n4, int nrhs, const float4 *A, long sa, long fa, const float4 *B, long fb, int k,
                   double *host_out);
lqcd_status bnorm_rdot32(lqcd_ctx *c, int nrhs, const float4 *x, long fx, const double2 *rho, long fr,
                         double *host_out);   // [r][0] = |x_r|^2, [r][1] = <rho_r, x_r>
lqcd_status bmulti_axpy32(lqcd_ctx *c, long n4, int nrhs, int k, const double *coef_host, const float4 *X, long sa,
                          long fa, float4 *y, long fy, double sign);
lqcd_status brho_update32(lqcd_ctx *c, int nrhs, const double *cR_host, const double *sx_host, float4 *x, long fx,
                          double2 *rho, long fr);   // rho_r -= cR_r x_r; x_r *= sx_r
lqcd_status bmulti_axpy_mixed(lqcd_ctx *c, int nrhs, int k, const double *coef_host, const float4 *X, long sa,
                              long fa, double2 *y, long fy);   // y_r += sum_i c_ri X_ir
lqcd_status blas_gamma5_native64(lqcd_ctx *c, long nhalf, const double2 *in, double2 *out);
lqcd_status blas_zero(lqcd_ctx *c, size_t bytes, void *p);

// sap
lqcd_status sap_axpby_native(lqcd_ctx *c, lqcd_prec p, const void *eta, void *r);
void sap_free_plans(lqcd_ctx *c);
lqcd_status sap_apply(lqcd_ctx *c, const lqcd_sap_params *sp, const void *eta_native,
                      void *psi_native, int nrhs = 1);
// batched operators over several lattices; hc: the batch's own context (stream,
// error text, launch counter); arenas hold the lattices' native full fields at
// offsets off[l] (in native spinor units of the precision)
struct DBatch;
lqcd_status dirac_batch_create(lqcd_ctx *hc, lqcd_ctx *const *ctx, int n, lqcd_prec p, const void *in, void *out,
                               const long *off, DBatch **out_b);
lqcd_status dirac_batch_D(lqcd_ctx *hc, DBatch *b, const int *active_dev);
void dirac_batch_free(DBatch *b);
struct SapBatch;
lqcd_status sap_batch_create(lqcd_ctx *hc, lqcd_ctx *const *ctx, int n, const lqcd_sap_params *sp, void *r,
                             void *psi, void *delta, const long *off, SapBatch **out_b);
lqcd_status sap_batch_apply(lqcd_ctx *hc, SapBatch *b, const void *eta, size_t bytes, const int *active_dev);
void sap_batch_free(SapBatch *b);
void chrono_free(lqcd_ctx *c);
// learned preconditioner
void net_free(lqcd_ctx *c);
lqcd_status net_apply_native(lqcd_ctx *c, const double2 *rho, double2 *phi, int nrhs);
// deflation
void dfl_free(lqcd_ctx *c);
// smoother: SAP (net = false) or the network (net = true) after the deflation step
lqcd_status dfl_precond_native(lqcd_ctx *c, const lqcd_sap_params *sp, const double2 *rho,
                               double2 *phi, int nrhs, bool net = false);
