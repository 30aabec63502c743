// Native FP16 storage with one FP32 scale per site (LQCD_F16S), and the FP16
// link and clover copies read by the F16S kernels.  Arithmetic stays FP32.
//
// Spinor half field (one parity, one right-hand side), 52 bytes per site:
//   uint4 q[3][Vh]   8 halves = 4 complex components each, canonical
//                    spin-colour order (q = 0: components 0..3, ...)
//   float s[Vh]      per-site scale = largest |real part| of the site's 24 reals
// The stored value is half * s, so every stored half lies in [-1, 1] and the
// rounding error of a site is relative to its own magnitude.
// Links: first two rows in FP16, uint2 [p][mu][3][Vh] (2 complex per uint2).
// Clover: packed Hermitian 6x6 pair in FP16, uint2 [18][Vh] per parity
// (block b: 9 uint2 = 6 real diagonal entries, then 15 complex upper entries).
#pragma once

#include <cuda_fp16.h>

#include "lqcd_internal.cuh"

// 16-byte storage unit of an F16S field (pointer arithmetic in these units)
struct h16s {
    uint4 v;
};
// one F16S half field in h16s units (Vh is a multiple of 8)
__host__ __device__ __forceinline__ long f16s_half_units(long Vh) { return 13 * Vh / 4; }

__device__ __forceinline__ cx<float> f16s_h2c(unsigned u, float s)
{
    __half2 h = *reinterpret_cast<__half2 *>(&u);
    float2 f = __half22float2(h);
    return mk(f.x * s, f.y * s);
}
__device__ __forceinline__ unsigned f16s_c2h(cx<float> v, float inv)
{
    __half2 h = __floats2half2_rn(v.re * inv, v.im * inv);
    return *reinterpret_cast<unsigned *>(&h);
}
__device__ __forceinline__ const float *f16s_scales(const h16s *f, long Vh)
{
    return reinterpret_cast<const float *>(reinterpret_cast<const uint4 *>(f) + 3 * Vh);
}
__device__ __forceinline__ float *f16s_scales(h16s *f, long Vh)
{
    return reinterpret_cast<float *>(reinterpret_cast<uint4 *>(f) + 3 * Vh);
}

// site r of a half field; RO = read-only data (through the non-coherent path)
template <bool RO>
__device__ __forceinline__ void f16s_load(const h16s *f, long Vh, long r, cx<float> v[12])
{
    const uint4 *q = reinterpret_cast<const uint4 *>(f);
    const float s = RO ? __ldg(f16s_scales(f, Vh) + r) : f16s_scales(f, Vh)[r];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        uint4 w = RO ? __ldg(q + k * Vh + r) : q[k * Vh + r];
        v[4 * k] = f16s_h2c(w.x, s);
        v[4 * k + 1] = f16s_h2c(w.y, s);
        v[4 * k + 2] = f16s_h2c(w.z, s);
        v[4 * k + 3] = f16s_h2c(w.w, s);
    }
}
__device__ __forceinline__ float f16s_maxabs(const cx<float> *v, int n)
{
    float m = 0.f;
    for (int i = 0; i < n; i++) m = fmaxf(m, fmaxf(fabsf(v[i].re), fabsf(v[i].im)));
    return m;
}
__device__ __forceinline__ void f16s_store(h16s *f, long Vh, long r, const cx<float> v[12])
{
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 12; i++) m = fmaxf(m, fmaxf(fabsf(v[i].re), fabsf(v[i].im)));
    const float inv = m > 0.f ? 1.f / m : 0.f;
    uint4 *q = reinterpret_cast<uint4 *>(f);
#pragma unroll
    for (int k = 0; k < 3; k++)
        q[k * Vh + r] = make_uint4(f16s_c2h(v[4 * k], inv), f16s_c2h(v[4 * k + 1], inv), f16s_c2h(v[4 * k + 2], inv),
                                   f16s_c2h(v[4 * k + 3], inv));
    f16s_scales(f, Vh)[r] = m;
}

// FP16 link (two stored rows, third = (row0 x row1)^*) of parity p, direction mu
__device__ __forceinline__ void f16s_link(const uint2 *U, long Vh, int p, int mu, long r, cx<float> u[3][3])
{
    const uint2 *b = U + (long)((p * 4 + mu) * 3) * Vh + r;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        uint2 t = __ldg(b + q * Vh);
        u[(2 * q) / 3][(2 * q) % 3] = f16s_h2c(t.x, 1.f);
        u[(2 * q + 1) / 3][(2 * q + 1) % 3] = f16s_h2c(t.y, 1.f);
    }
    su3_third_row(u);
}

// the 36 reals of clover block blk (FP16 copy)
__device__ __forceinline__ void f16s_clover(const uint2 *A, long Vh, long r, int blk, float v[36])
{
    const uint2 *b = A + (long)(9 * blk) * Vh + r;
#pragma unroll
    for (int q = 0; q < 9; q++) {
        uint2 t = __ldg(b + q * Vh);
        cx<float> a = f16s_h2c(t.x, 1.f), c = f16s_h2c(t.y, 1.f);
        v[4 * q] = a.re;
        v[4 * q + 1] = a.im;
        v[4 * q + 2] = c.re;
        v[4 * q + 3] = c.im;
    }
}
