// stencil.cuh -- per-point arithmetic shared by the step kernels.
//
// Arithmetic per point (FP32, FMA):
//   S_k = sum over the d axes of (P[+k] + P[-k]),  D_k = S_k - 2d P   (one rounding)
//   L'P = c1 D_1 + c2 D_2 + c3 D_3 + c4 D_4
//   Pn  = (w L'P + 2P - (1 - a) Pold) / (1 + a)       (a = 0: no division)
// Forming D_k before weighting keeps every large-magnitude sum exact or
// single-rounded, so a constant field gives L'P = 0 exactly and FP32 rounding
// does not act as a spurious mass term that drifts the phase over many steps.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fd_internal.h"

namespace fdk {

__device__ __forceinline__ float f4c(const float4 &v, int e)
{
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}

__device__ __forceinline__ float2 half2of(const float4 &v, int h)
{
    return h == 0 ? make_float2(v.x, v.y) : make_float2(v.z, v.w);
}

// x pair sums P[x+k] + P[x-k] for the two points (2h, 2h+1) of a thread whose
// row segment x-4 .. x+7 is xa[0..11].  Even k keeps both operands on aligned
// register pairs (one packed add); odd k straddles them (two scalar adds with
// the same rounding).
__device__ __forceinline__ float2 xpair2(const float (&xa)[12], int h, int k)
{
    const int i = 4 + 2 * h;
    if ((k & 1) == 0)
        return __fadd2_rn(make_float2(xa[i + k], xa[i + k + 1]), make_float2(xa[i - k], xa[i - k + 1]));
    return make_float2(xa[i + k] + xa[i - k], xa[i + k + 1] + xa[i - k + 1]);
}

// Damped leapfrog update of one point from its centre value, Pold, w, damping a
// and the four distance sums S_k over NDIM axes.
template <int NDIM>
__device__ __forceinline__ float update_point(const StepParams &prm, float p, float pold, float w,
                                              float a, float s1, float s2, float s3, float s4)
{
    constexpr float m = -2.0f * NDIM;
    float acc = prm.c1 * fmaf(m, p, s1);
    acc = fmaf(prm.c2, fmaf(m, p, s2), acc);
    acc = fmaf(prm.c3, fmaf(m, p, s3), acc);
    acc = fmaf(prm.c4, fmaf(m, p, s4), acc);
    const float num = fmaf(w, acc, fmaf(2.0f, p, -(1.0f - a) * pold));
    return a != 0.0f ? num / (1.0f + a) : num;
}

__device__ __forceinline__ void raise_error(int *err, volatile int *abort_flag, int code)
{
    *abort_flag = 1;
    atomicCAS(err, 0, code);
}

// One thread's 4 consecutive x points of a 2D tile held in shared memory: P
// box (TX+8) x (TZ+8) with a 4-point halo, Pold and w tiles TX x TZ.  Packed
// FP32 arithmetic in the rounding order of update_point<2>; sponge points use
// __fdividef.  Returns the new values in r[0] (points 0, 1) and r[1] (2, 3),
// and the stencil sums L'P of the same points in lp.
template <int TX>
__device__ __forceinline__ void tile2d_update(const float *sP, const float *sO, const float *sW, int tx, int tz,
                                              const float (&axv)[4], float azv, float c1, float c2, float c3,
                                              float c4, float2 (&r)[2], float2 (&lp)[2])
{
    constexpr int HX = TX + 8;
    const float *pl = sP + (tz + 4) * HX + 4 * tx + 4;
    const float4 xm = *reinterpret_cast<const float4 *>(pl - 4);
    const float4 xc = *reinterpret_cast<const float4 *>(pl);
    const float4 xp = *reinterpret_cast<const float4 *>(pl + 4);
    float4 zm[4], zp[4];
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
        zm[k - 1] = *reinterpret_cast<const float4 *>(pl - k * HX);
        zp[k - 1] = *reinterpret_cast<const float4 *>(pl + k * HX);
    }
    const float4 old = *reinterpret_cast<const float4 *>(sO + tz * TX + 4 * tx);
    const float4 wv = *reinterpret_cast<const float4 *>(sW + tz * TX + 4 * tx);
    const float xa[12] = {xm.x, xm.y, xm.z, xm.w, xc.x, xc.y, xc.z, xc.w, xp.x, xp.y, xp.z, xp.w};
    const float2 M = make_float2(-4.0f, -4.0f);
    const float2 NEG1 = make_float2(-1.0f, -1.0f);
    float2 acc[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float2 p2 = half2of(xc, h);
        float2 a2;
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
            const float2 sx = xpair2(xa, h, k);
            const float2 sz = __fadd2_rn(half2of(zp[k - 1], h), half2of(zm[k - 1], h));
            const float2 d = __ffma2_rn(M, p2, __fadd2_rn(sx, sz));
            const float ck = k == 1 ? c1 : k == 2 ? c2 : k == 3 ? c3 : c4;
            a2 = k == 1 ? __fmul2_rn(make_float2(ck, ck), d) : __ffma2_rn(make_float2(ck, ck), d, a2);
        }
        acc[h] = a2;
        lp[h] = a2;
    }
    if (axv[0] != 0.f || axv[1] != 0.f || axv[2] != 0.f || axv[3] != 0.f || azv != 0.f) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 p2 = half2of(xc, h), o2 = half2of(old, h), w2 = half2of(wv, h);
            const float a0 = axv[2 * h] + azv, a1 = axv[2 * h + 1] + azv;
            const float n0 = fmaf(w2.x, acc[h].x, fmaf(2.0f, p2.x, -(1.0f - a0) * o2.x));
            const float n1 = fmaf(w2.y, acc[h].y, fmaf(2.0f, p2.y, -(1.0f - a1) * o2.y));
            r[h] = make_float2(a0 != 0.0f ? __fdividef(n0, 1.0f + a0) : n0,
                               a1 != 0.0f ? __fdividef(n1, 1.0f + a1) : n1);
        }
    } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 p2 = half2of(xc, h);
            const float2 t = __ffma2_rn(NEG1, half2of(old, h), __fadd2_rn(p2, p2));
            r[h] = __ffma2_rn(half2of(wv, h), acc[h], t);
        }
    }
}

// Add the source amplitude to whichever of the 4 points is the source column.
__device__ __forceinline__ void add_source4(float2 (&r)[2], int e, float amp)
{
    if (e == 0) r[0].x += amp;
    if (e == 1) r[0].y += amp;
    if (e == 2) r[1].x += amp;
    if (e == 3) r[1].y += amp;
}

// Store 4 consecutive points of a dense row at dst (any alignment), of which the
// first is inside the row and `valid` are.
__device__ __forceinline__ void store4_dense(float *dst, const float2 (&v)[2], int valid, bool aligned)
{
    if (aligned && valid >= 4) {
        *reinterpret_cast<float4 *>(dst) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    } else {
        dst[0] = v[0].x;
        if (valid > 1) dst[1] = v[0].y;
        if (valid > 2) dst[2] = v[1].x;
        if (valid > 3) dst[3] = v[1].y;
    }
}

// grad[e] = fma(v[e], lp[e], grad[e]) for 4 consecutive points of a dense row at
// grad / lp (any alignment), of which the first is inside the row and `valid` are.
__device__ __forceinline__ void image4_dense(float *grad, const float *lp, const float2 (&v)[2], int valid,
                                             bool aligned)
{
    if (aligned && valid >= 4) {
        const float4 l = *reinterpret_cast<const float4 *>(lp);
        float4 g = *reinterpret_cast<const float4 *>(grad);
        g.x = fmaf(v[0].x, l.x, g.x);
        g.y = fmaf(v[0].y, l.y, g.y);
        g.z = fmaf(v[1].x, l.z, g.z);
        g.w = fmaf(v[1].y, l.w, g.w);
        *reinterpret_cast<float4 *>(grad) = g;
    } else {
        grad[0] = fmaf(v[0].x, lp[0], grad[0]);
        if (valid > 1) grad[1] = fmaf(v[0].y, lp[1], grad[1]);
        if (valid > 2) grad[2] = fmaf(v[1].x, lp[2], grad[2]);
        if (valid > 3) grad[3] = fmaf(v[1].y, lp[3], grad[3]);
    }
}

// Store 4 consecutive points, of which the first is known to be inside the row.
__device__ __forceinline__ void store4(float *dst, const float2 (&r)[2], int valid)
{
    if (valid >= 4) {
        *reinterpret_cast<float4 *>(dst) = make_float4(r[0].x, r[0].y, r[1].x, r[1].y);
    } else {
        dst[0] = r[0].x;
        if (valid > 1) dst[1] = r[0].y;
        if (valid > 2) dst[2] = r[1].x;
    }
}

}  // namespace fdk
