// fd_t2.cu -- two time steps per launch (temporal fusion) for 3D grids (sm_103a).
//
// One launch advances the damped leapfrog of the paper's section 7 (Eq. 1, the
// WaveSimulator::run() sequence) by two steps: from the levels P^{n-1}, P^n it
// writes P^{n+1} and P^{n+2}, reading P^{n-1}, P^n and w once and writing two
// levels, 20 bytes per point for two updates instead of 32.  The arithmetic per
// point and its rounding order are those of the single-step kernel, so two
// fused steps give bitwise the levels of two single steps.
//
// A CTA owns a 32 x 32 (x, y) column of the output and marches along z through
// bz planes.  Step one is evaluated on the column widened by the stencil radius
// (40 x 40 points), so that step two has the x/y neighbours of P^{n+1} without
// any exchange between CTAs; the widening is recomputed, not communicated.  At
// iteration j of the march:
//   - step one computes P^{n+1} on plane z0 - 4 + j of the widened column, from a
//     register queue of P^n along z (the thread's own 4 points, planes z0-8+j ..
//     z0+j), the x/y neighbours of P^n from a 48 x 48 TMA box of that plane, and
//     P^{n-1}, w from 40 x 40 boxes;
//   - the result goes to a shared-memory ring of P^{n+1} planes and, for the
//     column's own points, to a second register queue;
//   - step two computes P^{n+2} on plane z0 + j - 8 from that queue (z
//     neighbours), the ring plane written four iterations earlier (x/y
//     neighbours), P^n from the first queue and w from its ring.
// Points of the widened column outside the grid get P^{n+1} = 0, which is the
// zero halo that step two must see.  One CTA barrier per plane orders the
// P^{n+1} ring; after it, thread 0 issues the TMA loads of the stage kT2D
// planes ahead into slots that the barrier has just freed.  Every wait is
// bounded; on expiry the CTA raises the device error word, waits (bounded) for
// its own copies in flight and returns.

#include <algorithm>
#include <type_traits>

#include "fd_internal.h"
#include "ptx.cuh"
#include "stencil.cuh"

namespace fdk {

namespace {

constexpr int kT2X = 32, kT2Y = 32;          // output column
constexpr int kT2EQ = (kT2X + 8) / 4;        // quads per widened row (10)
constexpr int kT2EY = kT2Y + 8;              // widened rows (40)
constexpr int kT2Work = kT2EQ * kT2EY;       // step-one threads (400)
constexpr int kT2BX = kT2X + 16;             // P^n box: widened column + radius (48)
constexpr int kT2BY = kT2Y + 16;
constexpr int kT2PB = kT2BX * kT2BY;         // floats per P^n plane box
constexpr int kT2EB = (kT2X + 8) * kT2EY;    // floats per widened plane (P^{n-1}, w, P^{n+1})
constexpr int kT2EX = kT2X + 8;
constexpr int kT2D = 3;                      // stages issued ahead of the one consumed
constexpr int kT2SP1 = kT2D + 4;             // P^n ring: x/y use 4 planes after the queue fill
constexpr int kT2SP0 = kT2D;                 // P^{n-1} ring
constexpr int kT2SW = kT2D + 4;              // w ring: step two reads w 4 planes later
constexpr int kT2S2 = 5;                     // P^{n+1} ring: written at j, read at j + 4
constexpr int kT2NB = kT2D + 1;              // stage barriers
constexpr int kT2U = 4;                      // bodies per queue rotation

static_assert((kT2PB * 4) % 128 == 0 && (kT2EB * 4) % 128 == 0, "boxes keep 128-byte alignment");

}  // namespace

constexpr size_t t2_smem_floats()
{
    return (size_t)kT2SP1 * kT2PB + (size_t)(kT2SP0 + kT2SW + kT2S2) * kT2EB;
}

size_t step3d_t2_smem_bytes()
{
    return t2_smem_floats() * sizeof(float) + kT2NB * sizeof(uint64_t);
}

// L'P of the 4 points (packed pairs h = 0, 1) whose centre is c, x neighbours
// in xa (x-4 .. x+7), y neighbours ym[k-1] / yp[k-1] and z neighbours zm / zp at
// distance k, in the rounding order of the single-step kernel.
__device__ __forceinline__ void t2_lap(const float (&xa)[12], const float4 &c, const float4 (&ym)[4],
                                       const float4 (&yp)[4], const float4 (&zm)[4], const float4 (&zp)[4],
                                       const float2 (&C)[4], float2 (&acc)[2])
{
    const float2 M2 = make_float2(-6.0f, -6.0f);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float2 p2 = half2of(c, h);
        float2 a2;
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
            const float2 sxx = xpair2(xa, h, k);
            const float2 sy = __fadd2_rn(half2of(yp[k - 1], h), half2of(ym[k - 1], h));
            const float2 sz = __fadd2_rn(half2of(zp[k - 1], h), half2of(zm[k - 1], h));
            const float2 d = __ffma2_rn(M2, p2, __fadd2_rn(__fadd2_rn(sxx, sy), sz));
            a2 = k == 1 ? __fmul2_rn(C[0], d) : __ffma2_rn(C[k - 1], d, a2);
        }
        acc[h] = a2;
    }
}

// (w L'P + 2P - (1 - a) Pold) / (1 + a) for 4 points with damping a[e], in the
// single-step kernel's rounding (packed when no point is damped).
__device__ __forceinline__ void t2_update(const float4 &c, const float4 &old, const float4 &wv, const float (&a)[4],
                                          const float2 (&acc)[2], float2 (&r)[2])
{
    if (a[0] != 0.f || a[1] != 0.f || a[2] != 0.f || a[3] != 0.f) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 p2 = half2of(c, h), o2 = half2of(old, h), w2 = half2of(wv, h);
            const float a0 = a[2 * h], a1 = a[2 * h + 1];
            const float n0 = fmaf(w2.x, acc[h].x, fmaf(2.0f, p2.x, -(1.0f - a0) * o2.x));
            const float n1 = fmaf(w2.y, acc[h].y, fmaf(2.0f, p2.y, -(1.0f - a1) * o2.y));
            r[h] = make_float2(a0 != 0.0f ? __fdividef(n0, 1.0f + a0) : n0, a1 != 0.0f ? __fdividef(n1, 1.0f + a1) : n1);
        }
    } else {
        const float2 NEG1 = make_float2(-1.0f, -1.0f);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 p2 = half2of(c, h);
            const float2 t = __ffma2_rn(NEG1, half2of(old, h), __fadd2_rn(p2, p2));
            r[h] = __ffma2_rn(half2of(wv, h), acc[h], t);
        }
    }
}

__device__ __forceinline__ void t2_store(float *dst, const float2 (&r)[2], int x, int nx)
{
    if (x + 3 < nx) {
        *reinterpret_cast<float4 *>(dst) = make_float4(r[0].x, r[0].y, r[1].x, r[1].y);
    } else {
        dst[0] = r[0].x;
        if (x + 1 < nx) dst[1] = r[0].y;
        if (x + 2 < nx) dst[2] = r[1].x;
    }
}

__global__ void __launch_bounds__(kT2Threads, 1)
    step3d_t2_kernel(const __grid_constant__ CUtensorMap tmP1, const __grid_constant__ CUtensorMap tmP0,
                     const __grid_constant__ CUtensorMap tmW, const T2Params prm)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float *sP1 = reinterpret_cast<float *>(smem);
    float *sP0 = sP1 + kT2SP1 * kT2PB;
    float *sW = sP0 + kT2SP0 * kT2EB;
    float *sP2 = sW + kT2SW * kT2EB;
    uint64_t *full = reinterpret_cast<uint64_t *>(sP2 + kT2S2 * kT2EB);
    __shared__ int s_abort;

    const int tiles_x = (prm.nx + kT2X - 1) / kT2X;
    const int x0 = (blockIdx.x % tiles_x) * kT2X;
    const int y0 = (blockIdx.x / tiles_x) * kT2Y;
    const int z0 = blockIdx.y * prm.bz;
    const int z1 = min(prm.nz, z0 + prm.bz);
    const int NJ = z1 - z0 + 8;          // march iterations with compute (j = 0 .. NJ-1)
    const int NS = NJ + 8;               // stages: P^n planes z0-8 .. z1+7
    const int tid = threadIdx.x;

    // stage k: P^n plane z0-8+k (box with radius), and for k >= 8 P^{n-1} and w
    // of plane z0-12+k (the step-one plane of iteration k-8)
    int issued = 0;   // thread 0 only
    auto issue = [&](int k) {
        uint64_t *bar = &full[k % kT2NB];
        mbar_arrive_expect_tx(bar, (kT2PB + (k >= 8 ? 2 * kT2EB : 0)) * 4);
        tma_load_3d(sP1 + (k % kT2SP1) * kT2PB, &tmP1, bar, x0 - 8, y0 - 8, z0 - 8 + k);
        if (k >= 8) {
            tma_load_3d(sP0 + (k % kT2SP0) * kT2EB, &tmP0, bar, x0 - 4, y0 - 4, z0 - 12 + k);
            tma_load_3d(sW + (k % kT2SW) * kT2EB, &tmW, bar, x0 - 4, y0 - 4, z0 - 12 + k);
        }
        issued = k + 1;
    };

    if (tid == 0) {
        for (int b = 0; b < kT2NB; ++b)
            mbar_init(&full[b], 1);
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        prefetch_tensormap(&tmP1);
        prefetch_tensormap(&tmP0);
        prefetch_tensormap(&tmW);
        for (int k = 0; k < min(kT2D, NS); ++k)
            issue(k);
    }

    // receivers of the two levels this launch consumes (rows owed by the previous launch)
    {
        const int64_t nthr = (int64_t)gridDim.x * gridDim.y * blockDim.x;
        const int64_t first = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + tid;
        if (prm.trace_prev0)
            for (int64_t r = first; r < prm.nrec; r += nthr)
                prm.trace_prev0[r] = prm.P0[prm.rec_idx[r]];
        if (prm.trace_prev1)
            for (int64_t r = first; r < prm.nrec; r += nthr)
                prm.trace_prev1[r] = prm.P1[prm.rec_idx[r]];
    }

    const bool worker = tid < kT2Work;
    const int eq = tid % kT2EQ;
    const int ey = tid / kT2EQ;
    const bool inner = worker && eq >= 1 && eq <= kT2EQ - 2 && ey >= 4 && ey < kT2EY - 4;
    const int ex = x0 - 4 + 4 * eq;        // first of the thread's 4 points (widened column)
    const int eyg = y0 - 4 + ey;
    const bool y_in = eyg >= 0 && eyg < prm.ny;
    const int cB = (ey + 4) * kT2BX + 4 * eq + 4;   // centre in a P^n box
    const int cE = ey * kT2EX + 4 * eq;             // first point in a widened plane
    float axv[4] = {0.f, 0.f, 0.f, 0.f};
    bool x_in[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        x_in[e] = ex + e >= 0 && ex + e < prm.nx;
        if (prm.has_sponge && x_in[e])
            axv[e] = prm.ax[ex + e];
    }
    const float ayv = prm.has_sponge && y_in ? prm.ay[eyg] : 0.f;
    const bool store_any = inner && y_in && ex < prm.nx;
    const size_t plane_stride = (size_t)prm.ny * prm.px;
    const size_t col = (size_t)(y_in ? eyg : 0) * prm.px + (ex >= 0 ? ex : 0);
    const float2 C[4] = {make_float2(prm.c1, prm.c1), make_float2(prm.c2, prm.c2), make_float2(prm.c3, prm.c3),
                         make_float2(prm.c4, prm.c4)};

    float4 Q1[8 + kT2U];   // P^n of this column, planes z0-8+j .. z0+j in Q1[u .. 8+u]
    float4 Q2[8 + kT2U];   // P^{n+1} of this column, planes z0-12+j .. z0-4+j in Q2[u .. 8+u]
    // The rotations copy entries that the prologue has not filled yet; starting
    // from defined values keeps those copies (and everything derived from the
    // queues) well defined.
#pragma unroll
    for (int q = 0; q < 8 + kT2U; ++q) {
        Q1[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        Q2[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    bool ok = true;

    auto body = [&](int j, auto uu) {
        constexpr int u = decltype(uu)::value;
        const int k = j + 8;
        bool good = mbar_wait(&full[k % kT2NB], (k / kT2NB) & 1, &s_abort);
        if (good && worker) {
            Q1[8 + u] = *reinterpret_cast<const float4 *>(sP1 + (k % kT2SP1) * kT2PB + cB);
            if (j >= 0) {
                // ---- step one: P^{n+1} on plane zs of the widened column
                const int zs = z0 - 4 + j;
                const float *pl = sP1 + ((j + 4) % kT2SP1) * kT2PB + cB;
                const float4 xm = *reinterpret_cast<const float4 *>(pl - 4);
                const float4 xp = *reinterpret_cast<const float4 *>(pl + 4);
                float4 ym[4], yp[4], zm[4], zp[4];
#pragma unroll
                for (int q = 1; q <= 4; ++q) {
                    ym[q - 1] = *reinterpret_cast<const float4 *>(pl - q * kT2BX);
                    yp[q - 1] = *reinterpret_cast<const float4 *>(pl + q * kT2BX);
                    zm[q - 1] = Q1[4 + u - q];
                    zp[q - 1] = Q1[4 + u + q];
                }
                const float4 c = Q1[4 + u];
                const float xa[12] = {xm.x, xm.y, xm.z, xm.w, c.x, c.y, c.z, c.w, xp.x, xp.y, xp.z, xp.w};
                const float4 old = *reinterpret_cast<const float4 *>(sP0 + (k % kT2SP0) * kT2EB + cE);
                const float4 wv = *reinterpret_cast<const float4 *>(sW + (k % kT2SW) * kT2EB + cE);
                float2 acc[2], r[2];
                t2_lap(xa, c, ym, yp, zm, zp, C, acc);
                const bool zin = zs >= 0 && zs < prm.nz;
                float a[4];
                const float ayz = ayv + (prm.has_sponge && zin ? prm.az[zs] : 0.f);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    a[e] = x_in[e] && y_in && zin ? axv[e] + ayz : 0.f;
                t2_update(c, old, wv, a, acc, r);
                if (prm.src_on0 && zs == prm.sz && eyg == prm.sy && (unsigned)(prm.sx - ex) < 4u)
                    add_source4(r, prm.sx - ex, prm.amp0);
                // outside the grid the new level is zero (the rigid boundary of step two)
                if (!(y_in && zin)) {
                    r[0] = make_float2(0.f, 0.f);
                    r[1] = make_float2(0.f, 0.f);
                } else {
                    if (!x_in[0]) r[0].x = 0.f;
                    if (!x_in[1]) r[0].y = 0.f;
                    if (!x_in[2]) r[1].x = 0.f;
                    if (!x_in[3]) r[1].y = 0.f;
                }
                const float4 p2 = make_float4(r[0].x, r[0].y, r[1].x, r[1].y);
                *reinterpret_cast<float4 *>(sP2 + (j % kT2S2) * kT2EB + cE) = p2;
                if (inner) {
                    Q2[8 + u] = p2;
                    if (store_any && zs >= z0 && zs < z1)
                        t2_store(prm.out2 + (size_t)zs * plane_stride + col, r, ex, prm.nx);
                }
            }
        }
        if (good && inner && j >= 8) {
            // ---- step two: P^{n+2} on plane zc of the column itself
            const int zc = z0 + j - 8;
            const float *pl = sP2 + ((j - 4) % kT2S2) * kT2EB + cE;
            const float4 xm = *reinterpret_cast<const float4 *>(pl - 4);
            const float4 xp = *reinterpret_cast<const float4 *>(pl + 4);
            float4 ym[4], yp[4], zm[4], zp[4];
#pragma unroll
            for (int q = 1; q <= 4; ++q) {
                ym[q - 1] = *reinterpret_cast<const float4 *>(pl - q * kT2EX);
                yp[q - 1] = *reinterpret_cast<const float4 *>(pl + q * kT2EX);
                zm[q - 1] = Q2[4 + u - q];
                zp[q - 1] = Q2[4 + u + q];
            }
            const float4 c = Q2[4 + u];
            const float xa[12] = {xm.x, xm.y, xm.z, xm.w, c.x, c.y, c.z, c.w, xp.x, xp.y, xp.z, xp.w};
            const float4 wv = *reinterpret_cast<const float4 *>(sW + ((k - 4) % kT2SW) * kT2EB + cE);
            float2 acc[2], r[2];
            t2_lap(xa, c, ym, yp, zm, zp, C, acc);
            float a[4];
            const float ayz = ayv + (prm.has_sponge ? prm.az[zc] : 0.f);
#pragma unroll
            for (int e = 0; e < 4; ++e)
                a[e] = x_in[e] ? axv[e] + ayz : 0.f;
            t2_update(c, Q1[u], wv, a, acc, r);
            if (prm.src_on1 && zc == prm.sz && eyg == prm.sy && (unsigned)(prm.sx - ex) < 4u)
                add_source4(r, prm.sx - ex, prm.amp1);
            if (store_any)
                t2_store(prm.out3 + (size_t)zc * plane_stride + col, r, ex, prm.nx);
        }
        // one barrier per plane: the P^{n+1} plane is complete before step two reads
        // it, and every slot that stage k + kT2D reuses has been read for the last time
        if (__syncthreads_or(!good)) {
            ok = false;
            return;
        }
        if (tid == 0 && k + kT2D < NS)
            issue(k + kT2D);
    };

    for (int jg = -8; ok && jg < NJ; jg += kT2U) {
        body(jg, std::integral_constant<int, 0>{});
        if (ok && jg + 1 < NJ)
            body(jg + 1, std::integral_constant<int, 1>{});
        if (ok && jg + 2 < NJ)
            body(jg + 2, std::integral_constant<int, 2>{});
        if (ok && jg + 3 < NJ)
            body(jg + 3, std::integral_constant<int, 3>{});
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            Q1[q] = Q1[q + kT2U];
            Q2[q] = Q2[q + kT2U];
        }
    }
    if (!ok) {
        if (tid == 0) {
            raise_error(prm.err, &s_abort, kDevErrTimeout);
            // do not leave while copies into this CTA's shared memory may be in
            // flight: wait (bounded) for every issued stage not yet consumed
            int never = 0;
            for (int k = max(0, issued - kT2NB); k < issued; ++k)
                mbar_wait(&full[k % kT2NB], (k / kT2NB) & 1, &never, kWaitLimitCycles / 8);
        }
    }
}

cudaError_t step3d_t2_prepare()
{
    return cudaFuncSetAttribute(step3d_t2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)step3d_t2_smem_bytes());
}

cudaError_t launch_step3d_t2(const CUtensorMap &tmP1, const CUtensorMap &tmP0, const CUtensorMap &tmW,
                             const T2Params &p, int nchunks, cudaStream_t s)
{
    const int tiles = ((p.nx + kT2X - 1) / kT2X) * ((p.ny + kT2Y - 1) / kT2Y);
    step3d_t2_kernel<<<dim3(tiles, nchunks), kT2Threads, step3d_t2_smem_bytes(), s>>>(tmP1, tmP0, tmW, p);
    return cudaGetLastError();
}

}  // namespace fdk
