// fd_kernels.cu -- fused time-step kernels of the acoustic FD propagator (sm_103a).
//
// One launch performs one time step of the paper's WaveSimulator::run() loop
// (section 7): add_source, the z and x (and y) second derivatives, the time
// update and the rotation of levels, fused so that each grid point costs one
// read of P, Pold and w and one write of Pn (16 bytes) instead of the five
// field passes of the unfused routine sequence.  The receiver gather of the
// previous step rides along in the same launch.
//
// Arithmetic per point (FP32, FMA):
//   S_k = sum over the axes of (P[+k] + P[-k]),  D_k = S_k - 2d P   (one rounding)
//   L'P = c1 D_1 + c2 D_2 + c3 D_3 + c4 D_4
//   Pn  = (w L'P + 2P - (1 - a) Pold) / (1 + a)       (a = 0: no division)
// Forming D_k before weighting keeps every large-magnitude sum exact or
// single-rounded, so a constant field gives L'P = 0 exactly and FP32 rounding
// does not act as a spurious mass term that drifts the phase over many steps.

#include <algorithm>

#include "fd_internal.h"
#include "ptx.cuh"

namespace fdk {

__device__ __forceinline__ float f4c(const float4 &v, int e)
{
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
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

// Gather of the previous step's receiver row, spread over every thread of the grid.
__device__ __forceinline__ void gather_prev_row(const StepParams &prm)
{
    if (!prm.trace_prev)
        return;
    const int64_t nthr = (int64_t)gridDim.x * gridDim.y * blockDim.x;
    for (int64_t r = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
         r < prm.nrec; r += nthr)
        prm.trace_prev[r] = prm.P[prm.rec_idx[r]];
}

// ----------------------------------------------------------------------------- 3D

// A CTA owns the column [x0, x0+TX) x [y0, y0+TY) and output planes [z0, z1).
// Warps 0..NCW-1 are consumers (each thread: 4 consecutive x points of one row);
// warp NCW's lane 0 is the producer issuing TMA loads.  Ring stage k holds the
// haloed P plane z0-4+k and, for k >= 8, the Pold and w planes z0-8+k.  A
// consumer computing plane z = z0+j reads its z neighbours from a 9-deep
// register queue, its x/y neighbours from stage j+4 (plane z) and Pold, w from
// stage j+8, then frees stage j+4.
template <int TX, int TY, int S>
__global__ void __launch_bounds__(TX / 4 * TY + 32, 2)
    step3d_kernel(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmOld,
                  const __grid_constant__ CUtensorMap tmW, const StepParams prm)
{
    constexpr int QX = TX / 4;
    constexpr int NCONS = QX * TY;
    constexpr int NCW = NCONS / 32;
    constexpr int HX = TX + 8;
    constexpr int HY = TY + 8;
    constexpr int PBOX = HX * HY;
    constexpr int TBOX = TX * TY;
    constexpr uint32_t BYTES_P = PBOX * 4;
    constexpr uint32_t BYTES_T = TBOX * 4;
    static_assert(NCONS % 32 == 0, "consumer threads must fill warps");
    static_assert((PBOX * 4) % 128 == 0 && (TBOX * 4) % 128 == 0, "boxes keep 128-byte alignment");
    static_assert(S >= 5, "ring must hold planes z..z+4");

    extern __shared__ __align__(128) unsigned char smem[];
    float *sP = reinterpret_cast<float *>(smem);
    float *sO = sP + S * PBOX;
    float *sW = sO + S * TBOX;
    uint64_t *full = reinterpret_cast<uint64_t *>(sW + S * TBOX);
    uint64_t *empty = full + S;
    __shared__ int s_abort;

    const int tiles_x = (prm.nx + TX - 1) / TX;
    const int x0 = (blockIdx.x % tiles_x) * TX;
    const int y0 = (blockIdx.x / tiles_x) * TY;
    const int z0 = blockIdx.y * prm.bz;
    const int z1 = min(prm.nz, z0 + prm.bz);
    const int nb = z1 - z0;
    const int nstages = nb + 8;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();

    gather_prev_row(prm);

    if (warp == NCW) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            prefetch_tensormap(&tmP);
            prefetch_tensormap(&tmOld);
            prefetch_tensormap(&tmW);
            int issued = 0;
            for (int k = 0; k < nstages; ++k) {
                const int slot = k % S;
                if (k >= S && !mbar_wait(&empty[slot], ((k / S) - 1) & 1, &s_abort)) {
                    raise_error(prm.err, &s_abort, kDevErrTimeout);
                    break;
                }
                const int pz = z0 - 4 + k;
                const bool has_t = k >= 8;
                mbar_arrive_expect_tx(&full[slot], BYTES_P + (has_t ? 2 * BYTES_T : 0));
                tma_load_3d(sP + slot * PBOX, &tmP, &full[slot], x0 - 4, y0 - 4, pz);
                if (has_t) {
                    tma_load_3d(sO + slot * TBOX, &tmOld, &full[slot], x0, y0, pz - 4);
                    tma_load_3d(sW + slot * TBOX, &tmW, &full[slot], x0, y0, pz - 4);
                }
                issued = k + 1;
            }
            // Do not leave while copies into this CTA's shared memory are in flight:
            // wait (bounded, regardless of abort) for the newest use of every slot.
            int never = 0;
            for (int k = max(0, issued - S); k < issued; ++k)
                mbar_wait(&full[k % S], (k / S) & 1, &never);
        }
        return;
    }

    // -------------------------------------------------------------------- consumers
    const int tx = tid % QX;
    const int ty = tid / QX;
    const int x = x0 + 4 * tx;
    const int y = y0 + ty;
    const int cP = (ty + 4) * HX + 4 * tx + 4;   // centre float4 within a P box
    const int cT = ty * TX + 4 * tx;             // float4 within a Pold / w box
    const bool row_ok = y < prm.ny;

    float axv[4] = {0.f, 0.f, 0.f, 0.f};
    float ayv = 0.f;
    if (prm.has_sponge) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            axv[e] = x + e < prm.px ? prm.ax[x + e] : 0.f;
        ayv = row_ok ? prm.ay[y] : 0.f;
    }
    const bool x_band = axv[0] != 0.f || axv[1] != 0.f || axv[2] != 0.f || axv[3] != 0.f;

    float4 q[9];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int slot = k % S;
        ok = __all_sync(0xffffffffu, mbar_wait(&full[slot], (k / S) & 1, &s_abort));
        if (!ok)
            break;
        q[k] = *reinterpret_cast<const float4 *>(sP + slot * PBOX + cP);
        if (k < 4) {
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&empty[slot]);
        }
    }

    for (int j = 0; ok && j < nb; ++j) {
        const int k8 = j + 8;
        const int s8 = k8 % S;
        const int s4 = (j + 4) % S;
        ok = __all_sync(0xffffffffu, mbar_wait(&full[s8], (k8 / S) & 1, &s_abort));
        if (!ok)
            break;
        q[8] = *reinterpret_cast<const float4 *>(sP + s8 * PBOX + cP);
        const float *pl = sP + s4 * PBOX + cP;
        const float4 xm = *reinterpret_cast<const float4 *>(pl - 4);
        const float4 xc = *reinterpret_cast<const float4 *>(pl);
        const float4 xp = *reinterpret_cast<const float4 *>(pl + 4);
        float4 ym[4], yp[4];
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
            ym[k - 1] = *reinterpret_cast<const float4 *>(pl - k * HX);
            yp[k - 1] = *reinterpret_cast<const float4 *>(pl + k * HX);
        }
        const float4 old = *reinterpret_cast<const float4 *>(sO + s8 * TBOX + cT);
        const float4 wv = *reinterpret_cast<const float4 *>(sW + s8 * TBOX + cT);
        const int z = z0 + j;
        const float ayz = prm.has_sponge ? ayv + prm.az[z] : 0.f;
        const bool damped = x_band || ayz != 0.f;

        const float xa[12] = {xm.x, xm.y, xm.z, xm.w, xc.x, xc.y, xc.z, xc.w, xp.x, xp.y, xp.z, xp.w};
        float pn[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float s[4];
#pragma unroll
            for (int k = 1; k <= 4; ++k)
                s[k - 1] = ((xa[4 + e + k] + xa[4 + e - k]) + (f4c(yp[k - 1], e) + f4c(ym[k - 1], e))) +
                           (f4c(q[4 + k], e) + f4c(q[4 - k], e));
            const float a = damped ? axv[e] + ayz : 0.f;
            pn[e] = update_point<3>(prm, f4c(q[4], e), f4c(old, e), f4c(wv, e), a, s[0], s[1], s[2], s[3]);
        }
        if (prm.src_on && z == prm.sz && y == prm.sy && (unsigned)(prm.sx - x) < 4u) {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (prm.sx - x == e)
                    pn[e] += prm.src_amp;
        }
        if (row_ok && x < prm.nx) {
            float *dst = prm.out + ((size_t)z * prm.ny + y) * prm.px + x;
            if (x + 3 < prm.nx) {
                *reinterpret_cast<float4 *>(dst) = make_float4(pn[0], pn[1], pn[2], pn[3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (x + e < prm.nx)
                        dst[e] = pn[e];
            }
        }
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&empty[s4]);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            q[k] = q[k + 1];
    }
    if (ok) {
        for (int k = nb + 4; k < nb + 8; ++k) {
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&empty[k % S]);
        }
    } else {
        raise_error(prm.err, &s_abort, kDevErrTimeout);
    }
}

// ----------------------------------------------------------------------------- 2D

// A CTA owns one TX x TZ tile of the [nz][nx] grid.  One TMA transaction brings
// the haloed P tile and the Pold and w tiles; each thread computes 4
// consecutive x points of one row.
template <int TX, int TZ>
__global__ void __launch_bounds__(TX / 4 * TZ)
    step2d_kernel(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmOld,
                  const __grid_constant__ CUtensorMap tmW, const StepParams prm)
{
    constexpr int QX = TX / 4;
    constexpr int HX = TX + 8;
    constexpr int HZ = TZ + 8;
    constexpr uint32_t BYTES = (HX * HZ + 2 * TX * TZ) * 4;
    __shared__ __align__(128) float sP[HX * HZ];
    __shared__ __align__(128) float sO[TX * TZ];
    __shared__ __align__(128) float sW[TX * TZ];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_abort;

    const int tiles_x = (prm.nx + TX - 1) / TX;
    const int x0 = (blockIdx.x % tiles_x) * TX;
    const int z0 = (blockIdx.x / tiles_x) * TZ;
    const int tid = threadIdx.x;

    if (tid == 0) {
        mbar_init(&bar, 1);
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar, BYTES);
        tma_load_2d(sP, &tmP, &bar, x0 - 4, z0 - 4);
        tma_load_2d(sO, &tmOld, &bar, x0, z0);
        tma_load_2d(sW, &tmW, &bar, x0, z0);
    }
    gather_prev_row(prm);

    const int tx = tid % QX;
    const int tz = tid / QX;
    const int x = x0 + 4 * tx;
    const int z = z0 + tz;
    float axv[4] = {0.f, 0.f, 0.f, 0.f};
    float azv = 0.f;
    if (prm.has_sponge) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            axv[e] = x + e < prm.px ? prm.ax[x + e] : 0.f;
        azv = z < prm.nz ? prm.az[z] : 0.f;
    }
    const bool ok = __syncthreads_and(mbar_wait(&bar, 0, &s_abort));
    if (!ok) {
        if (tid == 0)
            raise_error(prm.err, &s_abort, kDevErrTimeout);
        return;
    }
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
    float pn[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float s[4];
#pragma unroll
        for (int k = 1; k <= 4; ++k)
            s[k - 1] = (xa[4 + e + k] + xa[4 + e - k]) + (f4c(zp[k - 1], e) + f4c(zm[k - 1], e));
        pn[e] = update_point<2>(prm, xa[4 + e], f4c(old, e), f4c(wv, e), axv[e] + azv, s[0], s[1], s[2],
                                s[3]);
    }
    if (prm.src_on && z == prm.sz && (unsigned)(prm.sx - x) < 4u) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (prm.sx - x == e)
                pn[e] += prm.src_amp;
    }
    if (z < prm.nz && x < prm.nx) {
        float *dst = prm.out + (size_t)z * prm.px + x;
        if (x + 3 < prm.nx) {
            *reinterpret_cast<float4 *>(dst) = make_float4(pn[0], pn[1], pn[2], pn[3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (x + e < prm.nx)
                    dst[e] = pn[e];
        }
    }
}

// ------------------------------------------------------------------------ helpers

__global__ void gather_kernel(const float *__restrict__ P, const int64_t *__restrict__ idx, int nrec,
                              float *__restrict__ out)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += gridDim.x * blockDim.x)
        out[r] = P[idx[r]];
}

__global__ void velocity_stats_kernel(const float *__restrict__ v, int nx, size_t rows, int px,
                                      unsigned *stats)
{
    unsigned vmax_bits = 0, bad = 0;
    const size_t n = (size_t)nx * rows;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / nx;
        const float x = v[row * px + (i - row * nx)];
        if (isfinite(x) && x > 0.f)
            vmax_bits = max(vmax_bits, __float_as_uint(x));   // positive floats order as their bits
        else
            ++bad;
    }
    for (int o = 16; o > 0; o >>= 1) {
        vmax_bits = max(vmax_bits, __shfl_xor_sync(0xffffffffu, vmax_bits, o));
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&stats[0], vmax_bits);
        if (bad)
            atomicAdd(&stats[1], bad);
    }
}

// w = (dt/h * v)^2 in FP64, rounded once to FP32; v and w share the pitched layout
// (v may alias w).
__global__ void compute_w_kernel(const float *v, float *w, int nx, size_t rows, int px, double dt_over_h)
{
    const size_t n = (size_t)nx * rows;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / nx;
        const size_t at = row * px + (i - row * nx);
        const double c = dt_over_h * (double)v[at];
        w[at] = (float)(c * c);
    }
}

// ------------------------------------------------------------------------ launchers

using Step3D = decltype(&step3d_kernel<kTX3, kTY3, kStages3>);

size_t step3d_smem_bytes()
{
    constexpr int PBOX = (kTX3 + 8) * (kTY3 + 8);
    constexpr int TBOX = kTX3 * kTY3;
    return (size_t)kStages3 * (PBOX + 2 * TBOX) * sizeof(float) + 2 * kStages3 * sizeof(uint64_t);
}

cudaError_t step3d_prepare()
{
    return cudaFuncSetAttribute(step3d_kernel<kTX3, kTY3, kStages3>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step3d_smem_bytes());
}

int step3d_blocks_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step3d_kernel<kTX3, kTY3, kStages3>, kThreads3,
                                                      step3d_smem_bytes()) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_step3d(const CUtensorMap &tmP, const CUtensorMap &tmOld, const CUtensorMap &tmW,
                          const StepParams &p, int nchunks, cudaStream_t s)
{
    const int tiles = ((p.nx + kTX3 - 1) / kTX3) * ((p.ny + kTY3 - 1) / kTY3);
    dim3 grid(tiles, nchunks);
    step3d_kernel<kTX3, kTY3, kStages3><<<grid, kThreads3, step3d_smem_bytes(), s>>>(tmP, tmOld, tmW, p);
    return cudaGetLastError();
}

cudaError_t launch_step2d(const CUtensorMap &tmP, const CUtensorMap &tmOld, const CUtensorMap &tmW,
                          const StepParams &p, cudaStream_t s)
{
    const int tiles = ((p.nx + kTX2 - 1) / kTX2) * ((p.nz + kTZ2 - 1) / kTZ2);
    step2d_kernel<kTX2, kTZ2><<<tiles, kThreads2, 0, s>>>(tmP, tmOld, tmW, p);
    return cudaGetLastError();
}

cudaError_t launch_gather(const float *P, const int64_t *idx, int nrec, float *out, cudaStream_t s)
{
    if (nrec <= 0)
        return cudaSuccess;
    const int blocks = min((nrec + 255) / 256, 1184);
    gather_kernel<<<blocks, 256, 0, s>>>(P, idx, nrec, out);
    return cudaGetLastError();
}

cudaError_t launch_velocity_stats(const float *v, int nx, size_t rows, int px, unsigned *stats,
                                  cudaStream_t s)
{
    const size_t n = (size_t)nx * rows;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 148 * 8);
    velocity_stats_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(v, nx, rows, px, stats);
    return cudaGetLastError();
}

cudaError_t launch_compute_w(const float *v, float *w, int nx, size_t rows, int px, double dt_over_h,
                             cudaStream_t s)
{
    const size_t n = (size_t)nx * rows;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 148 * 16);
    compute_w_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(v, w, nx, rows, px, dt_over_h);
    return cudaGetLastError();
}

}  // namespace fdk
