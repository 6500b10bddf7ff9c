// fd_unfused.cu -- the paper's routines one kernel each (section 7, Listing 3).
//
// WaveSimulator::run() calls add_source, fd_pzz, fd_pxx and fd_time, then
// swaps the levels.  fd_pzz and fd_pxx (and, in 3D, the y counterpart)
// materialise one second-derivative field each; fd_time combines them with P,
// Pold and w into Pn.  Run as separate kernels they move about 40 bytes per
// grid-point update in 2D (52 in 3D) against the fused step's 16; they are kept
// here, written the straightforward way, so that the difference can be
// measured on the same hardware.  The source is added to the new level after
// fd_time (the reading of the fused step), so both schedules compute the same
// recurrence; only the summation order of the axes differs.
//
// Each derivative kernel forms, per axis, D2 = sum_k c_k ((P[+k] + P[-k]) - 2 P)
// with P = 0 outside the grid, for 4 consecutive x points per thread with
// 16-byte loads.  The x kernel reads its neighbours from the same row; the y
// and z kernels march along their axis with the 9 values of the thread's
// column in registers, so each value is loaded about once.

#include <algorithm>

#include "fd.h"
#include "fd_internal.h"
#include "fd_model.h"
#include "fd_trace.h"

namespace fdk {

struct UnfusedParams {
    const float *P, *Pold, *w;
    float *out;                    // derivative field (D2 kernels) or Pn (time kernel)
    const float *d0, *d1, *d2;     // derivatives summed by the time kernel (d1 may be null in 2D)
    const float *ax, *ay, *az;
    int nx, ny, nz, px;
    int has_sponge;
    float c1, c2, c3, c4;
};

__device__ __forceinline__ float4 load4_or_zero(const float *P, long long row_base, int x, int nx)
{
    // x is a multiple of 4; rows are padded to px >= nx, with x + 3 < px
    if (x < 0 || x >= nx)
        return make_float4(0.f, 0.f, 0.f, 0.f);
    float4 v = *reinterpret_cast<const float4 *>(P + row_base + x);
    if (x + 3 >= nx) {
        if (x + 1 >= nx) v.y = 0.f;
        if (x + 2 >= nx) v.z = 0.f;
        if (x + 3 >= nx) v.w = 0.f;
    }
    return v;
}

__device__ __forceinline__ float comp(const float4 &v, int e)
{
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}

// D2 along x: a thread owns 4 consecutive x points of one row and reads its
// neighbours from the same row.
__global__ void __launch_bounds__(256) d2x_kernel(const UnfusedParams p)
{
    const int qx = (p.nx + 3) / 4;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long rows = (long long)p.nz * p.ny;
    if (i >= rows * qx)
        return;
    const int x = (int)(i % qx) * 4;
    const long long row = i / qx;
    const long long base = row * p.px;
    const float4 c = load4_or_zero(p.P, base, x, p.nx);
    const float4 m = load4_or_zero(p.P, base, x - 4, p.nx);
    const float4 q = load4_or_zero(p.P, base, x + 4, p.nx);
    const float a[12] = {m.x, m.y, m.z, m.w, c.x, c.y, c.z, c.w, q.x, q.y, q.z, q.w};
    float r[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float pc = a[4 + e];
        r[e] = p.c1 * fmaf(-2.f, pc, a[5 + e] + a[3 + e]);
        r[e] = fmaf(p.c2, fmaf(-2.f, pc, a[6 + e] + a[2 + e]), r[e]);
        r[e] = fmaf(p.c3, fmaf(-2.f, pc, a[7 + e] + a[1 + e]), r[e]);
        r[e] = fmaf(p.c4, fmaf(-2.f, pc, a[8 + e] + a[0 + e]), r[e]);
    }
    float *dst = p.out + base + x;
    if (x + 3 < p.nx) {
        *reinterpret_cast<float4 *>(dst) = make_float4(r[0], r[1], r[2], r[3]);
    } else {
        for (int e = 0; e < 4 && x + e < p.nx; ++e)
            dst[e] = r[e];
    }
}

// D2 along y (AXIS 1) or z (AXIS 2) by marching: a block of 32 x 8 threads, each
// thread 4 x points of one line along the axis (the lines of a block differ in
// the other transverse coordinate; a 2D grid, ny = 1, spreads them along x
// instead), kMarchLen points of the line per block with a 4-point halo at each
// end.  Same arithmetic and order as d2x_kernel, along the other axis.
constexpr int kMarchLen = 64;

template <int AXIS>
__global__ void __launch_bounds__(256) d2_march_kernel(const UnfusedParams p)
{
    const int extent = AXIS == 1 ? p.ny : p.nz;
    const int tdim = AXIS == 1 ? p.nz : p.ny;      // the other transverse coordinate
    const bool flat = tdim == 1;
    const int x = flat ? ((blockIdx.x * 8 + threadIdx.y) * 32 + threadIdx.x) * 4 : (blockIdx.x * 32 + threadIdx.x) * 4;
    const int t = flat ? 0 : blockIdx.y * 8 + threadIdx.y;
    if (x >= p.nx || t >= tdim)
        return;
    const int c0 = blockIdx.z * kMarchLen;
    const int c1 = min(extent, c0 + kMarchLen);
    const long long stride = AXIS == 1 ? (long long)p.px : (long long)p.ny * p.px;
    const long long base = AXIS == 1 ? (long long)t * p.ny * p.px : (long long)t * p.px;
    const float ck[4] = {p.c1, p.c2, p.c3, p.c4};
    float4 q[9];   // q[i] = P at coordinate c - 4 + i of this column
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = c0 - 4 + i;
        q[i] = c >= 0 && c < extent ? load4_or_zero(p.P, base + c * stride, x, p.nx) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int c = c0; c < c1; ++c) {
        q[8] = c + 4 < extent ? load4_or_zero(p.P, base + (c + 4) * stride, x, p.nx) : make_float4(0.f, 0.f, 0.f, 0.f);
        float r[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
#pragma unroll
            for (int k = 1; k <= 4; ++k) {
                const float d = fmaf(-2.f, comp(q[4], e), comp(q[4 + k], e) + comp(q[4 - k], e));
                r[e] = k == 1 ? ck[0] * d : fmaf(ck[k - 1], d, r[e]);
            }
        }
        float *dst = p.out + base + c * stride + x;
        if (x + 3 < p.nx) {
            *reinterpret_cast<float4 *>(dst) = make_float4(r[0], r[1], r[2], r[3]);
        } else {
            for (int e = 0; e < 4 && x + e < p.nx; ++e)
                dst[e] = r[e];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
            q[i] = q[i + 1];
    }
}

// Pn = (2P - (1 - a) Pold + w (d0 + d1 + d2)) / (1 + a), written over Pold.
__global__ void __launch_bounds__(256) time_kernel(const UnfusedParams p)
{
    const int qx = (p.nx + 3) / 4;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long rows = (long long)p.nz * p.ny;
    if (i >= rows * qx)
        return;
    const int x = (int)(i % qx) * 4;
    const long long row = i / qx;
    const int y = (int)(row % p.ny);
    const int z = (int)(row / p.ny);
    const long long at = row * p.px + x;
    const float4 P = *reinterpret_cast<const float4 *>(p.P + at);
    const float4 O = *reinterpret_cast<const float4 *>(p.Pold + at);
    const float4 W = *reinterpret_cast<const float4 *>(p.w + at);
    const float4 A = *reinterpret_cast<const float4 *>(p.d0 + at);
    const float4 C = *reinterpret_cast<const float4 *>(p.d2 + at);
    float4 B = make_float4(0.f, 0.f, 0.f, 0.f);
    if (p.d1)
        B = *reinterpret_cast<const float4 *>(p.d1 + at);
    float r[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float lap = (comp(A, e) + comp(B, e)) + comp(C, e);
        const float a = p.has_sponge ? p.ax[x + e] + p.ay[y] + p.az[z] : 0.f;
        const float num = fmaf(comp(W, e), lap, fmaf(2.0f, comp(P, e), -(1.0f - a) * comp(O, e)));
        r[e] = a != 0.0f ? __fdividef(num, 1.0f + a) : num;
    }
    float *dst = p.out + at;
    if (x + 3 < p.nx) {
        *reinterpret_cast<float4 *>(dst) = make_float4(r[0], r[1], r[2], r[3]);
    } else {
        for (int e = 0; e < 4 && x + e < p.nx; ++e)
            dst[e] = r[e];
    }
}

__global__ void add_source_kernel(float *Pn, long long at, float amp)
{
    Pn[at] += amp;
}

}  // namespace fdk

using namespace fdk;

static fd_status ensure_derivs(fd_model *m)
{
    const int naxes = m->d.ndim == 3 ? 3 : 2;
    for (int a = 0; a < 3; ++a) {
        if (a == 1 && naxes == 2)
            continue;
        if (!m->deriv[a]) {
            FD_CUDA(cudaMalloc((void **)&m->deriv[a], m->pitched * sizeof(float)), "derivative field");
            FD_CUDA(cudaMemsetAsync(m->deriv[a], 0, m->pitched * sizeof(float), m->stream), "derivative field");
        }
    }
    return FD_OK;
}

static UnfusedParams unfused_params(fd_model *m)
{
    float w4[4];
    fd_stencil_weights(w4);
    UnfusedParams p{};
    p.P = m->buf[m->cur];
    p.Pold = m->buf[m->cur ^ 1];
    p.w = m->w;
    p.ax = m->ax;
    p.ay = m->ay;
    p.az = m->az;
    p.nx = m->nx;
    p.ny = m->ny;
    p.nz = m->nz;
    p.px = m->px;
    p.has_sponge = m->has_sponge;
    p.c1 = w4[0];
    p.c2 = w4[1];
    p.c3 = w4[2];
    p.c4 = w4[3];
    return p;
}

// One 3D derivative routine through the step kernel's derivative mode: the haloed
// P ring of the fused step streams level n, and only sum_k c_k (P[+k] + P[-k] - 2P)
// along the axis is written, to deriv[axis].  x and z take their neighbours as
// the fused step does (from the ring plane and from the thread's z queue).  y
// runs as a z derivative over a view with y and z swapped (its tensor map and
// output strides permuted), so that it too marches with a register queue.
static cudaError_t launch_deriv3d(fd_model *m, int axis)
{
    if (axis == 1) {
        const uint64_t dims[3] = {(uint64_t)m->nx, (uint64_t)m->nz, (uint64_t)m->ny};
        const uint64_t strides[2] = {(uint64_t)m->ny * m->px * 4, (uint64_t)m->px * 4};
        const uint32_t halo[3] = {kTX3 + 8, kTY3 + 8, kPlanes3}, tile[3] = {kTX3, kTY3, kPlanes3};
        CUtensorMap tmP, tmT;
        if (!make_map_strided(&tmP, m->buf[m->cur], dims, strides, halo) ||
            !make_map_strided(&tmT, m->buf[m->cur ^ 1], dims, strides, tile))
            return cudaErrorInvalidValue;
        float w4[4];
        fd_stencil_weights(w4);
        StepParams p{};
        p.deriv_axis = 2;
        p.out = m->deriv[1];
        p.P = m->buf[m->cur];
        p.ax = m->ax;
        p.ay = m->ay;
        p.az = m->az;
        p.c1 = w4[0];
        p.c2 = w4[1];
        p.c3 = w4[2];
        p.c4 = w4[3];
        p.nx = m->nx;
        p.ny = m->nz;                 // the view's y is the grid's z
        p.nz = m->ny;                 // and its z (the march axis) the grid's y
        p.px = m->px;
        p.out_sy = (long long)m->ny * m->px;
        p.out_sz = m->px;
        p.err = m->d_err;
        int sms = 148;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
        const long long tiles = (long long)((m->nx + kTX3 - 1) / kTX3) * ((m->nz + kTY3 - 1) / kTY3);
        const long long slots = (long long)sms * step3d_blocks_per_sm();
        long long bz = (long long)m->ny * tiles / (6 * slots);
        bz = std::max(32LL, std::min<long long>(bz, m->ny));
        const int nchunks = (int)((m->ny + bz - 1) / bz);
        p.bz = (m->ny + nchunks - 1) / nchunks;
        return launch_step3d(tmP, tmT, tmT, p, nchunks, m->stream);
    }
    float w4[4];
    fd_stencil_weights(w4);
    StepParams p{};
    p.deriv_axis = axis;
    p.out = m->deriv[axis];
    p.P = m->buf[m->cur];
    p.ax = m->ax;
    p.ay = m->ay;
    p.az = m->az;
    p.c1 = w4[0];
    p.c2 = w4[1];
    p.c3 = w4[2];
    p.c4 = w4[3];
    p.nx = m->nx;
    p.ny = m->ny;
    p.nz = m->nz;
    p.px = m->px;
    p.bz = m->bz;
    p.err = m->d_err;
    const int c = m->cur;
    return launch_step3d(m->halo_map[c], m->tile_map[c ^ 1], m->w_map, p, m->nchunks, m->stream);
}

extern "C" fd_status fd_routine(fd_model *m, int routine)
{
    if (!m)
        return fail(FD_EINVAL, "NULL model");
    FD_CUDA(cudaSetDevice(m->device), "cudaSetDevice");
    if (routine < FD_ROUTINE_ADD_SOURCE || routine > FD_ROUTINE_SWAP ||
        (routine == FD_ROUTINE_PYY && m->d.ndim != 3))
        return fail(FD_EINVAL, "bad routine %d", routine);
    fd_status st = ensure_derivs(m);
    if (st)
        return st;
    UnfusedParams p = unfused_params(m);
    const long long threads = (long long)m->rows * ((m->nx + 3) / 4);
    const int blocks = (int)((threads + 255) / 256);
    cudaError_t e = cudaSuccess;
    switch (routine) {
    case FD_ROUTINE_PXX:
        if (m->d.ndim == 3) {
            e = launch_deriv3d(m, 0);
            break;
        }
        p.out = m->deriv[0];
        d2x_kernel<<<blocks, 256, 0, m->stream>>>(p);
        break;
    case FD_ROUTINE_PYY:
    case FD_ROUTINE_PZZ: {
        if (m->d.ndim == 3) {
            // the fused step's TMA ring, writing one axis's derivative only
            e = launch_deriv3d(m, routine == FD_ROUTINE_PYY ? 1 : 2);
            break;
        }
        const bool y = routine == FD_ROUTINE_PYY;
        p.out = m->deriv[y ? 1 : 2];
        const int qx = (m->nx + 3) / 4;
        const int extent = y ? m->ny : m->nz, tdim = y ? m->nz : m->ny;
        const dim3 block(32, 8);
        const dim3 grid(tdim == 1 ? (qx + 255) / 256 : (qx + 31) / 32, tdim == 1 ? 1 : (tdim + 7) / 8,
                        (extent + kMarchLen - 1) / kMarchLen);
        if (y)
            d2_march_kernel<1><<<grid, block, 0, m->stream>>>(p);
        else
            d2_march_kernel<2><<<grid, block, 0, m->stream>>>(p);
        break;
    }
    case FD_ROUTINE_TIME:
        p.out = m->buf[m->cur ^ 1];
        p.d0 = m->deriv[0];
        p.d1 = m->d.ndim == 3 ? m->deriv[1] : nullptr;
        p.d2 = m->deriv[2];
        time_kernel<<<blocks, 256, 0, m->stream>>>(p);
        break;
    case FD_ROUTINE_ADD_SOURCE:
        // into the level just written by the time routine (the Pold buffer)
        if (m->src_on && m->n < (int)m->amp.size())
            add_source_kernel<<<1, 1, 0, m->stream>>>(m->buf[m->cur ^ 1],
                                                     ((long long)m->sz * m->ny + m->sy) * m->px + m->sx,
                                                     m->amp[m->n]);
        else
            return FD_OK;
        break;
    case FD_ROUTINE_SWAP: {
        // receivers of the completed step, then the rotation Pold <- P, P <- Pn
        if (m->nrec > 0 && m->traces && m->n < m->trace_rows) {
            e = launch_gather(m->buf[m->cur ^ 1], m->d_rec, m->nrec, m->traces + (size_t)m->n * m->nrec,
                              m->stream);
            ++g_launches;
            if (e != cudaSuccess)
                return cuda_fail(e, "receiver gather");
        }
        m->cur ^= 1;
        ++m->n;
        m->pending_row = -1;
        return FD_OK;
    }
    default:
        break;
    }
    ++g_launches;
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "routine launch");
    return FD_OK;
}

extern "C" fd_status fd_step_unfused(fd_model *m, int nsteps)
{
    NvtxRange nvtx_range("fd_step_unfused");
    if (!m)
        return fail(FD_EINVAL, "NULL model");
    if (nsteps < 0)
        return fail(FD_EINVAL, "nsteps must be >= 0");
    if (m->pending_row >= 0) {
        // the fused path owes the gather of its last row: settle it first
        fd_status st = fd_step(m, 0);
        if (st)
            return st;
    }
    const int seq3[] = {FD_ROUTINE_PZZ, FD_ROUTINE_PXX, FD_ROUTINE_PYY, FD_ROUTINE_TIME, FD_ROUTINE_ADD_SOURCE,
                        FD_ROUTINE_SWAP};
    const int seq2[] = {FD_ROUTINE_PZZ, FD_ROUTINE_PXX, FD_ROUTINE_TIME, FD_ROUTINE_ADD_SOURCE, FD_ROUTINE_SWAP};
    for (int s = 0; s < nsteps; ++s) {
        if (m->d.ndim == 3) {
            for (int r : seq3) {
                fd_status st = fd_routine(m, r);
                if (st)
                    return st;
            }
        } else {
            for (int r : seq2) {
                fd_status st = fd_routine(m, r);
                if (st)
                    return st;
            }
        }
    }
    return FD_OK;
}
