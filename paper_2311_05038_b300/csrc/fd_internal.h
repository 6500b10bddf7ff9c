// fd_internal.h -- parameters and launchers shared by the host API and the kernels.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "fd.h"

namespace fdk {

constexpr int kRadius = 4;

// 3D step: a CTA owns a kTX3 x kTY3 column of the (x, y) plane and marches
// along z through bz planes, fed by two TMA rings in shared memory whose
// stages hold kPlanes3 consecutive planes each.
// Compile-time knobs (defaults are the tuned configuration).
#ifndef FD_TX3
#define FD_TX3 32
#endif
#ifndef FD_TY3
#define FD_TY3 16
#endif
#ifndef FD_STAGESP3
#define FD_STAGESP3 5
#endif
#ifndef FD_STAGEST3
#define FD_STAGEST3 2
#endif
#ifndef FD_QGROUP3
#define FD_QGROUP3 2
#endif
#ifndef FD_MINB3
#define FD_MINB3 4
#endif
constexpr int kTX3 = FD_TX3;
constexpr int kTY3 = FD_TY3;
constexpr int kPlanes3 = 2;              // z planes per TMA stage (the box depth)
constexpr int kStagesP3 = FD_STAGESP3;   // haloed P stages in flight
constexpr int kStagesT3 = FD_STAGEST3;   // Pold + w stages in flight
constexpr int kGroup3 = FD_QGROUP3;      // stages per unrolled z-queue rotation
constexpr int kMinBlocks3 = FD_MINB3;
constexpr int kThreads3 = kTX3 / 4 * kTY3;

// 2D step: a CTA owns a column of kZT2 tiles of kTX2 x kTZ2 points stacked along
// z (one tile when the grid would give fewer than kStackMinCtas2 such columns).
constexpr int kTX2 = 64;
constexpr int kTZ2 = 16;
constexpr int kZT2 = 8;
constexpr int kStackMinCtas2 = 4096;
constexpr int kThreads2 = kTX2 / 4 * kTZ2;

// Codes a kernel writes into the model's device error word.
constexpr int kDevErrTimeout = 1;

// Everything one time step needs besides the three tensor maps.
struct StepParams {
    float *out;               // Pn destination: the Pold buffer, pitched
    const float *P;           // level n, pitched (read by the receiver gather)
    const float *ax;          // damping a = dt * eta along x (px entries, 0 past nx)
    const float *ay;          // ... along y (ny entries)
    const float *az;          // ... along z (nz entries)
    float c1, c2, c3, c4;     // stencil weights
    int nx, ny, nz, px;       // extents and x pitch (elements)
    int bz;                   // z planes per CTA (3D)
    int has_sponge;
    int src_on, sx, sy, sz;   // source point, active this step if src_on
    float src_amp;            // dt^2 S(t_n) / h^d
    const int64_t *rec_idx;   // receivers' pitched linear indices
    int nrec;
    float *trace_prev;        // if set: trace_prev[r] = P[rec_idx[r]] (previous step's row)
    float *lp_out;            // if set (the *_lp launches): L'P of level n, dense [nz][ny][nx]
    const float *img_lp;      // if set (adjoint imaging launches): img_grad += Pn * img_lp,
    float *img_grad;          //   both dense [nz][ny][nx]
    int *err;                 // device error word
    int stall_stage = -1;     // test hook: CTA (0, 0) of the 3D step never issues this P stage (-1: none)
    int deriv_axis = -1;      // 0, 1, 2: write only the x / y / z second derivative of P to out (3D)
    long long out_sy = 0;     // derivative modes: element strides of out along the kernel's y and z
    long long out_sz = 0;     //   (0: the layout of P, px and ny * px)
};

// Two fused time steps per launch (3D): a CTA of kT2Threads threads owns a 32 x 32
// column and marches along z through bz planes.
constexpr int kT2Threads = 416;

struct T2Params {
    float *out2, *out3;       // P^{n+1} and P^{n+2} destinations (pitched; neither input buffer)
    const float *P0, *P1;     // levels n-1 and n (pitched; read by the receiver gathers)
    const float *ax, *ay, *az;
    float c1, c2, c3, c4;
    int nx, ny, nz, px;
    int bz;
    int has_sponge;
    int src_on0, src_on1, sx, sy, sz;   // source active in the first / second step
    float amp0, amp1;                   // its amplitudes dt^2 S(t_n) / h^3, dt^2 S(t_{n+1}) / h^3
    const int64_t *rec_idx;
    int nrec;
    float *trace_prev0;       // if set: trace_prev0[r] = P0[rec_idx[r]] (row owed for level n-1)
    float *trace_prev1;       // if set: trace_prev1[r] = P1[rec_idx[r]] (row owed for level n)
    int *err;
};

size_t step3d_t2_smem_bytes();
cudaError_t step3d_t2_prepare();
// tmP1: box 48 x 48 x 1 over level n; tmP0: box 40 x 40 x 1 over level n-1; tmW: 40 x 40 x 1 over w.
cudaError_t launch_step3d_t2(const CUtensorMap &tmP1, const CUtensorMap &tmP0, const CUtensorMap &tmW,
                             const T2Params &p, int nchunks, cudaStream_t s);

// One time step of up to kWide3Max 3D models in one launch (the batched 3D
// schedule): per model its three tensor maps and step parameters, its first CTA
// (cta_begin[nmodels] = total CTAs) and its CTAs per z chunk.
constexpr int kWide3Max = 48;
struct Wide3Params {
    CUtensorMap tmP[kWide3Max];
    CUtensorMap tmOld[kWide3Max];
    CUtensorMap tmW[kWide3Max];
    StepParams prm[kWide3Max];
    int cta_begin[kWide3Max + 1];
    int tiles[kWide3Max];
    int nmodels;
};
cudaError_t launch_wide3d(const Wide3Params &w, cudaStream_t s);
// The step parameters of one plain time step of model m at its current state
// (levels, step counter, source amplitude, owed receiver row).
void fill_step_params(fd_model *m, StepParams &p);

size_t step3d_smem_bytes();
cudaError_t step3d_prepare();
int step3d_blocks_per_sm();
// With p.lp_out set, the launch also writes the stencil sum L'P of level n; with
// p.img_grad set, it also adds Pn * p.img_lp to p.img_grad (the imaging condition).
cudaError_t launch_step3d(const CUtensorMap &tmP, const CUtensorMap &tmOld, const CUtensorMap &tmW,
                          const StepParams &p, int nchunks, cudaStream_t s);
cudaError_t launch_step2d(const CUtensorMap &tmP, const CUtensorMap &tmOld, const CUtensorMap &tmW,
                          const StepParams &p, cudaStream_t s);
cudaError_t launch_gather(const float *P, const int64_t *idx, int nrec, float *out, cudaStream_t s);
// Over the nx valid columns of a pitched [rows][px] velocity: stats[0] |= bit
// pattern of the largest finite positive value, stats[1] += count of entries
// that are not finite and positive.  stats must start at zero.
cudaError_t launch_velocity_stats(const float *v, int nx, size_t rows, int px, unsigned *stats,
                                  cudaStream_t s);
// w = (dt/h * v)^2 rounded to FP32 over the pitched layout (v may alias w).
cudaError_t launch_compute_w(const float *v, float *w, int nx, size_t rows, int px, double dt_over_h,
                             cudaStream_t s);

// Host helpers shared by the C ABI translation units.
// FP32 tensor map over a pitched field: rank 2 ([nz][px], extents nx, nz) or
// rank 3 ([nz][ny][px], extents nx, ny, nz), with box bx x by (x bz planes).
bool make_map(CUtensorMap *map, float *base, int ndim, int nx, int ny, int nz, int px, int bx, int by,
              int bz = 1);
// Rank-3 FP32 tensor map with explicit extents (x fastest), byte strides of the
// two outer dimensions (multiples of 16) and box.
bool make_map_strided(CUtensorMap *map, float *base, const uint64_t (&dims)[3], const uint64_t (&strides)[2],
                      const uint32_t (&box)[3]);
// Record a message for fd_last_error() and return st.
fd_status fail(fd_status st, const char *fmt, ...);
fd_status cuda_fail(cudaError_t e, const char *what);
extern std::atomic<uint64_t> g_launches;

// Return the fd_status of a failed CUDA call from the enclosing entry point.
#define FD_CUDA(call, what)                    \
    do {                                       \
        cudaError_t e_ = (call);               \
        if (e_ != cudaSuccess)                 \
            return fdk::cuda_fail(e_, what);   \
    } while (0)

}  // namespace fdk
