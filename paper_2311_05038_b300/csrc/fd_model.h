// fd_model.h -- the model object behind the opaque fd_model handle of fd.h.
//
// It plays the role of the paper's WaveSimulator (section 7, Listing 3): it
// owns the two wavefield levels, w = (dt v / h)^2, the sponge profiles, the
// source signature, the receiver list and the trace buffer of one shot.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "fd.h"

struct fd_model {
    fd_grid_desc d{};
    int nx = 0, ny = 0, nz = 0, px = 0;
    size_t rows = 0;       // nz * ny
    size_t pitched = 0;    // rows * px elements per field
    size_t npts = 0;       // nz * ny * nx
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t handoff = nullptr;   // fd_set_stream: orders the new stream after the old one

    float *buf[2] = {nullptr, nullptr};   // the two wavefield levels
    int cur = 0;                          // buf[cur] = P, buf[cur ^ 1] = Pold
    float *w = nullptr;
    float *ax = nullptr, *ay = nullptr, *az = nullptr;
    int has_sponge = 0;
    float vmax = 0.f;
    double sponge_vref = 0.0;  // velocity fixing the sponge strength (0: the model's vmax)
    int *d_err = nullptr;
    unsigned *d_stats = nullptr;

    CUtensorMap halo_map[2];   // haloed P box over buf[i]
    CUtensorMap tile_map[2];   // unhaloed box over buf[i] (as Pold)
    CUtensorMap w_map;
    int nchunks = 1;           // 3D: CTAs along z
    int bz = 1;

    int src_on = 0, sx = 0, sy = 0, sz = 0;
    std::vector<float> amp;    // dt^2 S(t_n) / h^d
    float *d_amp = nullptr;    // device copy of amp (read by batched launches)
    int amp_cap = 0;

    int nrec = 0;
    int64_t *d_rec = nullptr;  // pitched indices (device)
    int rec_cap = 0;
    // receivers grouped by grid point, for a deterministic injection (no atomics):
    // point u is d_inj_pt[u] (pitched), its receivers d_inj_rec[d_inj_beg[u] .. d_inj_beg[u+1])
    int64_t *d_inj_pt = nullptr;
    int *d_inj_beg = nullptr;
    int *d_inj_rec = nullptr;
    int ninj = 0;
    std::vector<int64_t> rec_dense;

    float *traces = nullptr;
    int trace_rows = 0;
    bool traces_owned = false;
    size_t trace_cap = 0;      // floats in an owned trace buffer
    float *stage = nullptr;    // velocity staging, kept once fd_set_velocity is used

    int stall_stage = -1;     // fd_debug_stall_stage
    int n = 0;
    int pending_row = -1;      // receiver row whose gather is still owed

    float *deriv[3] = {nullptr, nullptr, nullptr};   // Pxx, Pyy, Pzz of the unfused routines

    // Two steps per launch (fd_set_time_fusion, 3D): the launch writes both new
    // levels into two more buffers, which then trade places with buf[] (pointers
    // and tensor maps together).
    int tfuse = 1;
    float *xbuf[2] = {nullptr, nullptr};
    CUtensorMap xhalo_map[2], xtile_map[2];   // single-step maps over xbuf[i]
    CUtensorMap t2p1_map[2], t2e_map[2];      // fused-step maps over buf[i]: 48x48x1 and 40x40x1 boxes
    CUtensorMap xt2p1_map[2], xt2e_map[2];    // ... over xbuf[i]
    CUtensorMap t2w_map;                      // 40x40x1 box over w
    int t2_nchunks = 1, t2_bz = 1;
};
