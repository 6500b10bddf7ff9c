// fd_api.cu -- host side of the C ABI declared in include/fd.h.
//
// The model object plays the role of the paper's WaveSimulator (section 7,
// Listing 3): it owns the wavefields P and Pold, the velocity-derived w and the
// time step, and its fd_step() runs the routine sequence of run() -- here one
// fused kernel launch per time step, followed by the pointer swaps.  Inputs
// enter only through copying calls and outputs leave only through gather
// calls, the start/stop convention of section 5.
//
// Device layout: every field is [nz][ny][px] FP32 with a row pitch px = nx
// rounded up to 32 elements (128-byte rows, as TMA needs 16-byte strides).
// Columns past nx are never read by the stencil (the tensor maps stop at nx and
// zero-fill beyond), so the pitch is invisible to callers.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "fd.h"
#include "fd_internal.h"
#include "fd_model.h"
#include "fd_trace.h"

using namespace fdk;

// ------------------------------------------------------------------ errors & stats

static thread_local std::string g_last_error;
std::atomic<uint64_t> fdk::g_launches{0};

fd_status fdk::fail(fd_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

fd_status fdk::cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(FD_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(FD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}


// --------------------------------------------------------------- stencil weights

// Weights of the radius-4 centred second difference from Fornberg's closed
// form c_k = 2 (-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!), evaluated in FP64.
static double weight(int k)
{
    const int r = kRadius;
    double f[2 * kRadius + 1];
    f[0] = 1.0;
    for (int i = 1; i <= 2 * r; ++i)
        f[i] = f[i - 1] * i;
    const double sign = (k % 2 == 1) ? 1.0 : -1.0;
    return 2.0 * sign * f[r] * f[r] / ((double)k * k * f[r - k] * f[r + k]);
}

extern "C" double fd_cfl_limit(int ndim)
{
    if (ndim != 2 && ndim != 3)
        return -1.0;
    // lambda_1 = -(c_0 + 2 sum_k (-1)^k c_k) with c_0 = -2 sum_k c_k
    double sum = 0.0, alt = 0.0;
    for (int k = 1; k <= kRadius; ++k) {
        sum += weight(k);
        alt += ((k % 2) ? -1.0 : 1.0) * weight(k);
    }
    const double lambda1 = -(-2.0 * sum + 2.0 * alt);
    return 2.0 / std::sqrt(ndim * lambda1);
}

extern "C" fd_status fd_stencil_weights(float *out4)
{
    if (!out4)
        return fail(FD_EINVAL, "fd_stencil_weights: NULL output");
    for (int k = 1; k <= kRadius; ++k)
        out4[k - 1] = (float)weight(k);
    return FD_OK;
}

// ------------------------------------------------------------------ tensor maps

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// FP32 tensor map over a pitched field: rank 2 ([nz][px], extents nx, nz) or
// rank 3 ([nz][ny][px], extents nx, ny, nz), with the given box.
bool fdk::make_map(CUtensorMap *map, float *base, int ndim, int nx, int ny, int nz, int px, int bx, int by,
                   int bz)
{
    auto fn = encode_fn();
    if (!fn)
        return false;
    cuuint64_t dims[3];
    cuuint64_t strides[2];
    cuuint32_t box[3];
    cuuint32_t estr[3] = {1, 1, 1};
    cuuint32_t rank;
    if (ndim == 2) {
        rank = 2;
        dims[0] = nx;
        dims[1] = nz;
        strides[0] = (cuuint64_t)px * 4;
        box[0] = bx;
        box[1] = by;
    } else {
        rank = 3;
        dims[0] = nx;
        dims[1] = ny;
        dims[2] = nz;
        strides[0] = (cuuint64_t)px * 4;
        strides[1] = (cuuint64_t)px * ny * 4;
        box[0] = bx;
        box[1] = by;
        box[2] = bz;
    }
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// A rank-3 FP32 tensor map with explicit extents (x fastest) and byte strides of
// the two outer dimensions, for views whose outer axes are permuted.
bool fdk::make_map_strided(CUtensorMap *map, float *base, const uint64_t (&dims)[3], const uint64_t (&strides)[2],
                           const uint32_t (&box)[3])
{
    auto fn = encode_fn();
    if (!fn)
        return false;
    cuuint64_t d[3] = {dims[0], dims[1], dims[2]};
    cuuint64_t st[2] = {strides[0], strides[1]};
    cuuint32_t b[3] = {box[0], box[1], box[2]};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, d, st, b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ------------------------------------------------------------------------ model

static fd_status validate_desc(const fd_grid_desc *d)
{
    if (!d)
        return fail(FD_EINVAL, "NULL grid descriptor");
    if (d->ndim != 2 && d->ndim != 3)
        return fail(FD_EINVAL, "ndim must be 2 or 3 (got %d)", d->ndim);
    if (d->nx < 1 || d->ny < 1 || d->nz < 1)
        return fail(FD_EINVAL, "grid extents must be >= 1 (got %d x %d x %d)", d->nx, d->ny, d->nz);
    if (d->ndim == 2 && d->ny != 1)
        return fail(FD_EINVAL, "2D grids need ny == 1 (got %d)", d->ny);
    if (!(d->h > 0.0) || !std::isfinite(d->h) || !(d->dt > 0.0) || !std::isfinite(d->dt))
        return fail(FD_EINVAL, "h and dt must be positive and finite");
    if (d->sponge_width < 0)
        return fail(FD_EINVAL, "sponge_width must be >= 0");
    if (d->sponge_width > 0 && !(d->sponge_R > 0.0 && d->sponge_R < 1.0))
        return fail(FD_EINVAL, "sponge_R must lie in (0, 1)");
    const double npts = (double)d->nx * d->ny * d->nz;
    if (npts > 4.0e10)
        return fail(FD_EINVAL, "grid of %.3g points is too large", npts);
    return FD_OK;
}

// Damping profiles are allocated with zero padding past the grid, so that tile
// slices (up to 128 entries from a tile origin) can be copied without bounds checks.
static size_t profile_floats(int n)
{
    return ((size_t)n + 127) / 128 * 128 + 128;
}

// Per-axis damping a_i = dt * eta_max * (d_i / W)^2, d_i = max(W - i, i - (n-1-W), 0).
static std::vector<float> damping_profile(int n, int len, int W, double eta_max, double dt)
{
    std::vector<float> a(len, 0.f);
    if (W <= 0)
        return a;
    for (int i = 0; i < n; ++i) {
        const int d = std::max(std::max(W - i, i - (n - 1 - W)), 0);
        const double r = (double)d / W;
        a[i] = (float)(dt * eta_max * r * r);
    }
    return a;
}

static void free_model(fd_model *m)
{
    if (!m)
        return;
    cudaFree(m->buf[0]);
    cudaFree(m->buf[1]);
    cudaFree(m->w);
    cudaFree(m->ax);
    cudaFree(m->ay);
    cudaFree(m->az);
    cudaFree(m->d_err);
    cudaFree(m->d_stats);
    cudaFree(m->d_rec);
    cudaFree(m->d_inj_pt);
    cudaFree(m->d_inj_beg);
    cudaFree(m->d_inj_rec);
    cudaFree(m->d_amp);
    cudaFree(m->stage);
    for (float *d : m->deriv)
        cudaFree(d);
    cudaFree(m->xbuf[0]);
    cudaFree(m->xbuf[1]);
    if (m->traces_owned)
        cudaFree(m->traces);
    if (m->handoff)
        cudaEventDestroy(m->handoff);
    delete m;
}

// Damping profiles a = dt * eta per axis from the sponge strength of the model
// (its largest velocity, or the velocity fixed by fd_set_sponge_vmax).
static fd_status upload_damping(fd_model *m)
{
    const int W = m->d.sponge_width;
    m->has_sponge = W > 0;
    const double vref = m->sponge_vref > 0.0 ? m->sponge_vref : (double)m->vmax;
    const double eta_max = W > 0 ? 3.0 * vref * std::log(1.0 / m->d.sponge_R) / (2.0 * W * m->d.h) : 0.0;
    auto pax = damping_profile(m->nx, m->px, W, eta_max, m->d.dt);
    auto pay = damping_profile(m->ny, m->ny, m->d.ndim == 3 ? W : 0, eta_max, m->d.dt);
    auto paz = damping_profile(m->nz, m->nz, W, eta_max, m->d.dt);
    FD_CUDA(cudaMemcpyAsync(m->ax, pax.data(), pax.size() * 4, cudaMemcpyHostToDevice, m->stream), "sponge x");
    FD_CUDA(cudaMemcpyAsync(m->ay, pay.data(), pay.size() * 4, cudaMemcpyHostToDevice, m->stream), "sponge y");
    FD_CUDA(cudaMemcpyAsync(m->az, paz.data(), paz.size() * 4, cudaMemcpyHostToDevice, m->stream), "sponge z");
    FD_CUDA(cudaStreamSynchronize(m->stream), "velocity setup");
    return FD_OK;
}

// Load a dense velocity (host or device) into a staging copy, check it, and on
// success turn it into w and the sponge profiles.  Leaves the model untouched
// on failure.
static fd_status load_velocity(fd_model *m, const float *v, cudaMemcpyKind kind)
{
    NvtxRange nvtx_range("load_velocity");
    if (!v)
        return fail(FD_EINVAL, "NULL velocity");
    if (!m->stage)
        FD_CUDA(cudaMalloc((void **)&m->stage, m->pitched * sizeof(float)), "staging allocation");
    float *stage = m->stage;
    cudaError_t e = cudaMemcpy2DAsync(stage, (size_t)m->px * 4, v, (size_t)m->nx * 4, (size_t)m->nx * 4, m->rows,
                                      kind, m->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(m->d_stats, 0, 2 * sizeof(unsigned), m->stream);
    if (e == cudaSuccess) {
        e = launch_velocity_stats(stage, m->nx, m->rows, m->px, m->d_stats, m->stream);
        ++g_launches;
    }
    unsigned stats[2] = {0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(stats, m->d_stats, sizeof stats, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        return cuda_fail(e, "velocity upload");
    }
    if (stats[1] != 0) {
        return fail(FD_EINVAL, "velocity has %u entries that are not finite and positive", stats[1]);
    }
    float vmax;
    std::memcpy(&vmax, &stats[0], sizeof vmax);
    const double courant = (double)vmax * m->d.dt / m->d.h;
    const double lim = fd_cfl_limit(m->d.ndim);
    if (courant > lim) {
        return fail(FD_ECFL, "Courant number v_max dt / h = %.6g exceeds the stability limit %.6g", courant, lim);
    }
    e = launch_compute_w(stage, m->w, m->nx, m->rows, m->px, m->d.dt / m->d.h, m->stream);
    ++g_launches;
    if (e != cudaSuccess) {
        return cuda_fail(e, "computing w");
    }
    m->vmax = vmax;
    return upload_damping(m);
}

static fd_status create(const fd_grid_desc *desc, const float *v, cudaMemcpyKind kind, void *stream,
                        fd_model **out)
{
    if (!out)
        return fail(FD_EINVAL, "NULL output pointer");
    *out = nullptr;
    fd_status st = validate_desc(desc);
    if (st)
        return st;
    if (!v)
        return fail(FD_EINVAL, "NULL velocity");
    if (kind == cudaMemcpyHostToDevice) {
        // Host input: reject a bad model or an unstable time step before
        // touching the device (the device-side check repeats this).
        const size_t n = (size_t)desc->nx * desc->ny * desc->nz;
        float vmax = 0.f;
        size_t bad = 0;
        for (size_t i = 0; i < n; ++i) {
            const float x = v[i];
            if (std::isfinite(x) && x > 0.f)
                vmax = std::max(vmax, x);
            else
                ++bad;
        }
        if (bad)
            return fail(FD_EINVAL, "velocity has %zu entries that are not finite and positive", bad);
        const double courant = (double)vmax * desc->dt / desc->h;
        if (courant > fd_cfl_limit(desc->ndim))
            return fail(FD_ECFL, "Courant number v_max dt / h = %.6g exceeds the stability limit %.6g", courant,
                        fd_cfl_limit(desc->ndim));
    }

    fd_model *m = new fd_model();
    m->d = *desc;
    m->nx = desc->nx;
    m->ny = desc->ny;
    m->nz = desc->nz;
    m->px = (desc->nx + 31) / 32 * 32;
    m->rows = (size_t)m->nz * m->ny;
    m->pitched = m->rows * m->px;
    m->npts = m->rows * m->nx;
    m->stream = static_cast<cudaStream_t>(stream);

    auto bail = [&](fd_status s) {
        free_model(m);
        return s;
    };
    cudaError_t e = cudaGetDevice(&m->device);
    if (e != cudaSuccess)
        return bail(cuda_fail(e, "cudaGetDevice"));
    const size_t bytes = m->pitched * sizeof(float);
    if ((e = cudaMalloc((void **)&m->buf[0], bytes)) != cudaSuccess ||
        (e = cudaMalloc((void **)&m->buf[1], bytes)) != cudaSuccess ||
        (e = cudaMalloc((void **)&m->w, bytes)) != cudaSuccess ||
        (e = cudaMalloc((void **)&m->ax, profile_floats(m->px) * 4)) != cudaSuccess ||
        (e = cudaMalloc((void **)&m->ay, profile_floats(m->ny) * 4)) != cudaSuccess ||
        (e = cudaMalloc((void **)&m->az, profile_floats(m->nz) * 4)) != cudaSuccess ||
        (e = cudaMemsetAsync(m->ax, 0, profile_floats(m->px) * 4, m->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(m->ay, 0, profile_floats(m->ny) * 4, m->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(m->az, 0, profile_floats(m->nz) * 4, m->stream)) != cudaSuccess ||
        (e = cudaMalloc((void **)&m->d_err, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc((void **)&m->d_stats, 2 * sizeof(unsigned))) != cudaSuccess)
        return bail(cuda_fail(e, "device allocation"));
    if ((e = cudaMemsetAsync(m->buf[0], 0, bytes, m->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(m->buf[1], 0, bytes, m->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(m->w, 0, bytes, m->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(m->d_err, 0, sizeof(int), m->stream)) != cudaSuccess)
        return bail(cuda_fail(e, "device memset"));

    st = load_velocity(m, v, kind);
    if (st)
        return bail(st);
    // the staging copy is kept only by models whose velocity is replaced later
    cudaFree(m->stage);
    m->stage = nullptr;

    const int ndim = desc->ndim;
    bool ok = true;
    for (int i = 0; i < 2; ++i) {
        if (ndim == 3) {
            ok = ok && make_map(&m->halo_map[i], m->buf[i], 3, m->nx, m->ny, m->nz, m->px, kTX3 + 8, kTY3 + 8,
                                kPlanes3);
            ok = ok && make_map(&m->tile_map[i], m->buf[i], 3, m->nx, m->ny, m->nz, m->px, kTX3, kTY3, kPlanes3);
        } else {
            ok = ok && make_map(&m->halo_map[i], m->buf[i], 2, m->nx, 1, m->nz, m->px, kTX2 + 8, kTZ2 + 8);
            ok = ok && make_map(&m->tile_map[i], m->buf[i], 2, m->nx, 1, m->nz, m->px, kTX2, kTZ2);
        }
    }
    ok = ok && (ndim == 3 ? make_map(&m->w_map, m->w, 3, m->nx, m->ny, m->nz, m->px, kTX3, kTY3, kPlanes3)
                          : make_map(&m->w_map, m->w, 2, m->nx, 1, m->nz, m->px, kTX2, kTZ2));
    if (!ok)
        return bail(fail(FD_ECUDA, "cuTensorMapEncodeTiled failed"));

    if (ndim == 3) {
        if ((e = step3d_prepare()) != cudaSuccess)
            return bail(cuda_fail(e, "kernel attributes"));
        int sms = 148;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
        const long long tiles = (long long)((m->nx + kTX3 - 1) / kTX3) * ((m->ny + kTY3 - 1) / kTY3);
        const long long slots = (long long)sms * step3d_blocks_per_sm();
        // About six waves of CTAs, each marching at least 32 planes; grids whose
        // three fields fit in L2 may use chunks down to 8 planes (the extra halo
        // planes are re-read from L2), so that small shots still fill the GPU.
        const bool l2_resident = 3.0 * m->pitched * sizeof(float) <= 96.0 * 1048576.0;
        const long long bz_min = l2_resident ? 8 : 32;
        long long bz = (long long)m->nz * tiles / (6 * slots);
        bz = std::max(bz_min, std::min<long long>(bz, m->nz));
        m->nchunks = (int)((m->nz + bz - 1) / bz);
        m->bz = (m->nz + m->nchunks - 1) / m->nchunks;
    }
    *out = m;
    return FD_OK;
}

extern "C" fd_status fd_model_create(const fd_grid_desc *desc, const float *v_host, void *stream, fd_model **out)
{
    return create(desc, v_host, cudaMemcpyHostToDevice, stream, out);
}

extern "C" fd_status fd_model_create_dev(const fd_grid_desc *desc, const float *v_dev, void *stream,
                                         fd_model **out)
{
    return create(desc, v_dev, cudaMemcpyDeviceToDevice, stream, out);
}

extern "C" fd_status fd_model_destroy(fd_model *m)
{
    if (!m)
        return FD_OK;
    cudaSetDevice(m->device);
    cudaStreamSynchronize(m->stream);
    free_model(m);
    return FD_OK;
}

#define NEED_MODEL(m)                                              \
    do {                                                           \
        if (!(m))                                                  \
            return fail(FD_EINVAL, "NULL model");                  \
        cudaError_t e_ = cudaSetDevice((m)->device);               \
        if (e_ != cudaSuccess)                                     \
            return cuda_fail(e_, "cudaSetDevice");                 \
    } while (0)

extern "C" fd_status fd_set_velocity(fd_model *m, const float *v_host)
{
    NEED_MODEL(m);
    return load_velocity(m, v_host, cudaMemcpyHostToDevice);
}

extern "C" fd_status fd_set_velocity_dev(fd_model *m, const float *v_dev)
{
    NEED_MODEL(m);
    return load_velocity(m, v_dev, cudaMemcpyDeviceToDevice);
}

extern "C" fd_status fd_set_sponge_vmax(fd_model *m, double vmax)
{
    NEED_MODEL(m);
    if (!(vmax >= 0.0) || !std::isfinite(vmax))
        return fail(FD_EINVAL, "sponge velocity must be finite and >= 0");
    m->sponge_vref = vmax;
    return upload_damping(m);
}

static bool inside(const fd_model *m, int ix, int iy, int iz)
{
    return ix >= 0 && ix < m->nx && iy >= 0 && iy < m->ny && iz >= 0 && iz < m->nz;
}

extern "C" fd_status fd_set_source(fd_model *m, int ix, int iy, int iz, const float *wavelet_host, int nt)
{
    NEED_MODEL(m);
    if (nt < 0)
        return fail(FD_EINVAL, "nt must be >= 0");
    if (m->d.ndim == 2)
        iy = 0;
    if (nt == 0 || !wavelet_host) {
        m->src_on = 0;
        m->amp.clear();
        return FD_OK;
    }
    if (!inside(m, ix, iy, iz))
        return fail(FD_ERANGE, "source (%d, %d, %d) outside the %d x %d x %d grid", ix, iy, iz, m->nx, m->ny, m->nz);
    const double hd = m->d.ndim == 3 ? m->d.h * m->d.h * m->d.h : m->d.h * m->d.h;
    std::vector<float> amp(nt);
    for (int i = 0; i < nt; ++i)
        amp[i] = (float)(m->d.dt * m->d.dt * (double)wavelet_host[i] / hd);
    if (nt > m->amp_cap) {
        float *p = nullptr;
        FD_CUDA(cudaMalloc((void **)&p, (size_t)nt * sizeof(float)), "source allocation");
        cudaStreamSynchronize(m->stream);
        cudaFree(m->d_amp);
        m->d_amp = p;
        m->amp_cap = nt;
    }
    FD_CUDA(cudaMemcpyAsync(m->d_amp, amp.data(), (size_t)nt * sizeof(float), cudaMemcpyHostToDevice, m->stream),
            "source upload");
    FD_CUDA(cudaStreamSynchronize(m->stream), "source upload");
    m->amp.swap(amp);
    m->src_on = 1;
    m->sx = ix;
    m->sy = iy;
    m->sz = iz;
    return FD_OK;
}

extern "C" fd_status fd_set_receivers(fd_model *m, const int *xyz_host, int nrec)
{
    NEED_MODEL(m);
    if (nrec < 0 || (nrec > 0 && !xyz_host))
        return fail(FD_EINVAL, "bad receiver list");
    std::vector<int64_t> pit(nrec), dense(nrec);
    for (int r = 0; r < nrec; ++r) {
        const int ix = xyz_host[3 * r], iy = m->d.ndim == 3 ? xyz_host[3 * r + 1] : 0, iz = xyz_host[3 * r + 2];
        if (!inside(m, ix, iy, iz))
            return fail(FD_ERANGE, "receiver %d at (%d, %d, %d) outside the grid", r, ix, iy, iz);
        pit[r] = ((int64_t)iz * m->ny + iy) * m->px + ix;
        dense[r] = ((int64_t)iz * m->ny + iy) * m->nx + ix;
    }
    // receivers grouped by grid point (points ascending, receivers ascending within one)
    std::vector<int> order(nrec);
    for (int r = 0; r < nrec; ++r)
        order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pit[a] < pit[b]; });
    std::vector<int64_t> upt;
    std::vector<int> ubeg;
    for (int j = 0; j < nrec; ++j) {
        if (j == 0 || pit[order[j]] != pit[order[j - 1]]) {
            upt.push_back(pit[order[j]]);
            ubeg.push_back(j);
        }
    }
    ubeg.push_back(nrec);
    if (nrec > m->rec_cap) {
        int64_t *p = nullptr, *q = nullptr;
        int *b = nullptr, *o = nullptr;
        cudaError_t e = cudaMalloc((void **)&p, (size_t)nrec * sizeof(int64_t));
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&q, (size_t)nrec * sizeof(int64_t));
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&b, (size_t)(nrec + 1) * sizeof(int));
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&o, (size_t)nrec * sizeof(int));
        if (e != cudaSuccess) {
            cudaFree(p);
            cudaFree(q);
            cudaFree(b);
            cudaFree(o);
            return cuda_fail(e, "receiver allocation");
        }
        cudaStreamSynchronize(m->stream);
        cudaFree(m->d_rec);
        cudaFree(m->d_inj_pt);
        cudaFree(m->d_inj_beg);
        cudaFree(m->d_inj_rec);
        m->d_rec = p;
        m->d_inj_pt = q;
        m->d_inj_beg = b;
        m->d_inj_rec = o;
        m->rec_cap = nrec;
    }
    if (nrec > 0) {
        FD_CUDA(cudaMemcpyAsync(m->d_rec, pit.data(), (size_t)nrec * sizeof(int64_t), cudaMemcpyHostToDevice,
                                m->stream),
                "receiver upload");
        FD_CUDA(cudaMemcpyAsync(m->d_inj_pt, upt.data(), upt.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                m->stream),
                "receiver upload");
        FD_CUDA(cudaMemcpyAsync(m->d_inj_beg, ubeg.data(), ubeg.size() * sizeof(int), cudaMemcpyHostToDevice,
                                m->stream),
                "receiver upload");
        FD_CUDA(cudaMemcpyAsync(m->d_inj_rec, order.data(), (size_t)nrec * sizeof(int), cudaMemcpyHostToDevice,
                                m->stream),
                "receiver upload");
    }
    FD_CUDA(cudaStreamSynchronize(m->stream), "receiver upload");
    m->ninj = (int)upt.size();
    if (nrec != m->nrec) {
        // the trace layout changed: a caller buffer no longer fits, an owned one is re-laid out
        if (!m->traces_owned)
            m->traces = nullptr;
        m->trace_rows = 0;
    }
    m->nrec = nrec;
    m->rec_dense.swap(dense);
    m->pending_row = -1;
    return FD_OK;
}

extern "C" fd_status fd_set_trace_buffer(fd_model *m, float *traces_dev, int nt_rows)
{
    NEED_MODEL(m);
    if (nt_rows < 0)
        return fail(FD_EINVAL, "nt_rows must be >= 0");
    const size_t need = (size_t)nt_rows * m->nrec;
    m->pending_row = -1;
    m->trace_rows = 0;
    if (traces_dev || need == 0) {
        if (m->traces_owned) {
            cudaStreamSynchronize(m->stream);
            cudaFree(m->traces);
            m->traces_owned = false;
            m->trace_cap = 0;
        }
        m->traces = traces_dev;
    } else if (!m->traces_owned || m->trace_cap < need) {
        if (m->traces_owned) {
            cudaStreamSynchronize(m->stream);
            cudaFree(m->traces);
        }
        m->traces = nullptr;
        m->traces_owned = false;
        m->trace_cap = 0;
        FD_CUDA(cudaMalloc((void **)&m->traces, need * sizeof(float)), "trace allocation");
        m->traces_owned = true;
        m->trace_cap = need;
    }
    if (need > 0 && m->traces)
        FD_CUDA(cudaMemsetAsync(m->traces, 0, need * sizeof(float), m->stream), "trace clear");
    m->trace_rows = nt_rows;
    return FD_OK;
}

extern "C" fd_status fd_reset(fd_model *m)
{
    NEED_MODEL(m);
    const size_t bytes = m->pitched * sizeof(float);
    FD_CUDA(cudaMemsetAsync(m->buf[0], 0, bytes, m->stream), "reset");
    FD_CUDA(cudaMemsetAsync(m->buf[1], 0, bytes, m->stream), "reset");
    m->n = 0;
    m->pending_row = -1;
    return FD_OK;
}

extern "C" fd_status fd_set_wavefield(fd_model *m, const float *p_host, const float *pold_host, int n)
{
    NEED_MODEL(m);
    if (!p_host || !pold_host || n < 0)
        return fail(FD_EINVAL, "bad wavefield arguments");
    const size_t wb = (size_t)m->nx * 4, pb = (size_t)m->px * 4;
    FD_CUDA(cudaMemcpy2DAsync(m->buf[m->cur], pb, p_host, wb, wb, m->rows, cudaMemcpyHostToDevice, m->stream),
            "wavefield upload");
    FD_CUDA(cudaMemcpy2DAsync(m->buf[m->cur ^ 1], pb, pold_host, wb, wb, m->rows, cudaMemcpyHostToDevice,
                              m->stream),
            "wavefield upload");
    FD_CUDA(cudaStreamSynchronize(m->stream), "wavefield upload");
    m->n = n;
    m->pending_row = -1;
    return FD_OK;
}

static fd_status flush_pending(fd_model *m)
{
    if (m->pending_row < 0)
        return FD_OK;
    cudaError_t e = launch_gather(m->buf[m->cur], m->d_rec, m->nrec, m->traces + (size_t)m->pending_row * m->nrec,
                                  m->stream);
    ++g_launches;
    m->pending_row = -1;
    if (e != cudaSuccess)
        return cuda_fail(e, "receiver gather");
    return FD_OK;
}

void fdk::fill_step_params(fd_model *m, StepParams &p)
{
    float w4[4];
    fd_stencil_weights(w4);
    p = StepParams{};
    p.stall_stage = m->stall_stage;
    p.c1 = w4[0];
    p.c2 = w4[1];
    p.c3 = w4[2];
    p.c4 = w4[3];
    p.ax = m->ax;
    p.ay = m->ay;
    p.az = m->az;
    p.nx = m->nx;
    p.ny = m->ny;
    p.nz = m->nz;
    p.px = m->px;
    p.bz = m->bz;
    p.has_sponge = m->has_sponge;
    p.sx = m->sx;
    p.sy = m->sy;
    p.sz = m->sz;
    p.rec_idx = m->d_rec;
    p.nrec = m->nrec;
    p.err = m->d_err;
    const int c = m->cur;
    p.out = m->buf[c ^ 1];
    p.P = m->buf[c];
    p.src_on = m->src_on && m->n < (int)m->amp.size();
    p.src_amp = p.src_on ? m->amp[m->n] : 0.f;
    p.trace_prev = m->pending_row >= 0 ? m->traces + (size_t)m->pending_row * m->nrec : nullptr;
}

// Two fused steps: levels n+1, n+2 into the spare buffers, which then take the
// places of buf[] (with their maps).  The launch gathers the receiver rows still
// owed for its two input levels (pending_old from Pold, m->pending_row from P).
static fd_status step_pair(fd_model *m, int &pending_old)
{
    T2Params p{};
    float w4[4];
    fd_stencil_weights(w4);
    p.c1 = w4[0];
    p.c2 = w4[1];
    p.c3 = w4[2];
    p.c4 = w4[3];
    const int c = m->cur;
    p.P1 = m->buf[c];
    p.P0 = m->buf[c ^ 1];
    p.out2 = m->xbuf[0];
    p.out3 = m->xbuf[1];
    p.ax = m->ax;
    p.ay = m->ay;
    p.az = m->az;
    p.nx = m->nx;
    p.ny = m->ny;
    p.nz = m->nz;
    p.px = m->px;
    p.bz = m->t2_bz;
    p.has_sponge = m->has_sponge;
    p.sx = m->sx;
    p.sy = m->sy;
    p.sz = m->sz;
    const int na = (int)m->amp.size();
    p.src_on0 = m->src_on && m->n < na;
    p.amp0 = p.src_on0 ? m->amp[m->n] : 0.f;
    p.src_on1 = m->src_on && m->n + 1 < na;
    p.amp1 = p.src_on1 ? m->amp[m->n + 1] : 0.f;
    p.rec_idx = m->d_rec;
    p.nrec = m->nrec;
    p.trace_prev0 = pending_old >= 0 ? m->traces + (size_t)pending_old * m->nrec : nullptr;
    p.trace_prev1 = m->pending_row >= 0 ? m->traces + (size_t)m->pending_row * m->nrec : nullptr;
    p.err = m->d_err;
    cudaError_t e = launch_step3d_t2(m->t2p1_map[c], m->t2e_map[c ^ 1], m->t2w_map, p, m->t2_nchunks, m->stream);
    ++g_launches;
    if (e != cudaSuccess)
        return cuda_fail(e, "fused step kernel launch");
    // level n+1 (in xbuf[0]) becomes Pold, level n+2 (in xbuf[1]) becomes P
    std::swap(m->buf[c ^ 1], m->xbuf[0]);
    std::swap(m->halo_map[c ^ 1], m->xhalo_map[0]);
    std::swap(m->tile_map[c ^ 1], m->xtile_map[0]);
    std::swap(m->t2p1_map[c ^ 1], m->xt2p1_map[0]);
    std::swap(m->t2e_map[c ^ 1], m->xt2e_map[0]);
    std::swap(m->buf[c], m->xbuf[1]);
    std::swap(m->halo_map[c], m->xhalo_map[1]);
    std::swap(m->tile_map[c], m->xtile_map[1]);
    std::swap(m->t2p1_map[c], m->xt2p1_map[1]);
    std::swap(m->t2e_map[c], m->xt2e_map[1]);
    const bool rec = m->nrec > 0 && m->traces;
    pending_old = rec && m->n < m->trace_rows ? m->n : -1;
    m->pending_row = rec && m->n + 1 < m->trace_rows ? m->n + 1 : -1;
    m->n += 2;
    return FD_OK;
}

// nsteps time steps; if lp is set (nsteps == 1), the step also writes L'P of the
// level it consumes to lp; if img_grad is set (nsteps == 1), it adds Pn * img_lp
// to img_grad (all dense [nz][ny][nx]).
static fd_status step_n(fd_model *m, int nsteps, float *lp, const float *img_lp = nullptr,
                        float *img_grad = nullptr)
{
    int pending_old = -1;   // a receiver row of the Pold level still owed (after a fused pair)
    auto flush_old = [&]() -> fd_status {
        if (pending_old < 0)
            return FD_OK;
        cudaError_t e = launch_gather(m->buf[m->cur ^ 1], m->d_rec, m->nrec,
                                      m->traces + (size_t)pending_old * m->nrec, m->stream);
        ++g_launches;
        pending_old = -1;
        return e == cudaSuccess ? FD_OK : cuda_fail(e, "receiver gather");
    };
    int s0 = 0;
    if (m->tfuse == 2 && m->d.ndim == 3 && !lp && !img_grad && m->stall_stage < 0) {
        for (; s0 + 2 <= nsteps; s0 += 2)
            if (fd_status st = step_pair(m, pending_old))
                return st;
    }
    if (fd_status st = flush_old())
        return st;
    nsteps -= s0;
    StepParams p{};
    for (int s = 0; s < nsteps; ++s) {
        const int c = m->cur;
        fill_step_params(m, p);
        p.lp_out = lp;
        p.img_lp = img_lp;
        p.img_grad = img_grad;
        cudaError_t e = m->d.ndim == 3
                            ? launch_step3d(m->halo_map[c], m->tile_map[c ^ 1], m->w_map, p, m->nchunks, m->stream)
                            : launch_step2d(m->halo_map[c], m->tile_map[c ^ 1], m->w_map, p, m->stream);
        ++g_launches;
        if (e != cudaSuccess)
            return cuda_fail(e, "step kernel launch");
        m->cur ^= 1;
        m->pending_row = (m->nrec > 0 && m->traces && m->n < m->trace_rows) ? m->n : -1;
        ++m->n;
    }
    return flush_pending(m);
}

extern "C" fd_status fd_set_time_fusion(fd_model *m, int steps)
{
    NEED_MODEL(m);
    if (steps != 1 && steps != 2)
        return fail(FD_EINVAL, "fd_set_time_fusion: steps must be 1 or 2");
    if (steps == 2 && m->d.ndim != 3)
        return fail(FD_EINVAL, "fd_set_time_fusion: two fused steps need a 3D model");
    if (steps == 2 && !m->xbuf[0]) {
        const size_t bytes = m->pitched * sizeof(float);
        float *b[2] = {nullptr, nullptr};
        cudaError_t e = cudaMalloc((void **)&b[0], bytes);
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&b[1], bytes);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(b[0], 0, bytes, m->stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(b[1], 0, bytes, m->stream);
        if (e != cudaSuccess) {
            cudaFree(b[0]);
            cudaFree(b[1]);
            return cuda_fail(e, "fused-step buffers");
        }
        bool ok = true;
        for (int i = 0; i < 2; ++i) {
            ok = ok && make_map(&m->xhalo_map[i], b[i], 3, m->nx, m->ny, m->nz, m->px, kTX3 + 8, kTY3 + 8, kPlanes3);
            ok = ok && make_map(&m->xtile_map[i], b[i], 3, m->nx, m->ny, m->nz, m->px, kTX3, kTY3, kPlanes3);
            ok = ok && make_map(&m->xt2p1_map[i], b[i], 3, m->nx, m->ny, m->nz, m->px, 48, 48, 1);
            ok = ok && make_map(&m->xt2e_map[i], b[i], 3, m->nx, m->ny, m->nz, m->px, 40, 40, 1);
            ok = ok && make_map(&m->t2p1_map[i], m->buf[i], 3, m->nx, m->ny, m->nz, m->px, 48, 48, 1);
            ok = ok && make_map(&m->t2e_map[i], m->buf[i], 3, m->nx, m->ny, m->nz, m->px, 40, 40, 1);
        }
        ok = ok && make_map(&m->t2w_map, m->w, 3, m->nx, m->ny, m->nz, m->px, 40, 40, 1);
        if (!ok) {
            cudaFree(b[0]);
            cudaFree(b[1]);
            return fail(FD_ECUDA, "cuTensorMapEncodeTiled failed");
        }
        FD_CUDA(step3d_t2_prepare(), "fused-step kernel attributes");
        m->xbuf[0] = b[0];
        m->xbuf[1] = b[1];
        // about six waves of one-CTA-per-SM launches, each CTA marching at least 32 planes
        int sms = 148;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
        const long long tiles = (long long)((m->nx + 31) / 32) * ((m->ny + 31) / 32);
        long long bz = (long long)m->nz * tiles / (6LL * sms);
        bz = std::max(32LL, std::min<long long>(bz, m->nz));
        m->t2_nchunks = (int)((m->nz + bz - 1) / bz);
        m->t2_bz = (m->nz + m->t2_nchunks - 1) / m->t2_nchunks;
    }
    m->tfuse = steps;
    return FD_OK;
}

extern "C" fd_status fd_step(fd_model *m, int nsteps)
{
    NvtxRange nvtx_range("fd_step");
    NEED_MODEL(m);
    if (nsteps < 0)
        return fail(FD_EINVAL, "nsteps must be >= 0");
    return step_n(m, nsteps, nullptr);
}

extern "C" fd_status fd_step_lp(fd_model *m, float *lp_dev)
{
    NvtxRange nvtx_range("fd_step_lp");
    NEED_MODEL(m);
    if (!lp_dev)
        return fail(FD_EINVAL, "fd_step_lp: NULL output");
    return step_n(m, 1, lp_dev);
}

extern "C" fd_status fd_step_lp_n(fd_model *m, int nsteps, float *lp_buf)
{
    NvtxRange nvtx_range("fd_step_lp_n");
    NEED_MODEL(m);
    if (nsteps < 0 || (nsteps > 0 && !lp_buf))
        return fail(FD_EINVAL, "fd_step_lp_n: bad arguments");
    const size_t npts = (size_t)m->nx * m->ny * m->nz;
    for (int j = 0; j < nsteps; ++j)
        if (fd_status st = step_n(m, 1, lp_buf + (size_t)j * npts))
            return st;
    return FD_OK;
}

extern "C" fd_status fd_step_image(fd_model *m, const float *lp_dev, float *grad_dev)
{
    NvtxRange nvtx_range("fd_step_image");
    NEED_MODEL(m);
    if (!lp_dev || !grad_dev)
        return fail(FD_EINVAL, "fd_step_image: NULL argument");
    return step_n(m, 1, nullptr, lp_dev, grad_dev);
}

extern "C" fd_status fd_run_shot(fd_model *m, int nt, float *traces_dev)
{
    NvtxRange nvtx_range("fd_run_shot");
    NEED_MODEL(m);
    if (nt < 0)
        return fail(FD_EINVAL, "nt must be >= 0");
    fd_status st = fd_reset(m);
    if (st)
        return st;
    st = fd_set_trace_buffer(m, traces_dev, nt);
    if (st)
        return st;
    return fd_step(m, nt);
}

extern "C" fd_status fd_set_stream(fd_model *m, void *stream)
{
    NEED_MODEL(m);
    cudaStream_t to = static_cast<cudaStream_t>(stream);
    if (to == m->stream)
        return FD_OK;
    if (!m->handoff)
        FD_CUDA(cudaEventCreateWithFlags(&m->handoff, cudaEventDisableTiming), "cudaEventCreate");
    FD_CUDA(cudaEventRecord(m->handoff, m->stream), "cudaEventRecord");
    FD_CUDA(cudaStreamWaitEvent(to, m->handoff, 0), "cudaStreamWaitEvent");
    m->stream = to;
    return FD_OK;
}

extern "C" fd_status fd_stream_create(int priority, void **stream, int *greatest)
{
    if (!stream)
        return fail(FD_EINVAL, "fd_stream_create: NULL output");
    *stream = nullptr;
    int least = 0, most = 0;
    FD_CUDA(cudaDeviceGetStreamPriorityRange(&least, &most), "cudaDeviceGetStreamPriorityRange");
    const int p = std::min(least, std::max(most, priority));
    cudaStream_t s = nullptr;
    FD_CUDA(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, p), "cudaStreamCreateWithPriority");
    *stream = s;
    if (greatest)
        *greatest = most;
    return FD_OK;
}

extern "C" fd_status fd_stream_destroy(void *stream)
{
    if (!stream)
        return fail(FD_EINVAL, "fd_stream_destroy: NULL stream");
    FD_CUDA(cudaStreamDestroy(static_cast<cudaStream_t>(stream)), "cudaStreamDestroy");
    return FD_OK;
}

extern "C" fd_status fd_debug_stall_stage(fd_model *m, int stage)
{
    NEED_MODEL(m);
    if (stage < -1)
        return fail(FD_EINVAL, "fd_debug_stall_stage: stage must be >= -1");
    m->stall_stage = stage;
    return FD_OK;
}

extern "C" fd_status fd_debug_poison_padding(fd_model *m)
{
    NEED_MODEL(m);
    if (m->px == m->nx)
        return FD_OK;
    const size_t pitch = (size_t)m->px * sizeof(float);
    const size_t width = (size_t)(m->px - m->nx) * sizeof(float);
    float *fields[6] = {m->buf[0], m->buf[1], m->w, m->deriv[0], m->deriv[1], m->deriv[2]};
    for (float *f : fields)
        if (f)   // all-ones bytes are a NaN in FP32
            FD_CUDA(cudaMemset2DAsync(f + m->nx, pitch, 0xFF, width, m->rows, m->stream), "padding poison");
    return FD_OK;
}

extern "C" fd_status fd_gather_traces_async(fd_model *m, float *host_out, size_t cap)
{
    NvtxRange nvtx_range("fd_gather_traces");
    NEED_MODEL(m);
    const size_t need = (size_t)m->trace_rows * m->nrec;
    if (need > 0 && (!host_out || cap < need))
        return fail(FD_EINVAL, "trace output needs %zu floats (got %zu)", need, cap);
    if (m->pending_row >= 0)
        if (fd_status st = flush_pending(m))
            return st;
    if (need > 0 && m->traces)
        FD_CUDA(cudaMemcpyAsync(host_out, m->traces, need * sizeof(float), cudaMemcpyDeviceToHost, m->stream),
                "trace download");
    return FD_OK;
}

extern "C" fd_status fd_gather_traces(fd_model *m, float *host_out, size_t cap)
{
    if (fd_status st = fd_gather_traces_async(m, host_out, cap))
        return st;
    return fd_synchronize(m);
}

extern "C" fd_status fd_get_wavefield(fd_model *m, float *p_host, float *pold_host, size_t cap)
{
    NEED_MODEL(m);
    if (!p_host || cap < m->npts)
        return fail(FD_EINVAL, "wavefield output needs %zu floats (got %zu)", m->npts, cap);
    const size_t wb = (size_t)m->nx * 4, pb = (size_t)m->px * 4;
    FD_CUDA(cudaMemcpy2DAsync(p_host, wb, m->buf[m->cur], pb, wb, m->rows, cudaMemcpyDeviceToHost, m->stream),
            "wavefield download");
    if (pold_host)
        FD_CUDA(cudaMemcpy2DAsync(pold_host, wb, m->buf[m->cur ^ 1], pb, wb, m->rows, cudaMemcpyDeviceToHost,
                                  m->stream),
                "wavefield download");
    return fd_synchronize(m);
}

extern "C" fd_status fd_synchronize(fd_model *m)
{
    NEED_MODEL(m);
    FD_CUDA(cudaStreamSynchronize(m->stream), "stream synchronize");
    int err = 0;
    FD_CUDA(cudaMemcpy(&err, m->d_err, sizeof err, cudaMemcpyDeviceToHost), "error word");
    if (err) {
        cudaMemset(m->d_err, 0, sizeof(int));
        return fail(FD_ETIMEOUT, "a kernel gave up a bounded wait (device code %d)", err);
    }
    return FD_OK;
}

extern "C" fd_status fd_get_step(fd_model *m, int *n)
{
    if (!m || !n)
        return fail(FD_EINVAL, "NULL argument");
    *n = m->n;
    return FD_OK;
}

extern "C" fd_status fd_get_source_index(fd_model *m, int64_t *idx)
{
    if (!m || !idx)
        return fail(FD_EINVAL, "NULL argument");
    *idx = m->src_on ? ((int64_t)m->sz * m->ny + m->sy) * m->nx + m->sx : -1;
    return FD_OK;
}

extern "C" fd_status fd_get_receiver_indices(fd_model *m, int64_t *out, int cap)
{
    if (!m || (m->nrec > 0 && !out))
        return fail(FD_EINVAL, "NULL argument");
    if (cap < m->nrec)
        return fail(FD_EINVAL, "need room for %d indices", m->nrec);
    std::copy(m->rec_dense.begin(), m->rec_dense.end(), out);
    return FD_OK;
}

extern "C" fd_status fd_get_damping_profile(fd_model *m, int axis, float *out, int cap)
{
    NEED_MODEL(m);
    if (axis < 0 || axis > 2 || !out)
        return fail(FD_EINVAL, "bad axis or NULL output");
    const int n = axis == 0 ? m->nx : axis == 1 ? m->ny : m->nz;
    if (cap < n)
        return fail(FD_EINVAL, "need room for %d floats", n);
    const float *src = axis == 0 ? m->ax : axis == 1 ? m->ay : m->az;
    FD_CUDA(cudaMemcpyAsync(out, src, (size_t)n * 4, cudaMemcpyDeviceToHost, m->stream), "profile download");
    FD_CUDA(cudaStreamSynchronize(m->stream), "profile download");
    return FD_OK;
}

extern "C" uint64_t fd_kernel_launch_count(void)
{
    return g_launches.load();
}

extern "C" const char *fd_last_error(void)
{
    return g_last_error.c_str();
}
