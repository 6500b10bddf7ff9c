// fd_adjoint.cu -- the pieces of the reverse-time adjoint of the time step.
//
// Forward (fd_step):  (1 + a) P^{n+1} = 2 P^n - (1 - a) P^{n-1} + W L'P^n + (1 + a) s^n e_src,
// traces d^n = R P^{n+1}, W = diag(w), w = (dt v / h)^2 = dt^2 / (h^2 m), m = 1 / v^2.
// For J(d) with dJ/dd^n = g^n, the adjoint of this recurrence, written for
// psi = W lambda / (1 + a) (lambda the Lagrange multipliers), is the same damped
// leapfrog run backwards in time:
//   (1 + a) psi_k = 2 psi_{k+1} - (1 - a) psi_{k+2} + W L' psi_{k+1} + W R^T g^{k-1},
// so the adjoint wavefield advances with fd_step on a model with the same
// velocity, and the receiver residuals enter as w g / (1 + a) at the receiver
// points (fd_inject_receivers).  The gradient with respect to m is
//   dJ/dm = -(1/m) sum_{n=0}^{nt-1} psi_{n+1} (L' P^n)
// (damping profiles held fixed), accumulated by fd_imaging from a stored P^n or
// by fd_imaging_product from the L'P^n that fd_step_lp writes during the
// segment recompute (fd_adjoint_segment issues a whole segment).

#include <algorithm>

#include "fd.h"
#include "fd_internal.h"
#include "fd_model.h"
#include "fd_trace.h"

namespace fdk {

// The receiver terms w g / (1 + a) added to P, one thread per receiver point:
// the values of the receivers that share a point are summed first, in receiver
// order, so no atomics are needed and the result does not depend on thread
// timing.  With grad set, the injected value times lp is added to grad as well
// (dense indices), completing grad += P * lp for the level P had before the
// injection.
__global__ void inject_kernel(float *P, const float *w, const float *ax, const float *ay, const float *az,
                              const int64_t *pt, const int *beg, const int *rec, int npt, const float *values,
                              int nx, int ny, int px, int has_sponge, int ndim, const float *lp, float *grad)
{
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < npt; u += gridDim.x * blockDim.x) {
        const int64_t i = pt[u];
        float a = 0.f;
        if (has_sponge) {
            const int64_t row = i / px;
            const int x = (int)(i - row * px);
            const int y = ndim == 3 ? (int)(row % ny) : 0;
            const int z = ndim == 3 ? (int)(row / ny) : (int)row;
            a = ax[x] + (ndim == 3 ? ay[y] : 0.f) + az[z];
        }
        float g = values[rec[beg[u]]];
        for (int j = beg[u] + 1; j < beg[u + 1]; ++j)
            g += values[rec[j]];
        const float v = g * w[i];
        const float add = a != 0.f ? __fdividef(v, 1.0f + a) : v;
        P[i] += add;
        if (grad) {
            const int64_t row = i / px;
            const int64_t d = row * nx + (i - row * px);
            grad[d] = __fadd_rn(grad[d], __fmul_rn(add, lp[d]));
        }
    }
}

// grad[i] += psi[i] * (L'p)[i] over dense [nz][ny][nx] arrays p and grad; psi is pitched.
// L'p = sum over the axes of sum_k c_k ((p[+k] + p[-k]) - 2 p), zero outside the grid.
//
// A block of 32 x kImgRows threads owns a 32-wide x segment of kImgRows rows
// (y in 3D; in 2D the rows are further x segments) and marches along z through
// kImgChunk planes; each thread keeps the 9 values p[z-4 .. z+4] of its own
// column in registers, and reads its x and y neighbours through L1.
constexpr int kImgRows = 8;
constexpr int kImgChunk = 32;

template <int NDIM>
__global__ void __launch_bounds__(32 * kImgRows) imaging_kernel(const float *__restrict__ psi,
                                                                const float *__restrict__ p,
                                                                float *__restrict__ grad, int nx, int ny, int nz,
                                                                int px, float c1, float c2, float c3, float c4)
{
    const int x = NDIM == 3 ? blockIdx.x * 32 + threadIdx.x : (blockIdx.x * kImgRows + threadIdx.y) * 32 + threadIdx.x;
    const int y = NDIM == 3 ? blockIdx.y * kImgRows + threadIdx.y : 0;
    const int z0 = blockIdx.z * kImgChunk;
    const int z1 = min(nz, z0 + kImgChunk);
    if (x >= nx || y >= ny)
        return;
    const size_t plane = (size_t)nx * ny;
    const float *col = p + (size_t)y * nx + x;   // p[z][y][x] = col[z * plane]
    float q[9];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int z = z0 - 4 + i;
        q[i] = (z >= 0 && z < nz) ? col[(size_t)z * plane] : 0.f;
    }
    const float ck[4] = {c1, c2, c3, c4};
    for (int z = z0; z < z1; ++z) {
        q[8] = z + 4 < nz ? col[(size_t)(z + 4) * plane] : 0.f;
        const float *c = col + (size_t)z * plane;
        const float pc = q[4];
        float lap = 0.f;
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
            float s = (x + k < nx ? c[k] : 0.f) + (x - k >= 0 ? c[-k] : 0.f);
            s += q[4 + k] + q[4 - k];
            if (NDIM == 3)
                s += (y + k < ny ? c[(size_t)k * nx] : 0.f) + (y - k >= 0 ? c[-(ptrdiff_t)k * nx] : 0.f);
            lap = fmaf(ck[k - 1], fmaf(-2.0f * NDIM, pc, s), lap);
        }
        const size_t i = (size_t)z * plane + (size_t)y * nx + x;
        grad[i] = fmaf(psi[((size_t)z * ny + y) * px + x], lap, grad[i]);
#pragma unroll
        for (int i2 = 0; i2 < 8; ++i2)
            q[i2] = q[i2 + 1];
    }
}

// grad[i] += psi[i] * lp[i] with lp = L'P^n as written by fd_step_lp: dense
// grad and lp, pitched psi.  One block per group of rows, threads along x.
__global__ void __launch_bounds__(256) imaging_product_kernel(const float *__restrict__ psi,
                                                              const float *__restrict__ lp,
                                                              float *__restrict__ grad, int nx, size_t rows, int px)
{
    for (size_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const float *ps = psi + row * px;
        const float *l = lp + row * nx;
        float *g = grad + row * nx;
        for (int x = threadIdx.x; x < nx; x += blockDim.x)
            g[x] = fmaf(ps[x], l[x], g[x]);
    }
}

// v = m^(-1/2) for squared slowness m, in FP64 and rounded once to FP32 (a
// non-positive or non-finite m gives NaN, which model creation rejects).
__global__ void velocity_from_slowness_kernel(const float *__restrict__ m, float *__restrict__ v, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double x = (double)m[i];
        v[i] = x > 0.0 ? (float)(1.0 / sqrt(x)) : __int_as_float(0x7fc00000);
    }
}

// grad = -(acc_0 + ... + acc_{k-1}) / m: the images of k shot groups (consecutive
// arrays of n floats) summed in that order, then divided by m.
__global__ void gradient_from_image_kernel(const float *__restrict__ acc, int nacc, const float *__restrict__ m,
                                           float *__restrict__ grad, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float s = acc[i];
        for (int j = 1; j < nacc; ++j)
            s += acc[(size_t)j * n + i];
        grad[i] = -(s / m[i]);
    }
}

}  // namespace fdk

using namespace fdk;

extern "C" fd_status fd_get_wavefield_dev(fd_model *m, float *p_dev, float *pold_dev)
{
    if (!m || !p_dev)
        return fail(FD_EINVAL, "fd_get_wavefield_dev: NULL argument");
    FD_CUDA(cudaSetDevice(m->device), "cudaSetDevice");
    if (m->pending_row >= 0) {
        fd_status st = fd_step(m, 0);   // settle the owed receiver gather first
        if (st)
            return st;
    }
    const size_t wb = (size_t)m->nx * 4, pb = (size_t)m->px * 4;
    FD_CUDA(cudaMemcpy2DAsync(p_dev, wb, m->buf[m->cur], pb, wb, m->rows, cudaMemcpyDeviceToDevice, m->stream),
            "wavefield copy");
    if (pold_dev)
        FD_CUDA(cudaMemcpy2DAsync(pold_dev, wb, m->buf[m->cur ^ 1], pb, wb, m->rows, cudaMemcpyDeviceToDevice,
                                  m->stream),
                "wavefield copy");
    return FD_OK;
}

extern "C" fd_status fd_set_wavefield_dev(fd_model *m, const float *p_dev, const float *pold_dev, int n)
{
    if (!m || !p_dev || !pold_dev || n < 0)
        return fail(FD_EINVAL, "fd_set_wavefield_dev: bad arguments");
    FD_CUDA(cudaSetDevice(m->device), "cudaSetDevice");
    const size_t wb = (size_t)m->nx * 4, pb = (size_t)m->px * 4;
    FD_CUDA(cudaMemcpy2DAsync(m->buf[m->cur], pb, p_dev, wb, wb, m->rows, cudaMemcpyDeviceToDevice, m->stream),
            "wavefield copy");
    FD_CUDA(cudaMemcpy2DAsync(m->buf[m->cur ^ 1], pb, pold_dev, wb, wb, m->rows, cudaMemcpyDeviceToDevice,
                              m->stream),
            "wavefield copy");
    m->n = n;
    m->pending_row = -1;
    return FD_OK;
}

static fd_status inject(fd_model *m, const float *values_dev, const float *lp_dev, float *grad_dev)
{
    if (!m || (m->nrec > 0 && !values_dev))
        return fail(FD_EINVAL, "fd_inject_receivers: bad arguments");
    FD_CUDA(cudaSetDevice(m->device), "cudaSetDevice");
    if (m->nrec == 0)
        return FD_OK;
    if (m->pending_row >= 0) {
        fd_status st = fd_step(m, 0);   // the gather must read the level before injection
        if (st)
            return st;
    }
    const int blocks = std::min((m->ninj + 255) / 256, 1184);
    inject_kernel<<<blocks, 256, 0, m->stream>>>(m->buf[m->cur], m->w, m->ax, m->ay, m->az, m->d_inj_pt,
                                                 m->d_inj_beg, m->d_inj_rec, m->ninj, values_dev, m->nx, m->ny,
                                                 m->px, m->has_sponge, m->d.ndim, lp_dev, grad_dev);
    ++g_launches;
    FD_CUDA(cudaGetLastError(), "inject launch");
    return FD_OK;
}

extern "C" fd_status fd_inject_receivers(fd_model *m, const float *values_dev)
{
    return inject(m, values_dev, nullptr, nullptr);
}

extern "C" fd_status fd_inject_receivers_image(fd_model *m, const float *values_dev, const float *lp_dev,
                                               float *grad_dev)
{
    if (!lp_dev || !grad_dev)
        return fail(FD_EINVAL, "fd_inject_receivers_image: NULL argument");
    return inject(m, values_dev, lp_dev, grad_dev);
}

extern "C" fd_status fd_imaging(fd_model *adj, const float *p_dev, float *grad_dev)
{
    if (!adj || !p_dev || !grad_dev)
        return fail(FD_EINVAL, "fd_imaging: NULL argument");
    FD_CUDA(cudaSetDevice(adj->device), "cudaSetDevice");
    float w4[4];
    fd_stencil_weights(w4);
    const int nx = adj->nx, ny = adj->ny, nz = adj->nz;
    const dim3 block(32, kImgRows);
    const unsigned gz = (unsigned)((nz + kImgChunk - 1) / kImgChunk);
    if (adj->d.ndim == 3) {
        const dim3 grid((nx + 31) / 32, (ny + kImgRows - 1) / kImgRows, gz);
        imaging_kernel<3><<<grid, block, 0, adj->stream>>>(adj->buf[adj->cur], p_dev, grad_dev, nx, ny, nz, adj->px,
                                                           w4[0], w4[1], w4[2], w4[3]);
    } else {
        const dim3 grid((nx + 32 * kImgRows - 1) / (32 * kImgRows), 1, gz);
        imaging_kernel<2><<<grid, block, 0, adj->stream>>>(adj->buf[adj->cur], p_dev, grad_dev, nx, 1, nz, adj->px,
                                                           w4[0], w4[1], w4[2], w4[3]);
    }
    ++g_launches;
    FD_CUDA(cudaGetLastError(), "imaging launch");
    return FD_OK;
}

extern "C" fd_status fd_imaging_product(fd_model *adj, const float *lp_dev, float *grad_dev)
{
    if (!adj || !lp_dev || !grad_dev)
        return fail(FD_EINVAL, "fd_imaging_product: NULL argument");
    FD_CUDA(cudaSetDevice(adj->device), "cudaSetDevice");
    const int blocks = (int)std::min<size_t>(adj->rows, 148 * 64);
    imaging_product_kernel<<<blocks, 256, 0, adj->stream>>>(adj->buf[adj->cur], lp_dev, grad_dev, adj->nx, adj->rows,
                                                            adj->px);
    ++g_launches;
    FD_CUDA(cudaGetLastError(), "imaging product launch");
    return FD_OK;
}

extern "C" fd_status fd_adjoint_backward(fd_model *adj, int n0, int n1, const float *lp_buf, const float *g_dev,
                                         float *grad_dev)
{
    NvtxRange nvtx_range("fd_adjoint_backward");
    if (!adj || !lp_buf || !grad_dev || (adj->nrec > 0 && !g_dev))
        return fail(FD_EINVAL, "fd_adjoint_backward: NULL argument");
    if (n0 < 0 || n1 <= n0)
        return fail(FD_EINVAL, "fd_adjoint_backward: need 0 <= n0 < n1 (got %d, %d)", n0, n1);
    const size_t npts = (size_t)adj->nx * adj->ny * adj->nz;
    // grad += psi_k * L'P^{k-1}: the step adds its new level times L'P, the
    // injection adds its share, so the sum is (psi_k before + injected) * L'P
    for (int k = n1; k > n0; --k) {
        const float *lp = lp_buf + (size_t)(k - 1 - n0) * npts;
        if (fd_status st = fd_step_image(adj, lp, grad_dev))
            return st;
        if (fd_status st = fd_inject_receivers_image(
                adj, adj->nrec > 0 ? g_dev + (size_t)(k - 1) * adj->nrec : nullptr, lp, grad_dev))
            return st;
    }
    return FD_OK;
}

extern "C" fd_status fd_adjoint_segment(fd_model *fwd, fd_model *adj, int n0, int n1, float *lp_buf,
                                        const float *g_dev, float *grad_dev)
{
    NvtxRange nvtx_range("fd_adjoint_segment");
    if (!fwd || !adj || !lp_buf || !grad_dev || (adj->nrec > 0 && !g_dev))
        return fail(FD_EINVAL, "fd_adjoint_segment: NULL argument");
    if (n0 < 0 || n1 <= n0)
        return fail(FD_EINVAL, "fd_adjoint_segment: need 0 <= n0 < n1 (got %d, %d)", n0, n1);
    if (fwd->nx != adj->nx || fwd->ny != adj->ny || fwd->nz != adj->nz || fwd->d.ndim != adj->d.ndim)
        return fail(FD_EINVAL, "fd_adjoint_segment: models of different grids");
    if (fwd->stream != adj->stream)
        return fail(FD_EINVAL, "fd_adjoint_segment: the two models must share a stream");
    if (fwd->n != n0)
        return fail(FD_ESTATE, "fd_adjoint_segment: forward model at step %d, segment starts at %d", fwd->n, n0);
    const size_t npts = (size_t)fwd->nx * fwd->ny * fwd->nz;
    for (int j = 0; j < n1 - n0; ++j)
        if (fd_status st = fd_step_lp(fwd, lp_buf + (size_t)j * npts))
            return st;
    return fd_adjoint_backward(adj, n0, n1, lp_buf, g_dev, grad_dev);
}

extern "C" fd_status fd_velocity_from_slowness(const float *m_dev, float *v_dev, size_t n, void *stream)
{
    if (!m_dev || !v_dev || n == 0)
        return fail(FD_EINVAL, "fd_velocity_from_slowness: bad arguments");
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 148 * 16);
    velocity_from_slowness_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(m_dev, v_dev, n);
    ++g_launches;
    FD_CUDA(cudaGetLastError(), "slowness conversion launch");
    return FD_OK;
}

extern "C" fd_status fd_gradient_from_image(const float *acc_dev, int nacc, const float *m_dev, float *grad_dev,
                                            size_t n, void *stream)
{
    if (!acc_dev || nacc < 1 || !m_dev || !grad_dev || n == 0)
        return fail(FD_EINVAL, "fd_gradient_from_image: bad arguments");
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 148 * 16);
    gradient_from_image_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(acc_dev, nacc, m_dev,
                                                                                       grad_dev, n);
    ++g_launches;
    FD_CUDA(cudaGetLastError(), "gradient launch");
    return FD_OK;
}
