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
// accumulated by fd_imaging (damping profiles held fixed).

#include <algorithm>

#include "fd.h"
#include "fd_internal.h"
#include "fd_model.h"

namespace fdk {

// values[r] * w / (1 + a) added to P at receiver r (pitched indices).
__global__ void inject_kernel(float *P, const float *w, const float *ax, const float *ay, const float *az,
                              const int64_t *idx, int nrec, const float *values, int nx, int ny, int px,
                              int has_sponge, int ndim)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += gridDim.x * blockDim.x) {
        const int64_t i = idx[r];
        float a = 0.f;
        if (has_sponge) {
            const int64_t row = i / px;
            const int x = (int)(i - row * px);
            const int y = ndim == 3 ? (int)(row % ny) : 0;
            const int z = ndim == 3 ? (int)(row / ny) : (int)row;
            a = ax[x] + (ndim == 3 ? ay[y] : 0.f) + az[z];
        }
        const float v = values[r] * w[i];
        P[i] += a != 0.f ? __fdividef(v, 1.0f + a) : v;
    }
}

// grad[i] += psi[i] * (L'p)[i] over dense [nz][ny][nx] arrays p and grad; psi is pitched.
// L'p = sum over the axes of sum_k c_k ((p[+k] + p[-k]) - 2 p), zero outside the grid.
__global__ void __launch_bounds__(256) imaging_kernel(const float *__restrict__ psi, const float *__restrict__ p,
                                                      float *__restrict__ grad, int nx, int ny, int nz, int px,
                                                      int ndim, float c1, float c2, float c3, float c4)
{
    const long long n = (long long)nx * ny * nz;
    const float ck[4] = {c1, c2, c3, c4};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long row = i / nx;
        const int y = (int)(row % ny);
        const int z = (int)(row / ny);
        const float pc = p[i];
        float lap = 0.f;
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
            float s = (x + k < nx ? p[i + k] : 0.f) + (x - k >= 0 ? p[i - k] : 0.f);
            s += (z + k < nz ? p[i + (long long)k * nx * ny] : 0.f) + (z - k >= 0 ? p[i - (long long)k * nx * ny] : 0.f);
            if (ndim == 3)
                s += (y + k < ny ? p[i + (long long)k * nx] : 0.f) + (y - k >= 0 ? p[i - (long long)k * nx] : 0.f);
            lap = fmaf(ck[k - 1], fmaf(-2.0f * ndim, pc, s), lap);
        }
        grad[i] = fmaf(psi[row * px + x], lap, grad[i]);
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

extern "C" fd_status fd_inject_receivers(fd_model *m, const float *values_dev)
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
    const int blocks = std::min((m->nrec + 255) / 256, 1184);
    inject_kernel<<<blocks, 256, 0, m->stream>>>(m->buf[m->cur], m->w, m->ax, m->ay, m->az, m->d_rec, m->nrec,
                                                 values_dev, m->nx, m->ny, m->px, m->has_sponge, m->d.ndim);
    ++g_launches;
    FD_CUDA(cudaGetLastError(), "inject launch");
    return FD_OK;
}

extern "C" fd_status fd_imaging(fd_model *adj, const float *p_dev, float *grad_dev)
{
    if (!adj || !p_dev || !grad_dev)
        return fail(FD_EINVAL, "fd_imaging: NULL argument");
    FD_CUDA(cudaSetDevice(adj->device), "cudaSetDevice");
    float w4[4];
    fd_stencil_weights(w4);
    const long long n = (long long)adj->npts;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 148LL * 16);
    imaging_kernel<<<blocks, 256, 0, adj->stream>>>(adj->buf[adj->cur], p_dev, grad_dev, adj->nx, adj->ny, adj->nz,
                                                    adj->px, adj->d.ndim, w4[0], w4[1], w4[2], w4[3]);
    ++g_launches;
    FD_CUDA(cudaGetLastError(), "imaging launch");
    return FD_OK;
}
