/*
 * fd_oracle.c -- FP64 CPU reference propagator for the acoustic wave equation.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
 * and the benchmark's CPU-baseline / reference legs may load this library.  It
 * shares no code, header, table or constant with the CUDA path: the stencil
 * coefficients and the sponge profiles arrive as arguments, computed by
 * oracle/oracle.py from their own definitions.
 *
 * What it computes (paper section 7, Eq. 1, and the routine order of the
 * WaveSimulator::run() listing: add_source, fd_pzz, fd_pxx, fd_time, swaps):
 *
 *   P_tt = v^2 (P_xx + P_zz [+ P_yy]) + S(t) delta(x - x_s)
 *
 * discretised by the second-order leapfrog in time and a centred radius-r
 * stencil in space.  With the dimensionless stencil sum
 *
 *   L'P[i] = sum over axes of ( c_0 P[i] + sum_{k=1..r} c_k (P[i+k e] + P[i-k e]) )
 *
 * (P = 0 outside the grid: the rigid, zero-halo reading), w = (dt v / h)^2 and
 * the sponge damping a = dt (eta_x(ix) + eta_y(iy) + eta_z(iz)), one step maps
 * (P, Pold) at time levels n, n-1 to Pn at level n+1:
 *
 *   Pn = ( 2 P - (1 - a) Pold + w L'P ) / (1 + a)              (damped leapfrog)
 *   Pn[src] += dt^2 s[n] / h^d         (point source sampled at t_n = n dt)
 *   trace[n][r] = Pn[rec_r]            (receivers record the field at t_{n+1})
 *
 * With a = 0 the first line is the plain leapfrog 2P - Pold + dt^2 v^2 (P_xx +
 * P_zz).  The code is deliberately plain: one loop nest per step, a bounds test
 * per neighbour, no blocking, no fusion beyond the formula above, FP64
 * throughout.  OpenMP only splits the outermost (z) loop across threads.
 */
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* P at integer grid point (ix, iy, iz); zero outside the grid (rigid boundary). */
static double field_at(const double *P, long nx, long ny, long nz,
                       long ix, long iy, long iz)
{
    if (ix < 0 || ix >= nx || iy < 0 || iy >= ny || iz < 0 || iz >= nz)
        return 0.0;
    return P[(iz * ny + iy) * nx + ix];
}

/*
 * Dimensionless Laplacian sum L'P at one grid point: for each axis present,
 * c_0 P + sum_k c_k (P[+k] + P[-k]).  2D grids pass ny = 1 and ndim = 2, in
 * which case the y axis is not an axis of the operator.
 */
static double stencil_sum(const double *P, int ndim, long nx, long ny, long nz,
                          long ix, long iy, long iz, int radius, const double *c)
{
    double centre = field_at(P, nx, ny, nz, ix, iy, iz);
    double sum = 0.0;
    /* x axis */
    sum += c[0] * centre;
    for (int k = 1; k <= radius; ++k)
        sum += c[k] * (field_at(P, nx, ny, nz, ix + k, iy, iz) +
                       field_at(P, nx, ny, nz, ix - k, iy, iz));
    /* z axis */
    sum += c[0] * centre;
    for (int k = 1; k <= radius; ++k)
        sum += c[k] * (field_at(P, nx, ny, nz, ix, iy, iz + k) +
                       field_at(P, nx, ny, nz, ix, iy, iz - k));
    /* y axis, 3D only */
    if (ndim == 3) {
        sum += c[0] * centre;
        for (int k = 1; k <= radius; ++k)
            sum += c[k] * (field_at(P, nx, ny, nz, ix, iy + k, iz) +
                           field_at(P, nx, ny, nz, ix, iy - k, iz));
    }
    return sum;
}

/*
 * Advance the state (P, Pold) by nsteps leapfrog steps, starting at step index
 * n0 (so that the wavelet sample used by step n is wavelet[n]).
 *
 * ndim            2 or 3.  2D grids are [nz][nx] and must pass ny == 1.
 * nx, ny, nz      grid extents; arrays are [nz][ny][nx], x fastest.
 * h, dt           grid spacing (m) and time step (s).
 * radius, c       stencil radius r and coefficients c[0..r] of h^2 d2/dx2.
 * vel             velocity (m/s) per grid point.
 * eta_x/y/z       1D sponge damping rates (1/s) of length nx / ny / nz, or NULL
 *                 for none; eta_y is ignored in 2D.
 * six, siy, siz   source grid point (siy ignored in 2D); wavelet[0..nt_wavelet)
 *                 is S(t_n); steps n >= nt_wavelet inject nothing.  A NULL
 *                 wavelet means no source.
 * nrec, rec_xyz   receivers as (ix, iy, iz) triples (iy ignored in 2D).
 * P, Pold         in: levels n0 and n0-1; out: levels n0+nsteps and
 *                 n0+nsteps-1.
 * traces          [nsteps][nrec] output, or NULL.
 * nthreads        OpenMP threads for the z loop (<= 0: library default).
 *
 * Returns 0, or -1 for inconsistent arguments (nothing is modified then), or
 * -2 if scratch memory could not be allocated.
 */
int fdo_run(int ndim, int nx, int ny, int nz, double h, double dt,
            int radius, const double *c, const double *vel,
            const double *eta_x, const double *eta_y, const double *eta_z,
            int six, int siy, int siz, const double *wavelet, int nt_wavelet,
            int nrec, const int *rec_xyz,
            double *P, double *Pold, int n0, int nsteps,
            double *traces, int nthreads)
{
    if ((ndim != 2 && ndim != 3) || nx < 1 || ny < 1 || nz < 1 ||
        (ndim == 2 && ny != 1) || radius < 1 || !c || !vel || !P || !Pold ||
        nsteps < 0 || n0 < 0 || nrec < 0 || (nrec > 0 && !rec_xyz) ||
        !(h > 0.0) || !(dt > 0.0))
        return -1;
    if (ndim == 2) {
        siy = 0;
    }
    if (wavelet && (six < 0 || six >= nx || siy < 0 || siy >= ny || siz < 0 || siz >= nz))
        return -1;
    for (int r = 0; r < nrec; ++r) {
        int rx = rec_xyz[3 * r], ry = ndim == 3 ? rec_xyz[3 * r + 1] : 0, rz = rec_xyz[3 * r + 2];
        if (rx < 0 || rx >= nx || ry < 0 || ry >= ny || rz < 0 || rz >= nz)
            return -1;
    }

    const long npts = (long)nx * ny * nz;
    double *Pn = (double *)malloc(sizeof(double) * (size_t)npts);
    if (!Pn)
        return -2;
    double hd = ndim == 3 ? h * h * h : h * h;

#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif

    for (int s = 0; s < nsteps; ++s) {
        const int n = n0 + s;
#pragma omp parallel for schedule(static)
        for (long iz = 0; iz < nz; ++iz) {
            for (long iy = 0; iy < ny; ++iy) {
                for (long ix = 0; ix < nx; ++ix) {
                    long i = (iz * ny + iy) * nx + ix;
                    double lap = stencil_sum(P, ndim, nx, ny, nz, ix, iy, iz, radius, c);
                    double w = (dt * vel[i] / h) * (dt * vel[i] / h);
                    double eta = 0.0;
                    if (eta_x) eta += eta_x[ix];
                    if (eta_z) eta += eta_z[iz];
                    if (ndim == 3 && eta_y) eta += eta_y[iy];
                    double a = dt * eta;
                    Pn[i] = (2.0 * P[i] - (1.0 - a) * Pold[i] + w * lap) / (1.0 + a);
                }
            }
        }
        /* add_source: the point source enters the field of level n+1 */
        if (wavelet && n < nt_wavelet)
            Pn[((long)siz * ny + siy) * nx + six] += dt * dt * wavelet[n] / hd;
        /* receivers sample level n+1 */
        if (traces) {
            for (int r = 0; r < nrec; ++r) {
                long rx = rec_xyz[3 * r], ry = ndim == 3 ? rec_xyz[3 * r + 1] : 0, rz = rec_xyz[3 * r + 2];
                traces[(long)s * nrec + r] = Pn[(rz * ny + ry) * nx + rx];
            }
        }
        /* rotation: Pold <- P, P <- Pn */
        memcpy(Pold, P, sizeof(double) * (size_t)npts);
        memcpy(P, Pn, sizeof(double) * (size_t)npts);
    }
    free(Pn);
    return 0;
}

/* Threads an OpenMP parallel region would use (1 when built without OpenMP). */
int fdo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
