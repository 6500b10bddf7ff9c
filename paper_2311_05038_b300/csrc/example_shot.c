/*
 * example_shot.c -- one 3D shot through the C ABI of libfd (include/fd.h), with
 * no Python: a three-layer velocity model, a 15 Hz Ricker source near the top,
 * a plane of receivers, a 10-point sponge; the traces go to a binary file.
 * It is not part of libfd; it shows the boundary as a C caller sees it.
 *
 * Build (from the repository root, after building libfd.so):
 *   gcc -O2 -I include paper_2311_05038_b300/csrc/example_shot.c \
 *       -L paper_2311_05038_b300 -lfd -Wl,-rpath,$PWD/paper_2311_05038_b300 -lm -o example_shot
 * Run:
 *   ./example_shot traces.bin      (nt x nrec float32, row-major; nt and nrec on stdout)
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "fd.h"

#define CHECK(call)                                                          \
    do {                                                                     \
        fd_status st_ = (call);                                              \
        if (st_ != FD_OK) {                                                  \
            fprintf(stderr, "%s failed (%d): %s\n", #call, st_, fd_last_error()); \
            return 1;                                                        \
        }                                                                    \
    } while (0)

enum { NX = 96, NY = 80, NZ = 64, NT = 300, W = 10, STRIDE = 4 };

int main(int argc, char **argv)
{
    const double h = 10.0, vmax = 3000.0, f = 15.0;
    const double dt = 0.4 * h / vmax;   /* Courant number 0.4 */
    const double pi = 3.14159265358979323846;

    /* velocity [nz][ny][nx], x fastest: three flat layers */
    float *v = malloc(sizeof(float) * NX * NY * NZ);
    for (int z = 0; z < NZ; ++z)
        for (int i = 0; i < NX * NY; ++i)
            v[(size_t)z * NX * NY + i] = z < NZ / 3 ? 1800.0f : z < 2 * NZ / 3 ? 2400.0f : 3000.0f;

    /* Ricker wavelet of unit peak, delayed by 1.5 / f */
    float *wavelet = malloc(sizeof(float) * NT);
    for (int n = 0; n < NT; ++n) {
        double a = pi * f * (n * dt - 1.5 / f);
        a *= a;
        wavelet[n] = (float)((1.0 - 2.0 * a) * exp(-a));
    }

    /* receivers: every STRIDE-th point of the plane iz = W + 3 */
    const int nrec = (NX / STRIDE) * (NY / STRIDE);
    int *rec = malloc(sizeof(int) * 3 * nrec);
    int r = 0;
    for (int iy = 0; iy < NY; iy += STRIDE)
        for (int ix = 0; ix < NX; ix += STRIDE) {
            rec[3 * r] = ix;
            rec[3 * r + 1] = iy;
            rec[3 * r + 2] = W + 3;
            ++r;
        }

    fd_grid_desc desc = {3, NX, NY, NZ, h, dt, W, 1e-3};
    fd_model *m = NULL;
    CHECK(fd_model_create(&desc, v, NULL, &m));
    CHECK(fd_set_source(m, NX / 2, NY / 2, W + 6, wavelet, NT));
    CHECK(fd_set_receivers(m, rec, nrec));
    CHECK(fd_run_shot(m, NT, NULL));   /* library-owned trace buffer */

    float *traces = malloc(sizeof(float) * (size_t)NT * nrec);
    CHECK(fd_gather_traces(m, traces, (size_t)NT * nrec));
    CHECK(fd_model_destroy(m));

    double peak = 0.0;
    for (size_t i = 0; i < (size_t)NT * nrec; ++i)
        peak = fmax(peak, fabs(traces[i]));
    printf("nt %d nrec %d peak %.6e launches %llu\n", NT, nrec, peak,
           (unsigned long long)fd_kernel_launch_count());
    if (argc > 1) {
        FILE *out = fopen(argv[1], "wb");
        if (!out || fwrite(traces, sizeof(float), (size_t)NT * nrec, out) != (size_t)NT * nrec) {
            fprintf(stderr, "cannot write %s\n", argv[1]);
            return 1;
        }
        fclose(out);
    }
    free(traces);
    free(rec);
    free(wavelet);
    free(v);
    return 0;
}
