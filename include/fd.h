/*
 * fd.h -- C ABI of the B300 acoustic finite-difference propagator (libfd).
 *
 * The library advances the acoustic wave equation of the paper's proof of
 * concept (section 7, Eq. 1),
 *
 *     P_tt = v(x)^2 (P_xx + P_zz [+ P_yy]) + S(t) delta(x - x_s),
 *
 * with the routine sequence of its WaveSimulator::run() listing (add_source,
 * fd_pzz, fd_pxx, fd_time, then the two swaps), fused into one CUDA kernel per
 * time step on an sm_103a GPU.  One step maps the levels (P, Pold) at t_n,
 * t_{n-1} to Pn at t_{n+1}:
 *
 *     L'P  = sum_{k=1..4} c_k ( S_k - 2d P ),   S_k = sum over the d axes of
 *            P[i + k e] + P[i - k e],   c = (8/5, -1/5, 8/315, -1/560)
 *            (the radius-4 Taylor stencil; P = 0 outside the grid)
 *     Pn   = ( 2P - (1 - a) Pold + w L'P ) / (1 + a),   w = (dt v / h)^2,
 *            a = dt (eta_x(ix) + eta_y(iy) + eta_z(iz))   (sponge; a = 0 inside)
 *     Pn[src] += dt^2 S(t_n) / h^d                        (add_source)
 *     trace[n][r] = Pn[rec_r]                             (receivers, at t_{n+1})
 *     Pold <- P, P <- Pn                                  (the swaps)
 *
 * The sponge profile of each axis is eta_max (d / W)^2 for a point d =
 * max(W - i, i - (n - 1 - W), 0) points into a W-point band, with
 * eta_max = 3 v_max ln(1/R) / (2 W h).  The stencil order, boundary, sponge,
 * source scaling and receivers are not fixed by the paper; these are the
 * readings this library implements.
 *
 * Following the paper's start/stop convention (section 5), every input is
 * built on the host and copied in by the library ("copyFromHost"), and every
 * output leaves through an explicit gather call ("copyToHost").  The *_dev
 * variants take device pointers instead, for callers that keep data on the
 * GPU (e.g. PyTorch tensors); the library never takes ownership of them.
 *
 * Layout: every field is x-fastest, [nz][ny][nx] in 3D and [nz][nx] in 2D
 * (ny = 1), FP32.  Points are (ix, iy, iz) with iy = 0 in 2D.
 *
 * Errors: every entry point returns an fd_status; 0 is success, negative
 * values are errors.  No entry point aborts or throws; fd_last_error() gives a
 * message for the calling thread's last failure.  On a validation error
 * nothing is modified.
 *
 * Threading: a model is used from one host thread at a time; all its GPU work
 * is ordered on the stream given at creation.  Different models are
 * independent.
 */
#ifndef FD_H
#define FD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int fd_status;

#define FD_OK        0
#define FD_EINVAL   (-1)  /* bad dimensions, NULL pointer, bad size or count      */
#define FD_ECFL     (-2)  /* v_max dt / h above the leapfrog stability limit       */
#define FD_ERANGE   (-3)  /* source or receiver outside the grid                   */
#define FD_ENOMEM   (-4)  /* device allocation failed                              */
#define FD_EBUDGET  (-5)  /* request exceeds a caller-stated memory budget         */
#define FD_ECUDA    (-6)  /* a CUDA call failed (no device, launch error, ...)     */
#define FD_ETIMEOUT (-7)  /* a bounded device-side wait gave up                    */
#define FD_ESTATE   (-8)  /* call not valid in the model's current state           */

typedef struct fd_model fd_model;   /* opaque; owns its device wavefields */

/* Grid and discretisation of one model. */
typedef struct fd_grid_desc {
    int ndim;           /* 2 or 3                                                */
    int nx, ny, nz;     /* extents >= 1; ny must be 1 when ndim == 2             */
    double h;           /* grid spacing (m), > 0, the same on every axis         */
    double dt;          /* time step (s), > 0                                    */
    int sponge_width;   /* W >= 0 points of damping band on every face           */
    double sponge_R;    /* target reflection coefficient in (0, 1); used if W > 0 */
} fd_grid_desc;

/* Stability limit of the Courant number v_max dt / h for ndim = 2 or 3:
 * 2 / sqrt(ndim lambda_1), lambda_1 = -(c_0 + 2 sum_k (-1)^k c_k) of the
 * radius-4 stencil (the leapfrog condition omega dt <= 2).  Returns a negative
 * value for any other ndim. */
double fd_cfl_limit(int ndim);

/* The FP32 stencil weights c_1..c_4 the kernels use (host memory, 4 floats). */
fd_status fd_stencil_weights(float *out4);

/* Create a model: allocates the device fields P, Pold, w = (dt v / h)^2 and
 * the sponge profiles, computes w and the profiles on the device from the
 * velocity (m/s, [nz][ny][nx], copied), and sets P = Pold = 0, n = 0.
 * stream: a cudaStream_t (NULL = the legacy default stream) on which all of the
 * model's GPU work is ordered; the caller keeps it alive until destroy.
 * Errors: FD_EINVAL (bad desc, NULL pointers, non-positive or non-finite
 * velocity), FD_ECFL (v_max dt / h > fd_cfl_limit(ndim)), FD_ENOMEM, FD_ECUDA.
 * On success *out owns the device memory until fd_model_destroy. */
fd_status fd_model_create(const fd_grid_desc *desc, const float *v_host, void *stream,
                          fd_model **out);
/* As fd_model_create, but v_dev is a device pointer (dense [nz][ny][nx]). */
fd_status fd_model_create_dev(const fd_grid_desc *desc, const float *v_dev, void *stream,
                              fd_model **out);

/* Release everything the model owns (waits for its stream first).  NULL is a no-op. */
fd_status fd_model_destroy(fd_model *m);

/* Move the model's later GPU work to another stream (a cudaStream_t of the
 * model's device; NULL = the legacy default stream).  Work already enqueued
 * keeps its order: the library records an event on the old stream and makes
 * the new stream wait for it before anything the model enqueues later.  The
 * caller keeps the new stream alive until the model is destroyed or moved
 * again.  Not part of the paper's interface: a serving loop uses it to change
 * a shot's stream priority while the shot is running.  Errors: FD_EINVAL,
 * FD_ECUDA. */
fd_status fd_set_stream(fd_model *m, void *stream);

/* A non-blocking stream of the current device with the given priority (lower
 * numbers are scheduled first; values outside the device's range are clamped
 * to it), owned by the caller until fd_stream_destroy.  *greatest, if not NULL,
 * receives the device's highest priority (a negative number on current GPUs;
 * 0 is the default priority).  Errors: FD_EINVAL, FD_ECUDA. */
fd_status fd_stream_create(int priority, void **stream, int *greatest);
/* Destroy a stream from fd_stream_create (work already enqueued still runs). */
fd_status fd_stream_destroy(void *stream);

/* Replace the velocity model (same grid and dt); recomputes w and the sponge.
 * Same checks as create (FD_EINVAL, FD_ECFL).  Does not touch P, Pold or n. */
fd_status fd_set_velocity(fd_model *m, const float *v_host);
fd_status fd_set_velocity_dev(fd_model *m, const float *v_dev);

/* Fix the sponge strength to that of velocity vmax (m/s) instead of the model's
 * largest velocity, now and across later fd_set_velocity calls (0 restores the
 * default).  Lets the damping stay fixed while an inversion changes the model. */
fd_status fd_set_sponge_vmax(fd_model *m, double vmax);

/* Point source at (ix, iy, iz) with signature S(t_n) = wavelet[n], n < nt
 * (host, copied; steps n >= nt inject nothing).  nt = 0 or wavelet = NULL
 * removes the source.  FD_ERANGE if the point is outside the grid. */
fd_status fd_set_source(fd_model *m, int ix, int iy, int iz, const float *wavelet_host, int nt);

/* Receivers at nrec points given as (ix, iy, iz) int triples (host, copied).
 * nrec = 0 removes them.  FD_ERANGE if any point is outside the grid. */
fd_status fd_set_receivers(fd_model *m, const int *xyz_host, int nrec);

/* Trace buffer for the next steps: [nt_rows][nrec] FP32 on the device.  If
 * traces_dev is NULL the library allocates (and owns) it, else it writes into
 * the caller's buffer, which must stay valid while steps run.  Step n writes
 * row n (the model's step counter) when n < nt_rows. */
fd_status fd_set_trace_buffer(fd_model *m, float *traces_dev, int nt_rows);

/* P = Pold = 0 and step counter n = 0.  Source, receivers, traces kept. */
fd_status fd_reset(fd_model *m);

/* Set the state: P (level n) and Pold (level n-1), dense host arrays, and the
 * step counter n >= 0 (checkpoint resume / initial conditions). */
fd_status fd_set_wavefield(fd_model *m, const float *p_host, const float *pold_host, int n);

/* Advance nsteps >= 0 time steps, asynchronously on the model's stream. */
fd_status fd_step(fd_model *m, int nsteps);

/* Time steps per launch for later fd_step / fd_run_shot calls: 1 (the default)
 * or, for 3D models, 2.  With 2, one launch advances two steps (temporal fusion:
 * the first step is evaluated on each CTA's column widened by the stencil
 * radius, so the second has its neighbours without leaving the chip), reading
 * P^{n-1}, P^n and w once and writing P^{n+1} and P^{n+2}: 20 bytes per point
 * for two updates instead of 32.  The levels and traces are bitwise those of
 * single steps; an odd step count ends with one single step.  The first call
 * with 2 allocates two more wavefield buffers (2 x 4 nx*ny*nz bytes, padded
 * rows) kept until the model is destroyed.  The L'P and imaging steps of the
 * adjoint and the fd_debug_stall_stage hook always run single steps.  Errors:
 * FD_EINVAL (steps not 1 or 2, or 2 for a 2D model), FD_ECUDA / FD_ENOMEM. */
fd_status fd_set_time_fusion(fd_model *m, int steps);

/* One shot: reset, record into traces_dev ([nt][nrec] device buffer, or NULL
 * for a library-owned buffer), advance nt steps.  Asynchronous. */
fd_status fd_run_shot(fd_model *m, int nt, float *traces_dev);

/* Copy the recorded traces [rows][nrec] to host memory (cap = floats available;
 * FD_EINVAL if smaller than rows * nrec).  Synchronises the model's stream. */
fd_status fd_gather_traces(fd_model *m, float *host_out, size_t cap);
/* As fd_gather_traces, but only enqueues the copy on the model's stream and
 * returns: host_out holds the traces once the stream has reached the copy
 * (fd_synchronize, or an event), and must stay valid until then.  With pinned
 * host memory the copy overlaps kernels of other streams, e.g. the next shot
 * of a second model (with pageable memory CUDA may copy synchronously).
 * FD_EINVAL if cap is smaller than rows * nrec. */
fd_status fd_gather_traces_async(fd_model *m, float *host_out, size_t cap);

/* Copy P (level n) and, if pold_host is not NULL, Pold (level n-1) to dense
 * host arrays of cap floats each.  Synchronises the model's stream. */
fd_status fd_get_wavefield(fd_model *m, float *p_host, float *pold_host, size_t cap);

/* Wait for the model's stream; reports a device-side error flag if any kernel
 * raised one (FD_ETIMEOUT for a bounded wait that gave up). */
fd_status fd_synchronize(fd_model *m);

/* Introspection (host outputs): the step counter; the linear indices
 * (iz*ny + iy)*nx + ix of the source (-1 if none) and of each receiver; the
 * per-axis damping a = dt * eta as the kernels use it (axis 0 = x, 1 = y,
 * 2 = z; n_axis floats). */
fd_status fd_get_step(fd_model *m, int *n);
fd_status fd_get_source_index(fd_model *m, int64_t *idx);
fd_status fd_get_receiver_indices(fd_model *m, int64_t *out, int cap);
fd_status fd_get_damping_profile(fd_model *m, int axis, float *out, int cap);

/* ------------------------------------------------------------------ adjoint
 *
 * Building blocks of the reverse-time adjoint (gradient of a trace misfit with
 * respect to squared slowness m = 1/v^2).  The paper names imaging and
 * inversion only as uses of its simulator (section 8); the adjoint of the
 * time step is this library's.  With w = (dt v / h)^2 and damping a, the
 * adjoint of fd_step for dJ/dtrace^n = g^n is the same step run backwards in
 * time on psi (a model with the same velocity and no source), with
 * w g^{k-1} / (1 + a) added at the receivers after step k (fd_inject_receivers),
 * and dJ/dm = -(1/m) sum_n psi_{n+1} (L' P^n).  The gradient is accumulated by
 * fd_imaging (which evaluates L' from a stored P^n), by fd_imaging_product from
 * the L'P^n that fd_step_lp writes while the forward segment is recomputed, or,
 * cheapest, inside the adjoint step itself (fd_step_image with
 * fd_inject_receivers_image).  fd_adjoint_segment runs a whole checkpoint
 * segment; fd_step_lp_n and fd_adjoint_backward serve a run that keeps every
 * L'P^n instead of checkpoints. */

/* v_dev[i] = 1 / sqrt(m_dev[i]) for n device floats of squared slowness m
 * (s^2/m^2), in FP64 and rounded once to FP32; a non-positive m gives NaN, which
 * model creation then rejects.  Asynchronous on stream (a cudaStream_t; NULL =
 * the legacy default stream).  FD_EINVAL for NULL arrays or n = 0. */
fd_status fd_velocity_from_slowness(const float *m_dev, float *v_dev, size_t n, void *stream);
/* The gradient from accumulated images: grad_dev[i] = -(acc_0[i] + ... +
 * acc_{nacc-1}[i]) / m_dev[i], where acc_dev holds nacc consecutive arrays of n
 * floats (for instance one per group of shots run concurrently), each the sum
 * over its shots and time steps of psi_{n+1} L'P^n, summed in array order.
 * Asynchronous on stream.  FD_EINVAL for NULL arrays, nacc < 1 or n = 0. */
fd_status fd_gradient_from_image(const float *acc_dev, int nacc, const float *m_dev, float *grad_dev, size_t n,
                                 void *stream);

/* Copy P (level n) and, if pold_dev is not NULL, Pold to dense device arrays
 * [nz][ny][nx] (asynchronous on the model's stream). */
fd_status fd_get_wavefield_dev(fd_model *m, float *p_dev, float *pold_dev);
/* Set P, Pold from dense device arrays and the step counter n (asynchronous). */
fd_status fd_set_wavefield_dev(fd_model *m, const float *p_dev, const float *pold_dev, int n);
/* Add values_dev[r] * w / (1 + a) to P at each receiver r (values: nrec floats on
 * the device; the adjoint-source injection).  Receivers that share a grid point
 * have their values summed in receiver order first, so the result is the same
 * from run to run (no atomics). */
fd_status fd_inject_receivers(fd_model *m, const float *values_dev);
/* grad_dev += P_adj * (L' p_dev) over dense [nz][ny][nx] device arrays, where
 * P_adj is the current level of the model adj and L' the stencil sum. */
fd_status fd_imaging(fd_model *adj, const float *p_dev, float *grad_dev);
/* One time step, as fd_step(m, 1), that also writes L'P^n -- the stencil sum of
 * the level n it consumes, sum_k c_k D_k in the step's own FP32 arithmetic --
 * to lp_dev, a dense [nz][ny][nx] device array (asynchronous).  This is the
 * factor the imaging condition needs, produced while the forward segment is
 * recomputed, so the adjoint pass needs neither a copy of P^n nor a second
 * stencil. */
fd_status fd_step_lp(fd_model *m, float *lp_dev);   /* FD_EINVAL: NULL lp_dev (nx*ny*nz floats, the caller's) */
/* grad_dev += P_adj * lp_dev pointwise over dense [nz][ny][nx] device arrays,
 * where P_adj is the current level of adj and lp_dev comes from fd_step_lp
 * (asynchronous on adj's stream; one FMA per point).  Both arrays belong to
 * the caller.  FD_EINVAL for NULL arguments. */
fd_status fd_imaging_product(fd_model *adj, const float *lp_dev, float *grad_dev);
/* One time step, as fd_step(m, 1), that also adds Pn * lp_dev to grad_dev
 * pointwise (dense [nz][ny][nx] device arrays of the caller), Pn being the level
 * the step produces: the imaging condition fused into the adjoint step, one pass
 * over the grid instead of a step plus fd_imaging_product.  FD_EINVAL for NULL
 * arrays. */
fd_status fd_step_image(fd_model *m, const float *lp_dev, float *grad_dev);
/* As fd_inject_receivers, and adds each injected value times lp_dev at its
 * receiver point to grad_dev (dense arrays); after fd_step_image this makes the
 * gradient update (level + injection) * lp_dev.  FD_EINVAL for NULL arrays. */
fd_status fd_inject_receivers_image(fd_model *m, const float *values_dev, const float *lp_dev, float *grad_dev);
/* nsteps >= 0 calls of fd_step_lp, the j-th writing lp_buf + j * nx*ny*nz
 * (nsteps dense fields, the caller's): the forward pass of an adjoint that keeps
 * every L'P^n instead of checkpoints (HBM permitting).  FD_EINVAL for a NULL
 * buffer with nsteps > 0. */
fd_status fd_step_lp_n(fd_model *m, int nsteps, float *lp_buf);
/* The backward half of fd_adjoint_segment: for k = n1 down to n0 + 1 the adjoint
 * model adj takes one step (fd_step_image with lp_buf + (k-1-n0) * nx*ny*nz) and
 * receives g_dev + (k-1) * nrec (fd_inject_receivers_image), adding
 * psi_k * L'P^{k-1} to grad_dev.  With the L'P^n of a whole run stored by
 * fd_step_lp_n, one call with n0 = 0, n1 = nt needs no recompute.  FD_EINVAL for
 * bad arguments.  Asynchronous on adj's stream. */
fd_status fd_adjoint_backward(fd_model *adj, int n0, int n1, const float *lp_buf, const float *g_dev,
                              float *grad_dev);
/* One checkpoint segment [n0, n1) of the reverse-time adjoint, issued from the
 * host in one call (asynchronous; fwd and adj must share a stream and a grid).
 * The forward model fwd must be at step n0 (its levels n0 and n0-1 restored,
 * e.g. by fd_set_wavefield_dev); it advances n1 - n0 steps with fd_step_lp,
 * storing L'P^{n0+j} in lp_buf + j * nx*ny*nz (n1 - n0 dense fields, owned by
 * the caller).  Then for k = n1 down to n0 + 1 the adjoint model adj takes one
 * step, receives g_dev + (k-1) * nrec at its receivers, and psi_k * L'P^{k-1} is
 * added to grad_dev (fd_step_image, fd_inject_receivers_image).  Returns
 * FD_EINVAL for bad arguments, FD_ESTATE if fwd is not at step n0. */
fd_status fd_adjoint_segment(fd_model *fwd, fd_model *adj, int n0, int n1, float *lp_buf, const float *g_dev,
                             float *grad_dev);

/* --------------------------------------------------------- unfused routines
 *
 * The paper's routines one kernel each, as in its WaveSimulator::run()
 * (section 7, Listing 3): fd_pzz, fd_pxx (and, in 3D, the y counterpart) each
 * write one second-derivative field D2 = sum_k c_k ((P[+k] + P[-k]) - 2P);
 * fd_time writes Pn = (2P - (1 - a) Pold + w (Pxx [+ Pyy] + Pzz)) / (1 + a) over
 * Pold; add_source adds dt^2 S(t_n) / h^d to Pn; the swap gathers the step's
 * receivers and rotates the levels (step counter + 1).  The derivative fields
 * are allocated on first use.  This schedule moves ~40 B per update in 2D
 * (52 in 3D) against fd_step's 16 and exists for comparison on the same
 * hardware; it computes the same recurrence up to the order in which the axes
 * are summed.  Calls are asynchronous on the model's stream. */
#define FD_ROUTINE_ADD_SOURCE 0
#define FD_ROUTINE_PZZ        1
#define FD_ROUTINE_PXX        2
#define FD_ROUTINE_PYY        3
#define FD_ROUTINE_TIME       4
#define FD_ROUTINE_SWAP       5
/* One routine (FD_EINVAL for an unknown one, or PYY on a 2D model). */
fd_status fd_routine(fd_model *m, int routine);
/* nsteps steps of the sequence PZZ, PXX, [PYY,] TIME, ADD_SOURCE, SWAP. */
fd_status fd_step_unfused(fd_model *m, int nsteps);

/* ----------------------------------------------------------------- batches
 *
 * A batch advances many independent 2D shots (models) in one persistent,
 * cooperative kernel launch instead of one launch per shot and time step.  The
 * paper has no batching: this is the multi-shot form of the same time step
 * (section 7, Listing 3), with identical arithmetic, so every shot's
 * wavefield and traces are bitwise the same alone (fd_step) and in a batch.
 *
 * Work items are (shot, tile) pairs.  Each tile keeps a completed-step
 * counter in device memory; a tile starts step k + 1 only when it and its four
 * neighbours have completed step k (all waits are bounded; on expiry the
 * launch stops and fd_batch_step returns FD_ETIMEOUT).  Shots are advanced in
 * groups whose fields fit a stated budget, so a group stays in the 126 MB L2
 * across its time steps.  One launch advances every shot by up to
 * steps_per_launch steps; a run replays one captured CUDA graph node.
 *
 * The models stay owned by the caller and must outlive the batch.  A batch
 * call waits for the models' streams, runs on a stream of the batch's own and
 * returns when the work is done; meanwhile the models must not be used
 * otherwise. */
typedef struct fd_batch fd_batch;

typedef struct fd_batch_tuning {
    int tile;              /* schedule and tile shape (x by z): one persistent launch with
                              0 = 64 x 16, 1 = 64 x 32, 2 = 128 x 16 tiles; or one ordinary
                              launch per time step over all of a group's shots (tensor maps
                              in the launch parameters, up to 64 shots a launch) with
                              3 = 64 x 16, 4 = 64 x 32 tiles, or 5 / 6 / 7 = 64 x 16 tiles
                              in columns of 4 / 8 / 16 per CTA (double-buffered loads)       */
    int steps_per_launch;  /* time steps per persistent launch, >= 1 (persistent only)      */
    int ctas_per_sm;       /* resident CTAs per SM, 0 = as many as fit (persistent only)    */
    int group_mb;          /* L2 budget per shot group in MB, 0 = all shots in one group;
                              the groups run one after another                              */
} fd_batch_tuning;

/* Build a batch over nmodels models on the same device, all 2D or all 3D
 * (FD_EINVAL for a mix, NULL entries or a repeated model).  2D batches run the
 * schedule of their tuning.  3D batches run one launch per time step over up to
 * 48 models that still have steps to go, each CTA stepping its own model with
 * the single-shot 3D kernel (maps and parameters in the launch); their tuning
 * is not used, and fd_batch_autotune leaves it unchanged. */
fd_status fd_batch_create(fd_model *const *models, int nmodels, fd_batch **out);
fd_status fd_batch_destroy(fd_batch *b);
/* Set / read the tuning (validated; FD_EINVAL for out-of-range values). */
fd_status fd_batch_set_tuning(fd_batch *b, const fd_batch_tuning *t);
fd_status fd_batch_get_tuning(fd_batch *b, fd_batch_tuning *t);
/* Advance shot i by nsteps_each[i] steps (or every shot by nsteps when
 * nsteps_each is NULL), exactly as fd_step would, traces included.  Blocks
 * until done; returns FD_ETIMEOUT if a bounded device wait gave up. */
fd_status fd_batch_step(fd_batch *b, int nsteps, const int *nsteps_each);
/* Test hook for the failure path (persistent schedules, tiles 0-2): from the next fd_batch_step on, work item
 * stalled_item (0-based in the batch's (shot, tile) order; -1 clears it) never
 * runs, so its neighbours' bounded waits run out and the call returns
 * FD_ETIMEOUT with the context still usable.  After FD_ETIMEOUT the shots'
 * wavefields are undefined until reset. */
fd_status fd_batch_set_fault(fd_batch *b, int stalled_item);
/* Time every tuning candidate on trial_steps steps of this batch, keep the
 * fastest (cached per batch shape for the process) and write it to best.  The
 * candidates are every schedule and tile shape, group budgets of 0, 24, 48 and
 * 96 MB (those below the batch's footprint), and for the persistent schedules
 * 0 or 2 CTAs per SM and trial_steps, trial_steps / 2, trial_steps / 4 and the
 * current steps_per_launch (when shorter) steps per launch.  A trial cannot
 * time a launch longer than itself: when trial_steps steps per launch wins and
 * the current value is larger, the current value is kept (the wide schedules
 * also keep it; they do not use it).  FD_EINVAL for trial_steps < 1.  The
 * trial steps change the models' state: call fd_reset or fd_run_shot after.
 * A 3D batch has nothing to tune and is left unchanged. */
fd_status fd_batch_autotune(fd_batch *b, int trial_steps, fd_batch_tuning *best);

/* Allocation-free form of fd_batch_step.  The paper has no counterpart: it is
 * an entry point for callers that cannot allocate device memory once they are
 * running, such as a serving process whose memory pool already holds all the
 * device memory it was given, or a latency-bound loop that must not pay the
 * device-wide synchronisation that cudaMalloc and cudaFree imply.  Such a
 * caller creates its 2D models at start-up (fd_model_create and friends) and
 * advances them here: every model moves nsteps steps exactly as fd_step would,
 * traces included, in one persistent launch on the first model's stream; the
 * call returns when the work is done.
 *
 * No device or host memory is allocated.  The launch's scratch (shot
 * descriptors, tile table, receiver lists, per-tile step counters, launch
 * state, error word) lives in one static device array of about 1.8 MB that
 * every device loading the library holds until the process exits.  Limits:
 * at most 64 models, 32768 tiles of 64 x 16 points in total and 32768
 * receivers in total; larger requests return FD_EBUDGET and change nothing.
 * The first call on a device looks up the array's device address and sets the
 * kernel's shared-memory limit; the address is cached per device for the life
 * of the process, which assumes the device's primary context is never reset
 * (after cudaDeviceReset the cache is stale).  Every call synchronises the
 * models' streams and reads the error word back synchronously, so no call may
 * be made inside a stream capture, nor while another thread captures in
 * global mode.  Every call shares the array and leaves its tables there; the
 * call clears the counters, launch state and error word it uses before
 * launching.  Calls hold a process-wide lock until their kernel has finished,
 * so two calls of one process never overlap on the GPU; two processes have
 * separate arrays.  Host work per call is O(models + tiles + receivers).
 * Errors as fd_batch_step (FD_EINVAL, FD_EBUDGET, FD_ECUDA, FD_ETIMEOUT). */
fd_status fd_batch_step_noalloc(fd_model *const *models, int nmodels, int nsteps);

/* Test hook: fill the row padding of the model's device fields -- columns nx
 * .. px-1 of every row of P, Pold, w and any unfused derivative field, where
 * px is nx rounded up to 32 -- with NaN (asynchronous).  No kernel reads or
 * writes those columns, so results stay finite and unchanged; tests use this
 * in place of a memory checker.  fd_reset clears the padding again.  A no-op
 * when nx is a multiple of 32. */
fd_status fd_debug_poison_padding(fd_model *m);

/* Test hook for the step kernel's failure path: while stage >= 0, the first CTA
 * of every 3D step launch never issues the TMA load of its two-plane P stage
 * `stage` (counted from its first halo plane), so that CTA's bounded waits run
 * out (about 2 s): the kernel raises the device error word, its other CTAs
 * finish, and fd_synchronize returns FD_ETIMEOUT with the context still usable.
 * The wavefield is undefined afterwards until reset.  -1 clears the hook.
 * 2D models ignore it. */
fd_status fd_debug_stall_stage(fd_model *m, int stage);

/* Number of CUDA kernel launches this library has issued since load. */
uint64_t fd_kernel_launch_count(void);

/* Message for the calling thread's last error ("" if none). */
const char *fd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FD_H */
