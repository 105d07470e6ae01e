/*
 * teuk.h -- C ABI of the GB300 (sm_103a) Teukolsky time-domain solver.
 *
 * The library advances the (2+1)D Teukolsky equation for one azimuthal mode m
 * (Khanna & McKennon, arXiv 1001.3631, Sec. 2) with the two-step Lax-Wendroff
 * scheme of Eqs. (13)-(14), on the (r*, theta) grid of Eqs. (2)-(4), with the
 * boundary conditions stated after Eq. (14), plus a smeared point-particle
 * source.  Every step of the time loop runs in the library's CUDA kernels on
 * the device; host code only validates arguments, launches and copies.
 *
 * Conventions shared by every entry point:
 *   - Grid: r*_i = rstar_min + i dr*, i = 0 .. n_rstar-1, dr* = (rstar_max -
 *     rstar_min)/(n_rstar - 1); theta_j = (j + 1/2) pi / n_theta.
 *   - State layout on the host side, "u-layout": double [4][n_theta][n_rstar]
 *     holding {Phi_R, Phi_I, Pi_R, Pi_I} (the solution vector u of Eq. 9),
 *     Pi = d_t Phi + b d_r* Phi (Eq. 5).
 *   - Waveform record n: W_n[j] = Phi^n(r*_ext, theta_j), linear in r* between
 *     the two bracketing nodes, as FP64 (re, im) pairs [n_theta][2].
 *   - All host pointers are caller-owned; the library copies what it needs and
 *     keeps no host pointer past the call.  Device memory is owned by the
 *     context and released by teuk_destroy.
 *   - Work is queued on the caller's CUDA stream (the cuda_stream of
 *     teuk_create; NULL is the legacy default stream).  The context's CUDA graphs
 *     are captured on a private stream of its own and replayed on that stream.
 *     Calls that return host data synchronize that stream.
 *   - Every call returns a teuk_status; teuk_last_error() gives the message of
 *     the last failing call on that context.  Nothing aborts the process and
 *     no kernel traps: device-side failures are reported through a status
 *     word read at the next synchronizing call.  There is no CPU fallback: a
 *     missing or unusable GPU is TEUK_ECUDA.
 */
#ifndef TEUK_H
#define TEUK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TEUK_OK = 0,
    TEUK_EINVAL = 1,    /* invalid argument; nothing was changed or allocated */
    TEUK_ENOMEM = 2,    /* device allocation failed */
    TEUK_ECUDA = 3,     /* CUDA runtime error (no device, launch failure, ...) */
    TEUK_EUNSTABLE = 4, /* non-finite values found in the state or waveform */
    TEUK_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    TEUK_ESTATE = 6,    /* call not valid in the context's current state */
    TEUK_EBOUNDS = 7    /* checked builds: a device-side index check failed */
} teuk_status;

typedef enum {
    TEUK_FP64 = 0,        /* state, coefficients and arithmetic in FP64 */
    TEUK_FP32 = 1,        /* state and arithmetic in FP32 (coefficients rounded from FP64) */
    TEUK_FP32_KAHAN = 2,  /* FP32 arithmetic, state as compensated (hi, c) FP32 pairs */
    TEUK_FP64_DF = 3      /* FP64-equivalent: state, coefficients and arithmetic in
                           * double-float (hi + lo FP32 pairs, ~48 significant bits)
                           * on the FP32 units; the adjoint uses an FP64 co-state */
} teuk_precision;

/*
 * Problem statement of one instance (one mode, one orbit, one grid).
 * s, m, M, a: spin weight, azimuthal mode, Kerr mass and spin of Eq. (1); |a| < M.
 * rstar_min, rstar_max, n_rstar: radial grid (Eq. 2); n_rstar >= 8.
 * n_theta: angular cells; 4 <= n_theta <= 1024.
 * courant, dt_rule, dt: the time step.  dt > 0 is used as given; otherwise
 *   dt_rule 0: dt = courant * dr*  (the Courant factor read literally), or
 *   dt_rule 1: dt = courant * min(dr*, dtheta / (|m| + |s| + 2)), which keeps the
 *              explicitly integrated angular terms of Eq. (13)-(14) bounded.
 * rstar_ext: extraction radius, inside [rstar_min, rstar_max].
 * prec: arithmetic of this instance (all instances of a context must agree).
 * wave_capacity: number of waveform records kept on the device (a ring); 0 means
 *   4096.
 * slab_col0, slab_ncols: slab_ncols = 0 for the whole grid.  Otherwise the instance is a
 *   slab of the grid above (the r* decomposition of the grid over ranks): it owns the
 *   grid columns [slab_col0, slab_col0 + slab_ncols) (1 <= slab_col0, slab_col0 +
 *   slab_ncols <= n_rstar - 1, slab_ncols >= 2) and holds one more column on each side,
 *   the grid's end column or a halo that teuk_slab_import fills from the neighbouring
 *   slab after every step.  Its local column k is grid column slab_col0 - 1 + k; states
 *   (teuk_set_state / teuk_get_state) have slab_ncols + 2 columns.  Node positions,
 *   coefficients, source and time step are those of the whole grid, so slabs stepped one
 *   step at a time with their halos exchanged reproduce the whole grid bit for bit.
 */
typedef struct {
    int s, m;
    double M, a;
    double rstar_min, rstar_max;
    int n_rstar, n_theta;
    double courant;
    int dt_rule;
    double dt;
    double rstar_ext;
    int prec;
    int64_t wave_capacity;
    int slab_col0, slab_ncols;
} teuk_params;

/*
 * Synthetic particle source (the paper's source T is a Maple expression that is
 * not printed, Sec. 2.1 and Sec. 3): a particle on a prograde circular
 * equatorial orbit of radius r0, smeared by a 2D Gaussian in (r*, theta)
 * centred on (r*(r0), pi/2), truncated at 8 sigma:
 *   T_m = A_n exp(-i m (Omega t + phi0)) G,  Omega = M^(1/2)/(r0^(3/2) + a M^(1/2)),
 *   phi0 = a/(r_+ - r_-) ln((r0 - r_+)/(r0 - r_-)),
 * entering S_Pi as tau = 4 pi Delta (r^2 + a^2 cos^2) T_m / (Sigma^2 r^3).
 * Widths: sigma_*_abs > 0 in absolute units, else sigma_*_cells grid cells
 * (0 means 4 cells).
 */
typedef struct {
    double r0;
    double sigma_rstar_cells, sigma_theta_cells;
    double sigma_rstar_abs, sigma_theta_abs;
} teuk_orbit;

typedef struct teuk_ctx teuk_ctx;

/* Device-memory hooks (teuk_set_allocator): alloc returns `bytes` of device memory usable
 * in stream order on cuda_stream (a cudaStream_t), or NULL on failure; free releases a
 * block that alloc returned, in stream order on cuda_stream.  user is passed through. */
typedef void* (*teuk_alloc_fn)(size_t bytes, void* cuda_stream, void* user);
typedef void (*teuk_free_fn)(void* ptr, void* cuda_stream, void* user);

/* Route the device memory of contexts created from now on through the caller's allocator
 * (for example a framework's caching allocator, so that the library and the framework
 * share one pool); alloc = free = NULL restores the default, cudaMallocAsync /
 * cudaFreeAsync on the context's stream.  A context keeps the allocator it was created
 * with for all its allocations (state, tables, source, waveform ring, batched and adjoint
 * buffers) until teuk_destroy.  A NULL return from alloc makes the call that needed the
 * memory fail with TEUK_ENOMEM (teuk_create then frees what it had taken).  Not thread
 * safe against concurrent teuk_create.  TEUK_EINVAL if exactly one function is NULL. */
teuk_status teuk_set_allocator(teuk_alloc_fn alloc, teuk_free_fn free_fn, void* user);

/* Create a context of n_instances independent instances p[0 .. n_instances-1]
 * (uneven grids allowed), on the caller's stream (cudaStream_t passed as void*).
 * Builds the grids, inverts Eq. (2) for r at every node, forms the coefficient
 * tables, and zeroes the state; no source is set (tau = 0) until
 * teuk_set_source.  *out is NULL on failure.  Validation failures are
 * TEUK_EINVAL with nothing allocated. */
teuk_status teuk_create(const teuk_params* p, int n_instances, void* cuda_stream,
                        teuk_ctx** out);

/* Set the particle source of one instance.  amps: A_n for global step n < n_amps
 * (host, copied); steps n >= n_amps (or amps == NULL) use A_n = 1.
 * TEUK_EINVAL if r0 is not outside the horizon or the orbit is off the grid. */
teuk_status teuk_set_source(teuk_ctx* ctx, int instance, const teuk_orbit* orbit,
                            const double* amps, int64_t n_amps);

/* Moving particle (an eccentric or inclined orbit, the setting of Sec. 1): replace the
 * source of one instance by the same smeared particle following a sampled path.
 *   traj   host array [n_samples][4] = {r_p, theta_p, phi_p, A} at t = k dt/2,
 *          k = 0 .. n_samples-1 (copied; t counts from global step 0).
 *   widths Gaussian widths as in teuk_orbit (r0 ignored); NULL: 4 cells each.
 * The source at sample k is
 *   T_m = A_k exp(-i m phi_p,k) G(r* - r*(r_p,k), theta - theta_p,k)
 * (G the truncated 2D Gaussian above), entering S_Pi as tau of teuk_set_source.
 * Step n takes sample 2n in Eq. (13) (time t_n, half nodes) and sample 2n + 1 in
 * Eq. (14) (time t_n + dt/2, integer nodes); a sub-step with no sample has no
 * source.  A circular path r_p = r0, theta_p = pi/2, phi_p = Omega t + phi0 gives the
 * source of teuk_set_source.
 * Setup: one kernel tabulates, per step, the radial Gaussian factor of every column
 * and the angular factor of every row of the window that bounds the whole path, and
 * the complex amplitude of the two samples; the step kernels multiply them into a
 * static prefactor profile.  Device memory: about (n_samples / 2) x (2 window
 * columns + 2 window rows) values of the arithmetic type, plus 48 bytes a sample.
 * Synchronizes.  TEUK_EINVAL (source unchanged) if a sample is not finite, r_p is
 * not outside the horizon, theta_p is outside (0, pi), the path leaves the radial
 * grid, or n_samples < 1; TEUK_ENOMEM / TEUK_ECUDA on device failures (the instance
 * is then left without a source).  teuk_adjoint_n refuses instances with a moving
 * source (its gradients are those of the circular orbit); teuk_set_source replaces
 * the moving source. */
teuk_status teuk_set_trajectory(teuk_ctx* ctx, int instance, const teuk_orbit* widths,
                                const double* traj, int64_t n_samples);

/* Replace the state of one instance from host memory in u-layout (copied) and
 * set its time level to step0 (t = step0 dt).  Clears that instance's
 * waveform records.  Synchronizes.  The first call of teuk_set_state or
 * teuk_get_state on an instance allocates a device staging buffer of
 * 32 n_rstar n_theta bytes, kept until teuk_destroy. */
teuk_status teuk_set_state(teuk_ctx* ctx, int instance, const double* host_u, int64_t step0);

/* Copy the state of one instance to host memory in u-layout (through the staging
 * buffer described at teuk_set_state).  Synchronizes. */
teuk_status teuk_get_state(teuk_ctx* ctx, int instance, double* host_u);

/* Checkpoint and resume of one instance (no counterpart in the paper: long runs are
 * stopped and resumed).  The file holds the instance's parameters, its time level and
 * the planes of its current level in the library's own layout (the Kahan compensation
 * and the double-float low parts as stored), in one file.
 * teuk_save_state: writes path (created or truncated); synchronizes.
 * teuk_load_state: reads path into the instance.  The saved parameters must equal the
 * instance's (all of teuk_params but wave_capacity), else TEUK_EINVAL and nothing is
 * changed.  Sets the time level to the saved one and clears the waveform records, as
 * teuk_set_state does; with the same source and launch form the steps that follow are
 * bit for bit those that follow the save.  Synchronizes.
 * File errors (cannot open, short read or write, not a saved state): TEUK_EINVAL. */
teuk_status teuk_save_state(teuk_ctx* ctx, int instance, const char* path);
teuk_status teuk_load_state(teuk_ctx* ctx, int instance, const char* path);

/* Advance every instance by n full Lax-Wendroff steps (Eqs. 13-14), recording the
 * waveform at every time level.  Asynchronous on the context's stream.  A single
 * instance stepped one launch per step replays a CUDA graph of 64 launches (captured on
 * first use and again when the launch configuration changes; one per parity of the
 * buffer holding the state) for each whole 64 steps and launches the rest directly.  The
 * graphs are captured on a private stream of the context and replayed on its stream;
 * while the caller is capturing that stream every step is launched directly.  The
 * results are the same either way. */
teuk_status teuk_step_n(teuk_ctx* ctx, int64_t n);

/* Copy the waveform records of one instance to host memory: out [k][n_theta][2]
 * and, if out_scalar != NULL, w_n = sum_j W_n[j] sin(theta_j) dtheta as [k][2]
 * (FP64, j ascending).  Records are the time levels first_step .. first_step+k-1
 * where k = min(cap_steps, records held) and the records are the most recent
 * ones held (the ring keeps wave_capacity).  *n_written = k, *first_step is the
 * time level of the first record.  Synchronizes. */
teuk_status teuk_extract(teuk_ctx* ctx, int instance, double* out, double* out_scalar,
                         int64_t cap_steps, int64_t* n_written, int64_t* first_step);

/* The waveform summed over modes: the instances of the context are the modes m_i of
 * one problem (the same s, M, a, n_theta, time step and extraction radius; with
 * dt_rule 1 the step depends on |m|, so set dt), and the field of Eqs. (3)-(4),
 * Psi = sum_m e^{i m phi~} r^3 Phi_m, is formed at the extraction radius:
 *   out[k][j][l] = r_ext^3 sum_i e^{i m_i phi~_l} W_i[first + k][j]
 *   phi~_l = phi[l] + a/(r_+ - r_-) ln((r_ext - r_+)/(r_ext - r_-))      (Eq. 3)
 * for the time levels first .. first + n_records - 1 (each held by every instance,
 * see teuk_extract) and the azimuths phi[0 .. n_phi-1] (host), instances added in
 * index order, in one kernel.  out: host [n_records][n_theta][n_phi][2] (re, im).
 * Allocates and frees 16 n_records n_theta n_phi bytes of device memory; synchronizes.
 * TEUK_EINVAL if the instances are not modes of one problem, a record is not held,
 * or n_phi < 1. */
teuk_status teuk_mode_sum(teuk_ctx* ctx, const double* phi, int n_phi, int64_t first,
                          int64_t n_records, double* out);

/* Energy, linear momentum and angular momentum about the spin axis carried off by the
 * field of the context's instances, the modes m_i of one problem (as teuk_mode_sum, and
 * no two with the same m): the recoil of Sec. 2.2 (the system's kick velocity is
 * -P / M_total).  The paper prints no flux formula; these are Teukolsky and Press's
 * (1974, Kinnersley tetrad), from the records at the extraction radius r, taken far
 * from the source:
 *   r psi_4 = sum_i W_i e^{i m_i phi~} (r / (r - i a cos theta))^4   (psi_4 = rho^4 Psi,
 *             Psi = e^{i m phi~} r^3 Phi of Eq. 4; phi~ of Eq. 3 at r)
 *   N = int r psi_4 dt,  H = int N dt  (trapezoid rule from the record `first`)
 *   dE/dt = 1/(4 pi) oint |N|^2 dOmega,   dP/dt = 1/(4 pi) oint n |N|^2 dOmega,
 *   dJz/dt = -1/(4 pi) Re oint conj(N) d_phi H dOmega,
 * n = (sin th cos phi, sin th sin phi, cos th) in Boyer-Lindquist phi; theta by the
 * midpoint rule of the waveform sum (weights sin theta_j dtheta), the azimuth exactly.
 * Out (host): [n_records][10] FP64: dE/dt, dPx/dt, dPy/dt, dPz/dt, dJz/dt, E, Px, Py,
 * Pz, Jz at the time levels first .. first + n_records - 1 (totals from `first`).
 * In kernels: chunked time scans, each record's sums over modes and rows in a fixed
 * order, a block per quantity for the totals.  Allocates and frees at most 128 MB of
 * scan scratch plus 40 n_records ceil(n_theta / max(1, 256 / K)) + 80 n_records bytes
 * of device memory (K instances, at most 256); synchronizes.  TEUK_EINVAL if the
 * instances are not distinct modes of one problem or a record is not held. */
teuk_status teuk_radiated_flux(teuk_ctx* ctx, int64_t first, int64_t n_records, double* out);

/* Reverse-mode derivative of a waveform loss over the steps step0 .. step0+n-1 of
 * one instance (the transposed stencil of Eqs. 13-14, applied in kernels).
 *   grad_wave != NULL: host [n][n_theta][2] holding dL/dW for records step0+1 ..
 *     step0+n (real and imaginary parts); no forward state is needed because the
 *     step is linear; the context's state is not touched; *loss is not written.
 *   grad_wave == NULL: the built-in loss L = sum_{k=1..n} sum_j |r_ext^3 W_{step0+k}[j]|^2
 *     (psi = r^3 Phi, Eq. 4).  The instance's time level must be step0
 *     (else TEUK_ESTATE).  The forward sweep runs from the current state.
 *     ckpt_every <= 0: it keeps the cotangent of every record (16 n n_theta bytes)
 *     and the reverse sweep follows; ckpt_every = K > 0: it keeps a state
 *     checkpoint every K steps instead and the reverse sweep recomputes each
 *     segment's records from its checkpoint (one more forward sweep of work; the
 *     cotangent array is still n records long).  The state ends at step0 + n.
 * With a source, the reverse step stores the co-state over the source window into a
 * ring of at most 256 steps (32 MB at most), turned into gradients every ring's worth of
 * steps by one launch with a block per step.
 * Out (host): grad_amps[k] = dL/dA_{step0+k} (n values, may be NULL),
 *   *grad_r0 = dL/dr0 (may be NULL), *loss (built-in loss only, may be NULL).
 * The co-state is FP64 for TEUK_FP64 instances and compensated FP32 (the Kahan
 * scheme of the forward state) for the FP32 precisions; the gradient and loss sums
 * are FP64.  Synchronizes. */
teuk_status teuk_adjoint_n(teuk_ctx* ctx, int instance, int64_t step0, int64_t n,
                           int64_t ckpt_every, const double* grad_wave, double* grad_amps,
                           double* grad_r0, double* loss);

/* Wait for queued work, read the device status word and check the state of
 * every instance for non-finite values (TEUK_EUNSTABLE); a bounded device wait
 * that gave up is TEUK_ETIMEOUT; in a checked build, an index that failed its bounds
 * check is TEUK_EBOUNDS.  The status word is cleared once reported. */
teuk_status teuk_sync(teuk_ctx* ctx);

/* Halo exchange of slab instances (teuk_params.slab_ncols > 0), one column of the current
 * level in the state's own layout, device to device on the context's stream: planes
 * (1 for TEUK_FP32, else 2) one after the other, each pitch 16-byte nodes (pitch = n_theta
 * rounded up to a multiple of 32); teuk_slab_halo_bytes gives the size.
 *   teuk_slab_export: side 0 copies the first owned column, side 1 the last, to dev_buf.
 *   teuk_slab_import: side 0 fills the left halo, side 1 the right halo, from dev_buf
 *     (the column the neighbour exported at the same time level), and retakes the
 *     waveform record of that level if it reads the halo.
 * After each teuk_step_n(ctx, 1) every slab exports its two end columns and imports its
 * neighbours'; the caller moves the buffers (a device copy on one GPU, NCCL send / recv
 * or another transport between ranks).  The grid's own end columns are not imported:
 * they stay zero (the radial boundary condition).  TEUK_EINVAL for a non-slab instance,
 * a side other than 0 or 1, or a NULL buffer. */
teuk_status teuk_slab_halo_bytes(const teuk_ctx* ctx, int instance, int64_t* bytes);
teuk_status teuk_slab_export(teuk_ctx* ctx, int instance, int side, void* dev_buf);
teuk_status teuk_slab_import(teuk_ctx* ctx, int instance, int side, const void* dev_buf);

/* Time level (global step index) of one instance, and its time step dt. */
teuk_status teuk_get_time(const teuk_ctx* ctx, int instance, int64_t* step, double* dt);

/* Derived geometry of one instance: out[0..7] = {dr*, dtheta, dt, r_+, r_-, r_ext,
 * i_e, f_e} with r_ext = r(rstar_ext) (Eq. 2 inverted) and the extraction weights
 * W = (1 - f_e) Phi_{i_e} + f_e Phi_{i_e + 1}. */
teuk_status teuk_get_geometry(const teuk_ctx* ctx, int instance, double* out);

/* Launch configuration: r* columns per thread block ("strip"; a block holds one whole
 * theta column and streams along r*) for every instance (0 = automatic; a
 * per-instance choice from teuk_set_instance_tiling / teuk_autotune wins), and the
 * launch mode: steps_per_launch >= 1 launches one fused kernel per step (single-instance
 * contexts); 0 sends a single-instance context through the persistent batched kernel
 * that multi-instance contexts always use.  Results do not depend on either choice
 * (the per-point arithmetic is fixed). */
teuk_status teuk_set_tiling(teuk_ctx* ctx, int strip, int steps_per_launch);

/* Resident launches for a single-instance context whose grid fits the GPU's shared
 * memory (a not-in-the-paper launch form for small grids, such as 800 x 64): each
 * teuk_step_n becomes one cooperative launch in which every block keeps a run of r*
 * columns (with `halo` columns on each side) in shared memory for all n steps and
 * exchanges `halo` boundary columns with its neighbours through global memory every
 * `halo` steps, with bounded waits (TEUK_ETIMEOUT after about one second).  The state is
 * read once at the start and written once at the end; the results equal those of one
 * launch per step (the per-node arithmetic is the same).  halo = 0 turns it off.
 * Instances with a moving particle are still stepped one launch per step.
 * TEUK_EINVAL if the context has several instances or the grid does not fit (every
 * block must own >= halo columns, hold them in shared memory, and all blocks must be
 * resident at once).  Allocates the exchange slots (2 x blocks x 2 x halo columns).
 * teuk_set_resident_shape also sets the number of blocks per SM the column runs are cut
 * for (blocks_per_sm >= 1; teuk_set_resident takes 1): with several, the runs are
 * shorter and one block's halo wait overlaps another block's arithmetic on the same SM.
 * A shape that does not fit is TEUK_EINVAL. */
teuk_status teuk_set_resident(teuk_ctx* ctx, int halo);
teuk_status teuk_set_resident_shape(teuk_ctx* ctx, int halo, int blocks_per_sm);

/* Blocked launches for a single-instance context whose grid fits the GPU's shared memory
 * (a not-in-the-paper launch form for small grids): each launch advances `steps` steps
 * (the last one of a teuk_step_n the rest), every block holding its run of r* columns with
 * `steps` halo columns on each side in shared memory and computing the steps on the
 * shrinking region, the halos read from the previous launch's output; there is no
 * exchange and no wait between blocks (the launch boundary, with programmatic dependent
 * launch, is the synchronisation), and each launch writes the other state buffer.  The
 * results equal those of one launch per step.  Runs cut for blocks_per_sm blocks per SM
 * as in teuk_set_resident_shape.  steps = 0 turns it off; steps is at most 4; a shape that
 * does not fit is TEUK_EINVAL.  Allocates as teuk_set_resident does. */
teuk_status teuk_set_blocked(teuk_ctx* ctx, int steps, int blocks_per_sm);

/* Strip length (r* columns per block) of one instance (0 = back to the context default). */
teuk_status teuk_set_instance_tiling(teuk_ctx* ctx, int instance, int strip);

/* Autotuner of the strip length (r* columns per block), written to every instance
 * (chosen, may be NULL, receives them).  A single instance stepped one launch per step:
 * trial_steps steps of each candidate (1 .. 512 columns) and of resident launches with
 * halo 1 .. 4 and 1 .. 3 blocks per SM (teuk_set_resident_shape, where the grid fits) on
 * a scratch copy of the instance; the fastest is applied, and chosen[k] < 0 reports
 * resident launches with halo (-chosen[k]) % 16 and (-chosen[k]) / 16 + 1 blocks per SM.  Contexts that run the persistent kernels (several instances, or one with
 * steps_per_launch = 0): trial_steps steps of the whole context per candidate (16 .. 512),
 * one length for all instances first, then block-size class by class, on the live state,
 * which is restored afterwards from a snapshot (device memory for one copy of every
 * instance's state and waveform ring while the call runs).  The state, the time levels
 * and the waveform records are unchanged on return.  Synchronizes. */
teuk_status teuk_autotune(teuk_ctx* ctx, int trial_steps, int* chosen);

/* Testing aid for the bounded device waits of the batched kernel: work item
 * skip_release_item (numbered within a step, -1 = none) of the first step of each
 * call never publishes its completion, so the items that depend on it give up after
 * spin_limit polls (0 = the default of about one second) and the next teuk_sync
 * reports TEUK_ETIMEOUT; the state is then undefined until teuk_set_state.  With
 * resident launches (teuk_set_resident), block skip_release_item never publishes its
 * exchanged columns, and its neighbours' waits give up after about one second. */
teuk_status teuk_set_fault_injection(teuk_ctx* ctx, int64_t skip_release_item,
                                     long long spin_limit);

/* Testing aid for the bounded waits of the step kernels' column ring: while column >= 0,
 * the step kernels of one instance never copy that column of the input level into their
 * shared-memory ring (no copy is issued, so none is in flight), the blocks waiting for
 * it give up after about one second, and the next teuk_sync reports TEUK_ETIMEOUT; later
 * launches of the context return at once until the status has been read, and the state
 * is undefined until teuk_set_state.  column < 0 clears it. */
teuk_status teuk_set_fill_fault(teuk_ctx* ctx, int instance, int column);

/* Checked builds.  The library also builds as libteuk_check.so with TEUK_CHECK defined:
 * before each global-memory access of the time loop's kernels (state planes, TMA column
 * fills, coefficient tables, exchange buffers, co-state planes, waveform ring) the index
 * is tested against the extent of its buffer; a failure sets a bit of the device status
 * word and the access is skipped (a load gives zero), so nothing traps, and the next
 * teuk_sync returns TEUK_EBOUNDS.  (A skipped ring fill leaves its waiters to give up
 * after their bounded wait.)  No counterpart in the paper: a debugging aid standing in
 * for a device sanitizer.
 * teuk_checked_build: 1 in a checked build, 0 otherwise.
 * teuk_check_selftest: checked builds only (else TEUK_EINVAL): queues one kernel that
 * submits the index one past the end of instance 0's state plane to the bounds check,
 * without addressing it, so that the next teuk_sync returns TEUK_EBOUNDS. */
int teuk_checked_build(void);
teuk_status teuk_check_selftest(teuk_ctx* ctx);

/* Number of kernels the library launched on this context since creation. */
int64_t teuk_kernel_launches(const teuk_ctx* ctx);

/* Free all device memory of the context (synchronizes its stream).  NULL is a no-op. */
void teuk_destroy(teuk_ctx* ctx);

/* Message of the last failing call on ctx (or, when ctx == NULL, of the last failed
 * teuk_create or teuk_waveform_sum_noalloc).  Never NULL. */
const char* teuk_last_error(const teuk_ctx* ctx);

/* Largest n_records accepted by teuk_waveform_sum_noalloc. */
#define TEUK_NOALLOC_MAX_RECORDS 65536

/*
 * Allocation-free reduction of waveform records, for callers that must not allocate
 * device memory: for example an application that has given all device memory to
 * its own pool (so a cudaMalloc here would fail or fragment it), or a
 * latency-critical loop where a driver allocation, which may synchronize the
 * device, is not acceptable.  The paper has no counterpart; this is a service of
 * the library.
 *
 * Computes out_host[k] = sum_j W_k[j] sin(theta_j) dtheta (j ascending, FP64, with
 * theta_j = (j + 1/2) pi / n_theta), the same value teuk_extract returns in
 * out_scalar, for k = 0 .. n_records-1.
 *   wave_dev  device memory, [n_records][n_theta][2] doubles (re, im), caller-owned
 *   out_host  host memory, [n_records][2] doubles, caller-owned
 *   cuda_stream  the caller's stream (NULL: the legacy default stream); the call
 *             synchronizes it before returning
 * No device memory is allocated or freed: the intermediate results live in one
 * fixed device array of TEUK_NOALLOC_MAX_RECORDS (re, im) pairs (1 MiB) that every
 * GPU loading the library holds until the process exits.  n_records above that
 * size, n_theta outside [1, 1024] or NULL pointers are TEUK_EINVAL (message in
 * teuk_last_error(NULL)); CUDA failures are TEUK_ECUDA.
 * Every call looks up the array's device address on the current device (this
 * allocates nothing).  With lazy module loading (the CUDA default) the first call on a
 * device is what loads the library's device code there and places the array, so make
 * one call with n_records = 0 on each device (it does only that) before the region
 * that must not allocate, and before any stream capture.
 * All calls share the one array: calls whose GPU work overlaps (different streams
 * or threads at the same time) race on it and must be serialized by the caller.
 */
teuk_status teuk_waveform_sum_noalloc(const double* wave_dev, int64_t n_records, int n_theta,
                                      double* out_host, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* TEUK_H */
