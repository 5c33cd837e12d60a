/*
 * hram.h -- C-ABI of the B300 (sm_103a) planar WCSPH hydrodynamic-ram step.
 *
 * The library advances one case of the planar weakly compressible SPH model of
 * Alam, Biswas & Chakraborty ("Verification, Sensitivity, and Operating Limits
 * of a GPU-Accelerated Planar WCSPH Model for Hydrodynamic Ram"): a water
 * channel with Adami ghost walls, penetrated by a rigid disk with prescribed,
 * decelerating motion.  One step is U^{n+1} = T(L(G(U^n))) (Section 4.6):
 * ghost extrapolation G (Section 2.6, eqs. adami-p / adami-v), the fused
 * interaction sums L (Section 2.2: XSPH, momentum with Monaghan artificial
 * viscosity and a laminar term, continuity density, Tait pressure with the
 * cavitation cutoff) and the kick-drift-kick time advance T with the CFL gate
 * (Section 2.5, eq. cfl).  That is closure 0 (the default).  Closure 1 is
 * the paper's own closure: cubic B-spline, summation density, Mie-Grueneisen
 * EOS with an internal-energy equation (see hr_params.closure).  Every step
 * runs in CUDA kernels on the device; the host only launches a captured CUDA
 * graph.
 *
 * Conventions for every call:
 *   - SI units.  Fluid x in [0, Lx], y in [-W/2, W/2]; the disk moves along +x.
 *   - Host pointers are owned by the caller and are not retained after the
 *     call returns.  Arrays of 2-vectors are interleaved (x0, y0, x1, y1, ...).
 *     Per-particle arrays are in fluid-ID order (the order given at init).
 *   - All device work runs on the stream passed to hr_init_case, so it is
 *     ordered with the caller's other work on that stream.
 *   - Every call returns an int status: 0 = HR_OK, negative = error (the case
 *     may no longer be advanced), positive = warning bits (the state is valid).
 *     Device-side errors are sticky: once seen they are returned by every
 *     later call that synchronises.
 *   - No call reads the CUDA state of other cases; a case is not thread-safe.
 */
#ifndef HRAM_H
#define HRAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HR_MAX_PROBES 16

/* status codes */
#define HR_OK 0
#define HR_EINVAL (-1)    /* bad argument or parameter */
#define HR_ENOMEM (-2)    /* device allocation failed or workspace too small */
#define HR_ECUDA (-3)     /* a CUDA call failed */
#define HR_ENAN (-4)      /* NaN or Inf appeared in the fluid state */
#define HR_EDT (-5)       /* time step underflow (dt < 1e-14 s) */
#define HR_ETIMEOUT (-6)  /* a bounded device wait gave up (persistent batch barrier) */
#define HR_ERANGE (-7)    /* caller buffer too small */
#define HR_EIO (-8)       /* file error in save / load */
#define HR_ECHECK (-9)    /* an index check failed; only the bounds-checked build
                            (libhram_checked.so, compiled with -DHRAM_CHECKED)
                            checks every cell-list, sorted-array and ghost index
                            before use, skips the access and reports it here */
/* warning bits (positive) */
#define HR_WPENETRATION 1 /* fluid particles inside the disk circle */
#define HR_WOUTSIDE 2     /* particles left the computational box and were frozen */
#define HR_WPROBEFULL 4   /* probe history capacity reached; later samples dropped */

/* flags */
#define HR_FLAG_TIMING 1  /* record CUDA events around the step's kernel groups
                            (hr_kernel_times); each event inside the step graph
                            adds about 2.6 us to the step on a B300 */
#define HR_FLAG_TANGENT 2 /* carry tangent-linear derivatives along the run
                            (see hr_tangent_outputs); needs dt_mode 1 and
                            motion 0-2 */
#define HR_FLAG_STAGE_POS 4 /* interaction pass variant: a pass block whose
                            particles lie in one cell row copies the positions
                            of its three stencil rows to shared memory once and
                            tests its candidates there; the results are the
                            same bit for bit (a measured alternative, slower
                            or no faster on a B300; single-case steps only) */
#define HR_FLAG_STAGE_ALL 8 /* as HR_FLAG_STAGE_POS, with the velocities and
                            EOS records staged too (at most one of the two) */
#define HR_FLAG_NEWTON3 16 /* interaction pass variant: every fluid pair is
                            evaluated once (half stencil) and both particles
                            take their side of it, summed in a fixed order with
                            no floating-point atomics; results agree with the
                            plain pass to rounding and are reproducible.
                            Closure 0, cell_factor >= 1, single-case steps; not
                            with the tangent or reverse modes.  A cell denser
                            than the tiles hold makes the step return
                            HR_ERANGE */
#define HR_FLAG_PASS_LANES2 32 /* interaction pass variant: each particle's
                            candidates, pairs and ghosts split over 2 lanes
                            (sums combined in a fixed order; results agree with
                            the plain pass to rounding): a shorter critical
                            path for small, latency-bound cases.  cell_factor
                            >= 1, single-case steps; not with the tangent or
                            reverse modes.  At most one pass-variant flag */
#define HR_FLAG_PASS_LANES4 64 /* as HR_FLAG_PASS_LANES2 with 4 lanes */
#define HR_FLAG_PASS_SPLIT 128 /* run the interaction pass split: the interior
                            particles (no wall ghost in their cell stencil, not
                            near the disk) in one kernel that does not wait for
                            the ghost pass, and the boundary particles, listed by
                            the reorder, after the ghost pass on a
                            high-priority graph branch beside it.  Results are
                            the same bit for bit as the one-kernel pass.  By
                            default a case of at least 262,144 fluid particles
                            with the 3 x 3 stencil, no pass-variant flag and no
                            HR_FLAG_TANGENT runs split; this flag asks for it
                            at any size (same conditions otherwise) */
#define HR_FLAG_PASS_FUSED 256 /* never run the interaction pass split (not
                            with HR_FLAG_PASS_SPLIT) */
#define HR_FLAG_CLOSE_INLINE 512 /* close every step inside its own step graph.
                            By default a step graph leaves the step's close
                            (the reductions of the pass partials, the probes,
                            the FP64 accumulators, the CFL gate) to the next
                            step's graph, where it runs beside that step's
                            drift, which derives its dt from the maximum |v|
                            of the last pass directly; the library runs a
                            pending close itself before any call that reads,
                            saves, replaces or batches the case, so every
                            result is the same bit for bit.  Cases with
                            HR_FLAG_TANGENT or the two-way coupled disk
                            (motion 3, whose next step needs the close's
                            force) always close inline */

/* Case parameters.  Field meanings follow the paper's notation.
 *  dx, h_over_dx   particle spacing and smoothing length ratio (h = 1.3 dx)
 *  Lx, W           channel length and width
 *  wall_layers     ghost layers per side wall (0 = no side walls)
 *  end_walls       1 = also close x = 0 and x = Lx with ghost walls
 *  R_disk, v0, tau, t_ramp, x_c0, y_c0   disk radius, entry speed, decay time,
 *                  ramp time (Section 2.6.3), initial centre
 *  Ng              disk ghost count (Section 2.6.1); 0 = no disk
 *  motion          0 ramp x exponential decay, 1 ramp + quadratic drag
 *                  (Section 2.7, drag_M, drag_Cd, drag_R), 2 constant
 *                  acceleration a_const from rest, 3 ramp then two-way
 *                  coupling: M' dv/dt = -(force of the disk ghosts on the
 *                  fluid), M' = disk_density pi R^2 per unit depth
 *  rho0, c0, gamma Tait equation of state; p_cav cavitation cutoff
 *  alpha, eta2     artificial viscosity (eq. artificial-viscosity)
 *  eps_xsph        XSPH blending (eq. xsph); mu_lam dynamic viscosity
 *  gx, gy          body force; cfl the CFL number (eq. cfl)
 *  dt_mode         0 adaptive dt, 1 fixed dt = cfl h / (c0 + v0)
 *  rho_lo, rho_hi  density band as fractions of rho0 (0.5, 1.5)
 *  box_pad         computational-box padding (<= 0: default)
 *  cell_factor     cell side / 2h: >= 1 gives cells of side max(f, 1.001) 2h
 *                  and the 3 x 3 cell stencil; [0.5, 1) cells of side
 *                  max(f, 0.5005) 2h and the 5 x 5 stencil (smaller cells,
 *                  fewer candidates per particle, more cells to scan; not with
 *                  HR_FLAG_TANGENT, the staged pass variants, the reverse mode
 *                  or a persistent batch)
 *  probe_xy        wall probe points, n_probes of them
 *  probe_capacity  probe history rows kept on the device
 *  diag_every      record FP64 diagnostics every k steps (0 = never)
 *  flags           HR_FLAG_*
 *  disk_density    disk material density for motion 3 [kg/m^3]
 *  closure         0: Wendland C2 kernel, continuity density, Tait EOS (above);
 *                  1: the paper's own closure -- cubic B-spline (eq.
 *                  cubic-kernel), summation density with the band (eq.
 *                  density-sum), Mie-Grueneisen EOS (eq. eos) with C = c0 and
 *                  an internal-energy equation.  The input rho is then
 *                  ignored (the density is summed from the positions), the
 *                  internal energy starts at 0, and artificial viscosity uses
 *                  c = c0.  Closure 1 cases cannot be batched or run in
 *                  tangent mode.
 *  mg_S1, mg_gamma0, mg_a, mg_mu_max   Mie-Grueneisen S1, gamma0, a and the
 *                  compression cap on mu = rho/rho0 - 1 (1.979, 0.11, 3.0, 0.25)
 *  wall_reflect    1 = with wall_layers = 0 the side walls still reflect
 *                  particles (|y| > W/2: y pulled back to +-(W/2 - 1e-6 m),
 *                  v_y reversed), the paper's baseline hard wall without
 *                  ghosts (Section 2.6.2); it exerts no pressure, so the
 *                  wall impulse stays 0 */
typedef struct hr_params {
    double dx, h_over_dx, Lx, W;
    int32_t wall_layers, end_walls;
    double R_disk, v0, tau, t_ramp, x_c0, y_c0;
    int32_t Ng, motion;
    double a_const, drag_M, drag_Cd, drag_R;
    double rho0, c0, gamma, p_cav, alpha, eta2, eps_xsph, mu_lam, gx, gy, cfl;
    int32_t dt_mode, n_probes;
    double rho_lo, rho_hi, box_pad, cell_factor;
    double probe_xy[2 * HR_MAX_PROBES];
    int64_t probe_capacity;
    int32_t diag_every, flags;
    double disk_density;
    int32_t closure;
    double mg_S1, mg_gamma0, mg_a, mg_mu_max;
    int32_t wall_reflect;
} hr_params;

/* FP64 diagnostics (Section 2.10 and eq. energy-audit of Section 4.7). */
typedef struct hr_diag {
    double mass, px, py, KE, PE, E_el;
    double rho_min, rho_max, p_min, p_max, vmax_fluid;
    double n_in, penetrated, t, dt;
    double W_boundary, wall_impulse, dissipation, step;
} hr_diag;

typedef struct hr_case hr_case; /* opaque; owns or borrows all device memory */

/* Device bytes a case needs (one block, 256-byte aligned sub-buffers).
 * n_fluid: fluid particle count.  Returns HR_EINVAL for bad parameters. */
int hr_workspace_bytes(const hr_params *p, int64_t n_fluid, size_t *bytes);

/* Creates a case.  xy: n_fluid initial positions (float, host, ID order);
 * vel (n_fluid x 2) and rho (n_fluid) may be NULL for rest at rho0.
 * d_workspace: device memory of at least hr_workspace_bytes bytes owned by
 * the caller (it must outlive the case), aligned to 256 bytes (else
 * HR_EINVAL), or NULL to let the library allocate.
 * cuda_stream: a cudaStream_t (0 = legacy default stream).  Computes the
 * initial a, D rho, XSPH sums and dt (t = 0), captures the step graph and
 * synchronises.  On failure *out is NULL and nothing is retained. */
int hr_init_case(const hr_params *p, const float *xy, int64_t n_fluid, const float *vel,
                 const float *rho, void *d_workspace, size_t workspace_bytes,
                 void *cuda_stream, hr_case **out);

/* One time step U^{n+1} = T(L(G(U^n))) (operator order of Section 4.6; the
 * velocity Stoermer-Verlet advance with the CFL gate of Section 2.5, eq. cfl),
 * replayed from the captured step graph, asynchronous.  Returns the last
 * known status.  Unless the case was created with HR_FLAG_CLOSE_INLINE the
 * step's close runs with the next step or before the next call that reads
 * the case (HR_FLAG_CLOSE_INLINE). */
int hr_step(hr_case *c);

/* n_steps steps of hr_step (Sections 4.6 and 2.5); with t_end > 0 stops at
 * the first step that reaches t_end (n_steps <= 0 then means "until t_end"),
 * the event window of the paper's runs (Section 3).  Synchronises and
 * returns the device status. */
int hr_run(hr_case *c, int64_t n_steps, double t_end);

/* Waits for the case's work and returns the device status. */
int hr_sync(hr_case *c);

/* Probe pressure history (the wall pressure stations of Section 3, the
 * paper's PTn and PTf), row k = [p_probe0 .. p_probe(n-1)] after step k+1
 * (float, host, cap_rows x n_probes).  Each value is the Adami wall-ghost
 * formula (eq. adami-p with the wall at rest) evaluated at the probe point
 * over the end-of-step fluid, cutoff applied.  *n_rows = rows recorded. */
int hr_probe_pressure(hr_case *c, float *host_out, int64_t cap_rows, int64_t *n_rows);

/* Simulated time t^{k+1} after step k+1 (double, host): the time axis of the
 * probe histories (Section 3), a sum of the CFL steps of eq. cfl. */
int hr_probe_times(hr_case *c, double *host_out, int64_t cap, int64_t *n);

/* FP64 diagnostics of the current state (synchronises). */
int hr_diagnostics(hr_case *c, hr_diag *out);

/* Recorded periodic diagnostics (diag_every > 0): rows of 19 doubles in
 * hr_diag field order.  *n_rows = rows recorded. */
int hr_diag_history(hr_case *c, double *host_out, int64_t cap_rows, int64_t *n_rows);

/* Current fluid state in ID order (any pointer may be NULL): positions,
 * velocities, densities and the pressure of the equation of state (Section
 * 2.2: Tait with the cavitation cutoff for closure 0, eq. eos for closure 1)
 * at the end of the last step.  xy, vel: cap x 2; rho, p: cap.  cap must be
 * >= n_fluid (else HR_ERANGE).  Synchronises. */
int hr_get_state(hr_case *c, float *xy, float *vel, float *rho, float *p, int64_t cap);

/* Closure 1 only: specific internal energy e [J/kg] and its rate De [W/kg]
 * of the energy equation, in fluid-ID order (either pointer may be NULL),
 * cap >= n_fluid.  HR_EINVAL for a closure 0 case.  Synchronises. */
int hr_get_energy(hr_case *c, float *e, float *de, int64_t cap);

/* Replaces the fluid state (ID order, n == n_fluid), resets t = 0, the step
 * counter, probe history and accumulators, and recomputes a, D rho, X, dt as
 * hr_init_case does.  vel or rho may be NULL (rest, rho0). */
int hr_set_state(hr_case *c, const float *xy, const float *vel, const float *rho, int64_t n);

/* Ghost state of the last step (wall ghosts in wall-ID order, then disk
 * ghosts): xy, vel cap x 2; p, rho cap.  Synchronises. */
int hr_get_ghosts(hr_case *c, float *xy, float *p, float *rho, float *vel, int64_t cap);

/* Scalars: t, dt, step, xc, yc, vproj, aproj, Fdisk_x, Fdisk_y, Fwall,
 * W_boundary, wall_impulse, dissipation, diss_rate (14 doubles). */
int hr_get_scalars(hr_case *c, double *out, int n);

/* Counts: n_fluid, n_wall, n_disk, ncx, ncy, pass_blocks, 1 when the
 * interaction pass runs split (HR_FLAG_PASS_SPLIT), and 1 when the step
 * graphs defer each step's close to the next (not HR_FLAG_CLOSE_INLINE)
 * (8 int64; the first n of them are written). */
int hr_case_info(hr_case *c, int64_t *out, int n);

/* Neighbour sets of the current state as CSR over all points (fluid IDs,
 * then wall ghosts, then disk ghosts; fluid rows list fluid and ghost
 * neighbours, ghost rows list fluid neighbours; ids ascending).  offsets has
 * n_points + 1 entries.  With ids == NULL or cap too small only *n_pairs is
 * set (and HR_ERANGE returned when ids != NULL).  Synchronises. */
int hr_debug_neighbors(hr_case *c, int64_t *offsets, int32_t *ids, int64_t cap,
                       int64_t *n_pairs);

/* Durations (ms) of the last replayed step's kernel groups when the case was
 * created with HR_FLAG_TIMING: drift, sort, ghost, pass, finalize.  With the
 * deferred close (no HR_FLAG_CLOSE_INLINE) the drift group holds the previous
 * step's close and the finalize group is empty. */
int hr_kernel_times(hr_case *c, float *ms, int n);

/* Checkpoint / resume of the full state (positions, velocities, densities,
 * derivatives, time, dt, accumulators, probe history) in a binary file.
 * A loaded case continues bit-for-bit as the saved one would have. */
int hr_save_state(hr_case *c, const char *path);
int hr_load_state(hr_case *c, const char *path);

/* Batched runs: many cases advanced together, one launch per kernel per
 * step for all of them (the coefficient sweep of the sensitivity study,
 * Section 4.5: artificial viscosity, sound speed, cutoff, impact speed and
 * channel width varied per case).  Each case keeps its own cell grid, time
 * step, kinematics, probes and diagnostics; a case whose time reaches t_end
 * stops advancing while the others go on.  The cases stay owned by the
 * caller and must outlive the batch; they must all live on the current
 * device.  Read results with the per-case calls after hr_batch_run. */
typedef struct hr_batch hr_batch;

/* Groups n_cases existing cases into a batch that runs each one up to
 * simulated time t_end (> 0), captures the batched step graph.  schedule
 * orders the blocks of each batched launch: 0 case after case, 1 round robin
 * over the cases, 2 case after case from the largest down (results do not
 * depend on it; the autotuner picks the fastest).  cuda_stream: the stream
 * the batch runs on.  Allocates a small device block for the case tables.
 * HR_EINVAL if a case is a tangent case, is in an error state, or has a
 * different closure from cases[0] (one batch runs one closure: closure 1
 * batches add the batched summation density after the sort). */
int hr_batch_create(hr_case *const *cases, int n_cases, double t_end, int schedule,
                    void *cuda_stream, hr_batch **out);

/* The same sweep as one persistent launch (Section 4.5's sensitivity study
 * run as a batch): every case is given case_blocks[k] thread blocks of its
 * own (NULL: in proportion to the particle counts), all blocks stay
 * resident (a cooperative launch; the total may not exceed
 * hr_persist_capacity), and a case's blocks take it through the stages of
 * each step -- drift, cell scan, reorder, ghosts (eqs. adami-p / adami-v),
 * interaction pass (Section 2.2), closing reduction and CFL gate (eq. cfl)
 * -- meeting at a barrier of their own between stages, so cases of
 * different sizes and time steps run at their own pace.  Results are bit
 * for bit those of each case run alone.  Every barrier wait gives up after
 * spin_limit polls (<= 0: 2^24, about 2 s), and hr_batch_run /
 * hr_batch_step then return HR_ETIMEOUT and mark every case with it (the
 * cases stopped mid-step).  hr_batch_run runs the whole sweep (max_steps
 * <= 0) or max_steps steps of each case in one launch; hr_batch_step runs
 * one.  Same ownership and closure rules as hr_batch_create; t_end > 0;
 * every case takes the 3 x 3 stencil (cell_factor >= 1), else HR_EINVAL. */
int hr_batch_create_persistent(hr_case *const *cases, int n_cases, double t_end,
                               const int32_t *case_blocks, int64_t spin_limit, void *cuda_stream,
                               hr_batch **out);

/* Resident blocks the persistent batch may use on the current device (its
 * blocks per multiprocessor times the multiprocessor count), for closure 0
 * or 1. */
int hr_persist_capacity(int closure, int32_t *max_blocks);

/* One batched step (graph replay, or one step of a persistent batch). */
int hr_batch_step(hr_batch *b);

/* Steps until every case has reached t_end (or max_steps batched steps when
 * max_steps > 0); synchronises and returns the worst case status.
 * *steps_done = batched steps launched. */
int hr_batch_run(hr_batch *b, int64_t max_steps, int64_t *steps_done);

/* Number of cases that have reached t_end (synchronises). */
int hr_batch_done(hr_batch *b, int *n_done);

void hr_batch_destroy(hr_batch *b);

/* Tangent-linear (forward-mode) derivatives of two outputs of the run, for
 * a case created with HR_FLAG_TANGENT (dt_mode 1, motion 0-2).  The parameters
 * are theta = (alpha, c0, tau): the artificial-viscosity coefficient
 * (eq. artificial-viscosity, Section 2.2), the reference sound speed of the
 * Tait equation of state (which also sets the fixed step dt = C h / (c0 + v0))
 * and the decay time of motion 0, v = v0 min(t / t_ramp, 1) exp(-t / tau)
 * (eq. velocity-ramp times the exponential decay; motions 1 and 2 do not
 * depend on tau, so their tau-derivatives are zero).  The derivatives are those of
 * the discrete run itself: every step's kernels are differentiated with the
 * step's own neighbour sets and clamp decisions, from a state uploaded by
 * hr_init_case / hr_set_state that is taken as independent of theta.
 *   out[0]      peak probe-0 pressure P = max_n p_0(t^n) over the recorded
 *               history [Pa]
 *   out[1..3]   dP / d ln alpha, dP / d ln c0, dP / d ln tau  (theta_k dP/dtheta_k)
 *   out[4]      wall impulse J = sum_n dt^n F_wall^{n+1} [N s / m]
 *   out[5..7]   dJ / d ln alpha, dJ / d ln c0, dJ / d ln tau
 *   out[8]      history row of the peak (-1: no probe sample yet)
 * n >= 9 doubles; synchronises the case's stream.  HR_EINVAL if the case was
 * not created with HR_FLAG_TANGENT.  Batched runs do not take tangent cases,
 * and hr_load_state refuses them (a loaded state has no derivatives). */
int hr_tangent_outputs(hr_case *c, double *out, int n);

/* Reverse-mode (adjoint) derivatives of the same two outputs as
 * hr_tangent_outputs (the peak probe-0 pressure P and the wall impulse J)
 * with respect to theta = (alpha, c0, tau), for a case with closure 0,
 * dt_mode 1 and motion 0-2 (not created with HR_FLAG_TANGENT).  This is the
 * sensitivity study of Section 4.5 (the alpha sweep and Table
 * tab:alpha-sweep) as a gradient: the adjoint of the interaction pass
 * (Section 2.2), the ghost operator (eqs. adami-p / adami-v), the equation of
 * state and the time integrator (Section 2.5), swept backwards through the
 * run with the step's own neighbour sets, cell order and clamp / cutoff /
 * switch / reflection decisions, as the forward run took them.
 *
 * hr_adjoint_forward runs n_steps steps from the case's uploaded state (the
 * case must be at step 0: fresh from hr_init_case or hr_set_state), keeping a
 * checkpoint of the state every checkpoint_every steps.  out (n >= 3
 * doubles): [P, J, row of the peak in the probe history].  n_steps must not
 * exceed probe_capacity, and the case needs at least one probe.  The
 * library allocates the checkpoints, the records of one segment of
 * checkpoint_every steps and the adjoint buffers (about
 * (48 n_steps / checkpoint_every + 84 checkpoint_every + 300) bytes per fluid
 * particle) and keeps them until the next hr_adjoint_forward or
 * hr_destroy.  The last segment's steps run on the records as they go
 * (unless the case takes periodic diagnostics), so its reverse sweep needs no
 * recomputation.  Afterwards the case stands at step n_steps as after hr_run,
 * bit for bit.
 *
 * hr_adjoint_backward sweeps the run backwards: for each segment, last
 * first, it recomputes the segment's steps from its checkpoint (the last
 * segment's records are already there) and carries the adjoints of the state
 * from the end of each step to its start.  out (n
 * >= 6 doubles): [dP/d ln alpha, dP/d ln c0, dP/d ln tau, dJ/d ln alpha,
 * dJ/d ln c0, dJ/d ln tau] (theta_k d/d theta_k, as hr_tangent_outputs).  It
 * leaves the case's state as hr_adjoint_forward left it, and may be called
 * again.  HR_EINVAL without a preceding hr_adjoint_forward. */
int hr_adjoint_forward(hr_case *c, int64_t n_steps, int32_t checkpoint_every, double *out, int n);
int hr_adjoint_backward(hr_case *c, double *out, int n);

/* Neighbour counts of the current state without any device allocation.
 *
 * The paper has no counterpart; this is a library service.  hr_debug_neighbors
 * allocates device scratch with cudaMalloc on every call.  Some callers cannot
 * do that: a process whose device memory is fully reserved by another
 * allocator (a framework's caching allocator, a fixed pool handed out at
 * start-up), or code that must not change the device's allocation state while
 * it runs.  This entry point computes the same per-point neighbour counts
 * (counts[r] = offsets[r+1] - offsets[r] of hr_debug_neighbors, in the same
 * global point order: fluid IDs, then wall ghosts, then disk ghosts) into a
 * fixed device array that the library holds for the life of the process, then
 * copies them to host_counts (caller-owned, cap >= number of points).
 *
 * Limit: HR_STATIC_NEIGHBOR_MAX points (fluid + ghosts); larger cases are
 * rejected with HR_ERANGE before any device work.  The case's device (the one
 * current at hr_init_case) must be the current device: the array's address
 * differs between devices, and a call made with another device current
 * returns HR_EINVAL.  The fixed array (4 bytes
 * per point, 8 MiB) is resident on every device that loads the library until
 * the process exits.  The first call on a device looks up the array's device
 * address for that device (cudaGetSymbolAddress); make that first call before
 * any stream capture.  Every call overwrites entries [0, number of points) of
 * the shared array and leaves the rest as an earlier call left them; calls that
 * overlap on the GPU (other streams, other cases, other threads) race on it.
 * Synchronises the case's stream. */
#define HR_STATIC_NEIGHBOR_MAX (1 << 21)
int hr_neighbor_counts_static(hr_case *c, int32_t *host_counts, int64_t cap);

/* FP32 FMA rate of the current device in TFLOP/s (an FMA counted as two
 * operations), measured: a kernel of 16 independent FMA chains per thread on
 * 8 blocks of 256 threads per multiprocessor, as scalar fma.rn.f32 (packed
 * = 0) or as packed fma.rn.f32x2 (packed = 1), timed with CUDA events on
 * cuda_stream (NULL: the default stream).  The paper has no counterpart; the
 * interaction pass (Section 2.2) is an FP32 gather whose roofline is this
 * rate.  Allocates and frees a small device buffer; synchronises the
 * stream.  *tflops = 0 and a negative status on failure. */
int hr_fp32_rate(int packed, void *cuda_stream, double *tflops);

void hr_destroy(hr_case *c);
const char *hr_status_str(int status);

#ifdef __cplusplus
}
#endif
#endif /* HRAM_H */
