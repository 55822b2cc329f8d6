/*
 * epd_lb.h -- C ABI of the GB300 (sm_103a) hybrid Lattice-Boltzmann /
 * External-Potential-Dynamics time stepper of Heuser, Sevink and Schmid,
 * "Self-assembly of polymeric particles in Poiseuille flow: a hybrid Lattice
 * Boltzmann / External Potential Dynamics simulation study" (arXiv:1804.02883).
 *
 * One call of epd_lb_step advances every run of a handle by one time step of
 * the method (App. C, flow chart, with the omega-from-Phi inversion taken at
 * its starting guess, the auxiliary convection of omega):
 *   1. omega~ = omega - dt v . grad omega                    (App. C, item 1)
 *   2. Phi~ from omega~ by the single-chain solve           (Sec. 2, Eqs. (6)-(11))
 *   3. omega(t+dt) = omega~ - dt D_I Lap mu_I(Phi~)          (Sec. 2, Eq. (5); App. C)
 *   4. Phi(t+dt) from omega(t+dt)                            (Eqs. (6)-(11))
 *   5. polymer force from Phi(t+dt) - Phi~                   (Sec. 2, Eqs. (19)-(20))
 *   6. D2Q9 MRT collide-stream with that force plus the
 *      reverse-Poiseuille body force                         (Eqs. (12), (14)-(16), (23))
 * epd_lb_set_inversion switches to the exact step of App. C (convection of
 * Phi and the Fletcher-Reeves inversion in place of steps 1-2); the learned
 * surrogate (epd_lb_set_surrogate) can stand in for the solves; the analysis
 * calls (epd_lb_sigma_delta, epd_lb_width, epd_lb_particles) evaluate the
 * observables of Sec. 3 and Sec. 4; the epd_*3d entry points run the solve,
 * D3Q19 and the coupled step on 3D boxes with state in caller memory.
 *
 * Conventions for every entry point:
 *  - Return EPD_LB_OK (0) on success or a negative EPD_LB_E* code; the text
 *    of the last error of a handle is available from epd_lb_last_error.
 *  - Field layout is [field][y][x] with x fastest; x is the flow axis and y
 *    runs across the channel.  Species fields are ordered [A, B, S], velocity
 *    components [x, y], LB populations [i] in the D2Q9 order
 *      0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
 *  - Host buffers are caller-owned FP64 arrays; the library never frees caller
 *    memory.  *_dev variants take device pointers and work on the handle's
 *    stream.  Calls on one handle must not run concurrently.
 *  - Units: lengths in R_G, times in tau = R_G^2/D_S for the EPD part; the
 *    LB part is in lattice units (dx = dt = rho0 = 1).
 */
#ifndef EPD_LB_H
#define EPD_LB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    EPD_LB_OK = 0,
    EPD_LB_EINVAL = -1,      /* invalid argument or parameter set            */
    EPD_LB_ENOMEM = -2,      /* workspace too small or allocation failed     */
    EPD_LB_ECUDA = -3,       /* a CUDA runtime call failed                   */
    EPD_LB_ENONFINITE = -4,  /* non-finite value or Q <= 0 detected on device */
    EPD_LB_EUNSTABLE = -5,   /* Mach-number pre-flight refused the run       */
    EPD_LB_ETIMEOUT = -6,    /* a bounded device wait gave up                */
    EPD_LB_ENOTCONV = -7,    /* the CG inversion of the exact step did not converge */
    EPD_LB_ETOOLARGE = -8    /* problem needs more than the fixed scratch of
                                epd_prop_solve_noalloc                        */
};

enum {
    EPD_LB_PLAIN_FP64 = 0,   /* every field and transform in FP64            */
    EPD_LB_MIXED_FP32 = 1    /* propagators, LB populations and the EPD/force
                                transforms in FP32; fields omega and Phi,
                                contour sums, Q and masses in FP64.  The
                                step's second solve is computed as its
                                difference from the first (same result up to
                                rounding, FP32 relative to the change that
                                drives the force of Eqs. (19)-(20))          */
};

/*
 * Parameters of one run (Sec. 2 model, Sec. 3 and Sec. 4 set-up).
 *  nx, ny      grid sites per axis in [8, 2048], even and of the form 2^a 3^b 5^c
 *              (the paper's 150 x 150 included); nx is the flow axis.  Axes that
 *              are not powers of two take mixed-radix (2, 3, 4, 5) transforms in
 *              the streaming passes.
 *  ns          contour steps N_s in [2, 512]; even for MIXED_FP32 on
 *              power-of-two grids (the paper's N_s = N = 17 runs elsewhere)
 *  precision   EPD_LB_PLAIN_FP64 or EPD_LB_MIXED_FP32
 *  dx, dt, rg  grid spacing, time step, gyration radius R_G (paper: 1/3, 0.002, 1)
 *  n_seg       segments per chain N (paper: 17); the Boltzmann factor is exp(-N w ds/2)
 *  f_a         A-fraction q_A; the A block covers round(f_a ns) contour intervals
 *  phi_p       mean polymer volume fraction; the solvent has 1 - phi_p
 *  chi_*, kappa_h  Flory-Huggins and Helfand parameters of Eq. (1)
 *  d_s, d_p    diffusion constants of solvent and of both monomer species
 *  inv_beta_v  1/(beta v), the prefactor of the force of Eq. (20)
 *  gamma_s, gamma_b, gamma_g  MRT relaxation of shear, bulk and ghost modes
 *              (0, 0, 0 is BGK with tau = 1)
 *  f0          reverse-Poiseuille amplitude of Eq. (23) in units of f* = rho R_G / tau^2
 *  noise_amp   amplitude a of the initial noise omega_I = a U(-1, 1)
 *  seed        seed of the counter-based noise (splitmix64)
 *  junction_rule  the field at the A/B junction node s = q_A of the split step
 *              of Eq. (8) (Sec. 2 puts omega_A at s < q_A and omega_B
 *              otherwise): 0 literal (node j carries omega_A iff j < N_A, so
 *              the junction node takes omega_B); 1 segment-symmetric (both
 *              half-steps of the interval [s_j, s_{j+1}] use the field of its
 *              block, A iff j < N_A, the same from either chain end)
 *  reserved    0
 */
typedef struct epd_lb_params {
    int32_t nx, ny, ns, precision;
    double dx, dt, rg, n_seg, f_a, phi_p;
    double chi_ab, chi_as, chi_bs, kappa_h;
    double d_s, d_p, inv_beta_v;
    double gamma_s, gamma_b, gamma_g;
    double f0;
    double noise_amp;
    uint64_t seed;
    int32_t junction_rule, reserved;
} epd_lb_params;

typedef struct epd_lb epd_lb; /* opaque, library-owned */

/* Device workspace needed by epd_lb_init for nruns runs described by the
 * array p[0..nruns-1] (memory management, not in the paper).  Runs may differ in every parameter; runs sharing grid,
 * contour length, precision and model parameters are stepped as one batch. */
int epd_lb_workspace_bytes(const epd_lb_params *p, int32_t nruns, size_t *bytes);

/* Create a handle for nruns runs.  workspace: device memory of at least
 * epd_lb_workspace_bytes bytes, 256-byte aligned, owned by the caller and kept
 * alive until epd_lb_destroy; NULL lets the library cudaMalloc its own.
 * cuda_stream: a cudaStream_t created by the caller (not the legacy default
 * stream) on which every call of this handle is ordered; NULL lets the library
 * create a non-blocking stream.  Initialises every run (Sec. 3: omega noise
 * from the seed; Sec. 4: flow at the steady reverse-Poiseuille profile of
 * Eq. (24)) and solves Phi(0).  Fails with EPD_LB_EUNSTABLE when the expected
 * peak flow exceeds Mach 0.3. */
int epd_lb_init(const epd_lb_params *p, int32_t nruns, void *workspace, size_t workspace_bytes,
                void *cuda_stream, epd_lb **out);

/* Advance every run by nsteps time steps (the six operations listed at the
 * top, App. C).  Asynchronous on the handle's stream; the step sequence is
 * captured once into a CUDA graph and replayed. */
int epd_lb_step(epd_lb *h, int64_t nsteps);

/* Wait for the handle's stream and report device-side errors:
 * EPD_LB_ENONFINITE when a solve produced Q <= 0 or a non-finite Q (Q_P, Q_S
 * of Eqs. (9)-(11) are spatial means of positive propagators, so a
 * non-finite field anywhere reaches them), EPD_LB_ETIMEOUT when a bounded
 * device wait gave up. */
int epd_lb_sync(epd_lb *h);

/* Phi_{A,B,S}(t) of run `run` (3*ny*nx doubles) and q[0] = Q_P, q[1] = Q_S of
 * the solve that produced it (Q as spatial means, Eqs. (9)-(11)).  Either
 * pointer may be NULL.  Synchronous. */
int epd_lb_densities(epd_lb *h, int32_t run, double *phi, double *q);

/* omega (3*ny*nx; the fields conjugate to the densities, Sec. 2) and Phi
 * (3*ny*nx; Eqs. (9)-(11)) of run `run` into caller device memory (FP64,
 * asynchronous on the handle's stream); either pointer may be NULL. */
int epd_lb_fields_dev(epd_lb *h, int32_t run, double *omega_dev, double *phi_dev);

/* The intermediate fields of the last step of run `run` into caller device
 * memory (FP64, asynchronous on the handle's stream; either pointer may be
 * NULL): omega~ (the auxiliary-convected field, App. C item 1) and Phi~, its
 * densities (Eqs. (6)-(11)).  With epd_lb_fields_dev they give the
 * composition change Phi(t+dt) - Phi~ of the diffusion step that drives the
 * force (Eqs. (19)-(20)); on the grids of the differential second solve that
 * difference carries FP32 precision relative to itself. */
int epd_lb_step_fields_dev(epd_lb *h, int32_t run, double *omega_tilde_dev, double *phi_tilde_dev);

/* Fluid velocity u = (j + f/2)/rho of the last collision (the LB moments of
 * Eq. (12) with the force of Eq. (14), read in the Dunweg-Ladd form), lattice
 * units, 2*ny*nx doubles.  Synchronous. */
int epd_lb_velocity(epd_lb *h, int32_t run, double *v);

/* Asynchronous host-buffer variants for streaming a run's fields through
 * the step: epd_lb_set_omega_async replaces omega of run `run` (3*ny*nx
 * doubles, the fields conjugate to the densities, Sec. 2) and
 * epd_lb_densities_async reads Phi (3*ny*nx; Eqs. (9)-(11)) and q[2] =
 * (Q_P, Q_S); either output pointer may be NULL.  The copies are only
 * enqueued on the handle's stream, in order with epd_lb_step: the caller
 * keeps the host buffers alive and untouched until epd_lb_sync (or any
 * synchronous call) returns.  Page-locked host memory makes the copies
 * asynchronous; with pageable memory they complete before the call
 * returns. */
int epd_lb_set_omega_async(epd_lb *h, int32_t run, const double *omega);
int epd_lb_densities_async(epd_lb *h, int32_t run, double *phi, double *q);

/* Device-pointer variants of epd_lb_densities and epd_lb_velocity:
 * asynchronous copies on the handle's stream into caller device memory of
 * the same layout (FP64). */
int epd_lb_densities_dev(epd_lb *h, int32_t run, double *phi_dev, double *q_dev);
int epd_lb_velocity_dev(epd_lb *h, int32_t run, double *v_dev);

/* Full state of a run, what App. C carries from one step to the next:
 * omega (3n, Sec. 2), pre-collision LB populations (9n, Eq. (12): the
 * populations about to be collided at the next step) and the velocity handed
 * to the next convection step (2n, App. C item 1).  Any pointer may be NULL.
 * Synchronous. */
int epd_lb_get_state(epd_lb *h, int32_t run, double *omega, double *pop, double *vel);

/* Replace the state of a run (same layout as epd_lb_get_state).  A NULL
 * pointer keeps that part of the state.  Phi is not recomputed here: the next
 * epd_lb_step derives it from the new omega (epd_lb_solve gives it at once;
 * the exact step first recomputes Phi(t) of the new omega).
 * In EPD_LB_MIXED_FP32 the populations and velocity are rounded to FP32.  Host
 * buffers; the copies are staged through the workspace.  Synchronous. */
int epd_lb_set_state(epd_lb *h, int32_t run, const double *omega, const double *pop, const double *vel);

/* One single-chain solve, Eqs. (6)-(11), of run `run`'s grid and parameters
 * for the host fields omega (3n): phi (3n) and q[2] = (Q_P, Q_S).  Does not
 * change the run's state.  Synchronous. */
int epd_lb_solve(epd_lb *h, int32_t run, const double *omega, double *phi, double *q);

/* Per-run observables of the current state: out[0] = <Phi_A>, out[1] = <Phi_B>,
 * out[2] = <Phi_S> (each conserved by Eqs. (2) and (5)), out[3] = sigma of
 * Eq. (21), out[4] = LB mass / sites (conserved by Eq. (12)), out[5] = max |u|
 * (lattice), out[6] = Q_P, out[7] = Q_S (Eqs. (9)-(11)).  Sums in a fixed
 * order: a repeated call returns identical values.  Synchronous. */
int epd_lb_observables(epd_lb *h, int32_t run, double *out);

/* Checkpoint (no counterpart in the paper): serialise every run's state
 * (parameters, omega, the stored LB populations in the library's internal
 * representation, velocity; the state of App. C) to buf.
 * With buf == NULL only *len is set to the size needed.  Restoring with
 * epd_lb_load into a handle created with the same parameters recomputes Phi
 * and continues bit-identically. */
int epd_lb_save(epd_lb *h, void *buf, size_t *len);
int epd_lb_load(epd_lb *h, const void *buf, size_t len);

/* Kernel timing inside the captured step (a measurement service, no
 * counterpart in the paper).  epd_lb_enable_timing(h, 1)
 * re-captures the step graph with CUDA event-record nodes around launches of
 * the first batch's second single-chain solve and its LB collide-stream.
 * epd_lb_kernel_times waits for the stream and writes the durations of the
 * most recent step in milliseconds: ms[0..2] the propagator kernels, ms[3]
 * the LB collide-stream, ms[4] a flag.  With the streaming transform passes
 * (ms[4] = 0): ms[0] the row pass of contour node N_s/4, ms[1] the row pass
 * of node 3 N_s/4 + 1 (where the PLAIN_FP64 passes accumulate the contour
 * sums), ms[2] the column pass before it; in MIXED_FP32 these are passes of
 * the differential second solve.  With the cluster-resident solve (ms[4] = 1): ms[0]
 * its chain launches (the whole contour of both chains of every run, in one
 * launch or the phased schedule's several, see epd_lb_tiles; the
 * differential solve where the step uses one), ms[1] = ms[2] = 0. */
int epd_lb_enable_timing(epd_lb *h, int32_t on);
int epd_lb_kernel_times(epd_lb *h, double *ms);

/* Launch configuration chosen for a run's group (batching and tiling of the
 * hot path; not in the paper).  out[0]: solve path, 0 = streaming radix-2 /
 * mixed-radix passes, 1 = streaming radix-8 passes with the full contour history, 2 =
 * cluster-resident solve; out[1]: CTAs per cluster (path 2) or 0; out[2]: the
 * column tile width of the radix-8 column passes (EPD and streaming
 * propagator; 4, 8 or 16 columns), chosen at epd_lb_init by timing each
 * width on the group's own state, or 0 where those passes are not used
 * (EPD_LB_COLUMN_TILE=4|8|16 in the environment forces a width; every width
 * gives bit-identical results); out[3]: 1 if the step's second solve is the
 * differential one; out[4]: the column tile width of the streaming
 * propagator passes (path 1, tuned the same way), else 0; out[5]: launches
 * of the chain kernel per solve on path 2 (1, or 2 nruns when the group's
 * chains are one more than the 16-CTA clusters that fit at one CTA per SM:
 * the chains then take turns, each sitting out one launch; results do not
 * depend on it; EPD_LB_CHAIN_SCHEDULE=single|phased in the environment forces
 * one or the other), else 0.  out holds 6 values.  Returns EPD_LB_EINVAL for a
 * bad run index or NULL out. */
int epd_lb_tiles(epd_lb *h, int32_t run, int32_t *out);

/*
 * Learned density surrogate: a convolutional network that approximates the
 * map omega -> (Phi_A, Phi_B) of the single-chain solve, Eqs. (6)-(10), with
 * the exact means and the exact solvent density of Eq. (11).  Network: 3x3
 * convolutions with circular padding and dilations 1, 2, 2, 4 (tap (dy, dx)
 * of layer l reads the site r + d_l (dy, dx); receptive field +-9 sites),
 * channels 3 -> 32 -> 32 -> 32 -> 2, tanh after the first three; input
 * s_in (omega_c - <omega_c>), output Phi_c = <Phi_c> + s_out (y_c - <y_c>).
 * Parameters: epd_sur_num_params() FP32 values, per layer W[co][ci][3][3]
 * (tap = 3 (dy+1) + (dx+1)) then b[co].
 * Tensor-core kernels read BF16 copies of weights and activations and
 * accumulate in FP32.  Fields are [batch][species][ny][nx] FP64 on the device;
 * every call is asynchronous on cuda_stream; the workspace is caller-owned
 * device memory of epd_sur_workspace_bytes (training = 1 for the gradient and
 * training calls).  nx and ny must be multiples of 16.
 */
int32_t epd_sur_num_params(void);
int epd_sur_workspace_bytes(int32_t ny, int32_t nx, int32_t batch, int32_t training, size_t *bytes);
/* Densities of the surrogate for batch fields omega_dev -> phi_dev.  p gives
 * the grid, phi_p and the A-block fraction of the exact means. */
int epd_sur_forward(const epd_lb_params *p, int32_t batch, const float *params_dev, double s_in, double s_out,
                    const double *omega_dev, double *phi_dev, void *workspace, size_t workspace_bytes, void *cuda_stream);
/* Densities at omega_dev from the surrogate at omega0_dev to first order in
 * the field change: phi0_dev = the forward densities at omega0_dev, and
 * phi_dev = phi0_dev + s_out (dy_c - <dy_c>) for A and B, dy the network's
 * directional derivative (tangent pass, forward mode) along
 * omega_dev - omega0_dev; the solvent density from Eq. (11) at omega_dev.
 * The time stepper forms Phi(t+dt) from Phi~ this way.  Workspace as for
 * epd_sur_forward (training = 0). */
int epd_sur_tangent(const epd_lb_params *p, int32_t batch, const float *params_dev, double s_in, double s_out,
                    const double *omega0_dev, const double *omega_dev, double *phi0_dev, double *phi_dev, void *workspace,
                    size_t workspace_bytes, void *cuda_stream);
/* Loss L = mean over batch, A/B channels and sites of (y_c - (Phi_c - <Phi_c>)/s_out)^2
 * for the target densities phi_dev, and its gradient dL/dparams (FP32,
 * epd_sur_num_params values) to grad_dev; L to loss_dev[0]. */
int epd_sur_gradients(const epd_lb_params *p, int32_t batch, const float *params_dev, double s_in, double s_out,
                      const double *omega_dev, const double *phi_dev, float *grad_dev, double *loss_dev, void *workspace,
                      size_t workspace_bytes, void *cuda_stream);
/* epd_sur_gradients followed by one Adam step (beta 0.9, 0.999, eps 1e-8;
 * step counts from 1) on params_dev with moments adam_m_dev, adam_v_dev. */
int epd_sur_train_step(const epd_lb_params *p, int32_t batch, float *params_dev, float *adam_m_dev, float *adam_v_dev,
                       int32_t step, float lr, double s_in, double s_out, const double *omega_dev, const double *phi_dev,
                       double *loss_dev, void *workspace, size_t workspace_bytes, void *cuda_stream);

/* Let the surrogate stand in for both single-chain solves of epd_lb_step:
 * Phi~ is the surrogate at omega~ and Phi(t+dt) = Phi~ plus its tangent along
 * omega(t+dt) - omega~ (epd_sur_tangent).  Every exact_every-th step (and
 * while falling back) the exact step runs and also evaluates the surrogate
 * at omega~; its residual is the RMS difference of the A and B densities
 * relative to the RMS fluctuation of the exact ones (max over runs), and if
 * it exceeds residual_tol the following steps stay exact until a check
 * passes.  On the other steps both solves are the surrogate (Q_P, Q_S keep
 * their last exact values).  hold_force = 0: the polymer force of a
 * surrogate step comes from its own composition change Phi(t+dt) - Phi~
 * (Eqs. (19)-(20)); hold_force = 1: the LB keeps the force of the last exact
 * step.  (The force is the change over one diffusion step, and mu of
 * Eq. (1) nearly cancels in the incubation stage, so percent-level density
 * errors of a surrogate become large force errors, while the exact force
 * changes on the slow time scale of the composition.)  params_host: the
 * network's FP32 parameters (copied).  workspace: device memory of
 * epd_lb_surrogate_workspace_bytes bytes, caller-owned, kept alive while the
 * surrogate is attached.  exact_every = 0 detaches it. */
int epd_lb_surrogate_workspace_bytes(epd_lb *h, size_t *bytes);
int epd_lb_set_surrogate(epd_lb *h, const float *params_host, double s_in, double s_out, int32_t exact_every,
                         double residual_tol, int32_t hold_force, void *workspace, size_t workspace_bytes);
/* Controller statistics of epd_lb_set_surrogate (not in the paper): out[0]
 * steps taken with the surrogate attached, out[1] exact steps, out[2]
 * surrogate steps, out[3] exact steps forced by a failed check, out[4] last
 * residual (relative, as above), out[5] 1 if currently falling back. */
int epd_lb_surrogate_stats(epd_lb *h, double *out);

/* Exact step of App. C.  With max_iter > 0, epd_lb_step replaces steps 1-2
 * above by the convection of the composition fields and the inversion of the
 * density map (Sec. 2, integrator paragraph; App. C, items 1-3):
 *   Phi~ = Phi(t) - dt div(v Phi(t))       (convective part of Eq. (2), flux
 *                                           form, spectral derivatives),
 *   omega~ = Phi^{-1}(Phi~)                (Fletcher-Reeves CG from the
 *                                           auxiliary convection of omega),
 * and steps 3 and 5 use Phi(omega~).  CG minimises the convex function
 * G(omega) = <sum_I omega_I Phi~_I> + (phi_p/N) ln Q_P + (1 - phi_p) ln Q_S,
 * whose gradient is the density mismatch Phi~ - Phi(omega) over n; the line
 * search is one secant step between alpha = 0 and the previous step length
 * (1 at the first iteration); the direction restarts as the steepest descent
 * when it is not a descent direction.  Each iteration costs two single-chain
 * solves.  A run stops iterating when
 * sqrt(sum_I <(Phi~_I - Phi_I)^2>) < tol (N_tr = 1e-8 in the paper);
 * tol = 0 runs exactly max_iter iterations.  A step whose runs did not all
 * converge within max_iter iterations is completed and epd_lb_step returns
 * EPD_LB_ENOTCONV after it.  In MIXED_FP32 every density of the step is a
 * difference from the solve at the starting guess (so the mismatch carries
 * FP32 rounding relative to the changes only); excludes the surrogate
 * (EPD_LB_EINVAL).  The step is then enqueued eagerly
 * (no graph) and synchronises once per iteration when tol > 0.
 * max_iter = 0 (the default) restores the truncated step. */
int epd_lb_set_inversion(epd_lb *h, int32_t max_iter, double tol);
/* Of the last exact step of run `run` (App. C items 2-3): out[0] CG
 * iterations, out[1] the residual at the starting guess, out[2] the final
 * residual.  Synchronous. */
int epd_lb_inversion_stats(epd_lb *h, int32_t run, double *out);

/* Analysis of the polymer distribution Phi_P = Phi_A + Phi_B of the current
 * state (Phi is first recomputed if epd_lb_set_state replaced omega).  All
 * synchronous, host outputs. */
/* sigma_Delta of Eq. (22): *out = <|Phi_P(run_a) - Phi_P(run_b)|>, e.g. a run
 * with and one without the LB coupling (inv_beta_v = 0) from the same
 * initial state.  The runs need the same grid (EPD_LB_EINVAL otherwise). */
int epd_lb_sigma_delta(epd_lb *h, int32_t run_a, int32_t run_b, double *out);
/* Y_2^P of Eq. (30): the width of the polymer distribution across the flow,
 * read for the reverse-Poiseuille box as two channels of width L_y/2 centred
 * at L_y/4 and 3 L_y/4, y the distance from the nearest centre, rows at
 * (y + 1/2) dx: *out = sqrt(sum y^2 Phi_P / (phi_p sum y^2)); 1 for a
 * uniform distribution, below 1 when polymer gathers at the channel centres. */
int epd_lb_width(epd_lb *h, int32_t run, double *out);
/* Particles (Sec. 4): connected clusters of sites with Phi_P >= threshold
 * (0.5 in the paper; must be > 0), sites connected to their 4 nearest
 * neighbours across the periodic boundaries, numbered in the order of each
 * cluster's first site (row-major).  *count = the number of particles; for
 * particle k < max_particles, stats[10 k + 0..9] = sites, content
 * N = sum Phi_P, centre x, centre y (in R_G, in [0, L)), G_xx, G_xy, G_yy of
 * the gyration tensor of Eq. (27) (site positions (x, y) dx, separations the
 * shortest periodic ones: exact for particles narrower than half the box),
 * R and c of Eq. (28), c_rel of Eq. (29).  labels (ny*nx int32, may be NULL):
 * each site's particle number or -1.  The tensor's moments are FP64 atomic
 * sums (order-dependent in the last bits). */
int epd_lb_particles(epd_lb *h, int32_t run, double threshold, int32_t max_particles, int32_t *count,
                     double *stats, int32_t *labels);

/* Self-test of the failure path of the cluster solve's exchanges (failure
 * detection, not in the paper): one CTA
 * waits, with the same bounded wait as every exchange of the solve, on a
 * barrier that nothing arrives on; after limit_ms milliseconds (1..2000, at
 * the device's base clock) it gives up and sets the error bit that
 * epd_lb_sync reports as EPD_LB_ETIMEOUT.  *timed_out = 1 when that bit was
 * set.  The context stays usable.  Synchronous on cuda_stream. */
int epd_selftest_bounded_wait(int32_t limit_ms, void *cuda_stream, int32_t *timed_out);

/* Text of the last error on the handle (never NULL; not in the paper). */
const char *epd_lb_last_error(const epd_lb *h);

/* Release the handle (and its workspace if the library allocated it; not in
 * the paper). */
void epd_lb_destroy(epd_lb *h);

/*
 * Stateless single-chain solve on a 3D box, the extension the paper names in
 * Sec. 2 and Sec. 5: Eqs. (6)-(11) on nz x ny x nx sites (layout
 * [species][z][y][x]), the Fourier factor exp(-R_G^2 (kx^2 + ky^2 + kz^2) ds).
 * p gives nx, ny and every other parameter as for the 2D solve; nz is even,
 * of the form 2^a 3^b 5^c, at most 2048, and nx ny nz at most 2^22 sites.
 * omega_dev (3 nz ny nx doubles) -> phi_dev (the same), q_dev[2] = (Q_P, Q_S).
 * The streaming passes run over three views of the box (z pillars, y columns
 * of each plane, x rows carrying the node factors, history and contour
 * sums).  workspace_dev: epd_prop_solve3d_workspace_bytes bytes, 256-byte
 * aligned; EPD_LB_EINVAL for an unsupported box, EPD_LB_ENOMEM for a short
 * workspace.  Asynchronous on cuda_stream (may be NULL).
 */
int epd_prop_solve3d_workspace_bytes(const epd_lb_params *p, int32_t nz, size_t *bytes);
int epd_prop_solve3d(const epd_lb_params *p, int32_t nz, const double *omega_dev, double *phi_dev, double *q_dev,
                     void *workspace_dev, size_t workspace_bytes, void *cuda_stream);

/*
 * One coupled step on an nz x ny x nx box (the extension to 3D, Sec. 2 and
 * Sec. 5), in the order of the 2D step: auxiliary convection of omega with
 * the 3D spectral gradient, the 3D single-chain solve at omega~, the
 * diffusion step with the 3D Laplacian, the 3D solve at omega(t + dt), the
 * force of Eqs. (19)-(20) with i k / |k|^2 in 3D plus the reverse-Poiseuille
 * body force of Eq. (23) along x (a function of y), one D3Q19 update
 * (epd_lb3d_step).  EPD transforms in FP64, the solves in p->precision.
 * State on the device, updated in place: omega_dev [3][z][y][x], pop_dev
 * [19][z][y][x] (pre-collision, the order of epd_lb3d_step), vel_dev
 * [3][z][y][x] (the velocity handed to the convection, lattice units).
 * Outputs: phi_dev [3][z][y][x] = Phi(t + dt), q_dev[2], force_dev
 * [3][z][y][x] = the polymer force (lattice units).  workspace_dev:
 * epd_step3d_workspace_bytes bytes, 256-byte aligned.  Size rules of
 * epd_prop_solve3d.  Asynchronous on cuda_stream.
 */
int epd_step3d_workspace_bytes(const epd_lb_params *p, int32_t nz, size_t *bytes);
int epd_step3d(const epd_lb_params *p, int32_t nz, double *omega_dev, double *pop_dev, double *vel_dev, double *phi_dev,
               double *q_dev, double *force_dev, void *workspace_dev, size_t workspace_bytes, void *cuda_stream);

/*
 * One D3Q19 collide-stream on an nz x ny x nx box (the three-dimensional LB
 * scheme the paper names for the extension to 3D, Sec. 2), FP64: the
 * collision in the mode form of the D2Q9 update (u = (j + f/2)/rho, j* =
 * j + f, stress relaxed about rho c_s^2 I + rho u u by gamma_s and gamma_b of
 * p, Sigma of Eq. (15) with its d = 3 constants, ghosts scaled by gamma_g),
 * then streaming out_i(r + c_i) = n_i*(r), periodic.  pop_in_dev, pop_out_dev:
 * 19 nz ny nx doubles, [i][z][y][x], velocity order 0:(0,0,0), 1-6:
 * (+-1,0,0) (0,+-1,0) (0,0,+-1) in that order, 7-18: (1,1,0) (-1,-1,0)
 * (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1)
 * (0,1,-1) (0,-1,1); distinct buffers.  force_dev: total force [3][z][y][x]
 * (lattice units); vel_dev: u at the collision [3][z][y][x].  nz and the
 * size rules as for epd_prop_solve3d.  Asynchronous on cuda_stream.
 */
int epd_lb3d_step(const epd_lb_params *p, int32_t nz, const double *pop_in_dev, const double *force_dev,
                  double *pop_out_dev, double *vel_dev, void *cuda_stream);

/*
 * Stateless single-chain solve on device pointers (Sec. 2, Eqs. (6)-(11)):
 * omega_dev (3*ny*nx doubles) -> phi_dev (3*ny*nx doubles), q_dev[2] =
 * (Q_P, Q_S).  workspace_dev of epd_prop_solve_workspace_bytes bytes holds the
 * propagator history and the transform buffers; cuda_stream may be NULL (the
 * legacy default stream).  Asynchronous.
 */
int epd_prop_solve_workspace_bytes(const epd_lb_params *p, size_t *bytes);
int epd_prop_solve(const epd_lb_params *p, const double *omega_dev, double *phi_dev, double *q_dev,
                   void *workspace_dev, size_t workspace_bytes, void *cuda_stream);

/*
 * Allocation-free variant of epd_prop_solve (the paper has no counterpart;
 * this is a service for callers).
 *
 * Some callers cannot allocate device memory at the moment they need a
 * solve: plug-ins whose host framework owns every byte of the device through
 * its own pool, and real-time loops that must not pay for, or be serialised
 * by, cudaMalloc / cudaFree.  This entry point takes the same inputs and outputs as
 * epd_prop_solve (device pointers, caller-owned) but no workspace: its
 * scratch (propagator history, contour sums, transform tables, partial sums)
 * lives in one fixed array of EPD_PROP_SOLVE_NOALLOC_MAX_BYTES in the
 * library's device image.  Every GPU that loads the library holds that array
 * until the process exits.  The call makes no cudaMalloc, cudaFree or other
 * allocating call, on the device or through any library.
 *
 * Limits and behaviour:
 *  - The scratch needed is about nx*ny*(16 + (ns/2 + 3)*2*b) + 40 KiB bytes,
 *    b = 4 (EPD_LB_MIXED_FP32) or 8 (EPD_LB_PLAIN_FP64): e.g. 128 x 128 with
 *    ns = 64 fits in either precision, 256 x 512 does not.  A problem that
 *    does not fit is rejected with EPD_LB_ETOOLARGE before any work.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, which may load the library's device code) with
 *    that device current.  Later calls reuse the address, which belongs to the device's
 *    current context: after cudaDeviceReset (or any other teardown of that
 *    context) the stored address is stale and later calls in the same
 *    process are not valid.
 *  - All calls on one device share the array and it keeps the contents of
 *    the last call; each call re-initialises what it reads.  Two calls that
 *    can overlap on the GPU (different streams without ordering between
 *    them, or different host threads) race on the scratch and give wrong
 *    results: order them on one stream or serialise them.
 *  - The device-side error word of the solve (Q <= 0 or not finite) lives
 *    in the private scratch, so this call cannot report it: after the stream
 *    has completed, check that q_dev holds positive, finite Q_P and Q_S.
 *  - Asynchronous on cuda_stream (NULL: the legacy default stream).  Returns
 *    EPD_LB_EINVAL for bad parameters or NULL pointers, EPD_LB_ETOOLARGE if
 *    the scratch needed exceeds EPD_PROP_SOLVE_NOALLOC_MAX_BYTES, EPD_LB_ECUDA
 *    if a CUDA call fails.
 */
#define EPD_PROP_SOLVE_NOALLOC_MAX_BYTES (16u << 20)
int epd_prop_solve_noalloc(const epd_lb_params *p, const double *omega_dev, double *phi_dev, double *q_dev,
                           void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* EPD_LB_H */
