/*
 * lbve.h -- C ABI of the GB300 coupled viscoelastic lattice Boltzmann step.
 *
 * The library advances the coupled time step of Yu, Chen, Wang, Yuan & Shu,
 * "An improved lattice Boltzmann method with a novel conservative boundary
 * scheme for viscoelastic fluid flows" (arXiv 2508.16997):
 *   - a D2Q9 two-relaxation-time regularised (TRT-RLB) hydrodynamic lattice
 *     with the third-order Hermite equilibrium, the Galilean correction G_i,
 *     the local polymer-stress source T_i and the Hermite forcing F_i
 *     (Sec. 3.1, eqs. eq_ev_f, eq2, eq_ev_f0, eq4a-d, eq5, eq6);
 *   - three TRT-RLB convection-diffusion lattices for A_xx, A_xy, A_yy with
 *     the Oldroyd-B source Phi_ab, the auxiliary term G~_i, the source F~_i
 *     and its backward time difference (Sec. 3.2, eqs. eq_g0, eq_geq,
 *     eq_p_neq_m, eq_p_G_1, eq_p_F);
 *   - conservative non-equilibrium bounce-back (CNEBB) for the conformation
 *     lattices and wet-node non-equilibrium bounce-back (Zou-He) for the
 *     hydrodynamic lattice on flat walls (Sec. 3.3; Secs. 4.2-4.3);
 *   - optional solid masks (obstacles such as the cylinder of Sec. 4.3):
 *     CNEBB for the conformation lattices and linear interpolated
 *     bounce-back, at a per-link wall fraction q, for the hydrodynamic
 *     lattice, from a compact list of the fluid nodes next to the mask, with
 *     the momentum-exchange force on the solid (eq_F_x).
 *
 * Conventions shared by every entry point
 *   - Return value: LBVE_OK (0) or a negative LBVE_ERR_* code.  No C++
 *     exception crosses the ABI.  lbve_error_string() names a code;
 *     lbve_last_error() gives a one-line detail for the calling thread.
 *   - Grids are nx x ny nodes, periodic in x.  In y either periodic, or
 *     wet-node walls on rows y = 0 and y = ny - 1 (solid beyond them).  A
 *     solid mask may add interior solid nodes.
 *   - Host arrays are row-major [component][y][x], x fastest, float64,
 *     regardless of the storage precision of the instance.
 *   - The library never allocates device memory.  The caller allocates one
 *     device workspace of lbve_workspace_bytes() bytes and keeps it alive
 *     until lbve_destroy(); the library carves every buffer out of it.
 *   - All device work is enqueued on the caller's CUDA stream (cudaStream_t
 *     passed as void*).  lbve_step and lbve_fields(_many) with device output
 *     are asynchronous.  The calls that synchronise the stream are the set-up
 *     calls (lbve_create, lbve_set_geometry(_many), lbve_set_inlet,
 *     lbve_set_wall_distances, lbve_autotune), the adjoint
 *     (lbve_adjoint_step, lbve_adjoint_step_ex), the reads (lbve_status,
 *     lbve_fields(_many) with host output, lbve_totals, lbve_residual,
 *     lbve_profile_read), lbve_save, lbve_load and lbve_profile.
 *   - Lattice units: dx = dt = 1, rho_0 = 1, c_s^2 = 1/3.
 */
#ifndef LBVE_H
#define LBVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define LBVE_OK 0
#define LBVE_ERR_ARG (-1)       /* invalid argument or parameter            */
#define LBVE_ERR_CUDA (-2)      /* a CUDA runtime call or launch failed     */
#define LBVE_ERR_NONFINITE (-3) /* a field became NaN or Inf                */
#define LBVE_ERR_TIMEOUT (-4)   /* reserved for a bounded device-side wait;
                                   no entry point waits on the device, so
                                   none returns it                          */
#define LBVE_ERR_GEOMETRY (-5)  /* geometry not supported / inconsistent    */
#define LBVE_ERR_WORKSPACE (-6) /* workspace missing, too small, misaligned */
#define LBVE_ERR_STATE (-7)     /* call out of order (e.g. step before init)*/

/* ---- storage / arithmetic precision of an instance ---------------------- */
#define LBVE_FP64 0     /* populations stored and computed in float64        */
#define LBVE_FP32_DEV 1 /* float32 storage of deviations from the rest state
                           (f_i - w_i, g_i - w_i delta_c), float32 arithmetic,
                           float64 for conserved totals and wall balances     */
#define LBVE_DF32 2     /* float32 pairs (hi + lo, about 48 significant bits)
                           for storage and arithmetic: error-free float32
                           transformations on the float32 pipe, 8 bytes per
                           value as float64.  Oldroyd-B instances with flat
                           walls or periodic rows only (no solid mask, open
                           channel, FENE model or eq_p_G form); not covered
                           by the adjoint.  The paper has no counterpart: a
                           precision choice of this implementation.          */

/* Number of doubles returned by lbve_totals(). */
#define LBVE_NTOTALS 14

/* One problem statement (Sec. 2.4-2.5 of the paper), lattice units.
 * Derived on the host in float64:
 *   U_c = Ma c_s, nu_0 = U_c L_c / Re, nu_s = beta nu_0, mu_p = (1-beta) nu_0,
 *   tau_s1 = 3 nu_s + 1/2, tau_s2 = Lambda_s/(tau_s1 - 1/2) + 1/2,
 *   kappa = nu_s / Sc, tau_p1 = 3 kappa + 1/2,
 *   tau_p2 = Lambda_p/(tau_p1 - 1/2) + 1/2, lambda = Wi L_c / U_c. */
typedef struct {
  int32_t nx, ny;     /* nodes (ny >= 3 when walled)                        */
  int32_t periodic_y; /* 1: periodic in y; 0: walls on rows 0 and ny-1      */
  int32_t precision;  /* LBVE_FP64, LBVE_FP32_DEV or LBVE_DF32              */
  double beta;        /* viscosity ratio mu_s/mu_0, 0 < beta <= 1 (eqb7)    */
  double Wi;          /* Weissenberg number (eqb6), > 0                     */
  double Re;          /* Reynolds number (eqb5), > 0                        */
  double Sc;          /* Schmidt number (eqb8), > 0                         */
  double Ma;          /* Mach number (eq_Mach), > 0                         */
  double Lc;          /* characteristic length in lattice units, > 0       */
  double Lambda_s;    /* hydrodynamic magic parameter (Sec. 3.1), > 0       */
  double Lambda_p;    /* conformation magic parameter (Sec. 3.2), > 0       */
  double Fx, Fy;      /* uniform body force, used when no force field given */
  int32_t tile_tx;    /* tile width in nodes along x for the step kernel:
                         0 = library default (min(32, nx)), else 1..48
                         (float32; 1..128 for float64) and
                         <= nx (e.g. a width lbve_autotune() returned).  A
                         pure performance setting: each node's update does
                         not depend on the tiling; only the summation order
                         of the float64 totals follows the tiles.  The
                         workspace size does not depend on it.  A float64
                         batch with fewer 256-node tiles than the GPU's 152
                         SMs runs 64-thread tiles (TX x 64/TX) unless one of
                         its float64 instances asks for a width above 32.  */
  int32_t max_wall_nodes; /* capacity for a solid mask: the most fluid nodes
                         next to solid nodes (nodes with a solid neighbour
                         along any lattice direction) lbve_set_geometry may
                         install; 0 = no mask.  Costs nx*ny bytes plus 144
                         bytes per wall node of workspace.                 */
  int32_t open_x;     /* 0: periodic in x.  1: open channel (Sec. 4.3 set-up):
                         inlet column x = 0 with the profile of
                         lbve_set_inlet() (u = 0, A = I until set), outlet
                         column x = nx - 1 at density 1; nx >= 5.  Every
                         population of the two columns follows from the
                         neighbouring column by non-equilibrium
                         extrapolation: inlet f = f^eq(rho_f, u_in) + f_f -
                         f^eq(rho_f, u_f), g = g^eq(A_in, u_in) + g_f -
                         g^eq(phi_f, u_f); outlet f = f^eq(1, u_f) + f_f -
                         f^eq(rho_f, u_f), g = g_f (zero gradient).  The
                         columns' wall-row corners take the same rule;
                         gradients along x are one-sided there.            */
  int32_t model;      /* constitutive function F(A) of the conformation
                         equation and the Kramers stress (Sec. 2; eqb4 is
                         model 0): 0 Oldroyd-B F = A - I; 1 FENE-P
                         F = A/(1 - tr A/L2) - I/(1 - 2/L2); 2 FENE-CR
                         F = (A - I) L2/(L2 - tr A).                        */
  int32_t gtilde;     /* auxiliary term G~_i: 0 incompressible form eq_p_G_1,
                         1 the density-gradient form eq_p_G (F - c_s^2
                         grad rho, gradients as for u).                     */
  double L2;          /* FENE extensibility L^2 (> 2) for models 1 and 2.   */
} lbve_params;

typedef struct lbve_handle lbve_handle;

/* Bytes of device workspace needed for n_instances problems p[0..n-1].
 * Pure host computation.  Errors: LBVE_ERR_ARG for invalid parameters. */
int lbve_workspace_bytes(const lbve_params* p, int32_t n_instances, size_t* bytes);

/* Tile-width autotuner (the paper has no counterpart: the step kernel's
 * tiling is an implementation choice).  Times the batch p[0..n-1] with
 * candidate tile widths -- the widths 8, 16, 32 (float32; up to 128 for
 * float64) that fit nx,
 * or nx itself when nx < 8 -- and writes the fastest width of each instance
 * to tile_tx_out[0..n-1] (never 0).  Instances with the same candidates,
 * precision and wall layout share one width; one pass of coordinate descent
 * over these classes keeps a width only when the whole batch gets more than
 * 1% faster.  Each timing is trial_steps (1..100000) steps of lbve_step()
 * from the rest state with the uniform force of p, after as many warm-up
 * steps, best of two.
 *   d_workspace: >= lbve_workspace_bytes(p, n) bytes of device memory,
 *                256-byte aligned; used as scratch and left undefined, so it
 *                must not belong to a live handle (a handle may be created
 *                on it afterwards).
 *   cuda_stream: the stream the trials run on; synchronised.  The call
 *                refuses (LBVE_ERR_STATE) while that stream is capturing.
 * Errors: LBVE_ERR_ARG, LBVE_ERR_WORKSPACE, LBVE_ERR_STATE, LBVE_ERR_CUDA. */
int lbve_autotune(const lbve_params* p, int32_t n_instances, void* d_workspace, size_t bytes,
                  void* cuda_stream, int32_t trial_steps, int32_t* tile_tx_out);

/* Create a handle for n_instances independent problems p[0..n-1] that are
 * advanced together, one launch per precision per time step.
 *   d_workspace: device pointer, >= lbve_workspace_bytes() bytes, 256-byte
 *                aligned, owned by the caller, alive until lbve_destroy().
 *   cuda_stream: cudaStream_t (or NULL for the legacy default stream).
 * Copies the parameter tables to the device (on the stream).  The
 * instances are not initialised until lbve_set_geometry().
 * Errors: LBVE_ERR_ARG, LBVE_ERR_WORKSPACE, LBVE_ERR_CUDA. */
int lbve_create(const lbve_params* p, int32_t n_instances, void* d_workspace, size_t bytes,
                void* cuda_stream, lbve_handle** out);

/* Set the geometry, body force and initial state of instance inst and reset
 * its time to 0 (Sec. 4.2: unit density, zero velocity, identity
 * conformation and equilibrium populations unless init_fields is given).
 *   solid_mask : host uint8 [ny][nx], nonzero = solid node, or NULL for
 *                none.  Solid nodes take no part in the update and report
 *                zero fields; they are left out of the totals.  At each
 *                fluid node x next to the mask, every link i with x - e_i
 *                solid is a wall link: its hydrodynamic population is
 *                completed by linear interpolated bounce-back at wall
 *                fraction q (1/2, i.e. half-way bounce-back, until
 *                lbve_set_wall_distances() sets it), its three conformation
 *                populations by CNEBB (Sec. 3.3) with u at x; velocity
 *                gradients next to solid nodes are one-sided.
 *                LBVE_ERR_GEOMETRY if the instance has max_wall_nodes = 0
 *                or fewer than the mask's wall nodes, if a walled domain
 *                has solid nodes on rows 0-2 or ny-3..ny-1 (an open channel
 *                on columns 0-2 or nx-3..nx-1), if a fluid node
 *                has solid nodes on both ends of one lattice line, or if no
 *                fluid node is left.
 *   body_force : host float64 [2][ny][nx], or NULL for the uniform (Fx, Fy).
 *   init_fields: host float64 [6][ny][nx] = rho, ux, uy, Axx, Axy, Ayy, or
 *                NULL for rho = 1, u = 0, A = I.
 * Populations start at the equilibria (eq2, eq_geq) of the initial fields;
 * the history of the CDE source is set so that its time difference is zero
 * on the first step.  Host arrays may be freed when the call returns.
 * The geometry is checked on the host before anything changes; the values
 * of body_force and init_fields on the device after their upload: a value
 * that is not finite or an initial density that is not > 0 returns
 * LBVE_ERR_ARG and leaves the instance uninitialised (its previous state is
 * lost; lbve_step returns LBVE_ERR_STATE until the instance is set again).
 * Errors: LBVE_ERR_ARG, LBVE_ERR_GEOMETRY, LBVE_ERR_CUDA. */
int lbve_set_geometry(lbve_handle* h, int32_t inst, const uint8_t* solid_mask,
                      const double* body_force, const double* init_fields);

/* lbve_set_geometry for the n instances insts[0..n-1] in one call:
 * instance insts[j] takes solid_masks[j], body_forces[j] and init_fields[j]
 * (each as in lbve_set_geometry; a NULL list stands for n NULL pointers).
 * Every upload and initialisation is enqueued first and the stream is
 * synchronised once, at the end, so that the copies of one instance overlap
 * the host work of the next (with pinned host arrays the uploads are
 * asynchronous DMA; the arrays may be freed when the call returns).  Lists
 * of 16 or more instances are uploaded in chunks on the handle's internal
 * side stream, which waits for the caller's stream first; each chunk's
 * launches run on the caller's stream once its uploads are done.
 *   insts: host int32 [n], distinct instances (a repeated or out-of-range
 *          entry returns LBVE_ERR_ARG before anything changes).
 * Instances are enqueued in list order.  A geometry rejected on the host or
 * a CUDA error at list position j leaves insts[j..n-1] unchanged (insts[j]
 * uninitialised after a CUDA error) and still finishes insts[0..j-1]; a
 * CUDA error in the launches that follow the uploads leaves every staged
 * instance uninitialised.
 * Values rejected on the device (as in lbve_set_geometry) leave exactly the
 * rejected instances uninitialised; the others are set.  The return value is
 * the error of the first failing instance in list order (LBVE_OK if none),
 * and lbve_status bit 1 marks every instance whose values were rejected.
 * Errors: LBVE_ERR_ARG, LBVE_ERR_GEOMETRY, LBVE_ERR_CUDA. */
int lbve_set_geometry_many(lbve_handle* h, int32_t n, const int32_t* insts,
                           const uint8_t* const* solid_masks, const double* const* body_forces,
                           const double* const* init_fields);

/* Inlet profile of an open channel (open_x = 1): host float64 [5][ny] =
 * u_x, u_y, A_xx, A_xy, A_yy on the inlet column, rows 0..ny-1 (e.g. the
 * fully developed Oldroyd-B channel profile of Sec. 4.3).  Takes effect from
 * the next step; synchronises the stream.
 * Errors: LBVE_ERR_ARG (null, not finite), LBVE_ERR_GEOMETRY (not open),
 * LBVE_ERR_CUDA. */
int lbve_set_inlet(lbve_handle* h, int32_t inst, const double* inlet);

/* Wall fractions of curved walls (Sec. 4.3): for each of the n_links links
 * (node[j] = y nx + x of a fluid node, dir[j] in 1..8 with x - e_dir a solid
 * node of the mask), the fraction q[j] in (0, 1] of the link from the node
 * toward the solid node at which the wall lies.  Links not named keep their
 * fraction (1/2 after lbve_set_geometry).  q < 1/2 interpolates with the
 * fluid node x + e_dir (half-way bounce-back where that node is solid).
 * D2Q9 directions: e_1 = (1,0), e_2 = (0,1), e_3 = (-1,0), e_4 = (0,-1),
 * e_5 = (1,1), e_6 = (-1,1), e_7 = (-1,-1), e_8 = (1,-1).  Host arrays,
 * synchronises the stream.
 * Errors: LBVE_ERR_ARG (ranges, q), LBVE_ERR_GEOMETRY (no mask, not a wall
 * link), LBVE_ERR_CUDA. */
int lbve_set_wall_distances(lbve_handle* h, int32_t inst, int32_t n_links, const int32_t* node,
                            const int32_t* dir, const double* q);

/* Advance every instance by n_steps >= 0 time steps (asynchronous on the
 * stream).  The last step of the call also refreshes the macroscopic fields,
 * the float64 totals, the residual and the non-finite flags.  Runs of 32
 * non-final steps are replayed from a CUDA graph captured on first use (a
 * driver-managed object owned by the handle, released by lbve_destroy).
 * Errors: LBVE_ERR_STATE if an instance was never initialised,
 * LBVE_ERR_CUDA if a launch failed. */
int lbve_step(lbve_handle* h, int64_t n_steps);

/* Per-launch timing of the step kernel (the paper has no counterpart: a
 * measurement facility).  Synchronises the stream and arms CUDA events
 * around each of the next max_launches launches of the plain (unmasked) step
 * kernel of each precision, recorded on the handle's stream; the earlier
 * events are released.  While armed, lbve_step launches every step directly
 * instead of replaying its graph, so that each launch gets its own events.
 * max_launches = 0 disarms and releases the events.  Launches beyond
 * max_launches run untimed.
 * Errors: LBVE_ERR_ARG (max_launches outside [0, 2^20]), LBVE_ERR_STATE (the
 * stream is capturing), LBVE_ERR_CUDA. */
int lbve_profile(lbve_handle* h, int32_t max_launches);

/* Read the launches timed since lbve_profile() for the step kernel of one
 * precision (LBVE_FP64, LBVE_FP32_DEV or LBVE_DF32) and kind (final_step = 0: the
 * ordinary steps; 1: the last step of each lbve_step call, which also writes
 * the float64 fields and partial sums): their number, the sum of their
 * durations and the shortest and longest (ms; ms_min, ms_max may be NULL).
 * Each kind is armed for max_launches launches.  Waits for the last timed
 * launch to finish.  Zero launches when nothing was armed or no instance has
 * that precision.
 * Errors: LBVE_ERR_ARG, LBVE_ERR_CUDA. */
int lbve_profile_read(lbve_handle* h, int32_t precision, int32_t final_step, int32_t* launches,
                      double* ms_total, double* ms_min, double* ms_max);

/* Synchronise the stream and copy per-instance status flags into
 * flags[0..n-1] (bit 0: a non-finite field was seen at the end of an
 * lbve_step call; bit 1: the last lbve_set_geometry of the instance
 * rejected its force or initial fields).  Returns LBVE_ERR_NONFINITE if bit 0
 * of any flag is set. */
int lbve_status(lbve_handle* h, int32_t* flags);

/* Macroscopic fields of instance inst at its current time:
 * [6][ny][nx] float64 = rho, ux, uy (eq_ev_f0), Axx, Axy, Ayy (sum of g).
 * on_device = 0: out is host memory (the call synchronises the stream);
 * on_device = 1: out is device memory (asynchronous device-to-device copy). */
int lbve_fields(lbve_handle* h, int32_t inst, double* out, int32_t on_device);

/* lbve_fields for the n instances insts[0..n-1]: outs[j] (host or device
 * as on_device says, [6][ny][nx] float64 of instance insts[j]) receives its
 * fields.  All copies are enqueued first; with host outputs the stream is
 * synchronised once, at the end.  The arguments are checked before any copy
 * starts.  Errors: LBVE_ERR_ARG (null list or output, instance out of
 * range), LBVE_ERR_STATE (an instance never initialised), LBVE_ERR_CUDA. */
int lbve_fields_many(lbve_handle* h, int32_t n, const int32_t* insts, double* const* outs,
                     int32_t on_device);

/* Float64 totals of instance inst at its current time (synchronises):
 *   out[0..2]  sum rho, sum rho ux, sum rho uy  (rho u as in eq_ev_f0)
 *   out[3..5]  sum A_xx, sum A_xy, sum A_yy
 *   out[6..8]  CNEBB wall "in" of the last step, per conformation lattice:
 *              what the completion added back at wall nodes
 *   out[9..11] CNEBB wall "out" of the last step: post-collision populations
 *              that left wall nodes toward the wall (Sec. 3.3); in == out
 *   out[12..13] force of the fluid on the solid mask over the last step by
 *              momentum exchange (eq_F_x), x and y; 0 without a mask.
 * Sums run over fluid nodes; flat walls and mask walls both count in
 * out[6..11]. */
int lbve_totals(lbve_handle* h, int32_t inst, double out[LBVE_NTOTALS]);

/* Residual of instance inst (synchronises): max over nodes of
 * |u(t) - u(t')| / U_c, where t is the current time and t' the time at the
 * end of the previous lbve_step call (eq_err / 2eq4 when the calls advance
 * T_c steps each). */
int lbve_residual(lbve_handle* h, int32_t inst, double* out);

/* Current time step of instance inst. */
int lbve_time(lbve_handle* h, int32_t inst, int64_t* t);

/* Host bytes of a saved state of every instance of h (lbve_save/lbve_load). */
int lbve_state_bytes(lbve_handle* h, size_t* bytes);

/* Checkpoint: copy every instance's current state -- 36 post-collision
 * populations, 5 history values and the force (storage precision), the
 * float64 fields, the time and the set-up flags -- into host_buf
 * (>= lbve_state_bytes()).  Synchronises the stream. */
int lbve_save(lbve_handle* h, void* host_buf, size_t bytes);

/* Resume: restore a state saved by lbve_save() into a handle created with the
 * same parameters (checked: instance count, grid, precision, walls).  The
 * continuation is bit-identical to the saved run's.  Synchronises.
 * Errors: LBVE_ERR_ARG on a size or parameter mismatch, LBVE_ERR_CUDA. */
int lbve_load(lbve_handle* h, const void* host_buf, size_t bytes);

/* Bytes of device workspace lbve_adjoint_step() needs for instance inst and
 * a trajectory of n_steps >= 1 steps (sqrt(n_steps) checkpoints and one
 * recomputed segment of stored states, plus the adjoint fields).  Host only. */
int lbve_adjoint_workspace_bytes(lbve_handle* h, int32_t inst, int64_t n_steps, size_t* bytes);

/* Bytes of adjoint workspace for a checkpoint interval of `interval` steps
 * (1 <= interval <= n_steps): ceil(n_steps/interval) stored states plus a
 * recomputed segment of `interval` states.  The paper has no counterpart:
 * it trades memory for recomputation.  lbve_adjoint_step() takes the
 * shortest interval whose workspace fits the bytes it is given, so a caller
 * with memory to spare passes more: interval 1 stores every forward state and
 * recomputes none (about n_steps x 41 planes of the storage precision).  The
 * gradient does not depend on the interval (every state is recomputed by the
 * same step from the same predecessor).  Host only.
 * Errors: LBVE_ERR_ARG. */
int lbve_adjoint_workspace_bytes_interval(lbve_handle* h, int32_t inst, int64_t n_steps,
                                          int64_t interval, size_t* bytes);

/* Gradient of a loss L on the fields at time n_steps with respect to the
 * per-node body force of instance inst, by a discrete adjoint of every step
 * (the reverse of each stage of the coupled step of Secs. 3.1-3.3: collisions,
 * source, finite-difference gradients, Zou-He and CNEBB completions, pull
 * streaming) with sqrt(n_steps) checkpointing and recomputation.
 * Open channels (Sec. 4.3 set-up) are covered: the inlet and outlet columns'
 * completion from the neighbouring column is reversed too, with the inlet
 * profile held fixed.  Models other than Oldroyd-B and the eq_p_G form are
 * refused (LBVE_ERR_ARG); a solid mask is covered (see
 * lbve_adjoint_step_ex).
 * The trajectory is the one that lbve_set_geometry(h, inst, NULL, <current
 * force of inst>, init_fields) followed by lbve_step(n_steps) produces; the
 * forward states are recomputed in the adjoint workspace (the instance's own
 * state is not touched).
 *   init_fields  : host float64 [6][ny][nx] initial fields, or NULL for rho = 1,
 *                  u = 0, A = I (as in lbve_set_geometry)
 *   d_dL_dfields : device float64 [6][ny][nx], dL/d(rho, ux, uy, Axx, Axy, Ayy)
 *                  at time n_steps
 *   d_ws, bytes  : device workspace >= lbve_adjoint_workspace_bytes(), 256-byte
 *                  aligned, owned by the caller; the shortest checkpoint
 *                  interval (down to 1) whose workspace fits `bytes` is used
 *                  (lbve_adjoint_workspace_bytes_interval)
 *   d_dL_dforce  : device float64 [2][ny][nx], overwritten with dL/dF (the
 *                  derivative with respect to a per-node force, also when the
 *                  instance uses a uniform force)
 * Computed in the instance's precision.  Synchronises the stream.
 * Errors: LBVE_ERR_ARG, LBVE_ERR_STATE, LBVE_ERR_WORKSPACE, LBVE_ERR_CUDA. */
int lbve_adjoint_step(lbve_handle* h, int32_t inst, const double* init_fields,
                      const double* d_dL_dfields, int64_t n_steps, void* d_ws, size_t bytes,
                      double* d_dL_dforce);

/* The adjoint with the solid mask's losses and parameters: as
 * lbve_adjoint_step(), with
 *   d_dL_dfields : as there, or NULL for no field term;
 *   dL_ddrag     : host float64 [2], dL/d(F_x, F_y) of the force on the solid
 *                  over the last step (lbve_totals() out[12..13], eq_F_x), or
 *                  NULL; needs a solid mask;
 *   d_dL_dq      : device float64 [8][ny][nx] or NULL; written with dL/dq of
 *                  each wall link's fraction q (plane i-1 at node k for the
 *                  link (k, i) of lbve_set_wall_distances; zero elsewhere) --
 *                  the gradient with respect to the wall geometry; needs a
 *                  solid mask.
 * At least one of d_dL_dfields and dL_ddrag must be given.  The forward
 * states are recomputed with the wall pass; the reverse passes differentiate
 * the interpolated bounce-back, CNEBB at the mask and the one-sided
 * gradients next to solid nodes.
 * Errors: as lbve_adjoint_step(); LBVE_ERR_GEOMETRY for drag or q gradients
 * without a mask. */
int lbve_adjoint_step_ex(lbve_handle* h, int32_t inst, const double* init_fields,
                         const double* d_dL_dfields, const double* dL_ddrag, int64_t n_steps,
                         void* d_ws, size_t bytes, double* d_dL_dforce, double* d_dL_dq);

/* Float64 sums of a macroscopic field array, computed WITHOUT ALLOCATING any
 * device memory.  The paper has no counterpart: this serves callers that
 * cannot call cudaMalloc -- a framework whose own allocator owns all device
 * memory and forbids side allocations, a latency-critical loop that cannot
 * afford the device synchronisation of cudaMalloc/cudaFree, or a caller that
 * holds a field array but no lbve workspace.
 *   d_fields: device float64 [6][ny][nx] = rho, ux, uy, Axx, Axy, Ayy (the
 *             layout lbve_fields() writes with on_device = 1); read only.
 *   d_out   : device float64 [6], written: sum rho, sum rho ux, sum rho uy,
 *             sum Axx, sum Axy, sum Ayy (the quantities of lbve_totals()
 *             out[0..5], summed in a different fixed order).
 * Asynchronous on cuda_stream (a cudaStream_t, NULL for the default stream).
 * Scratch: one file-scope static device array of 16384 partial records
 * (1 MiB) that every GPU loading the library keeps until the process exits;
 * it limits a call to nx * ny <= 16,777,216 nodes (LBVE_ERR_ARG beyond).  The
 * first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process; make that first call before any stream capture, and do not
 * call the entry point after cudaDeviceReset (the array may then move).  Every call shares the array and
 * leaves its records behind; each call overwrites the records it reads, so
 * nothing needs clearing, but calls that overlap on the GPU (other streams,
 * other threads) race on it and must be serialised by the caller.
 * Errors: LBVE_ERR_ARG (null pointer, bad size, over the limit),
 * LBVE_ERR_CUDA (device query, symbol lookup or launch failed); every error
 * leaves its detail in lbve_last_error(). */
int lbve_field_totals_noalloc(const double* d_fields, int32_t nx, int32_t ny, double* d_out,
                              void* cuda_stream);

/* Release the handle (host memory only; the workspace stays the caller's).
 * Synchronises the stream. */
void lbve_destroy(lbve_handle* h);

/* Static name of a return code, and a detail line for the calling thread. */
const char* lbve_error_string(int code);
const char* lbve_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBVE_H */
