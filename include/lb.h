/*
 * lb.h - C ABI of the GB300 lattice Boltzmann + raspberry-colloid library.
 *
 * The library advances a D3Q19 lattice Boltzmann fluid coupled by point
 * friction to rigid "raspberry" colloids, the method of Ustach & Faller,
 * "The Raspberry model for protein-like particles: ellipsoids and confinement
 * in cylindrical pores" (arXiv:1604.01829):
 *   - fluid: streaming along the discrete velocity links and a collision that
 *     relaxes towards equilibrium on one time scale (BGK) or mode by mode
 *     (multiple relaxation times), deterministic or with thermal noise;
 *     boundary nodes reflect what streams into them (Sec. 1.1);
 *   - coupling: each bead feels F = -gamma (v - u(r,t)) + f_s with u
 *     interpolated from the nearest nodes, Eq. (latticeboltzmannfriction)
 *     in Sec. 1.1; -F goes back to the same nodes;
 *   - bodies: beads are virtual sites of a rigid body whose centre of mass
 *     moves by velocity Verlet and whose orientation is a quaternion
 *     (Sec. 1.2, Sec. 2.3);
 *   - pores: cylindrical walls with boundary nodes half a grid spacing
 *     outside the wall (Sec. 2.3).
 *
 * Units: lattice units throughout (grid spacing 1, time step 1, fluid mass
 * per node rho0). Node (x, y, z), 0 <= x < nx etc., has its centre at
 * (x + 1/2, y + 1/2, z + 1/2) and linear index x + nx (y + ny z).
 * Populations are exchanged as double arrays [19][N] in the velocity order
 * of lb_lattice().
 *
 * Conventions: every call returns an lb_status; none aborts, prints or
 * throws. Inputs are copied (the caller keeps ownership of its buffers);
 * outputs go to caller-owned buffers. Pointer arguments are HOST pointers
 * unless the name says otherwise. The library owns all device memory it
 * allocates; lb_destroy frees it. A handle is not thread-safe: one host
 * thread at a time per handle. Device work is issued on the stream given at
 * creation (or a private stream); calls that return data to the host
 * synchronise that stream.
 */
#ifndef LB_H
#define LB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx *lb_handle;

typedef enum {
    LB_OK = 0,
    LB_ERR_ARG = 1,      /* invalid argument or unsupported combination   */
    LB_ERR_OOM = 2,      /* device or host allocation failed              */
    LB_ERR_CUDA = 3,     /* a CUDA call failed (message in lb_last_error) */
    LB_ERR_UNSTABLE = 4, /* non-finite mass or momentum detected          */
    LB_ERR_TIMEOUT = 5,  /* a bounded device wait ran out                 */
    LB_ERR_STATE = 6     /* call not valid in the current state           */
} lb_status;

typedef struct {
    int nx, ny, nz;          /* lattice size, each >= 2                              */
    int precision;           /* 64: FP64 populations; 32: FP32 populations stored as
                                f_i - w_i rho0 (compute in FP32, bodies and
                                reductions in FP64)                                  */
    int collision;           /* 0: BGK (Sec. 1.1 single time scale); 1: MRT          */
    double tau;              /* BGK relaxation time (> 1/2)                          */
    double gamma_shear;      /* MRT: non-equilibrium part of each mode is multiplied */
    double gamma_bulk;       /*   by its rate per step, m* - m_eq = g (m - m_eq);     */
    double gamma_odd;        /*   |g| < 1. Shear: g = (6 nu - 1)/(6 nu + 1).          */
    double gamma_even;       /*   odd / even: kinetic (ghost) modes.                  */
    double rho0;             /* reference density (> 0)                              */
    double kT;               /* thermal energy; > 0 enables fluctuating MRT modes
                                and bead noise (MRT only)                            */
    double gamma_bead;       /* bead friction gamma of Eq. (latticeboltzmannfriction),
                                lattice units (>= 0)                                 */
    unsigned long long seed; /* Philox4x32-10 key                                    */
    unsigned int instance;   /* third Philox counter word (independent replicas)     */
    double body_force[3];    /* uniform force density on every fluid node            */
    int compensate_force;    /* 1: add -sum(F_ext of free bodies)/N_fluid to the
                                fluid so the total momentum stays constant           */
    int md_substeps;         /* MD substeps per LB step, 1-4 (0 = 1; the paper's MD step
                                is half the LB step: 2). Each substep moves the bodies by
                                dt = 1/n and couples the beads to this LB step's fluid
                                (bead noise of variance 2 kT gamma / dt); the fluid
                                receives every substep's bead forces times dt. Not with
                                the adjoint; in a batch every instance has the same.   */
} lb_params;

/* Creates a lattice with every population at rest, f_i = w_i rho0.
 * cuda_stream: a cudaStream_t to issue work on, or NULL for a private stream.
 * On success *out holds the new handle. Errors: LB_ERR_ARG (bad params),
 * LB_ERR_OOM, LB_ERR_CUDA (no device, launch failure). */
lb_status lb_create(const lb_params *params, void *cuda_stream, lb_handle *out);

/* Frees all device and host memory of the handle. NULL is accepted. */
lb_status lb_destroy(lb_handle h);

/* Cylindrical pore (Sec. 2.3): wall along `axis` (0 x, 1 y, 2 z) through the
 * box centre; a node whose centre lies at distance >= radius from the axis is
 * a boundary node, so the first boundary node along a lattice direction sits
 * half a grid spacing outside the wall. Populations streaming into boundary
 * nodes return to their origin reversed (halfway bounce-back). Only before
 * the first lb_step. Errors: LB_ERR_ARG, LB_ERR_STATE. */
lb_status lb_set_pore(lb_handle h, double radius, int axis);

/* Moving walls for the Stokes-flow resistance set-up (Sec. 2.3: boundary
 * nodes along the +y and -y faces with an imposed fluid velocity, the colloid
 * held fixed in between): the planes y = -1/2 and y = ny - 1/2 bound the
 * fluid and move with the tangential velocities u_lo[3] and u_hi[3] (y
 * components must be 0); the box stays periodic in x and z. A population
 * streaming into a wall returns reversed with the wall's momentum,
 * f_opp(i) = f*_i - 6 w_i rho0 (c_i . u_wall) (moving-wall halfway
 * bounce-back); a node beyond a wall carries the wall's velocity in the bead
 * interpolation and takes no spread force. Mass stays exact. Only before the
 * first lb_step and without a pore (LB_ERR_STATE); LB_ERR_ARG for a normal
 * velocity component or ny < 2. Not available to lb_adjoint_drag. */
lb_status lb_set_channel_walls(lb_handle h, const double u_lo[3], const double u_hi[3]);

/* Repulsive pore wall for the raspberries (Sec. 2.3: beads placed around the
 * pore surface, a given distance apart, interacting with the colloid beads by
 * a purely repulsive WCA potential with sigma = r_bead + r_pore_bead).
 * Reading: the wall beads sit on the cylinder of radius R_pore + r_pore_bead
 * around the pore axis (so that they touch the hydrodynamic wall), in rings
 * of round(2 pi (R_pore + r_pore_bead) / spacing) beads at
 * (k + 1/2) L / round(L / spacing) along the axis (L the box length along
 * it). Each colloid bead at distance d < 2^(1/6) sigma from a wall bead gets
 * F = 24 epsilon (2 (sigma/d)^12 - (sigma/d)^6) d_vec / d^2 (minimum image
 * along the axis); the force and its torque go to the body, not to the
 * fluid, and are not part of lb_forces' per-bead friction forces. Needs a
 * pore (else LB_ERR_STATE); spacing = 0 removes the wall beads; LB_ERR_ARG
 * for spacing < 0, negative radii or a zero sigma, epsilon < 0. Lattice units
 * (the paper's 5 nm spacing, r_p = 6.25 nm, r_r = 0.5 nm, epsilon = kT). */
lb_status lb_set_pore_beads(lb_handle h, double spacing, double r_pore_bead, double r_bead, double epsilon);

/* Adds a rigid raspberry (Sec. 1.2): nbeads body-frame bead offsets
 * beads_body_xyz[3*nbeads] relative to the centre of mass X[3], orientation
 * q[4] = (w, x, y, z) (normalised by the library), mass and principal
 * moments inertia[3] (body axes = principal axes), constant external force
 * F_ext[3] and torque T_ext[3] (lab frame, may be NULL = 0). fixed = 1 holds
 * the body's position, orientation and velocities (a fixed colloid in flow);
 * fixed = 2 integrates translation only, the orientation held and omega = 0
 * (a colloid pulled along a body axis, the case the adjoint differentiates).
 * *body_id receives the body index (0, 1, ...). Only before the first lb_step.
 * Errors: LB_ERR_ARG, LB_ERR_STATE. */
lb_status lb_add_raspberry(lb_handle h, const double *beads_body_xyz, int nbeads,
                           const double X[3], const double q[4], double mass,
                           const double inertia[3], const double F_ext[3],
                           const double T_ext[3], int fixed, int *body_id);

/* Sets the kinematic state of a body: centre X, velocity V, orientation q,
 * body-frame angular velocity w (any pointer may be NULL = unchanged). */
lb_status lb_set_body_state(lb_handle h, int body_id, const double X[3], const double V[3],
                            const double q[4], const double w[3]);

/* Replaces the external forces and torques of the first nbodies bodies from
 * F_ext[3*nbodies], T_ext[3*nbodies] (lab frame; T_ext may be NULL = 0); the
 * next lb_step uses them. The values are copied before the call returns
 * (into host-mapped memory that the next step's prologue reads, after
 * waiting for steps already queued to have read the previous ones; where
 * that memory could not be allocated, by copies queued on the stream, which
 * read the caller's arrays later). Errors: LB_ERR_ARG (bad count, NULL
 * F_ext, non-finite values). */
lb_status lb_set_external_forces(lb_handle h, int nbodies, const double *F_ext, const double *T_ext);

/* Advances nsteps LB steps. One step: (1) bodies half-kick and drift,
 * (2) virtual sites, (3) bead coupling with trilinear interpolation and
 * spread, (4) fused collision + in-place streaming with halfway
 * bounce-back, (5) bodies second half-kick. Asynchronous on the handle's
 * stream. Errors: LB_ERR_ARG (nsteps < 0), LB_ERR_CUDA. */
lb_status lb_step(lb_handle h, int nsteps);

/* Total force F[3] and torque T[3] (lab frame, about the centre of mass) on
 * body_id from the last step: sum of bead forces plus F_ext / T_ext, the
 * quantity of Eq. (stokesflow). per_bead_xyz (may be NULL) receives the
 * 3*nbeads bead forces of that body. Synchronises. */
lb_status lb_forces(lb_handle h, int body_id, double F[3], double T[3], double *per_bead_xyz);

/* F[3*nbodies], T[3*nbodies] for the first nbodies bodies (as lb_forces,
 * every body in one call: after a step the totals and the device error word
 * are read from host-mapped memory the step wrote, without a copy).
 * Synchronises; returns LB_ERR_TIMEOUT / LB_ERR_STATE as lb_forces. */
lb_status lb_forces_all(lb_handle h, int nbodies, double *F, double *T);

/* One round of a host control loop in one call: lb_set_external_forces(h,
 * nbodies, F_ext, T_ext) (skipped when F_ext is NULL), lb_step(h, nsteps),
 * then lb_forces_all(h, nbodies, F, T) (skipped when F and T are both NULL),
 * with the same arguments, layouts ([3 nbodies] each, lab frame) and errors
 * as those three calls; the first failing part's status is returned and the
 * later parts are not run. Host arrays are the caller's and are used only
 * during the call. Synchronises when F or T is given. */
lb_status lb_step_io(lb_handle h, int nsteps, int nbodies, const double *F_ext, const double *T_ext, double *F,
                     double *T);

/* Body state X[3], V[3], q[4], body-frame w[3] (any may be NULL). */
lb_status lb_get_body(lb_handle h, int body_id, double X[3], double V[3], double q[4], double w[3]);

/* Pre-collision populations of the current step as double [19][N]
 * (n == 19*N). Boundary-node entries are unspecified. Synchronises. */
lb_status lb_get_populations(lb_handle h, double *host, size_t n);

/* Replaces the pre-collision populations of the current step. */
lb_status lb_set_populations(lb_handle h, const double *host, size_t n);

/* Pre-collision populations of `count` nodes given by linear index
 * nodes[count] into out[19*count] (node-major). Synchronises. */
lb_status lb_sample_populations(lb_handle h, const long long *nodes, int count, double *out);

/* Bead force density spread onto the nodes by the last step (the force the
 * last collision used, without body_force), as double [3][N]. */
lb_status lb_get_node_force(lb_handle h, double *host, size_t n);

/* Fluid mass sum f and momentum sum c f of the pre-collision populations,
 * reduced in FP64. Returns LB_ERR_UNSTABLE if either is not finite. */
lb_status lb_conservation(lb_handle h, double *mass, double mom[3]);

typedef struct {
    long long nodes, fluid_nodes, step;
    int nbodies, nbeads, precision;
    size_t device_bytes;
} lb_info_t;

lb_status lb_info(lb_handle h, lb_info_t *info);

/* Choice of the fused collide-and-stream kernel: variant 0 = automatic
 * (currently the plain kernel, the faster one measured on GB300), 1 = plain
 * per-thread loads, 2 = TMA-staged
 * (FP32 storage, no pore, nx % 4 == 0, else LB_ERR_ARG). stages (0 = auto,
 * 2-6) sets the depth of the shared-memory ring of row segments, ctas_per_sm
 * (0 = auto) the persistent grid. Results do not depend on the choice. */
lb_status lb_set_kernel_variant(lb_handle h, int variant, int stages, int ctas_per_sm);

/* Checkpoint and resume. A checkpoint holds the whole state a later step
 * depends on: the populations in the storage precision (bit for bit), the
 * step counter (which is also the Philox counter of the noise), every body's
 * state, the per-bead forces, and the spread-force buffers with their tile
 * flags and lists (the previous step's force enters the next interpolation).
 * Loading it into a handle created with the same parameters (lattice,
 * precision, collision, seed, pore or walls) and the same bodies and beads
 * resumes the run exactly: the same steps then give the same results, up to
 * the summation order of the bead-force atomics. The trajectory recorder is
 * not part of a checkpoint. lb_checkpoint_size: bytes needed (uploads the
 * bodies on the first call); lb_checkpoint_save: into a caller-owned host
 * buffer of at least that size (synchronises); lb_checkpoint_load: from such
 * a buffer. Errors: LB_ERR_ARG (null or short buffer, not a checkpoint),
 * LB_ERR_STATE (taken from a lattice with other parameters or bodies),
 * LB_ERR_CUDA. The layout is this library's own and may change between
 * versions. */
lb_status lb_checkpoint_size(lb_handle h, size_t *bytes);
lb_status lb_checkpoint_save(lb_handle h, void *host, size_t bytes);
lb_status lb_checkpoint_load(lb_handle h, const void *host, size_t bytes);

/* Limit, in SM clock cycles, of each bounded device wait (the TMA-staged
 * kernel's wait for a stage's copies; 0 = the default of about 2 s). A wait
 * that runs out stops its thread block (after its copies in flight have
 * landed) and sets the handle's device error word; the next synchronising
 * call (lb_forces, lb_forces_all, lb_conservation) returns LB_ERR_TIMEOUT once
 * and clears it. The lattice state is then partly stepped and should be
 * restored (lb_set_populations). No effect on the plain kernel, which does not
 * wait. Errors: LB_ERR_ARG for cycles < 0. */
lb_status lb_set_wait_limit(lb_handle h, long long cycles);

/* Kernel timing: when on, CUDA events bracket every launch of the fused
 * collide-and-stream kernel on the handle's stream. lb_kernel_time returns
 * (synchronising) the summed device time in ms and the number of timed
 * launches since the last call, then resets the counters. */
lb_status lb_set_timing(lb_handle h, int on);
lb_status lb_kernel_time(lb_handle h, double *total_ms, long long *launches);

/* Message of the last failed call on h (or of the last failed lb_create when
 * h is NULL). Owned by the library, valid until the next call. */
const char *lb_last_error(lb_handle h);
const char *lb_status_string(lb_status s);

/* Adjoint of the deterministic step (kT = 0; every body fixed (1) or
 * translation-only (2)). Runs nsteps steps from the current state (the
 * handle ends exactly where lb_step(h, nsteps) would leave it) and returns
 * J = mean over the last `window` steps of component `axis` of the velocity
 * of body `body` (the terminal velocity of a colloid pulled by F_ext, whose
 * drag is F_ext / J as in Eq. (stokesflow)), dJ/dgamma (bead friction of
 * Eq. (latticeboltzmannfriction)) and, if dJ_dbeads is not NULL, dJ/ds for
 * every body-frame bead offset of every body (3 per bead, in the order the
 * beads were added). checkpoints: snapshot slots of the two-level schedule
 * (0 = ceil(sqrt(nsteps))); memory ~ (checkpoints + nsteps/checkpoints)
 * lattice states, cost ~ two forward sweeps plus one reverse sweep.
 * Errors: LB_ERR_ARG, LB_ERR_OOM, LB_ERR_CUDA. */
lb_status lb_adjoint_drag(lb_handle h, int nsteps, int window, int body, int axis, int checkpoints,
                          double *J, double *dJ_dgamma, double *dJ_dbeads);

/* Checkpointing schedules of the adjoint sweep (the states a reversed step
 * needs are kept or recomputed; the paper itself has no adjoint).
 *   LB_ADJ_TWO_LEVEL: `snapshots` slots (0 = ceil(sqrt(nsteps))) hold one
 *     state every K = ceil(nsteps/slots) steps during the forward sweep; each
 *     segment is re-run from its slot with every step taped, then reversed.
 *     Memory ~ (slots + K) states, cost one extra forward sweep.
 *   LB_ADJ_BINOMIAL: at most `snapshots` states (>= 1; 0 = 16), the start
 *     state included, placed by the binomial rule of Griewank and Walther
 *     (revolve): with s states and r repetitions, C(s + r, s) steps can be
 *     reversed, so r is the smallest repetition count with
 *     C(s + r, s) >= nsteps, and no step is re-run more than r times. Each
 *     reversed step re-runs only its body prologue and bead coupling from the
 *     restored state (the reverse pass needs no stored populations). Memory
 *     (snapshots + 1) states, cost about r forward sweeps. */
#define LB_ADJ_TWO_LEVEL 0
#define LB_ADJ_BINOMIAL 1
typedef struct {
    int schedule;   /* LB_ADJ_TWO_LEVEL or LB_ADJ_BINOMIAL */
    int snapshots;  /* see above */
} lb_adjoint_opts;

/* Where the time of one lb_adjoint_drag_ex call went (device times from
 * CUDA events on the handle's stream). */
typedef struct {
    double alloc_ms;          /* host time allocating the workspace; 0 when a
                                 previous call's workspace was reused */
    double forward_ms;        /* the first forward sweep (to the first reversed step) */
    double recompute_ms;      /* re-run forward steps, taping, saves and restores after it */
    double reverse_ms;        /* the reverse-pass kernels alone */
    long long forward_steps;  /* steps of the first sweep */
    long long recompute_steps;/* forward steps re-run after it (a turn's prologue and
                                 coupling are not counted) */
    long long reversed_steps;
    double workspace_bytes;   /* device memory held by the adjoint's workspace */
} lb_adjoint_stats;

/* lb_adjoint_drag with a chosen schedule (opts NULL = two-level with
 * ceil(sqrt(nsteps)) slots) and, if stats is not NULL, the time split above
 * (the events cost a little; stats = NULL times nothing). The workspace
 * (snapshots, tapes, adjoint fields) stays allocated with the handle and is
 * reused by later calls that need no more of it; lb_destroy frees it.
 * Results are those of lb_adjoint_drag up to the summation order of
 * atomics in re-run steps. Errors: as lb_adjoint_drag; LB_ERR_ARG for an
 * unknown schedule or snapshots < 0. */
lb_status lb_adjoint_drag_ex(lb_handle h, int nsteps, int window, int body, int axis, const lb_adjoint_opts *opts,
                             double *J, double *dJ_dgamma, double *dJ_dbeads, lb_adjoint_stats *stats);

/* ------------------------------------------------------------------ batches
 * Many independent lattices of uneven size advanced together: the same step
 * as above for every instance (Sec. 1.1, Eq. (latticeboltzmannfriction),
 * Sec. 2.3), with one launch per kernel per step for all instances and the
 * step sequence replayed from a CUDA graph. Instance k reproduces what a
 * single handle with params[k] computes. */
typedef struct lb_batch_ctx *lb_batch_handle;

/* params[n]: one parameter set per instance (all with the same precision,
 * collision type and thermal noise on/off; sizes, rates, seeds, forces may
 * differ). cuda_stream as for lb_create. Errors: LB_ERR_ARG, LB_ERR_OOM,
 * LB_ERR_CUDA. */
lb_status lb_batch_create(const lb_params *params, int n, void *cuda_stream, lb_batch_handle *out);
lb_status lb_batch_destroy(lb_batch_handle h);
/* As lb_set_pore / lb_add_raspberry for instance `inst` (before the first
 * step); *body_id is the body's index within its instance. From the first
 * step on, a pore instance stores its fluid nodes only (populations set
 * before are carried over; wall nodes read back as fluid at rest), which
 * limits its cross-section to 65534 fluid positions (the first step returns
 * LB_ERR_ARG for a larger one). */
/* Pore-wall beads of one instance, as lb_set_pore_beads (after its pore,
 * before the first step). */
lb_status lb_batch_set_pore_beads(lb_batch_handle h, int inst, double spacing, double r_pore_bead,
                                  double r_bead, double epsilon);
lb_status lb_batch_set_pore(lb_batch_handle h, int inst, double radius, int axis);
lb_status lb_batch_add_raspberry(lb_batch_handle h, int inst, const double *beads_body_xyz, int nbeads,
                                 const double X[3], const double q[4], double mass, const double inertia[3],
                                 const double F_ext[3], const double T_ext[3], int fixed, int *body_id);
/* Advances every instance nsteps steps (pairs of steps as one graph launch). */
lb_status lb_batch_step(lb_batch_handle h, int nsteps);
lb_status lb_batch_forces(lb_batch_handle h, int inst, int body_id, double F[3], double T[3]);
lb_status lb_batch_get_body(lb_batch_handle h, int inst, int body_id, double X[3], double V[3], double q[4],
                            double w[3]);
lb_status lb_batch_get_populations(lb_batch_handle h, int inst, double *host, size_t n);
lb_status lb_batch_set_populations(lb_batch_handle h, int inst, const double *host, size_t n);
/* Work schedule of the fluid kernel: tile_nodes (64, 128, 256) consecutive
 * nodes of one instance per CTA iteration, blocks_per_sm resident CTAs of
 * the persistent grid (tile_nodes * blocks_per_sm <= 2048; each step's grid is
 * further capped at the CTAs of that step's kernel that fit at once), order 0 =
 * tiles dealt round-robin to CTAs, 1 = contiguous chunks, 2 = no persistent
 * grid: one CTA per tile, left to the hardware block scheduler
 * (blocks_per_sm is then not used). Results do not depend on it. */
lb_status lb_batch_set_schedule(lb_batch_handle h, int tile_nodes, int blocks_per_sm, int order);
/* Measures every schedule for trial_steps steps on a snapshot of the state
 * (restored afterwards, so the simulation is unchanged), keeps the fastest;
 * chosen[3] (may be NULL) receives it, *best_ms_per_step its step time. */
lb_status lb_batch_autotune(lb_batch_handle h, int trial_steps, int chosen[3], double *best_ms_per_step);
lb_status lb_batch_info(lb_batch_handle h, long long *total_nodes, long long *step, int schedule[3]);
/* Kernel timing of the batched fluid kernel (steps run without the graph
 * while on), as lb_set_timing / lb_kernel_time. */
lb_status lb_batch_set_timing(lb_batch_handle h, int on);
lb_status lb_batch_kernel_time(lb_batch_handle h, double *total_ms, long long *launches);
/* Checkpoint and resume of a whole batch, as lb_checkpoint_* for one lattice:
 * every instance's populations, the bodies, the last per-bead forces, both
 * spread-force pools with their tile flags and lists, and the step count, in
 * a caller-owned host buffer of lb_batch_checkpoint_size bytes (save
 * synchronises). A batch built with the same instances (sizes, pores, seeds,
 * instance numbers, in the same order) and the same bodies and beads loads it
 * and resumes the run: the same steps give the same results up to the
 * summation order of the bead-force atomics. Not saved: the trajectory
 * recorder and the schedule (neither changes results). Errors: LB_ERR_ARG
 * (null or short buffer, not a batch checkpoint), LB_ERR_STATE (taken from a
 * batch with other instances or bodies), LB_ERR_CUDA. */
lb_status lb_batch_checkpoint_size(lb_batch_handle h, size_t *bytes);
lb_status lb_batch_checkpoint_save(lb_batch_handle h, void *host, size_t bytes);
lb_status lb_batch_checkpoint_load(lb_batch_handle h, const void *host, size_t bytes);
const char *lb_batch_last_error(lb_batch_handle h);

/* Allocation-free mass and momentum reduction. The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc, either
 * because another allocator (for example a caching allocator) already holds
 * the device's free memory, or because they must not let an allocation
 * synchronise the device while a simulation runs. It allocates nothing: its
 * per-block partial sums live in a static device array of
 * LB_NOALLOC_MAX_BLOCKS * 4 doubles (256 KiB), which every GPU that loads the
 * library keeps until the process exits.
 *
 * d_populations: DEVICE pointer to a population array laid out like the
 * library's own, [19][nx*ny*nz], doubles (precision 64) or deviations
 * f_i - w_i rho0 as floats (precision 32), in the in-place streaming layout
 * after an even (odd_parity = 0) or odd (odd_parity = 1) number of steps.
 * pore_radius > 0 excludes the wall nodes of a pore along pore_axis, as
 * lb_set_pore defines them. d_out: DEVICE pointer to 4 doubles receiving
 * {sum f, sum c_x f, sum c_y f, sum c_z f} over the fluid nodes. Work is
 * queued on cuda_stream (NULL = legacy default stream) without waiting.
 * err (may be NULL) receives a message of at most err_len bytes on failure.
 * Lattices of more than LB_NOALLOC_MAX_NODES nodes are rejected with
 * LB_ERR_ARG. Lattices with moving channel walls (lb_set_channel_walls) are
 * not supported: at odd parity their wall rows hold the wall's momentum
 * terms, which this reduction does not add back. All calls share the one
 * scratch array, so calls that overlap on the GPU race and give wrong sums.
 * Each call made outside stream capture looks up the array's device address
 * with the current device (so a reset of the device's primary context is
 * harmless); a call made while cuda_stream is being captured uses the
 * address found by the device's last call outside capture, so make one call
 * on each device before capturing (LB_ERR_STATE otherwise). */
#define LB_NOALLOC_NODES_PER_BLOCK 4096
#define LB_NOALLOC_MAX_BLOCKS 8192
#define LB_NOALLOC_MAX_NODES (LB_NOALLOC_NODES_PER_BLOCK * LB_NOALLOC_MAX_BLOCKS)
lb_status lb_moments_noalloc(const void *d_populations, int precision, int nx, int ny, int nz,
                             int odd_parity, double rho0, double pore_radius, int pore_axis,
                             double *d_out, void *cuda_stream, char *err, size_t err_len);

/* ---------------------------------------------------------------------
 * Trajectories and their mean squared displacements (Sec. 2.4-2.7: the
 * transport of a raspberry is measured from its centre and orientation
 * recorded at a fixed interval).
 *
 * lb_record_bodies: from the next step on, every `every` steps (the step
 * count after a step is a multiple of `every`) the step prologue writes the
 * centre X (unwrapped, lattice units) and orientation q (w, x, y, z) of
 * every body into a device ring of `capacity` records, without host
 * synchronisation. every = 0 turns recording off and frees the ring;
 * calling it again restarts the ring. LB_ERR_ARG for every < 0,
 * capacity < 1 when every > 0, or no bodies; LB_ERR_OOM if the ring
 * ([capacity][nbodies][7] doubles) does not fit. */
lb_status lb_record_bodies(lb_handle h, int every, int capacity);
/* The records of one body still in the ring, oldest first (at most
 * max_records, the most recent ones): steps[k] (step count of record k),
 * X[3k..3k+2], q[4k..4k+3]; any of the three may be NULL. *count receives
 * the number written. */
lb_status lb_get_trajectory(lb_handle h, int body_id, int max_records, long long *steps, double *X, double *q,
                            int *count);
/* The same for the batched handle (all instances share the step count). */
lb_status lb_batch_record_bodies(lb_batch_handle h, int every, int capacity);
lb_status lb_batch_get_trajectory(lb_batch_handle h, int inst, int body_id, int max_records, long long *steps,
                                  double *X, double *q, int *count);

/* Mean squared displacements of nbodies trajectories on the GPU.
 * X: host [nbodies][nrec][3] centres (unwrapped), q: host [nbodies][nrec][4]
 * unit quaternions (w, x, y, z; lab = R(q) body), records equally spaced.
 * For every body b and lag l = 1..max_lag records, averaged over the
 * nrec - l time origins, out[(b*max_lag + l-1)*LB_MSD_COLS + c] holds
 *   c = 0-2  squared lab-frame displacement per lab axis, Eq. (dt_lab);
 *   c = 3-5  squared displacement of the body-frame trajectory per body axis:
 *            increments R(q_{n-1})^T (X_n - X_{n-1}) summed over the records,
 *            Eqs. (labdisp), (quat), (bodyframedisplacement),
 *            (bodyframetrajectory), (dt_body);
 *   c = 6    squared angle between p(t) and p(t+l), p = R(q) p_ref (p_ref a
 *            body-frame reference vector), Eq. (delta_theta);
 *   c = 7-9  squared change of the summed body-frame angular displacements
 *            about body axis x, y, z (projection method of the SI section
 *            "Body-frame angular displacement"; Eqs.
 *            (bodyframerotdisplacement), (bodyframerottrajectory)).
 * Divide by the paper's denominators for diffusivities (Eq. (dt_lab): sum of
 * c = 0-2 over 6 tau; Eq. (dt_body): 2 tau per axis; Eq. (dr_lab): 6 tau;
 * Eq. (dr_body): 3 tau). The stream may be NULL. Errors: LB_ERR_ARG
 * (null pointers, nrec < 2, max_lag outside [1, nrec), nbodies outside
 * [1, 65535], p_ref zero), LB_ERR_OOM, LB_ERR_CUDA; the message goes to
 * err (err_len bytes, may be NULL). Allocates and frees its own device
 * memory (inputs, a work array of 9 doubles per record, the output). */
#define LB_MSD_COLS 10
lb_status lb_msd_trajectory(const double *X, const double *q, int nrec, int nbodies, int max_lag,
                            const double p_ref[3], double *out, void *cuda_stream, char *err, size_t err_len);

/* Pore-frame mean squared displacements of one trajectory on the GPU
 * (Sec. 2.8 and the SI "Pore-frame coordinate determination"). X: host
 * [nrec][3] centres at a fixed interval in a box nx*ny*nz with a pore of
 * radius R_pore along `axis` through the box centre. Centres relative to the
 * axis give x^c, y^c (across it, in the order x, y, z of the remaining two
 * axes) and theta = atan2(y^c, x^c); each interval's displacement is rotated
 * by P(theta) = [[cos, sin, 0], [-sin, cos, 0], [0, 0, 1]] at the start of
 * the interval (x^p radial, y^p azimuthal, z^p axial) and summed, Eq.
 * (poreframedisplacement). Every record t with radial coordinate r(t) <
 * R_pore falls in bin floor(r(t) / R_pore * nbins) and its sub-trajectory
 * adds (X^p(t + l) - X^p(t))^2 to that bin, Eq. (poreframetrajectory):
 * out[(b*max_lag + l-1)*3 + c] is the mean over the counts[b*max_lag + l-1]
 * origins of bin b (0 where there are none). Readings: theta at the start
 * of the interval; the matrix's x_1 = y_1 = 1. Errors as lb_msd_trajectory
 * (nbins 1-4096); allocates its own device memory. */
lb_status lb_pore_msd(const double *X, int nrec, int nx, int ny, int nz, int axis, double R_pore, int nbins,
                      int max_lag, double *out, long long *counts, void *cuda_stream, char *err, size_t err_len);

/* Raspberry shell construction (Sec. 2.1 and the SI section "Details for
 * ellipsoidal raspberry construction"): beads on an ellipsoid
 * x^2/a^2 + y^2/b^2 + z^2/c^2 = 1 (body frame, centred at the origin) spread
 * evenly by an MD-style relaxation. Each bead is pulled to its nearest surface
 * point r_s by U = k |r - r_s|^2 (Eq. (harmonic_sphere) generalised); r_s =
 * (x a^2/(t + a^2), y b^2/(t + b^2), z c^2/(t + c^2)) (Eq. (xtoxs)) with t the
 * root of F(t) = sum (x a/(t + a^2))^2 - 1 (Eq. (bisection), read without the
 * printed "+1", which contradicts Eq. (xtoxs)) found by bisection on
 * [-m^2 + m |x_m|, a_max |r|] (m the smallest semi-axis, x_m the coordinate
 * along it): 64 halvings in FP64, 40 in FP32. Beads of one shell repel
 * pairwise with WCA (sigma, epsilon, cut at 2^(1/6) sigma). Damped leapfrog,
 * unit mass, zero initial velocity: v <- (1 - eta dt) v + dt F, r <- r + dt v.
 * After `steps` steps each bead is optionally replaced by its nearest surface
 * point. Paper values: eta = 1000, sigma = 1.4, epsilon = 0.1, dt = 0.001,
 * about 1e7 steps; k is not given (1000 is a reasonable choice). */
typedef struct {
    double k_surface;        /* harmonic restraint constant k (> 0)                  */
    double sigma, epsilon;   /* WCA size and energy between beads of a shell (> 0)   */
    double dt, eta;          /* time step (> 0) and damping (eta dt in [0, 2])       */
    long long steps;         /* relaxation steps (>= 0)                              */
    int precision;           /* 64: FP64 arithmetic; 32: FP32 arithmetic (positions
                                are returned as doubles either way)                  */
    int project_final;       /* 1: end with every bead on its nearest surface point  */
    int pair_search;         /* 0: automatic (cell list when it fits in shared memory
                                and a shell has 1024 beads or more, or 256 or more with
                                at most two shells per SM); 1: all pairs; 2: cell list
                                (cells at least as wide as the WCA range, rebuilt every
                                step; a step with a bead outside the box 1.25 a + 1
                                around the centre tests all pairs). The results agree
                                to summation order.                                   */
} lb_shell_params;

/* Relax nshells independent shells in one launch (one thread block per
 * shell). axes: host [nshells][3] semi-axes (a, b, c > 0); counts: host
 * [nshells] beads per shell (1 to LB_SHELL_MAX_BEADS each); xyz: host
 * [sum counts][3], shell after shell: the initial positions on entry, the
 * relaxed positions on return (the caller draws the initial positions, e.g.
 * seeded random points near the surface). The stream may be NULL. Errors:
 * LB_ERR_ARG (null pointers, nshells outside [1, 65535], counts, axes or
 * parameters out of range), LB_ERR_OOM, LB_ERR_CUDA, LB_ERR_UNSTABLE (a
 * non-finite position: the step is too large for the stiffness); on error
 * xyz is left unchanged. The message goes to err (err_len bytes, may be
 * NULL). Allocates and frees its own device memory and synchronises the
 * stream. Cost per step and shell: O(n) with the cell list, O(n^2) when
 * testing all pairs, n = beads of the shell. */
#define LB_SHELL_MAX_BEADS 4096
lb_status lb_relax_shells(int nshells, const double *axes, const int *counts, double *xyz,
                          const lb_shell_params *params, void *cuda_stream, char *err, size_t err_len);

/* Host-only: the velocity set c[19*3], weights w[19] and opposite-link table
 * opp[19] the library uses. Needs no GPU. Returns 19. */
int lb_lattice(int *c, double *w, int *opp);

#ifdef __cplusplus
}
#endif

#endif /* LB_H */
