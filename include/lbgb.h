/*
 * lbgb.h -- C ABI of the GB300 (sm_103a) colloidal two-component Shan-Chen
 * lattice-Boltzmann library (method of Bonaccorso et al., "LBsoft: a parallel
 * open-source software for simulation of colloidal systems",
 * arXiv:2004.04080).
 *
 * One library context owns one D3Q19 lattice of nx*ny*nz sites on one GPU,
 * with two fluid components and up to max_colloids rigid spheres.  Each call
 * of lb_step advances the whole coupled system by the paper's time step
 * (Sec. 3.1, particle sequence): moments (Eqs. 6, 7, 14), fluid-node
 * destruction and creation under moving particles (Eqs. 24, 25), particle
 * pair forces (Eqs. 26, 27), wetting virtual densities and Shan-Chen forces
 * (Eqs. 11, 20, 21), collision with the exact-difference source (Eqs. 13-16),
 * halfway bounce-back on particles and walls with the link forces
 * (Eqs. 8, 9, 17-19, 22, 23), Svanberg rotational leap-frog (Eqs. 28-35) and
 * streaming (Eq. 3).
 *
 * Conventions shared by every entry point:
 *  - Site index s = x + nx*(y + ny*z); fields are flat arrays of length
 *    N = nx*ny*nz; vector fields are structure-of-arrays [3][N].
 *  - Particle arrays are [n][3] (quaternions [n][4] as q0,q1,q2,q3, scalar
 *    first), double precision, in lattice units.
 *  - Host pointers are owned by the caller; the library copies from or into
 *    them before the call returns (synchronously on the context stream).
 *  - Device memory: the library allocates nothing.  The caller allocates one
 *    device workspace of lb_workspace_bytes() bytes (256-byte aligned) and
 *    keeps it alive until lb_destroy; all kernels run on the CUDA stream
 *    given to lb_create (NULL = legacy default stream).
 *  - Errors: every call returns LB_OK (0) or a negative LB_ERR_* code; no
 *    exception crosses the ABI.  lb_last_error() gives a text for the last
 *    failure of a context.  Device-detected conditions (non-finite or
 *    negative density, overlapping particles) are read back once at the end
 *    of lb_step.
 */
#ifndef LBGB_H
#define LBGB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx; /* opaque; created by lb_create */

enum {
    LB_OK = 0,
    LB_ERR_ARG = -1,       /* invalid argument                               */
    LB_ERR_STATE = -2,     /* call out of order or capacity exceeded         */
    LB_ERR_CUDA = -3,      /* a CUDA runtime call failed                      */
    LB_ERR_NOMEM = -4,     /* workspace too small                             */
    LB_ERR_NONFINITE = -5, /* a density became non-finite or negative         */
    LB_ERR_OVERLAP = -6,   /* two particles claimed the same lattice node     */
    LB_ERR_TIMEOUT = -7    /* reserved: no call returns it (no kernel spin-waits) */
};

/* Storage precision of the populations.  LB_FP64 and LB_FP32 compute in the
 * storage type; LB_FP16 stores each population as the half-precision
 * deviation f_i - w_i rho0^k and computes in FP32.  Particle state, particle
 * force/torque sums and the global reductions are FP64 in every mode. */
enum { LB_FP64 = 0, LB_FP32 = 1, LB_FP16 = 2 };

/* Flag or-ed into the prec argument of lb_workspace_bytes and lb_create: a
 * lattice of one fluid component (the single-component benchmark of
 * Sec. 5.1, App. D test 1).  It holds the populations of component A only
 * (19 per site), has no Shan-Chen force (G, zeta ignored), no particles
 * (max_colloids must be 0; lb_add_colloids returns LB_ERR_ARG), walls and
 * velocity faces on z (open types 0 and 2), and no adjoint (LB_ERR_STATE).
 * lb_init_fields ignores rhoB (which may be NULL); lb_get_fields returns
 * rhoB = 0; lb_get_populations accepts k = 0 only; lb_get_owner returns -1
 * everywhere.  The step is Eqs. 5-7 and 16 with one component (the body force
 * of Eq. 15 as F = rho g) and push streaming with the wall rule of Eq. 9. */
enum { LB_ONE_COMPONENT = 0x100 };

/* Physical parameters (paper App. A "LB" and "MD" rooms; lattice units). */
typedef struct {
    double tau[2];          /* BGK relaxation time per component (Eq. 4), > 1/2   */
    double G;               /* Shan-Chen coupling G_C (Eq. 11); repulsive for G>0 */
    double zeta[2];         /* wetting constant per component (Eq. 20)            */
    double rho0[2];         /* reference density: FP16 deviation shift, and the  */
                            /* refill density of a node with no fluid neighbour  */
    int bc[3];              /* 1 periodic, 0 wall; walls only along z (bc[2])    */
    double wall_u_lo[3];    /* velocity of the wall at z = -1/2 (Eq. 9)          */
    double wall_u_hi[3];    /* velocity of the wall at z = nz - 1/2              */
    double body_force[3];   /* force per unit mass on the fluid ("force ext")    */
    double hertz_K;         /* Hertz constant K (Eq. 26); 0 disables              */
    double hertz_sigma;     /* contact distance: force acts for r < sigma         */
    double hertz_rcap;      /* r is floored at rcap in the force magnitude       */
    int lub_on;             /* lubrication (Eq. 27) on/off                        */
    double lub_hn, lub_hmin, lub_scale; /* cut-off gap, gap floor, prefactor    */
    double side_wall_k;     /* soft harmonic particle-wall spring; 0 disables    */
    double side_wall_d;     /* it pushes when a centre is closer than d to a wall */
    int rotate;             /* integrate angular velocity and orientation        */
    /* Janus wettability (Sec. 5.1 colloid benchmarks; App. A wettability
     * angle): with janus != 0 a particle node whose direction from the
     * centre makes the polar angle theta with the particle's first body axis
     * x* (first column of R(q), Eq. 31) uses the wetting constants
     * s zeta[0] and -s zeta[1] in Eq. 20, where s goes from -1 to 1 across
     * [janus_theta0 - janus_width/2, janus_theta0 + janus_width/2] along the
     * cubic smoothstep (a step at janus_theta0 for width 0).  Degrees;
     * janus_width >= 0. */
    int janus;
    double janus_theta0, janus_width;
    /* Particle pair list (App. A, the MD room's rcut and delr directives):
     * pairs are listed within max(rcut, the interaction range) + delr, where
     * the interaction range is hertz_sigma and, with lubrication, 2 R_max +
     * lub_hn; the list is rebuilt only when a particle has moved more than
     * delr / 2 since the last build (delr = 0: every step).  The forces are
     * evaluated with their own cut-offs on the listed pairs, so rcut and
     * delr change the cost, never the result.  Both >= 0. */
    double rcut, delr;
    /* Open z faces (Sec. 2.2; App. A open-boundary directives), with bc[2]
     * = 0.  open[0] (z = -1/2) and open[1] (z = nz - 1/2): 0 a wall moving
     * at wall_u (Eq. 9); 1 pressure: anti-bounce-back of Eq. 10 with the
     * face density open_rho[face][k] and u_w the velocity of the boundary
     * node (Eq. 14); 2 velocity: Eq. 9 with u_w = wall_u and the density of
     * the boundary node (the wall rule); 3 equilibrium: the incoming
     * populations are f^eq(open_rho[face][k], wall_u).  A pressure or
     * equilibrium face carries open_rho into the Shan-Chen force of Eq. 11.
     * open_extrap = 1 takes u_w of a pressure face and rho_w of a velocity
     * face at the face itself, extrapolated to first order from the
     * boundary node b and the next interior node b + 1 along z (Sec. 2.2):
     * q_w = q_b + (q_b - q_{b+1}) / 2, with q_b alone where b + 1 is a
     * particle node or nz < 2; 0 (the default) takes q_b.  Walls and
     * equilibrium faces ignore it.  The adjoint accepts walls and velocity
     * faces without extrapolation only. */
    int open[2];
    double open_rho[2][2];
    int open_extrap;
} lb_params;

/* Device workspace size for a lattice; *bytes receives the size.  prec may
 * carry LB_ONE_COMPONENT.  Returns LB_ERR_ARG for a non-positive size, an
 * unknown precision, or particles on a one-component lattice. */
int lb_workspace_bytes(int nx, int ny, int nz, int prec, int max_colloids, size_t *bytes);

/* Create a context on the calling thread's current CUDA device.
 * d_workspace: device pointer, 256-byte aligned, >= lb_workspace_bytes bytes,
 * owned by the caller.  cuda_stream: a cudaStream_t or NULL.
 * Lattice sides must be >= 4; nx must be a multiple of 4; nx*ny*nz below
 * 2^31 - 4096 (LB_ERR_ARG otherwise: sites are indexed in 32 bits). */
int lb_create(int nx, int ny, int nz, int prec, int max_colloids, void *d_workspace,
              size_t bytes, void *cuda_stream, lb_ctx **out);

/* Set the parameters (copied).  Must precede lb_init_fields. */
int lb_set_params(lb_ctx *ctx, const lb_params *p);

/* Initialise populations to f^eq(rho^k, u) (Eq. 5) on every site.
 * rhoA, rhoB: [N] host arrays; u: [3][N] host array or NULL for rest.
 * Removes any particles (their node map is cleared). */
int lb_init_fields(lb_ctx *ctx, const double *rhoA, const double *rhoB, const double *u);

/* Append n particles (total <= max_colloids) and map their solid nodes
 * (Sec. 2.4: node solid iff |x - r_p|^2 < R_p^2, minimum image); fluid on the
 * newly solid nodes is removed without momentum bookkeeping.
 * pos, radius, mass required; vel = v(-1/2), omega, quat may be NULL (zero,
 * zero, identity).  A mass of +inf makes a particle immobile.
 * Positions are wrapped into the box along periodic axes; along a wall axis
 * they must lie in [0, n-1].  2R+5 must be smaller than each periodic side. */
int lb_add_colloids(lb_ctx *ctx, int n, const double *pos, const double *vel,
                    const double *omega, const double *quat, const double *radius,
                    const double *mass);

/* Advance nsteps time steps.  Returns LB_ERR_NONFINITE / LB_ERR_OVERLAP if the
 * device flagged the condition during these steps (state then undefined). */
int lb_step(lb_ctx *ctx, int nsteps);

/* Densities rho^k and the half-force-corrected mixture velocity
 * u = sum_k (j^k + F^k/2) / rho (Sec. 2.3) of the current state, with the
 * forces evaluated on the current node map.  Solid nodes read zero.
 * Any output pointer may be NULL. */
int lb_get_fields(lb_ctx *ctx, double *rhoA, double *rhoB, double *u);

/* Particle state: position r(t), velocity v(t-1/2), angular velocity
 * omega(t-1/2), orientation q(t), and the total force / torque of Eq. 35 used
 * by the last step.  Any pointer may be NULL.  Returns the particle count. */
int lb_get_colloids(lb_ctx *ctx, double *pos, double *vel, double *omega, double *quat,
                    double *force, double *torque);

/* One per-particle force term of the last step, [n][3]:
 * 0 F_liq(t+1/2) (Eq. 22), 1 T_liq (Eq. 23), 2 F_d, 3 T_d (Eq. 24),
 * 4 F_c, 5 T_c (Eq. 25), 6 F_s, 7 T_s (Eq. 21 summed over the frontier),
 * 8 pair + side-wall force (Eqs. 26-27), 9 total force, 10 total torque. */
int lb_get_colloid_terms(lb_ctx *ctx, int which, double *out);

/* Global FP64 sums over fluid nodes: out[0..1] mass of A and B,
 * out[2..4] sum_k j^k, out[5..7] sum_k (j^k + F^k/2). */
int lb_get_totals(lb_ctx *ctx, double *out);

/* Raw populations of component k as FP64, [19][N] (for tests). */
int lb_get_populations(lb_ctx *ctx, int k, double *out);

/* Node map: -1 fluid, else the index of the owning particle, [N]. */
int lb_get_owner(lb_ctx *ctx, int *out);

/* Kernel timing.  While enabled, lb_step records a CUDA event pair on the
 * context stream around every launch of the fused lattice kernel (the
 * collide + Shan-Chen + stream + bounce-back kernel, the dominant one, with
 * the small wall kernel that follows it in the lean form; LB_KERNEL_FUSED)
 * and around the full density pass that precedes it when particles are
 * present (LB_KERNEL_DENSITY; see lb_fused_kernel).
 * lb_profile(ctx, 1) enables and clears the records, lb_profile(ctx, 0)
 * disables them; lb_profile_read_kernel waits for the recorded events of one
 * kernel kind (LB_ERR_ARG for another value) and returns its summed time
 * (ms) and the number of timed launches (at most 16384 are kept per record);
 * lb_profile_read is the fused-kernel record. */
enum { LB_KERNEL_FUSED = 0, LB_KERNEL_DENSITY = 1, LB_KERNEL_KINDS = 2 };

/* Rounding of the FP16 deviation storage (the precision forms; the paper
 * stores FP64).  LB_ROUND_STOCHASTIC (the default of an LB_FP16 context)
 * rounds every population stored by the time step up or down with
 * probability given by the value's position between the two neighbouring half
 * values (the hardware's stochastic-rounding conversion, with bits from a
 * counter-based hash of site, step and `seed`), so that the expected stored
 * value is the FP32 one: a population that stays the same from step to step
 * is then not rounded the same way every step (rounding to nearest makes the
 * error of such a population a bias that grows with the number of steps).
 * LB_ROUND_NEAREST stores half(f_i - w_i rho0^k) rounded to nearest.  The
 * sequence of bits is fixed by `seed` and the number of steps since this call
 * or since lb_init_fields (the default seed is a fixed constant).  No effect
 * on LB_FP32 / LB_FP64 contexts.  The adjoint functions return LB_ERR_STATE
 * while stochastic rounding is on (their forward recomputation would not
 * reproduce the recorded steps): an FP16 adjoint needs LB_ROUND_NEAREST.
 * LB_ERR_ARG for another mode. */
enum { LB_ROUND_NEAREST = 0, LB_ROUND_STOCHASTIC = 1 };
int lb_set_rounding(lb_ctx *ctx, int mode, unsigned long long seed);
int lb_profile(lb_ctx *ctx, int enable);
int lb_profile_read(lb_ctx *ctx, double *total_ms, long long *launches);
int lb_profile_read_kernel(lb_ctx *ctx, int kernel, double *total_ms, long long *launches);

/* ---- Reverse mode (adjoint) of the time step, for immobile particles ----
 * With every particle immobile (added with infinite mass and zero velocity and
 * angular velocity) the node map is static and one time step is a smooth map
 * f(t) -> f(t+1) of the populations (Sec. 2.3, Eqs. 5-7, 11, 13-16; bounce-back
 * Eqs. 8, 9, 17; link forces Eqs. 19, 22) with parameters tau_A, tau_B, G,
 * zeta_A, zeta_B.  lb_adjoint_step maps dJ/df(t+1) to dJ/df(t) and adds the
 * step's parameter gradients; the caller keeps the states f(t) (checkpoints
 * plus recomputation) and chains the steps backwards.  The adjoint functions
 * return LB_ERR_STATE when a particle is mobile.
 *
 * A population state is 2 x 19 x (padded plane) values of the storage type
 * (lb_state_bytes); lb_get_state / lb_set_state copy the current populations
 * to / from such a caller device buffer (device to device, synchronous).
 * An adjoint field holds lambda_i(x) = L_i(x) + R(x) in the compute type
 * (FP64 for LB_FP64, FP32 otherwise): 2 x 19 planes L then 2 planes R
 * (lb_adjoint_bytes: *field_bytes); adjoint calls also need one scratch
 * buffer of *scratch_bytes.  All buffers are caller-owned device memory. */
int lb_state_bytes(const lb_ctx *ctx, size_t *bytes);
int lb_get_state(lb_ctx *ctx, void *d_dst);
int lb_set_state(lb_ctx *ctx, const void *d_src);
int lb_adjoint_bytes(const lb_ctx *ctx, size_t *field_bytes, size_t *scratch_bytes);

/* Seed for the interface measure A = sum_x (1 - phi^2), phi =
 * (rho_A - rho_B)/(rho_A + rho_B) over fluid nodes of the current state:
 * writes weight * dA/df into d_adj and A into *value (host). */
int lb_adjoint_seed(lb_ctx *ctx, double weight, void *d_adj, void *d_scratch, double *value);

/* One step backwards.  d_state: the populations f(t) at the start of the step
 * being reversed; d_adj_in: dJ/df(t+1); d_adj_out (distinct): receives
 * dJ/df(t).  dJdF: host [n][3] array dJ/dF_liq,p of this step's link forces
 * (Eq. 22), or NULL.  grads: host array of 5 to which dJ/d(tau_A, tau_B, G,
 * zeta_A, zeta_B) of this step are added.  Synchronous. */
int lb_adjoint_step(lb_ctx *ctx, const void *d_state, const void *d_adj_in, void *d_adj_out, void *d_scratch,
                    const double *dJdF, double *grads);

/* As lb_adjoint_step, without a host round trip: d_dJdF is a device array
 * [n][3] (or NULL) and the call is asynchronous on the context stream.  The
 * parameter gradients accumulate on the device (in d_scratch; lb_adjoint_seed
 * clears them) until a call with grads != NULL adds the accumulated sums to
 * grads (host, 5) and clears them; that call waits for the stream. */
int lb_adjoint_step_async(lb_ctx *ctx, const void *d_state, const void *d_adj_in, void *d_adj_out,
                          void *d_scratch, const double *d_dJdF, double *grads);

/* dJ/dF_liq for J = weight * sum_p sqrt(|F_p|^2 + eps^2) (the per-step term
 * of a mean drag magnitude): d_dJdF[p] = weight F_p / sqrt(|F_p|^2 + eps^2),
 * d_F and d_dJdF device arrays [n][3] of the current particles; eps >= 0.
 * Asynchronous on the context stream. */
int lb_drag_gradient(lb_ctx *ctx, const double *d_F, double weight, double eps, double *d_dJdF);

/* Record during the next nsteps time steps of lb_step: the populations f(t)
 * at the start of each step into d_states (consecutive blocks of
 * lb_state_bytes) and the link forces F_liq (Eq. 22) after each step into
 * d_forces ([nsteps][n][3] doubles); either may be NULL.  Device-to-device
 * copies on the context stream, so a checkpointed reverse sweep needs no host
 * round trip per step.  nsteps <= 0 stops a recording. */
int lb_record(lb_ctx *ctx, void *d_states, double *d_forces, int nsteps);

/* dJ/drho^k(0) for initial populations f = f^eq(rho^k, 0) (Eq. 5):
 * d_grad (device, [2][N] doubles) = sum_i w_i lambda_i(0); zero on particle
 * nodes (their initial fluid is removed by the first map). */
int lb_adjoint_initial(lb_ctx *ctx, const void *d_adj, double *d_grad);

/* Global FP64 sums of a population array that the caller holds on the
 * device, computed without allocating any device memory and without a
 * context.  The paper has no counterpart: this is a convenience for callers
 * that cannot allocate at the point of the call (for example a monitor running
 * between the time steps of an application whose device memory belongs to its
 * own pool, where a cudaMalloc would synchronise the device and bypass the
 * pool) and that hold no workspace.
 *   d_pops: populations [2][19][plane_stride] in the storage type of prec
 *           (LB_FP16: half deviations f - w_i rho0^k), site s = x + nx(y + ny z);
 *   d_mask: N bytes, nonzero = particle node (skipped), or NULL;
 *   rho0:   host array of 2 reference densities (needed for LB_FP16 only);
 *   d_out:  device array of 5 doubles: mass of A and B, sum_k j^k (x, y, z).
 * The scratch is a static device array of per-plane partials (320 KiB on each
 * device that loads the library, kept until exit): nz must be <= 4096,
 * otherwise LB_ERR_ARG.  The first call in each CUDA context looks up that
 * array's address and should come before any stream capture; a device reset
 * replaces the context, and the next call then looks it up again.  Calls share
 * the array,
 * so calls that overlap on the GPU race; calls ordered on one stream do not.
 * Runs asynchronously on cuda_stream; returns LB_ERR_ARG / LB_ERR_CUDA on bad
 * arguments or a failed launch. */
int lb_totals_static(const void *d_pops, int prec, int nx, int ny, int nz, long long plane_stride,
                     const unsigned char *d_mask, const double *rho0, double *d_out, void *cuda_stream);

/* Number of kernel launches issued by this context since creation. */
long long lb_launch_count(const lb_ctx *ctx);

/* Number of particle pair-list builds so far (see lb_params.rcut / delr);
 * synchronises the context's stream.  -1 for a null context. */
long long lb_pair_list_builds(lb_ctx *ctx);

/* Which fused lattice kernel lb_step launches in the context's present state
 * (the sequence of Sec. 3.1 is the same for all; they differ in how the
 * moments and the Shan-Chen halo densities of Eq. 11 reach the collision):
 *  LB_FUSED_MOMENTUM  tau_A = tau_B = 1, with or without particles: a
 *      density pass writes rho^k and j^k of every node (Eqs. 6-7), the
 *      class of every link (fluid-fluid, fluid-particle) is kept with the
 *      node map; the lean lattice kernel collides every node from the
 *      moments (Eq. 16 at omega = 1), staging the halo of rho^k in shared
 *      memory with asynchronous copies, pushes the links and bounces those
 *      into particle nodes (Eqs. 17-19, 22, 23); a small kernel then applies
 *      the rules of the z faces (Eqs. 9, 10);
 *  LB_FUSED_TWO_PASS  particles, other tau: a density pass writes rho^k, the
 *      fused kernel re-reads the populations;
 *  LB_FUSED_PLAIN     no particles, other tau: one pass, halo densities
 *      formed from the neighbours' populations;
 *  LB_FUSED_SINGLE    a one-component lattice (LB_ONE_COMPONENT): one pass,
 *      one thread per site.
 * Returns the code, or LB_ERR_ARG for a NULL context. */
enum { LB_FUSED_MOMENTUM = 1, LB_FUSED_TWO_PASS = 2, LB_FUSED_PLAIN = 3, LB_FUSED_SINGLE = 4 };
int lb_fused_kernel(const lb_ctx *ctx);


/* Release the context (not the caller's workspace). */
int lb_destroy(lb_ctx *ctx);

/* Text of the last error of ctx ("" if none); valid until the next call. */
const char *lb_last_error(const lb_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBGB_H */
