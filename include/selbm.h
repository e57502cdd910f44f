/*
 * selbm.h - C ABI of the GB300 filtered spectral-element lattice Boltzmann
 * library (method of Zhao, Patel, Lin, Min, Lee, "A flux bounce-back scheme for
 * the filtered Spectral Element Lattice Boltzmann Method", arXiv 2509.19171).
 *
 * One handle = one simulation on one GPU.  Every entry point returns an int
 * status (SELBM_OK = 0, negative = error; selbm_last_error() gives the text)
 * unless stated otherwise.  The synchronising calls selbm_sync and
 * selbm_diagnostics return the positive SELBM_OK_FALLBACK instead of SELBM_OK
 * when the learned filter control's drift fallback is engaged.  All work is enqueued on the CUDA stream given to
 * selbm_create(); calls that return data to the host synchronise that stream.
 * Input arrays are copied; the caller keeps ownership of every pointer it
 * passes.  Output buffers are caller-owned and must be large enough.
 *
 * Population order (the index alpha of every state array): velocities sorted
 * by speed class |e|^2 = 0, 1, 2, 3 and, inside a class, by the ternary code
 * (e_x+1) + 3 (e_y+1) + 9 (e_z+1) ascending.  selbm_lattice_table() returns
 * the table.  Node order inside an element: i + (N+1) j + (N+1)^2 k, r index
 * fastest (Sec. 2.2 of the paper).
 */
#ifndef SELBM_H
#define SELBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct selbm selbm_t; /* opaque; owned by the library */

enum {
  SELBM_OK_FALLBACK = 1,    /* OK; the learned control's drift fallback has switched it off and the
                               paper's fixed filter runs for the rest of the run */
  SELBM_OK = 0,
  SELBM_ERR_ARG = -1,       /* bad argument (NULL, size out of range, unsupported option) */
  SELBM_ERR_MESH = -2,      /* non-positive Jacobian, unmatched periodic nodes, bad tags */
  SELBM_ERR_CUDA = -3,      /* a CUDA call failed (text in selbm_last_error) */
  SELBM_ERR_NONFINITE = -4, /* the state holds NaN or Inf */
  SELBM_ERR_TIMEOUT = -5,   /* a bounded device wait gave up */
  SELBM_ERR_STATE = -6      /* call out of order (e.g. step before init) */
};

enum { SELBM_D2Q9 = 0, SELBM_D3Q19 = 1, SELBM_D3Q27 = 2 };

/* Storage / arithmetic form of the hot path. */
enum {
  SELBM_FP64 = 0,   /* state f stored and updated in FP64 */
  SELBM_FP32DEV = 1 /* deviations g = f - t_alpha rho0 stored and updated in FP32;
                       metrics and matrices built in FP64 */
};

/*
 * Conforming quad (dim 2) / hex (dim 3) mesh given by element corners.
 *  verts[e][c][k]   corner c = a + 2b (+4g), a,b,g in {0,1} <-> r,s(,t) = -1/+1
 *  curved[e][f]     1: face f lies on the circle/cylinder x^2 + y^2 = radius^2
 *                   (axis z); the edge(s) of that face in the x-y plane are
 *                   circular arcs with the angle linear in the reference
 *                   coordinate; curved 3D elements are extrusions along z.
 *                   Face ids: 0 r=-1, 1 r=+1, 2 s=-1, 3 s=+1, 4 t=-1, 5 t=+1.
 *                   May be NULL (all flat).
 *  face_bc[e][f]    0: interior or periodic face; k >= 1: wall k (flux
 *                   bounce-back, Sec. 2.2.1) moving with wall_velocity[k-1].
 *                   May be NULL (no walls).
 *  period[k]        periodic length along axis k, 0 if not periodic.
 *  origin[k]        domain origin along axis k (for periodic wrapping).
 * The element map is the Gordon-Hall blend of the (straight or arc) edges in
 * (r, s), linear in t; GLL nodes that coincide (modulo periods) are one node.
 */
typedef struct {
  int32_t dim;
  int32_t nelem;
  const double *verts;
  const int32_t *curved;
  const int32_t *face_bc;
  const double *period;
  const double *origin;
  int32_t nwalls;
  const double *wall_velocity; /* [nwalls][dim] */
  double radius;
} selbm_mesh;

/*
 * General curved, unstructured quad (dim 2) / hex (dim 3) mesh given by the GLL node
 * coordinates of its isoparametric element maps (Sec. 2.2) and its face connectivity.
 *  order            N_g, 1 <= N_g <= 14: the map of element e is the tensor-product Lagrange
 *                   interpolant through xyz at the (N_g+1)^dim GLL nodes (N_g = 1: trilinear);
 *                   the solver's own GLL nodes (order N of selbm_params) are interpolated
 *                   from it, and the metrics are GLL derivatives of the interpolated map.
 *  xyz[e][k][p]     coordinate k of node p = i + (N_g+1) j (+ (N_g+1)^2 l), r index fastest.
 *  face_nbr[e][f]   element across face f (face ids as in selbm_mesh: 0 r=-1, 1 r=+1,
 *                   2 s=-1, 3 s=+1, 4 t=-1, 5 t=+1), or -1 on the domain boundary.  Periodic
 *                   faces name their partner (an element may be its own neighbour).
 *  face_nbr_face[e][f]  the neighbour's face id.
 *  face_orient[e][f]    how the face's nodes meet the neighbour's.  Face coordinates
 *                   (a, b) of face f are its two tangential node indices in increasing axis
 *                   order (faces 0, 1: (j, l); 2, 3: (i, l); 4, 5: (i, j); in 2D the single
 *                   tangential index a).  Node (a, b) of face f of e is node (a', b') of face
 *                   face_nbr_face of the neighbour, where (u, v) = (b, a) if bit 0 of the code
 *                   is set, else (a, b); a' = N - u if bit 1 is set, else u; b' = N - v if bit
 *                   2 is set, else v.  In 2D only bit 1 may be set.
 *  face_bc[e][f]    0: interior, periodic or open face; k >= 1: wall k (flux bounce-back,
 *                   Sec. 2.2.1) moving with wall_velocity[k-1].  May be NULL (no walls).
 * Nodes are identified through the connectivity alone (no coordinate matching); the setup
 * checks that the pairs are mutual and that matched nodes differ by one translation per face
 * (zero inside the domain, a period across periodic faces), else SELBM_ERR_MESH.
 */
typedef struct {
  int32_t dim;
  int32_t nelem;
  int32_t order;
  const double *xyz;
  const int32_t *face_nbr;
  const int8_t *face_nbr_face;
  const int8_t *face_orient;
  const int32_t *face_bc;
  int32_t nwalls;
  const double *wall_velocity; /* [nwalls][dim] */
} selbm_mesh_nodes;

/*
 * Explicit modal filter (Sec. 2.4): sigma_k = 1 for k <= kc, else
 *  shape 0 (paper): 1 - gamma r^2;  shape 1: (1 - gamma)^(r^p);  r = (k-kc)/(N-kc).
 * Applied to every population, element by element, once per step after the
 * last Runge-Kutta stage, in the hierarchical basis 1, xi, L_k - L_{k-2}.
 * gamma = 0 disables it.  kc must satisfy 1 <= kc < N (real values allowed).
 */
typedef struct {
  int32_t shape;
  double gamma;
  double kc;
  double p;
} selbm_filter;

typedef struct {
  int32_t lattice;        /* SELBM_D2Q9 / D3Q19 / D3Q27 (dim must match the mesh) */
  int32_t order;          /* polynomial order N, 2 <= N <= 14 (3D: the element tile must fit in shared memory) */
  double nu;              /* kinematic viscosity; lambda = nu / cs^2, tau = lambda / dt */
  double dt;              /* > 0: time step; <= 0: dt = cfl * smallest GLL node spacing */
  double cfl;
  double rho0;            /* reference density of the wall term and of the FP32 deviations */
  int32_t precision;      /* SELBM_FP64 or SELBM_FP32DEV */
  selbm_filter filter;
  double body_accel[3];   /* g: body force F = rho g (Sec. 3.5), split into F* and F** */
} selbm_params;

/*
 * Build the handle: GLL tables, element map, metrics (all FP64), global node
 * numbering, assembly map, wall tables; allocate device state.  The hot path
 * runs on `cuda_stream` (a cudaStream_t, NULL = legacy default stream).
 * Errors: SELBM_ERR_ARG, SELBM_ERR_MESH, SELBM_ERR_CUDA; *out is NULL then.
 */
int selbm_create(const selbm_mesh *mesh, const selbm_params *params, void *cuda_stream, selbm_t **out);
/* The same for a mesh given by GLL node coordinates and face connectivity (selbm_mesh_nodes). */
int selbm_create_nodes(const selbm_mesh_nodes *mesh, const selbm_params *params, void *cuda_stream, selbm_t **out);
void selbm_destroy(selbm_t *h);
/* Text of the last error on this handle (or of the last failed create when h is NULL). */
const char *selbm_last_error(const selbm_t *h);

/*
 * Sizes and scalars: out_i[0..8] = E, Np, Q, G (unique nodes), dim, N,
 * precision, steps taken, step form (0: whole-element stage kernels, 1:
 * population-split stages after a per-element prologue); out_d[0..3] = dt,
 * tau, lambda, time.
 */
int selbm_info(const selbm_t *h, int64_t out_i[9], double out_d[4]);
/* Lattice table: e[Q][3] (zero-padded in 2D), t[Q], opposite[Q]. */
int selbm_lattice_table(const selbm_t *h, int32_t *e, double *t, int32_t *opp);
/* Physical coordinates of every local node, host buffer [E][Np][dim]. */
int selbm_node_coords(const selbm_t *h, double *xyz);

/*
 * Initial state f_bar = f^eq(rho, u) - dt/2 F** (Sec. 2.1, f at equilibrium).
 * rho [E][Np], u [E][Np][dim]; host pointers, or device pointers when
 * on_device = 1.  Copies of a shared node take the value of its first copy
 * (lowest e, then lowest local index).
 */
int selbm_init(selbm_t *h, const double *rho, const double *u, int on_device);
/* Set / read the full state f_bar, layout [Q][E][Np] FP64 (read: filtered, as after a step). */
int selbm_set_state(selbm_t *h, const double *f, int on_device);
int selbm_get_state(selbm_t *h, double *f, int on_device);

/*
 * Advance nsteps time steps (Sec. 2, summary list): BGK collision with F**,
 * three Shu-Osher SSPRK3 stages of the weak advection with F* and the flux
 * bounce-back wall flux (or the four printed stages, see selbm_set_time_scheme),
 * assembly of shared nodes, explicit filter.  Each step is launched as a captured
 * CUDA graph after one eager step of its kind.
 * Asynchronous: enqueues the work and returns.  Errors: SELBM_ERR_STATE
 * (not initialised), SELBM_ERR_CUDA (launch failure).
 */
int selbm_step(selbm_t *h, int64_t nsteps);

/* Density and velocity rho = sum f_bar, rho u = sum e f_bar (Eqs. pressure, momentum)
 * at every local node: rho [E][Np], u [E][Np][dim]. */
int selbm_moments(selbm_t *h, double *rho, double *u, int on_device);

/*
 * Non-equilibrium second moment at every local node (Sec. 3.3, the stress recovered from the
 * higher moments of the distribution): Pi_ij = tau / (tau + 1/2) sum_a e_ai e_aj (f_bar_a -
 * f_bar_a^eq), f_bar^eq = f^eq - dt/2 F** at the node's (rho, u) and force; the factor turns
 * the non-equilibrium part of f_bar into that of f.  To leading order -Pi is the viscous
 * stress rho nu (d_i u_j + d_j u_i); in planar shear flow -Pi_xx carries the normal stress
 * -2 mu lambda (u')^2.  Read from the filtered state, as selbm_moments.  pi [E][Np][dim][dim],
 * host or device (on_device = 1).  Errors: SELBM_ERR_ARG, SELBM_ERR_STATE, SELBM_ERR_CUDA.
 */
int selbm_stress(selbm_t *h, double *pi, int on_device);

/* Replace the filter (Sec. 2.4); takes effect from the next step. */
int selbm_set_filter(selbm_t *h, const selbm_filter *filter);
/*
 * Time scheme of the streaming step (Sec. 2.2.2).  0 (default): the Shu-Osher three-stage
 * SSPRK3 that the text names.  1: the four stages exactly as printed,
 *   f1 = f0 + dt/3 L f0,  f2 = f1 - 3dt/4 L(f0 - f1),  f3 = f2 + 2dt/3 L(f0 - f1 + f2),
 *   f  = f3 - dt/4 L(f0 - f1 + f2 - f3),
 * f0 the collided state, L applied to each combination as a whole (its force and
 * wall-velocity terms once per application); for a linear L (no force, walls at rest) this is
 * the fourth-order Taylor polynomial of exp(dt L).  Taken literally the four applications
 * weight a source term of L by 1/3 - 3/4 + 2/3 - 1/4 = 0.  2: the printed stages with L's
 * source terms (F*, moving-wall velocity) kept only for the arguments whose weights sum to
 * one (f0 and f0 - f1 + f2) and dropped for the differences (f0 - f1, f0 - f1 + f2 - f3):
 * fourth order in time for an affine L, steady states of L kept exactly.  The first call
 * with 1 or 2 allocates four more state arrays (4 Q G reals), freed by selbm_destroy.  Takes
 * effect from the next step.  Errors: SELBM_ERR_ARG (h NULL, scheme not 0, 1 or 2),
 * SELBM_ERR_CUDA (allocation failure).
 */
int selbm_set_time_scheme(selbm_t *h, int scheme);
/* Replace the body acceleration g (F = rho g). */
int selbm_set_body_force(selbm_t *h, const double g[3]);
/*
 * Per-node body acceleration field on top of g (Sec. 4, pipe flow: the divergence-free
 * perturbation force F' of the first three eddy turnover times, applied through the same
 * force split as the body force).  The acceleration at unique node x_g becomes
 * g + A(t) S_g, with A(t) = sin(2 pi t / period) while t < t_end and 0 afterwards
 * (period <= 0: A = 1 while t < t_end).  t is the time at the start of a step (the clock
 * of selbm_info, reset by selbm_init) and the force is frozen through the step.
 * S: host buffer [E][Np][dim] FP64 in acceleration units, copied; copies of a shared node
 * take the value of their first copy (lowest e, then lowest local index).  S = NULL
 * removes the field.  Takes effect from the next step and in selbm_init.  The first call
 * allocates 3 G reals of device memory, freed by selbm_destroy.  Errors: SELBM_ERR_ARG
 * (h NULL, period or t_end NaN), SELBM_ERR_CUDA (allocation or copy failure).
 */
int selbm_set_force_field(selbm_t *h, const double *S, double period, double t_end);

/*
 * Diagnostics of the current (filtered) state, FP64 quadrature sums:
 * out[0] mass = sum_g M_g rho, out[1..3] momentum sum M rho u,
 * out[4] kinetic energy sum M rho0 |u|^2 / 2, out[5] viscous dissipation integral
 * eps = 2 mu sum_i (d_i u_i)^2 - (2/3) mu (div u)^2 + mu sum_{i<j} (d_i u_j + d_j u_i)^2
 * (mu = rho0 nu; Sec. 3.4 with the square of the divergence term), quadrature over
 * element-local nodes with GLL derivatives, out[6] dt, out[7] time.
 * Returns SELBM_ERR_NONFINITE if the state holds NaN/Inf, SELBM_OK_FALLBACK when the
 * learned control's drift fallback is engaged.
 */
int selbm_diagnostics(selbm_t *h, double out[8]);
/*
 * Pipe-flow statistics (Sec. 4, turbulent pipe: tau_w evaluated at the boundary nodes,
 * mean axial velocity averaged in space and time), of the current (filtered) state.
 *
 * selbm_wall_stress: wall shear stress along the direction dir (normalised here), the
 * average over every wall face, weighted by the surface quadrature weights w_s J_s, of
 * -mu n . grad(u . dir) at the face's GLL nodes; n is the outward unit normal, the
 * gradient is the element's GLL derivative with the chain rule, mu = rho0 nu.  A node on
 * several wall faces contributes once per face.  *tau = 0 on meshes without walls.
 * For the pipe, tau_w of the paper (mu (sin theta du_z/dy + cos theta du_z/dx)) with
 * dir = the axis.  Errors: SELBM_ERR_ARG (NULL or zero dir), SELBM_ERR_STATE, SELBM_ERR_CUDA.
 *
 * selbm_radial_profile: unique nodes binned by their distance r from the line through
 * origin along axis, bin = min(floor(r nbins / radius), nbins - 1); mean[b] = sum M_g
 * (u_g . axis) / mass[b], mass[b] = sum M_g (lumped mass), host buffers of nbins
 * values (mean[b] = 0 for an empty bin).  Time averages are the caller's: average the
 * mean profiles of successive calls weighted by mass.  1 <= nbins <=
 * SELBM_PROFILE_MAX_BINS.  Errors as selbm_wall_stress.
 */
#define SELBM_PROFILE_MAX_BINS 2048
int selbm_wall_stress(selbm_t *h, const double dir[3], double *tau);
int selbm_radial_profile(selbm_t *h, const double origin[3], const double axis[3], double radius, int nbins,
                         double *mean, double *mass);

/* ------------------------------------------------------------------------
 * Learned per-element filter control.  Not in the paper, whose fixed explicit
 * filter (Sec. 2.4) is the fallback.  Per element and step, before the filter:
 * features x = [log10(E_k(rho - rho0) + 1e-30), log10(E_k(|u|) + 1e-30)], k = 0..N,
 * with E_k the sum of squared modal coefficients (hierarchical basis of the
 * filter) whose largest index is k; scaled input s = 2 (x - lo)/(hi - lo) - 1;
 * network 2(N+1) -> 64 tanh -> 64 tanh -> 2 with bfloat16 weights (FP32
 * arithmetic in the FP32 form, FP64 in the FP64 form); gamma = 0.5
 * sigmoid(o0), kc = 2 + (N-3) sigmoid(o1); the element is filtered with the
 * paper's quadratic transfer function at (gamma, kc).  Parameter vector (FP32):
 * W1[64][nin], b1[64], W2[64][64], b2[64], W3[2][64], b3[2], nin = 2(N+1).
 * Fallback to the fixed filter: per element when any feature leaves [lo, hi];
 * for the rest of the run when the relative change of the mass between steps
 * exceeds mass_bound, or (runs without body force, ke_bound > 0) the kinetic
 * energy grows by more than ke_bound relative between steps; ke_bound <= 0
 * disables the kinetic-energy criterion (weakly compressible runs exchange
 * kinetic and acoustic energy, so it is off by default in the binding).
 * ------------------------------------------------------------------------ */

/* Enable the learned control (host arrays: params [selbm_mlp_nparams(2(N+1))],
 * lo/hi [2(N+1)]).  Weights are rounded to bfloat16 (nearest, ties to even). */
int selbm_set_learned_filter(selbm_t *h, const float *params, const float *lo, const float *hi, double mass_bound,
                             double ke_bound);
/* Back to the fixed filter. */
int selbm_clear_learned_filter(selbm_t *h);
/* out[0] = global fallback flag, out[1] = element-steps that kept the fixed filter
 * since the last call (counter reset), out[2] = 1 if the learned control is on. */
int selbm_learned_status(selbm_t *h, int64_t out[4]);
/* Transfer functions sigma[E][N+1] chosen by the last control pass (host buffer). */
int selbm_element_sigma(selbm_t *h, double *sigma);
/* Features of the state the next filter acts on (the state before the pending filter of
 * the last step, i.e. what the learned control sees), device buffer feat[E][2(N+1)] (float). */
int selbm_features(selbm_t *h, float *feat);
/* Per-element error sum wJ ((rho - rho_ref)^2 + |u - u_ref|^2) of h against ref, a
 * handle on the same mesh at a higher order whose fields are interpolated element by
 * element to h's GLL nodes; device buffer err[E] (double).  Allocates temporaries. */
int selbm_element_errors(selbm_t *h, selbm_t *ref, double *err);

/* MLP training (device pointers; scaled inputs x [M][nin], targets y [M][2] = (gamma*, kc*)).
 * loss = mean(((gamma - gamma*)/0.5)^2 + ((kc - kc*)/(N-3))^2). */
int selbm_mlp_nparams(int32_t nin);
/* Mean loss and its gradient over all M samples (FP32, deterministic order). */
int selbm_mlp_grad(const float *params, int32_t nin, int32_t order, const float *x, const float *y, int64_t M,
                   float *grad, float *loss, void *cuda_stream);
/* (gamma, kc) per sample -> out [M][2]; bf16 = 1 rounds the weights to bfloat16. */
int selbm_mlp_forward(const float *params, int32_t nin, int32_t order, const float *x, int64_t M, int32_t bf16,
                      float *out, void *cuda_stream);
/* Adam (0.9, 0.999, 1e-8) on minibatches of `batch` samples in a fresh shuffled order per
 * epoch (Feistel permutation keyed by seed and epoch); *adam_t counts updates (in/out);
 * loss_hist (host, [epochs], may be NULL) gets the mean minibatch loss per epoch.
 * Allocates its scratch. */
int selbm_mlp_train(float *params, float *m, float *v, int32_t nin, int32_t order, const float *x, const float *y,
                    int64_t M, int32_t batch, int32_t epochs, float lr, uint64_t seed, int64_t *adam_t,
                    float *loss_hist, void *cuda_stream);

/*
 * Dry run of selbm_create's host setup, without touching the GPU: validates
 * the mesh and reports out_i[0..5] = E, Np, Q, G (unique nodes), Gb (nodes on
 * element boundaries), affine (1 if every element has constant metrics);
 * out_d[0..3] = smallest GLL node spacing, sum of the assembled lumped mass
 * (domain measure), number of wall-face nodes, sum of wall surface weights.
 * Errors as selbm_create (SELBM_ERR_ARG / SELBM_ERR_MESH), text in selbm_last_error(NULL).
 */
int selbm_mesh_check(const selbm_mesh *mesh, int32_t lattice, int32_t order, int64_t out_i[6], double out_d[4]);
/* The same dry run for a selbm_mesh_nodes mesh. */
int selbm_mesh_check_nodes(const selbm_mesh_nodes *mesh, int32_t lattice, int32_t order, int64_t out_i[6],
                           double out_d[4]);

/*
 * Per-kernel device timers (tracing).  selbm_timers(h, 1) resets and starts
 * recording a CUDA event pair around every hot-path launch on the handle's
 * stream; selbm_timers(h, 0) stops.  selbm_timers_read synchronises the
 * stream and returns, per kernel kind k, the summed device time ms[k] and the
 * launch count n[k] since the last reset:
 *   k = 0: stage kernel, stage 1 (whole-element form: filter + collision +
 *          streaming RHS; population-split form: streaming RHS only)
 *   k = 1: stage kernel, stages 2 and 3
 *   k = 2: assembly kernel (all stages)
 *   k = 3: learned filter control (features, network, filter, drift check; in
 *          the population-split form also the collision and the assembly of
 *          the filtered copies of shared nodes)
 *   k = 4: population-split form: prologue (fixed filter + collision, or the
 *          collision alone when no filter is pending)
 * The population-split form is the default for hexahedral meshes at the
 * compiled orders (D3Q19: N = 4, 7; D3Q27: N = 5, 7), in both precisions.
 */
#define SELBM_TIMER_KINDS 5
int selbm_timers(selbm_t *h, int enable);
int selbm_timers_read(selbm_t *h, double ms[SELBM_TIMER_KINDS], int64_t n[SELBM_TIMER_KINDS]);

/*
 * Allocation-free integrals of a caller-owned state.  The paper has no
 * counterpart: this entry exists for callers that cannot let the library
 * allocate device memory -- e.g. an application whose own memory pool has
 * already reserved the GPU's memory, or a per-step monitoring hook inside a
 * time loop where cudaMalloc/cudaFree would add an implicit device
 * synchronisation.  selbm_diagnostics needs a handle, and selbm_create
 * allocates; this call does not allocate anything.
 *
 * Inputs (device pointers): f [Q][nelem][np] FP64 populations f_bar at the
 * element-local nodes (the layout of selbm_get_state), w [nelem][np] the
 * quadrature weight of each local node (rho_i rho_j rho_k J for conforming
 * elements, so that copies of a shared node add up to its assembled mass).
 * Output (device pointer): out[0] = sum w rho, out[1..3] = sum w rho u,
 * out[4] = sum w rho0 |u|^2 / 2, out[5] = number of non-finite entries of f.
 * Enqueued on cuda_stream (a cudaStream_t, NULL = legacy default stream);
 * returns without synchronising.
 *
 * Scratch: per-element partial sums in one fixed device array inside the
 * library (SELBM_NOALLOC_MAX_ELEMS x 6 doubles = 3 MiB), held by every GPU
 * that loads the library until the process exits.  nelem above
 * SELBM_NOALLOC_MAX_ELEMS returns SELBM_ERR_ARG with no device work.  Every
 * call overwrites the partials it reads, so nothing carries over between
 * calls, but all calls share the one array: calls that overlap on the GPU
 * (e.g. on two streams at once) race and must be serialised by the caller.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is kept for the life of the
 * process: it does not survive a cudaDeviceReset of that device, so a process
 * that resets a device must not call this entry point on it afterwards.
 * Errors: SELBM_ERR_ARG (NULL pointer, bad sizes or lattice), SELBM_ERR_CUDA
 * (address lookup or launch failed).
 */
#define SELBM_NOALLOC_MAX_ELEMS 65536
int selbm_integrals_noalloc(int32_t lattice, int32_t nelem, int32_t np, const double *f, const double *w,
                            double rho0, double *out, void *cuda_stream);

/* Block until all work on the handle's stream is done; returns the first CUDA error seen,
 * else SELBM_OK_FALLBACK when the learned control's drift fallback is engaged, else SELBM_OK. */
int selbm_sync(selbm_t *h);

#ifdef __cplusplus
}
#endif
#endif /* SELBM_H */
