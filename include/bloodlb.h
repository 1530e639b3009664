/*
 * bloodlb.h -- C ABI of the GB300 (sm_103a) library for the coupled time step
 * of Janoschek, Toschi & Harting, "A simplified particulate model for
 * coarse-grained hemodynamics simulations" (arXiv:1005.2594):
 * a D3Q19 lattice-BGK plasma (Sec. II) with rigid ellipsoidal cells coupled
 * by moving-boundary bounce-back, fill/drain and contact links (Sec. II), and
 * Berne-Pechukas-scaled Hookean cell-cell and cell-wall potentials (Sec. III).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Status: every int-returning call returns BL_OK (0) or a negative BL_E*
 *   code.  Errors are sticky per context: after a failure every later call
 *   returns the same code until bl_destroy; bl_last_error() names the cause.
 *   Device-side failures (unstable fluid, list overflow) are raised by the
 *   kernels into a status word and reported by bl_sync() and by the next
 *   call that waits on the stream.
 * Ownership: the library owns all of its device memory (allocated in
 *   bl_lb_init / bl_particles_set, released by bl_destroy).  Caller pointers
 *   are borrowed for the duration of the call only.
 * Streams: every call of a context is ordered on the CUDA stream given to
 *   bl_lb_init (NULL = the legacy default stream).  Inside a step the cell
 *   list, the potentials and the contact sums run on two more streams of the
 *   context (created at the highest priority) beside the lattice sweep, and
 *   the claims beside the pending moving-boundary terms; steps replay
 *   captured graphs on a fourth stream.  All are
 *   forked from and joined back to the caller's stream with events, so work
 *   the caller enqueues later still follows the step.  A context is not
 *   thread-safe; use one context per stream.
 * Lattice: nodes are numbered n = x + nx (y + ny z), x fastest.  A
 *   non-periodic axis carries solid wall layers at index 0 and N-1; faces
 *   are numbered x-,x+,y-,y+,z-,z+ = wall ids 0..5.  Owner codes: -1 fluid,
 *   -2-w wall with id w (0..7), k >= 0 cell k.
 * Directions: r = 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = (1,1,0),
 *   (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1),
 *   (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1).  Weights 1/3, 1/18, 1/36
 *   (Sec. II, after Eq. neq).
 * Cells: X centre, q unit quaternion (w,x,y,z) whose rotation takes e_z to
 *   the symmetry axis, V linear velocity, L lab-frame angular momentum.
 *   A time step takes X(t), q(t), V(t-1/2), L(t-1/2) to the next level.
 * Units: lattice units (dx = dt = 1).
 */
#ifndef BLOODLB_H
#define BLOODLB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BL_OK 0
#define BL_EINVAL (-1)     /* bad argument, size or parameter */
#define BL_ENOMEM (-2)     /* device allocation failed */
#define BL_EUNSTABLE (-3)  /* rho <= 0, NaN, |u| above the Mach guard in a fluid node, or a cell
                              faster than half a node per step */
#define BL_EOVERFLOW (-4)  /* an internal list exceeded its capacity */
#define BL_EBARRIER (-5)   /* a bounded device-side wait timed out */
#define BL_ECUDA (-6)      /* a CUDA runtime call failed */
#define BL_ESTATE (-7)     /* call out of order (e.g. step before particles_set with cells) */

#define BL_STORE_F32 0  /* populations stored as FP32 (shifted by alpha_r rho_bar) */
#define BL_STORE_BF16 1 /* shifted populations stored as BF16, collided in FP32 */
#define BL_STORE_F16 2  /* shifted populations stored as FP16 (scaled by 2^10), collided in FP32 */

typedef struct bl_ctx bl_ctx;

/* Lattice and fluid (Sec. II; tau = 1 and rho_bar = 1 in every run of the
   paper, Sec. IV).  The body force g is an acceleration: force density rho g,
   applied with the Guo scheme, u = (j + rho g / 2) / rho. */
typedef struct {
  int nx, ny, nz;          /* lattice size, each >= 1 */
  int periodic[3];         /* 1 periodic, 0 wall layers at 0 and N-1 */
  double wall_vel[8][3];   /* velocity of wall id 0..7 (moving bounce-back, Eq. c) */
  double tau;              /* BGK relaxation time (Eq. col), > 1/2 */
  double rho0;             /* rho_bar: initial density, fill density (Sec. II) */
  double g[3];             /* body-force acceleration on the fluid */
  int store_dtype;         /* BL_STORE_* */
  int body_force_on_cells; /* 1: cells also feel m g (tube flow of Sec. IV) */
} bl_lb_params;

/* Cells (Sec. II fluid coupling, Sec. III potentials).  The strength of the
   pair potential is eps (1 - chi^2 (o_i.o_j)^2)^(-nu/2) eps2^mu, eps2 being
   the bracket of Eq. (sigma) with chi_prime; the paper's Berne-Pechukas form
   is nu = 1, mu = 0. */
typedef struct {
  double R_par, R_perp;     /* half-axes of the fluid-coupling ellipsoid */
  double sig_par, sig_perp; /* half-axes of the potential (Eq. sigma) */
  double eps, eps_w, sig_w; /* epsbar, epsbar_w, wall sphere radius (1/2) */
  double mu, nu, chi_prime; /* Gay-Berne exponents of the strength */
  double r_cut;             /* neighbour-list radius (the potential is compact) */
  double rho_p;             /* cell density; mass rho_p 4/3 pi R_perp^2 R_par */
  int move_particles;       /* 0: cells held fixed (forces still computed); 1: free cells; 2: prescribed
                               motion, the cells keep the V and Omega = I_lab^-1 L of their last set
                               (forces computed and reported, not applied) */
  int reserved;
} bl_particle_params;

/* Creates a context: allocates the population field (19 x N in the storage
   type, single AA buffer), the owner map, and sets resting fluid
   n = n^eq(rho_bar, 0) on all non-wall nodes (the paper starts from rest,
   Sec. IV).  cuda_stream is a cudaStream_t or NULL.  *out receives the
   context, or NULL on failure (status returned). */
int bl_lb_init(bl_ctx **out, const bl_lb_params *p, void *cuda_stream);

/* Adds static walls: mask is a host array of N bytes; mask[n] = k in 1..8
   makes node n a wall with id k-1 (0 leaves the node unchanged).  Call
   before bl_particles_set.  The surface wall nodes (walls linked to a
   non-wall node, Sec. III) are rebuilt. */
int bl_walls_set(bl_ctx *c, const uint8_t *mask);

/* Sets the cells: host arrays X (n x 3), q (n x 4), V (n x 3), L (n x 3).
   The first call (or a call with a different n) discretises from scratch
   (lowest index wins on overlap), deletes the fluid of covered nodes and
   gives no impulses.  A later call with the same n re-discretises against
   the current owner map with the first-arrival rule and fill/drain
   impulses, exactly as a time step does (Sec. II).  n may be 0.
   The first call waits for the device; a later call is enqueued on the
   stream and returns at once (its device errors surface at the next
   bl_sync); the host arrays may be reused when it returns.
   Requirements (BL_EINVAL otherwise): r_cut >= max(R_par, R_perp) + 1, so
   that the cells covering a node lie in the cell-list bins around it; every
   periodic length >= 2 max(R_par, R_perp) + 4, so that a cell does not
   reach its own periodic image. */
int bl_particles_set(bl_ctx *c, int n, const bl_particle_params *pp, const double *X, const double *q,
                     const double *V, const double *L);

/* Enqueues nsteps coupled time steps on the context stream (no host sync):
   collide + stream + bounce-back + momentum exchange + contact links, cell
   list, pair and wall potentials, leap-frog, re-discretisation with
   fill/drain.  The moving-boundary term of the populations a step bounces
   off cells is added when the next step reads them (Eqs. c, lbe-bb-corr
   with the half-step cell velocity of the implicit coupling): between steps
   it is held per fluid node, and every read-out of populations or fields
   adds it first, so what the caller sees is the state after the whole step.
   With timing off, pairs of steps are launched as one CUDA
   graph and a last single step as a one-step graph (captured on first use,
   and again when the cell arrays or parameters, the walls, the sweep variant
   or the attached network change).  Returns the sticky status known so far
   (device errors of this call surface at the next bl_sync). */
int bl_step(bl_ctx *c, int nsteps);

/* Moments of the current populations: rho (N doubles) and
   u = (j + rho g / 2) / rho (N x 3 doubles) on fluid nodes, 0 elsewhere;
   owner (N int32).  Any pointer may be NULL.  on_device = 1: the pointers
   are device memory (e.g. CUDA tensors) written on the context stream;
   on_device = 0: host memory, the call waits. */
int bl_fields_get(bl_ctx *c, double *rho, double *u, int32_t *owner, int on_device);

/* Cell read-out after the last step (host arrays, n x 3 / n x 4, any may be
   NULL): F, T = total force and torque used by the last integration (links,
   potentials, fill/drain impulses, body force); X, q, V, L = current state.
   Waits on the stream. */
int bl_forces_get(bl_ctx *c, double *F, double *T, double *X, double *q, double *V, double *L);

/* Parts of the last step's force (host, n x 3 each, any may be NULL):
   Fh/Th link force (bounce-back momentum exchange Eq. deltap plus contact
   links Eq. deltapppp), Fp/Tp potentials (Eqs. phi-sigmaw), Om angular
   velocity I_lab^-1 L used for the rotation; PF/PT fill/drain impulses
   waiting for the next integration. */
int bl_force_parts_get(bl_ctx *c, double *Fh, double *Th, double *Fp, double *Tp, double *Om, double *PF,
                       double *PT);

/* Momentum given to each wall id by its bounce-back links, summed over the
   steps since the previous call (or since bl_lb_init), then reset (8 x 3
   doubles, host); the momentum-transfer observable of Eq. (mu). */
int bl_wall_momentum_get(bl_ctx *c, double *wallmom);

/* Lees-Edwards shear (Sec. IV, the plane Couette cells of its rheology):
   the periodic images of the box along x slide past each other in z, the
   image above moving with velocity offset U (lattice units, |U| < 0.3) and
   displaced by U t after t steps.  A population crossing the plane between
   x = nx-1 and x = 0 comes from the neighbouring image, from a point U t
   along z from its periodic source (linear interpolation between the two
   nearest nodes), its equilibrium part carried into this image's frame,
   n + n^eq(rho, u -+ U e_z) - n^eq(rho, u) with its source node's moments
   (reading Q25).  A free cell whose centre comes closer than d_reflect to
   the plane (x = -1/2) while moving toward it has its x velocity negated
   before it moves (Sec. IV; the step's coupling used the solved velocity);
   d_reflect <= 0 takes max(sigma_perp, max(R_perp, R_par) + 1), so that no
   cell covers a node beside the plane.  Every axis must be periodic and no
   wall mask set (BL_EINVAL / BL_ESTATE); a node beside the plane that is not
   fluid during a step is reported by bl_sync as BL_ESTATE.  A later call
   sets a new U and restarts t and the momentum sums.  The sweep keeps its
   variant; two small passes over the two planes follow each sweep. */
int bl_lees_edwards_set(bl_ctx *c, double U, double d_reflect);

/* The z-momentum moved along +x across the sheared plane, summed over the
   steps since bl_lees_edwards_set, and the number of steps (host scalars).
   Per step it is the flux of the crossing post-collision populations, the
   mean of its value in the frame below the plane and in the frame above it;
   in steady shear it is -mu gamma_dot l_y l_z, so that Eq. (mu) reads
   mu_app = -Delta p_LE / (l_y l_z gamma_dot).  Waits on the stream. */
int bl_lees_edwards_get(bl_ctx *c, double *P_sum, int64_t *steps);

/* Checkpoint of the fluid: node-major host array N x 19 doubles, the
   unshifted populations n_r(x, t) in the direction order above; non-fluid
   nodes read as 0 and are ignored on set. */
int bl_populations_get(bl_ctx *c, double *pop);
int bl_populations_set(bl_ctx *c, const double *pop);

/* Boundary links (fluid node y, direction r with y + c_r solid, owner of
   y + c_r) and contact links (node x of cell p, r, owner of x + c_r, a wall
   or another cell) of the current owner map, as int32 triples in (node, r)
   order, built by warp-level stream compaction.  Writes min(count, cap)
   triples to the host array out and the full count to *count. */
int bl_boundary_links_get(bl_ctx *c, int32_t *out, int64_t cap, int64_t *count);
int bl_contact_links_get(bl_ctx *c, int32_t *out, int64_t cap, int64_t *count);

/* The bounce links of the last step's lattice sweep, as the step sums the
   link momentum of Eq. (deltap) over them and gives them the moving-boundary
   term of Eq. (c): the sweep writes, for every fluid node next to a cell, one
   record per cell into that cell's list.  Read out as (fluid node y,
   direction r with y + c_r inside cell p, p) int32 triples in (node, r)
   order: the boundary links whose owner is a cell, of the owner map the
   last step started from.  Empty before the first step after cells are set.
   Writes min(count, cap) triples to the host array out and the full count to
   *count; BL_EOVERFLOW if a list outgrew its capacity. */
int bl_cell_links_get(bl_ctx *c, int32_t *out, int64_t cap, int64_t *count);

/* Cell list of the current positions in canonical (bin, id) order:
   nb_k = max(1, floor(N_k / r_cut)), bin_k = floor((X_k / N_k) nb_k)
   clamped; start has nb0 nb1 nb2 + 1 entries, ids n entries (host).
   Pass start = ids = NULL to query nb only. */
int bl_cell_list_get(bl_ctx *c, int32_t nb[3], int32_t *start, int32_t *ids);

/* Cell-list build that allocates nothing, for callers that cannot call
   cudaMalloc (device memory already given to their own pool allocator, or a
   time loop that must avoid the synchronisation an allocation can cause).
   The paper has no counterpart: it is an interface of this library.  Builds
   the list of bl_cell_list_get for n cells at device positions X (n x 3
   doubles in [0, dims)) into device arrays start (nb0 nb1 nb2 + 1 int32) and
   ids (n int32) on cuda_stream; nb receives the bin counts (host).  Scratch
   lives in a fixed array reserved on every GPU that loads the library
   (2.25 MiB, held until exit): at most 65536 cells and 262144 bins, larger
   requests return BL_EINVAL (nb is then left untouched).  The first call on
   a device looks up that array and should come before any stream capture;
   the address is cached per device for the life of the process, which
   assumes the device's primary context and no cudaDeviceReset in between.
   Calls that overlap on the GPU share the array and race.  No context is needed; errors are returned, not
   kept. */
int bl_cell_list_build_static(const double *X, int n, const int32_t dims[3], double r_cut, int32_t nb[3],
                              int32_t *start, int32_t *ids, void *cuda_stream);

/* Sweep variants of the lattice sweep (the same arithmetic, other thread
   mappings): 0 one node per thread; 1, 2 (FP32 storage only) a software
   pipeline that walks 4 or 8 z planes per thread block and copies the next
   node's populations into shared memory while the current one is collided;
   3, 4 (any storage) a pipeline over 8 or 4 z planes whose row segments are
   fetched by bulk asynchronous copies (TMA) two planes ahead; 5 (any
   storage) a persistent grid of as many blocks as the device holds, each
   walking its share of the rows through one bulk-copy pipeline.  3 to 5
   need rows of a multiple of 16 bytes (nx a multiple of 4 in FP32, of 8 in
   BF16 / FP16; otherwise they run as variant 0).  A context that was given
   no variant chooses: with cells, 0 (the boundary work of a suspension
   falls unevenly on the warps, and the block-wide barriers of 1 to 5 make
   every warp wait for the slowest); without cells, 3 where the rows allow
   it, else FP32 with 1 and 16-bit storage with 0.  bl_sweep_variant sets
   one and keeps it (BL_EINVAL for an unknown variant, or variant 1 or 2
   with 16-bit storage).  A bounded wait for the bulk copies that gives up
   makes the next bl_sync return BL_EBARRIER.
   bl_autotune times every variant the storage type allows over trial_steps
   steps (>= 2; the context advances by those steps, so call it before the
   steps that count), keeps the fastest and writes its number to *choice
   (may be NULL).  The paper has no counterpart: these are interfaces of
   this library. */
int bl_sweep_variant(bl_ctx *c, int variant);
int bl_autotune(bl_ctx *c, int trial_steps, int *choice);

/* Ensembles: n independent contexts (different lattices, cells, parameters;
   one device) advanced together.  bl_ensemble_step(e, k) advances every
   member by k steps; pairs of steps of all members run as one CUDA graph
   whose branches are the members' steps, so that small lattices fill the
   GPU together; it is ordered after the work already enqueued on each
   member's stream and on cuda_stream, and each member's later work follows
   it.  The ensemble borrows the contexts: they must outlive it, and a
   member with timing enabled makes the step return BL_ESTATE.  Errors of a
   member are reported by bl_ensemble_step / bl_ensemble_sync (the first
   one).  The paper has no counterpart (a batching interface of this
   library). */
/* ---------------------------------------------------------------------
   Indexed lattice of vessel networks (closing discussion of the paper: the
   method joined to an indexed LB scheme for digitised vessel networks).
   Only the fluid nodes of a lattice with walls are stored and swept, so
   memory and time scale with the lumen, not the bounding box.  The update is
   the dense lattice's plasma update of Sec. II (moments, Guo forcing, BGK
   toward the third-order equilibrium, mid-link bounce-back with the
   moving-wall term C, the walls' momentum); cells are not coupled to it.
   Fluid nodes are numbered in dense node order (x fastest); a table gives
   each one's 18 neighbours.  Walls: the face layers of non-periodic axes
   (ids 0..5, first walled axis in x, y, z order) and a mask of N bytes as
   for bl_walls_set (value k in 1..8: wall id k - 1, overriding). */
typedef struct bl_sparse bl_sparse;

/* Host only (no device work): the index of a lattice.  With dense_of and nbr
   NULL, *n_fluid receives the number of fluid nodes.  Otherwise *n_fluid
   must hold their capacity (>= that number; BL_EINVAL if smaller) and
   receives the number; dense_of[i] is the dense index x + nx (y + ny z) of
   fluid node i, nbr[(r - 1) n_fluid + i] (r = 1..18, the direction
   numbering above) the fluid index of node i + c_r, or -1 - w for a wall of
   id w.  Either array may be NULL.  mask may be NULL. */
int bl_sparse_index_build(const bl_lb_params *p, const uint8_t *mask, int64_t *n_fluid, int32_t *dense_of,
                          int32_t *nbr);

/* Creates an indexed lattice: builds the index on the host, uploads it and
   sets resting fluid n^eq(rho_bar, 0).  Storage 19 x n_fluid elements of
   p->store_dtype plus 18 x n_fluid int32.  cuda_stream as in bl_lb_init. */
int bl_sparse_init(bl_sparse **out, const bl_lb_params *p, const uint8_t *mask, void *cuda_stream);
/* nsteps steps (pairs of steps replay one CUDA graph). */
int bl_sparse_step(bl_sparse *s, int nsteps);
/* rho (N) and u = (j + rho g / 2) / rho (N x 3) on the dense grid, zero at
   walls; host (on_device 0) or device pointers.  Waits on the stream. */
int bl_sparse_fields_get(bl_sparse *s, double *rho, double *u, int on_device);
/* populations n_r (N x 19 host doubles on the dense grid, zero at walls) as
   the next step reads them; set writes those of the fluid nodes. */
int bl_sparse_populations_get(bl_sparse *s, double *pop);
int bl_sparse_populations_set(bl_sparse *s, const double *pop);
/* momentum given to each wall id since the previous call, then reset (8 x 3). */
int bl_sparse_wall_momentum_get(bl_sparse *s, double *wallmom);
/* waits for the stream; BL_EUNSTABLE if a node went unstable */
int bl_sparse_sync(bl_sparse *s);
int64_t bl_sparse_nodes(const bl_sparse *s);
int64_t bl_sparse_launch_count(const bl_sparse *s);
const char *bl_sparse_last_error(const bl_sparse *s);
void bl_sparse_destroy(bl_sparse *s);

typedef struct bl_ens bl_ens;
int bl_ensemble_create(bl_ens **out, bl_ctx *const *ctxs, int n, void *cuda_stream);
int bl_ensemble_step(bl_ens *e, int nsteps);
int bl_ensemble_sync(bl_ens *e);
void bl_ensemble_destroy(bl_ens *e);

/* Learned near-contact correction (the paper motivates it and leaves it open:
   two cells closer than the lattice resolves have no fluid node between them
   and no lubrication force, Sec. II).  A network 14 -> 64 -> 64 -> 6 with tanh
   hidden layers, BF16 weights and activations on the tensor cores, FP32
   accumulation and FP32 master parameters.
   Features of the ordered pair (i, j), in the body frame of i: R_i^T r
   (r = X_j - X_i, minimum image), q_i^* q_j with w >= 0, the gap
   |r| - sigma_R (the contact distance of Eq. sigma built from R_par, R_perp),
   R_i^T (V_j - V_i), R_i^T (W_j - W_i).  Outputs: the force and torque
   correction on i in the body frame of i.
   Parameters (host arrays of float): theta = W1 (64 x 14), b1 (64),
   W2 (64 x 64), b2 (64), W3 (6 x 64), b3 (6), row-major, 5510 values;
   norm = input means (14), input scales (14), output means (6), output
   scales (6): the network sees (x - mean) / scale and its output is
   y~ scale + mean.  Scales must be > 0.
   bl_mlp_forward: x (B x 14) and y (B x 6) are device arrays (FP32) on the
   model's stream.  bl_mlp_grad: loss (mean over the B samples of the squared
   error of the scaled outputs summed over the six) and its gradient with
   respect to theta for targets y (device); loss and grad (5510) are host
   pointers, may be NULL (then the call does not wait); the gradient stays on
   the device for bl_mlp_adam, which takes one Adam step with it.
   bl_mlp_params_set resets the Adam moments. */
typedef struct bl_mlp bl_mlp;
int bl_mlp_create(bl_mlp **out, void *cuda_stream);
int bl_mlp_params_set(bl_mlp *m, const float *theta, const float *norm);
int bl_mlp_params_get(bl_mlp *m, float *theta, float *norm);
int bl_mlp_forward(bl_mlp *m, const float *x, int B, float *y);
int bl_mlp_grad(bl_mlp *m, const float *x, const float *y, int B, float *loss, float *grad);
int bl_mlp_adam(bl_mlp *m, float lr, float beta1, float beta2, float eps);
int bl_mlp_sync(bl_mlp *m);
void bl_mlp_destroy(bl_mlp *m);

/* Uses model m (NULL: none, the plain method) in every later step of
   context c: after the potentials, every ordered pair of cells with
   gap_lo <= gap < gap_hi (lattice units; gap as in bl_pair_features) and
   relative speed |V_j - V_i| in [speed_lo, speed_hi] gets the network's
   force and torque correction, rotated to the lab frame and added to the
   potential part of the step's force (bl_force_parts_get Fp / Tp); every
   other pair keeps the plain method (a network is not used outside the
   gaps and speeds it was trained on).  bl_mlp_attach(c, m, cut) is the range
   gap < cut at any speed.  BL_EINVAL unless gap_lo < gap_hi, |gap_hi| <
   1000 and 0 <= speed_lo <= speed_hi.  The model must outlive its use; the
   step runs it on the context's streams. */
int bl_mlp_attach_range(bl_ctx *c, bl_mlp *m, double gap_lo, double gap_hi, double speed_lo, double speed_hi);
int bl_mlp_attach(bl_ctx *c, bl_mlp *m, double gap_cut);

/* Features of n ordered pairs (device array of n x 2 int32 cell indices) from
   the current cell state, into the device array out (n x 14 float), on the
   context stream; invalid pairs (an index out of range, i == j) give zeros. */
int bl_pair_features(bl_ctx *c, const int32_t *pairs, int n, float *out);

/* Kernel timing with CUDA events.  While enabled, steps are enqueued one
   kernel group at a time (no graph), each group bracketed by an event pair
   on the stream it runs on, and the lattice sweep runs alone: the side
   streams start when it ends (in a replayed graph they run beside it), so
   that its time is the kernel's own.  Groups: 0 fused
   collide/stream/bounce-back with the cell-link records (the lattice
   sweep), 1 cell list, 2 pair + wall potentials (1 and 2 on a side
   stream), 3 link sums + half-step solve + leap-frog + claims + pending
   moving-boundary term, 4 contact sums (second side stream) + resolve with
   fill/drain + neighbour words.  bl_timing_read waits, then writes per
   group the summed milliseconds and the number of timed launches (arrays
   of ngroups), and clears the sums. */
int bl_timing_enable(bl_ctx *c, int enable);
int bl_timing_read(bl_ctx *c, double *ms, int64_t *count, int ngroups);

/* Number of kernels this context has launched since bl_lb_init. */
int64_t bl_launch_count(const bl_ctx *c);

/* Waits for the stream; returns the sticky status including device errors. */
int bl_sync(bl_ctx *c);

/* Human-readable cause of the sticky error ("" if none). */
const char *bl_last_error(const bl_ctx *c);

/* Releases all device memory of the context; c may be NULL. */
void bl_destroy(bl_ctx *c);

#ifdef __cplusplus
}
#endif

#endif /* BLOODLB_H */
