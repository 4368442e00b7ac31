/*
 * ib_cav.h -- C ABI of the B300 library for coupling-aware Vanka (CAV) multigrid
 * preconditioning of the reduced Eulerian velocity-pressure immersed-boundary system.
 *
 * The system (Sec. 2, Eq. Eul_schur) is K_E x = b with
 *     K_E = [[A, G], [-D, 0]],  A = A0 - dt E_E,  A0 = (rho/dt) I - mu L,  E_E = S E J,
 * on a periodic N x N MAC grid of [0, L)^2 with h = L / N.  Unknown vectors have length
 * 3 N^2 and are laid out as three blocks u | v | p, entry (i, j) of a block at j N + i;
 * u_{ij} sits at (i h, (j+1/2) h), v_{ij} at ((i+1/2) h, j h), p_{ij} at the cell centre.
 *
 * Conventions shared by every call
 *   - Every call returns ib_status; nothing throws or aborts across the ABI.  On a non-OK
 *     status ib_last_error() returns a thread-local message.
 *   - Descriptor structs and the marker arrays they point to are HOST memory, read during
 *     the call and not retained.
 *   - Vectors named b, x, r, z, w, y are caller-owned DEVICE buffers of FP64 (3 N_l^2
 *     entries on level l), unless a descriptor says otherwise.  They must not alias unless
 *     a call says so.
 *   - Calls are ordered on the given CUDA stream (0 = legacy default stream).  Set-up calls
 *     and fgmres_solve synchronise that stream before returning; sweep-level calls do not.
 *   - Handles (ib_system, cav_hierarchy) are library-owned: created by *_setup, released by
 *     *_destroy, and hold device memory of the device current at set-up time.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef IB_CAV_H
#define IB_CAV_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IB_OK = 0,
  IB_ERR_INVALID = 1,   /* bad argument, size or descriptor field                       */
  IB_ERR_OOM = 2,       /* device allocation failed                                       */
  IB_ERR_CUDA = 3,      /* a CUDA runtime call or kernel launch failed                    */
  IB_ERR_SINGULAR = 4,  /* a local patch matrix had a zero pivot (Sec. 3.3 factorisation)  */
  IB_ERR_NOCONV = 5,    /* FGMRES stopped at maxit above tolerance; x holds the last iterate */
  IB_ERR_TIMEOUT = 6,   /* a bounded device-side wait ran out (about a second); the call's
                           output is not valid, the device stays usable                   */
  IB_ERR_INTERNAL = 7   /* a device-side consistency check failed (e.g. a stencil window) */
} ib_status;

/* Message for the last non-OK status returned on the calling thread ("" if none). */
const char* ib_last_error(void);
/* ABI version of this header: 5 (4: ib_grid_desc.bc, ib_test_wait_stall; 5: fgmres_desc.loop,
 * ibnet_inner). */
int ib_abi_version(void);
/* Number of kernels this library has launched in this process (host-side count; a graph
 * replay adds the kernels it ran). */
int64_t ib_launch_count(void);

/* ------------------------------------------------------------------ system (Sec. 2) */

typedef enum { IB_FORCE_TARGET = 0, IB_FORCE_MEMBRANE = 1, IB_FORCE_BEAM = 2, IB_FORCE_FIBER = 3 } ib_force_law;

/* Boundary conditions of the Eulerian grid (ABI 4):
 *   periodic  the periodic square of Sec. 2 (every experiment of Sec. 5.1 and 5.2);
 *   channel   the flow-past-a-fiber channel of Sec. 5.3: periodic in x, a prescribed inflow
 *             (u, v) = (0, -U(t)) on the top wall y = L, a traction outflow on y = 0 whose
 *             traction carries the backflow term (rho/2) min(u.n, 0) u.  The unknowns are the
 *             periodic grid's (3 N^2: the outflow row's v faces are unknowns, the top wall's
 *             are prescribed).  K_E holds the rows with homogeneous boundary data, closed by
 *             ghost values:  u_{i,N} = -u_{i,N-1},  v_{i,N} = 0,
 *                            u_{i,-1} = u_{i,0} + v_{i,0} - v_{i-1,0},
 *                            v_{i,-1} = v_{i,0} + u_{i+1,-1} - u_{i,-1},
 *                            p_{i,-1} = (2 mu / h)(v_{i,1} - v_{i,-1}) - p_{i,0};
 *             the boundary data enter the right-hand side (ib_channel_rhs).  The pressure is
 *             determined: no mean is removed and the coarsest solve has no border.  On the
 *             coarse levels a v face next to the top wall takes half the coarse face below it
 *             and the pressure prolongation is clamped in y; the inflow row's Vanka patches
 *             have four unknowns and an outflow-row v face has one incident cell.  Markers
 *             must stay at least 2.5 h from both walls (their supports do not wrap).        */
typedef enum { IB_BC_PERIODIC = 0, IB_BC_CHANNEL = 1 } ib_bc;

typedef struct {
  int32_t N;       /* cells per direction (>= 8; even to allow coarsening)              */
  double L;        /* side of the square                                                 */
  double rho, mu, dt;
  int32_t bc;      /* ib_bc (ABI 4)                                                      */
} ib_grid_desc;

/* Force laws (Lagrangian elasticity matrix E, acting identically on x and y):
 *   target   E = -k_target I                                  (Sec. 5.2)
 *   membrane E = k_stretch/ds^2 * cyclic [1 -2 1] - k_target I (Eq. disc_force_law)
 *   beam     E = k_stretch/ds^2 [1 -2 1] - k_bend/ds^4 [1 -4 6 -4 1] - k_target I, cyclic
 *                                                             (Sec. 5.2)
 * membrane and beam require closed = 1.  The tether source k_target X_target enters the
 * right-hand side only (ib_force, ib_step_rhs).
 * fiber (ABI 3, Sec. 5.3): an open chain (closed = 0, M odd >= 3, midpoint m = M / 2) with
 *   the energies  E_b = k_bend/(2 ds^5) sum_k (D_k x D_{k+1})^2,  D_k = X_{k+1} - X_k,
 *                 E_s = k_stretch/(2 ds) sum_k (|D_k| - ds)^2,
 *                 E_p = k_pos/2 |X_m - X_c|^2,  E_t = k_tan/2 |(X_{m+1} - X_{m-1})/(2 ds) - e_x|^2;
 *   force F = -(1/ds) grad (E_b + E_s + E_p + E_t) and E = dF/dX (the Newton tangent, which
 *   couples x and y), both at X_lin; S and J stay at X.  k_target must be 0.            */
typedef struct {
  int32_t M;             /* number of Lagrangian markers (0 allowed: no structure)      */
  int32_t closed;        /* 1: the marker chain is a closed curve                        */
  int32_t law;           /* ib_force_law                                                 */
  const double* X;       /* host, 2M doubles interleaved (x0, y0, x1, y1, ...): X^n      */
  const double* omega;   /* host, M quadrature weights omega_k                            */
  double ds;             /* uniform Lagrangian spacing used by the force stencils         */
  double k_target, k_stretch, k_bend;  /* k_target != 0 tethers every marker on any law */
  const double* X_target;  /* host, 2M interleaved, nullable: tether targets (source term) */
  /* fiber law only (ABI 3): */
  const double* X_lin;   /* host, 2M interleaved, nullable (= X): where F and E are taken  */
  double k_pos, k_tan;   /* midpoint clamp stiffnesses K_p, K_t                            */
  double clamp_x, clamp_y;  /* the clamp point X_c                                         */
} ib_structure_desc;

typedef struct ib_system ib_system;

/* Builds S^n, J^n at X (Peskin four-point kernel), E, and E_E = S E J on the device
 * (Sec. 2, Eq. intro_saddle).  *out receives a new handle. */
ib_status ib_setup(const ib_grid_desc* grid, const ib_structure_desc* structure,
                   cudaStream_t stream, ib_system** out);
/* A new configuration for the same grid (a Newton iterate or the next time step, Sec. 5.3):
 * S^n, J^n, E and E_E are rebuilt at sd's markers in place of the previous ones, which are
 * released.  Hierarchies built on this system before the call keep the E_E they copied at
 * set-up: they go on preconditioning with the configuration they were built from (FGMRES
 * accepts such a lagged preconditioner) until rebuilt with cav_setup.  On failure the
 * handle keeps its previous configuration.  Synchronises the device. */
ib_status ib_update_structure(ib_system* sys, const ib_structure_desc* structure, cudaStream_t stream);
/* y = K_E x on the finest grid (Eq. Eul_schur). */
ib_status ib_apply(const ib_system* sys, const double* x, double* y, cudaStream_t stream);
/* r = b - K_E x on the finest grid. */
ib_status ib_residual(const ib_system* sys, const double* b, const double* x, double* r,
                      cudaStream_t stream);
void ib_destroy(ib_system* sys);

/* Lagrangian / Eulerian transfers at the system's configuration X^n (Sec. 2) and the pieces
 * of a semi-implicit time step (Eqs. im_disc_mom, im_disc_advec, Eul_schur).
 * Lagrangian vectors F, U are device buffers of 2M doubles, x components then y components. */
/* F = E X^n + k_target X_target; for the fiber law, its nonlinear force F(X_lin). */
ib_status ib_force(const ib_system* sys, double* F, cudaStream_t stream);
/* f = S F on the 2 N^2 velocity faces (f: device, u block then v block). */
ib_status ib_spread(const ib_system* sys, const double* F, double* f, cudaStream_t stream);
/* U = J u from the velocity blocks of u (device, >= 2 N^2 entries). */
ib_status ib_interp(const ib_system* sys, const double* u, double* U, cudaStream_t stream);
/* Right-hand side of Eq. Eul_schur for one step: b_vel = (rho/dt) u_prev + f_body
 * + S F with F as ib_force returns it, b_p = 0.  u_prev (3 N^2) and f_body (2 N^2) are
 * device buffers and may be NULL (zero). */
ib_status ib_step_rhs(const ib_system* sys, const double* u_prev, const double* f_body, double* b,
                      cudaStream_t stream);
/* X^{n+1} = X^n + dt J u (Eq. im_disc_advec) into X_next (host, 2M interleaved); syncs. */
ib_status ib_advect(const ib_system* sys, const double* u, double* X_next, cudaStream_t stream);

/* Channel time step of Sec. 5.3 (ABI 4; IB_BC_CHANNEL systems only).  The base right-hand
 * side of the step t^n -> t^{n+1}:  b = [(rho/dt) u^n - rho N[u^n] ; 0] + g, N[u] = (u.grad)u
 * (explicit, centred, each component averaged from its four neighbours onto the other's
 * faces, with the previous inflow -U_prev on the top wall), g the boundary vector of the
 * inflow v = -U_next on the top wall and of the outflow traction (rho/2) min(u^n.n, 0) u^n
 * (u^n extrapolated to the wall as (3 u_0 - u_1)/2).  w_n (3 N^2) and b are device buffers. */
ib_status ib_channel_rhs(const ib_system* sys, const double* w_n, double U_next, double U_prev, double* b,
                         cudaStream_t stream);
/* Right-hand side of one Newton system of the step (Eqs. im_disc_mom, im_disc_advec, Sec.
 * 5.3) at the iterate w (device, 3 N^2) whose configuration X_k = X^n + dt J^n u_k was given
 * to the system as X_lin:  rhs = b_base + [S^n F(X_k) - dt E_E(X_k) u_k ; 0].  The linear
 * system is K_E(X_k) w' = rhs, and K_E(X_k) w - rhs is the Newton residual at w itself.  Any
 * force law (the fiber law's F and tangent are those of X_lin).  rhs must not alias. */
ib_status ib_newton_rhs(const ib_system* sys, const double* b_base, const double* w, double* rhs,
                        cudaStream_t stream);
/* r = b - K_E x and *norm = ||r||_2 (host; reduced on the device in a fixed order; syncs). */
ib_status ib_residual_norm(const ib_system* sys, const double* b, const double* x, double* r, double* norm,
                           cudaStream_t stream);

/* -------------------------------------------------------- hierarchy (Sec. 3, Sec. 4) */

/* Patch family of the smoothing levels (Sec. 3):
 *   CAV    one patch per cell, Eq. cav_patch_set;
 *   VANKA  one standard 5-unknown patch per cell, B(1,0);
 *   BOX    B(b,o) (ABI 3): the grid cut into b x b blocks, in lexicographic order of their
 *          lower-left cells; each block's patch holds every unknown of the cells within o
 *          layers of it (periodic), and its correction is injected only into the unknowns of
 *          the unexpanded block (restricted injection, Sec. 3.3).  The box smoother is the
 *          multiplicative one, so it needs smoother = CAV_SMOOTH_COLOURED on every level
 *          (coloured_levels 0), FP32 or FP64 inverses, and every smoothing level with
 *          N_l divisible by b and b + 2 o < N_l; otherwise IB_ERR_INVALID.               */
typedef enum { CAV_PATCH_CAV = 0, CAV_PATCH_VANKA = 1, CAV_PATCH_BOX = 2 } cav_patch_kind;
typedef enum { CAV_PREC_FP64 = 0, CAV_PREC_FP32 = 1, CAV_PREC_BF16 = 2 } cav_precision;
/* Smoother of every level:
 *   additive  the weighted additive sweep of Eq. additive_cav_saddle (alpha, Theta = 1/count);
 *   coloured  the multiplicative sweep of Sec. 3.3 with the patches visited class by class:
 *             the patches are split at set-up into classes whose members share no unknown
 *             and are not coupled by any entry of K_E (the Stokes stencils plus E_E's
 *             structural pattern), by first-fit greedy colouring visiting the enlarged
 *             patches in cell order, then the standard ones; inside a class every patch
 *             solves its local residual b_p - (K_E w)_p from the current iterate and adds its
 *             correction (no damping, alpha unused).  Within a class the order is
 *             immaterial, so the result is the sequential multiplicative sweep in
 *             class-by-class order.                                                      */
typedef enum { CAV_SMOOTH_ADDITIVE = 0, CAV_SMOOTH_COLOURED = 1 } cav_smoother;
/* The coloured smoother with BF16 inverses is rejected (IB_ERR_INVALID): rounding the
 * equilibrated inverses to 8 significant bits makes the undamped multiplicative sweep
 * diverge (the FP64 oracle with BF16-rounded inverses diverges the same way). */

typedef struct {
  int32_t kind;        /* cav_patch_kind: CAV (Eq. cav_patch_set), standard Vanka B(1,0)
                          or box B(b,o)                                                    */
  int32_t coarsest_N;  /* halve while N_l / 2 >= coarsest_N (the paper uses 8)             */
  int32_t nu_pre, nu_post;  /* sweeps per level in the V-cycle                             */
  double alpha;        /* relaxation factor of Eq. additive_cav_saddle                     */
  int32_t precision;   /* cav_precision of the stored enlarged-patch inverses              */
  int32_t autotune;    /* 1: time the patch-apply kernel variants on each level's patches at
                          set-up and keep the fastest (all variants give identical bits)   */
  int32_t krylov_capacity;  /* > 0: reserve FGMRES workspace for this many iterations at
                               set-up (0: on the first solve)                              */
  int32_t smoother;    /* cav_smoother (ABI 2)                                              */
  int32_t coloured_levels;  /* coloured smoother: how many levels, from the finest, use it;
                               the coarser smoothing levels use the additive sweep (0: all)  */
  int32_t nu_additive; /* coloured smoother: sweeps per side on its additive levels
                          (0: nu_pre / nu_post)                                             */
  int32_t box_b, box_o; /* BOX patches: block size b >= 1 and overlap o >= 0 (ABI 3; the
                           paper's comparator is B(4,2)); ignored by the other kinds      */
} cav_desc;

typedef struct cav_hierarchy cav_hierarchy;

typedef struct {
  int32_t N;             /* cells per direction on this level                              */
  int32_t n_patches;     /* one patch per cell (N^2) on smoothing levels, or per block (box
                            patches); 1 on the coarsest                                    */
  int32_t n_enlarged;    /* patches that are not a standard 5-unknown Vanka patch (every box
                            patch)                                                          */
  int32_t max_n;         /* largest patch size                                              */
  int64_t sum_n;         /* sum of patch sizes                                              */
  int64_t sum_n2;        /* sum of squared patch sizes                                      */
  int64_t enlarged_sum_n, enlarged_sum_n2;  /* over the patches stored with their own inverse:
                            the enlarged ones, and on a Vanka level with structure the Vanka
                            patches whose unknowns have E_E rows                            */
  int64_t inverse_bytes; /* bytes of the stored inverses (padded layout)                    */
  int64_t ee_nnz;        /* structural nonzeros of E_E on this level                        */
  int32_t ee_rows;       /* velocity rows of E_E with at least one nonzero                  */
  int32_t ee_window;     /* max per-axis index offset between a row and a column of E_E     */
  int32_t is_coarsest;
  int32_t apply_variant;     /* patch-apply kernel variant in use (0 unless autotuned)        */
  float apply_us[5];         /* autotuner's time per launch of each variant (0: not timed)    */
  int32_t n_colours;         /* colour classes of the coloured smoother (0 for additive) (ABI 2) */
  int32_t sweep_form;        /* additive levels (ABI 5): 0 the sweep's parts as separate kernels,
                                1 one fused cooperative kernel (residual, patch apply, scatter
                                and mean removal between grid-wide barriers; same bits)       */
  float sweep_us[2];         /* the set-up's timing of one sweep in each form (0: not timed)  */
} cav_level_info;

/* Builds the level hierarchy, Galerkin E_E^(l-1) = R E_E^(l) P, the patch sets and their
 * equilibrated LU inverses (Sec. 3.2, 3.3, 4) as batched FP64 device kernels, then stores
 * the enlarged-patch inverses in desc->precision.  Level 0 is the finest grid.  With
 * desc->autotune the set-up also times, per additive level, the patch-apply variants and the
 * sweep as separate kernels or one fused kernel, and keeps the fastest (all give the same
 * bits).  Test hooks read from the environment at each call (not part of the method):
 * CAV_FACTOR_GLOBAL=1 factorises every patch with the one-CTA global-memory kernel;
 * CAV_SWEEP_FORM=fused or =separate forces the sweep's form on every additive level. */
ib_status cav_setup(const ib_system* sys, const cav_desc* desc, cudaStream_t stream,
                    cav_hierarchy** out);
/* Numerical re-set-up (ABI 4): when sys's finest E_E has the structural pattern the hierarchy
 * was built from -- the next Newton iterate of a time step, whose S^n and J^n are unchanged and
 * whose force law keeps its band, or a step whose markers stayed within their cells -- the
 * patch sets, colour classes, transfers and captured V-cycle graphs are kept and only the
 * numbers are recomputed into the existing buffers: E_E on every level (Galerkin, Sec. 4), the
 * patch inverses (equilibration and Gauss-Jordan, Sec. 3.3), their storage precision, and the
 * coarsest inverse.  The result is the one cav_setup would build for sys, bit for bit.  sys
 * must have the grid and parameters of the hierarchy's system; the hierarchy is then bound
 * to sys.  IB_ERR_INVALID (hierarchy unchanged) when the pattern differs: call cav_setup.
 * Synchronises the stream. */
ib_status cav_refactor(cav_hierarchy* h, const ib_system* sys, cudaStream_t stream);
ib_status cav_num_levels(const cav_hierarchy* h, int32_t* levels);
ib_status cav_get_level_info(const cav_hierarchy* h, int32_t level, cav_level_info* info);
/* Host copies of the patch sets of one smoothing level in cell order c = j N + i (block
 * order for box patches), each sorted ascending: offsets[n_patches + 1] (int64),
 * dofs[sum_n] (int32).  Pass NULL arrays to query n_patches and sum_n only. */
ib_status cav_patch_export(const cav_hierarchy* h, int32_t level, int64_t* offsets,
                           int32_t* dofs, int32_t* n_patches, int64_t* sum_n);
/* Host copy of the colour class of every patch of one smoothing level, in patch order
 * (cell order c = j N + i, or block order for box patches; coloured smoother only):
 * colour_of_cell[n_patches].  NULL: query *n_colours only.  IB_ERR_INVALID for an additive
 * hierarchy. */
ib_status cav_colour_export(const cav_hierarchy* h, int32_t level, int32_t* colour_of_cell,
                            int32_t* n_colours);
/* Host copy of E_E on one level as CSR over all 2 N_l^2 velocity rows (columns sorted):
 * rowptr[2 N_l^2 + 1], cols[nnz], vals[nnz].  NULL arrays: query *nnz only. */
ib_status cav_ee_export(const cav_hierarchy* h, int32_t level, int64_t* rowptr,
                        int32_t* cols, double* vals, int64_t* nnz);
/* One CAV sweep on level `level`, w updated in place, then the mean pressure removed
 * (Sec. 3.3).  Additive smoother (Eq. additive_cav_saddle):
 *   r = b - K_E w;  w <- w + alpha sum_i R_i^T Theta_i K_{E,i}^{-1} R_i r,
 *   Theta_i = 1 / patch count per unknown.
 * Coloured smoother: for each colour class in turn, for every patch p of the class at once,
 *   w_p <- w_p + K_{E,p}^{-1} (b - K_E w)_p  (multiplicative Schwarz, Sec. 3.3). */
ib_status cav_sweep(const cav_hierarchy* h, int32_t level, const double* b, double* w,
                    cudaStream_t stream);
/* cav_sweep, cav_sweep_noalloc and vcycle_apply then synchronise the stream and read the
 * hierarchy's device status word: IB_ERR_TIMEOUT if a bounded wait of a kernel ran out (the
 * word is cleared).  While the stream is being captured into a CUDA graph they skip that
 * check (and the synchronisation); the next fgmres_solve or checked call reports it. */
/* r = b - K_E^(l) w on level l (rediscretised Stokes part plus Galerkin E_E). */
ib_status cav_residual(const cav_hierarchy* h, int32_t level, const double* b, const double* w,
                       double* r, cudaStream_t stream);
/* bc = R r: velocity by (1/4) P^T of RT0 prolongation, pressure by cell averaging (Sec. 4);
 * r on level l, bc on level l + 1. */
ib_status cav_restrict(const cav_hierarchy* h, int32_t level, const double* r, double* bc,
                       cudaStream_t stream);
/* w += P xc: RT0 velocity and bilinear pressure prolongation (Sec. 4); xc on level l + 1. */
ib_status cav_prolong_add(const cav_hierarchy* h, int32_t level, const double* xc, double* w,
                          cudaStream_t stream);
/* z = bordered direct solve on the coarsest level (Sec. 4): [[K, e],[e^T, 0]] [z; l] = [r; 0]. */
ib_status cav_coarse_solve(const cav_hierarchy* h, const double* r, double* z, cudaStream_t stream);
/* z = B r: one V-cycle (nu_pre, nu_post sweeps per level, zero initial guess) (Sec. 4). */
ib_status vcycle_apply(const cav_hierarchy* h, const double* r, double* z, cudaStream_t stream);
void cav_destroy(cav_hierarchy* h);

/* Allocation-free sweep.  Same result as cav_sweep (the same kernels run in the same
 * order), but its scratch -- the residual (and its FP32 copy), the packed patch corrections
 * and the partial sums of the pressure mean (with the coloured smoother: the partial sums
 * only) -- lives in a fixed 8 MiB device array inside this library
 * (CAV_NOALLOC_SCRATCH_DOUBLES doubles) instead of buffers reserved per hierarchy.  It is for
 * callers that cannot let a call allocate device memory: code that runs with all device
 * memory already handed to its own pool or budget, where a cudaMalloc would fail or
 * fragment it, and code that cannot afford the implicit device synchronisation that
 * cudaMalloc and cudaFree may cause.  The paper has no counterpart: it is an interface
 * variant of cav_sweep, not a step of the method.
 *   - The call allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *   - Every GPU that loads the library holds the array until the process exits.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     and caches it; make that first call before any stream capture.
 *   - A level needs 3 N_l^2 + (enlarged-patch unknowns) + (partial sums) doubles, plus
 *     3 N_l^2 / 2 (an FP32 copy of the residual) on levels with FP32 or BF16 inverses, each
 *     part rounded up to 32; larger levels are rejected with IB_ERR_INVALID and a message
 *     giving both sizes.
 *   - All calls share the one array and it keeps the last call's contents (every part is
 *     fully written before it is read, so nothing needs clearing); calls whose work overlaps
 *     on the GPU (other streams, other host threads) race on it and must be serialised by
 *     the caller.
 *   - The current device must be the one the hierarchy was built on. */
#define CAV_NOALLOC_SCRATCH_DOUBLES 1048576
ib_status cav_sweep_noalloc(const cav_hierarchy* h, int32_t level, const double* b, double* w,
                            cudaStream_t stream);

/* Live timing of the finest level's batched patch-apply launches (the sweep's dominant
 * kernel).  enable = 1 starts recording a CUDA event pair around each such launch, on the
 * stream it is launched on (up to 8192 launches); cav_profile_read waits for the recorded
 * events, returns the number of launches and their summed duration in milliseconds, and
 * clears the record.  Not part of the paper's method: instrumentation for roofline
 * reporting. */
ib_status cav_profile(cav_hierarchy* h, int32_t enable);
ib_status cav_profile_read(cav_hierarchy* h, int32_t* launches, double* total_ms);

/* -------------------------------------------------------------- Krylov (Sec. 5) */

typedef struct {
  double rtol;       /* stop when ||r_k||_2 <= rtol ||ref||_2                           */
  int32_t maxit;     /* no restarts                                                      */
  int32_t rel_to;    /* 0: ref = b, 1: ref = r_0                                         */
  int32_t host_io;   /* 1: b and x are HOST pointers; the call copies them to and from
                        the device inside the call                                       */
  int32_t loop;      /* 0: host-driven iterations (the host reads one small record per
                        iteration); 1: device-driven (ABI 5): the whole solve -- or, in
                        fgmres_solve_batched, the whole batch -- is one CUDA graph launch
                        whose iterations run under a conditional while node, the
                        convergence test setting the loop condition on the device.  The
                        graph is built on the first call and cached with the first
                        hierarchy while the systems, hierarchies, vectors, rtol, maxit and
                        rel_to stay the same (ib_update_structure and cav_refactor make the
                        next call rebuild it).  Results are bitwise those of loop = 0.
                        Device buffers only (host_io must be 0).                          */
} fgmres_desc;

typedef struct {
  int32_t iters, converged;
  double relres_est;   /* |g_{k+1}| / ||ref|| from the Givens recurrence                  */
  double relres_true;  /* ||b - K_E x|| / ||ref|| recomputed at exit                      */
} fgmres_info;

/* Right-preconditioned flexible GMRES with the CAV V-cycle (Sec. 5): x holds the initial
 * guess on entry and the solution on exit.  history (host, nullable, maxit + 1 doubles)
 * receives the relative residual estimate per iteration.  Returns IB_ERR_NOCONV when maxit
 * is reached above tolerance, and also when an iteration's preconditioned vector is not
 * finite (a diverging V-cycle): the solve then stops there, x holds the iterate of the
 * iterations before it and ib_last_error() says so (x and info valid in both cases).
 * Returns IB_ERR_TIMEOUT (info filled, x not valid) when a bounded device wait ran out in
 * any V-cycle of the solve.  Synchronises the stream. */
ib_status fgmres_solve(const ib_system* sys, const cav_hierarchy* h, const double* b, double* x,
                       const fgmres_desc* desc, fgmres_info* info, double* history,
                       cudaStream_t stream);

/* Many independent systems solved together (batched, uneven sizes): the same FGMRES as
 * fgmres_solve for each (systems[i], hierarchies[i], b[i], x[i]), advanced in lockstep with
 * every system on its own library-owned stream so that their V-cycle graphs and Krylov
 * kernels overlap on the device (desc->loop = 0), or as one CUDA graph launch whose branches
 * are the systems' device-driven solves (desc->loop = 1).  Each system stops at its own
 * convergence; infos[i] is filled for every i.  Results are bitwise those of fgmres_solve.
 * Device buffers only (host_io must be 0); a hierarchy may appear once per call.  Waits on `stream` before
 * starting and synchronises everything before returning.  IB_ERR_NOCONV if any system
 * stopped at maxit. */
ib_status fgmres_solve_batched(int32_t count, const ib_system* const* systems,
                               const cav_hierarchy* const* hierarchies, const double* const* b,
                               double* const* x, const fgmres_desc* desc, fgmres_info* infos,
                               cudaStream_t stream);

/* Test hook, not part of the method (ABI 4): while enable != 0 every bounded device-side
 * wait for data in the patch-apply and class-step kernels (a TMA copy landing, a gathered
 * vector) ignores its barrier and runs out after about 2^20 clock cycles, so that tests can
 * check that IB_ERR_TIMEOUT comes back through the calls above without faulting or hanging
 * the device.  Copies already in flight still land before a kernel's blocks exit.  Process
 * wide; call with 0 to restore normal waits. */
ib_status ib_test_wait_stall(int32_t enable);

/* ------------------------------------------------------ learned initial guess (CNN)
 * Not from the paper: a small convolutional network that predicts each time step's initial
 * FGMRES guess from the previous three steps' solutions (u, v, p) and spread Lagrangian
 * forces (f_u, f_v), trained on solutions the solver produced.  FP32, periodic (circular)
 * 3x3 convolutions: conv(in_ch -> hidden) GELU, (n_hidden - 1) x [conv(hidden -> hidden)
 * GELU], conv(hidden -> out_ch).  Tensors are device FP32 [batch][channel][N][N]; parameters
 * are one flat vector, per layer W[cout][cin][3][3] then b[cout].  Loss: mean squared error. */
typedef struct ibnet ibnet;
typedef struct {
  int32_t in_ch, hidden, n_hidden, out_ch;
  uint64_t seed;   /* weight initialisation (splitmix64) */
} ibnet_desc;
ib_status ibnet_create(const ibnet_desc* desc, ibnet** out);
void ibnet_destroy(ibnet* net);
int64_t ibnet_num_params(const ibnet* net);
ib_status ibnet_get_params(const ibnet* net, float* host);
ib_status ibnet_set_params(ibnet* net, const float* host);   /* also resets Adam state */
ib_status ibnet_forward(ibnet* net, const float* in, float* out, int32_t batch, int32_t N,
                        cudaStream_t stream);
/* Loss and all parameter gradients for one batch (host copies; syncs). */
ib_status ibnet_gradients(ibnet* net, const float* in, const float* target, int32_t batch,
                          int32_t N, float* loss, float* grads, cudaStream_t stream);
/* Forward, backward and one Adam step (beta 0.9 / 0.999, eps 1e-8); loss (host) optional. */
ib_status ibnet_train_step(ibnet* net, const float* in, const float* target, int32_t batch,
                           int32_t N, float lr, float* loss, cudaStream_t stream);
/* in (15 x N x N) from three steps x_0, x_1, x_2 (hist_x, device, 3 N^2 FP64, oldest first)
 * and spread forces f_0, f_1, f_2 (hist_f, device, 2 N^2 FP64): three groups of channels
 * (u, v, p, f_u, f_v) holding x_1 - x_0 | f_1 - f_0, then x_2 - x_1 | f_2 - f_1, then
 * x_2 | f_2, each divided by in_scale[c]. */
ib_status ibnet_pack_input(int32_t N, const double* const* hist_x, const double* const* hist_f,
                           const float* in_scale, float* out, cudaStream_t stream);
/* in (5 K x N x N) from K <= 4 steps x_0 .. x_{K-1} (hist_x, device 3 N^2, oldest first) and
 * spread forces f_0 .. f_{K-1} (hist_f, device 2 N^2) in difference form (ABI 4): channel
 * groups holding the backward differences of order K - 1, ..., 1, 0 in time at the newest
 * step of (u, v, p, f_u, f_v) (order 0: the newest fields), each divided by in_scale[c]. */
ib_status ibnet_pack_history(int32_t N, int32_t K, const double* const* hist_x, const double* const* hist_f,
                             const float* in_scale, float* out, cudaStream_t stream);
/* target (3 x N x N) = (x_new - base) / out_scale per field (u, v, p), where base is x_prev,
 * the linear extrapolation 2 x_prev - x_prev2 when x_prev2 is not NULL, or the quadratic
 * extrapolation 3 x_prev - 3 x_prev2 + x_prev3 when x_prev3 is not NULL too (ABI 4). */
ib_status ibnet_pack_target(int32_t N, const double* x_new, const double* x_prev,
                            const double* x_prev2, const double* x_prev3, const float* out_scale,
                            float* out, cudaStream_t stream);
/* out (host) = <a, b> over n FP32 values, products and sums in FP64 in a fixed order
 * (ABI 5): used to fit the scale of the network's correction on held-out steps.  Uses a
 * scratch buffer of the network (one call at a time per network); synchronises the stream. */
ib_status ibnet_inner(ibnet* net, int64_t n, const float* a, const float* b, double* out,
                      cudaStream_t stream);
/* x_out = base + out_scale * delta per field (base as above; delta NULL: base alone): the
 * predicted initial guess. */
ib_status ibnet_apply_delta(int32_t N, const double* x_prev, const double* x_prev2,
                            const double* x_prev3, const float* delta, const float* out_scale,
                            double* x_out, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* IB_CAV_H */
