/*
 * hydro.h -- C ABI of the GB300 (sm_103a) hydro step library.
 *
 * The library evaluates, for every leaf sub-grid of an adaptive octree, the
 * per-sub-grid step of the fully three-dimensional reconstruction scheme of
 * Octo-Tiger's hydro module (arXiv 2107.10987, Sec. III-B): PPM reconstruction
 * (Colella & Woodward 1984, with its optional contact steepening) along the
 * 13 lines through cell centres to the 26 face, edge and vertex points of
 * each cell, the Kurganov-Tadmor (2000)
 * central flux at the 9 points of every face, the Newton-Cotes (Simpson)
 * face sum, the flux divergence, rotating-frame and spin-torque sources
 * (rotating frame: Sec. I), and the maximum signal speed for the CFL time
 * step; plus the SSP-RK3 stage update with the dual-energy tracer resync of
 * Bryan et al. (1995) (three hydro iterations per step: Sec. IV-A.2).
 *
 * Data layout (all FP64, C order, x fastest; N = 8 or 16 interior cells per
 * sub-grid edge, fixed per context):
 *   U     [n_sub][F][S][S][S]  cell averages with G = 3 ghost layers,
 *                              S = N + 2G, F = 9 + n_species fields in the order
 *                              rho, s_x, s_y, s_z, E, tau, z_x, z_y, z_z, species...
 *   dUdt  [n_sub][F][N][N][N]
 *   amax  [n_sub]
 *   origin[n_sub][3] lower corner of each sub-grid's interior; h [n_sub] cell width
 *   g     [n_sub][3][N][N][N]  optional gravitational acceleration
 * Device pointers unless stated; every buffer is owned by the caller, the
 * library never frees or reallocates one.  The library owns the context, its
 * scratch buffers and the device status word.
 *
 * Streams: every call is asynchronous on the given stream (a cudaStream_t
 * passed as void*, NULL = legacy default stream) and never synchronises the
 * device.  One context per stream; a context is not thread-safe.
 *
 * Errors: 0 on success, a negative HYDRO_E* code otherwise.  Argument errors
 * are detected on the host before any launch.  Faults found on the device
 * (non-positive density or pressure, NaN, an expired bounded wait) never
 * trap: they set bits in the context's device status word, read back by
 * hydro_status() after the caller has synchronised the stream.
 */
#ifndef HYDRO_GB300_H
#define HYDRO_GB300_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define HYDRO_OK 0
#define HYDRO_EINVAL (-1)   /* bad layout, size, pointer alignment or argument */
#define HYDRO_ECUDA (-2)    /* a CUDA call failed; hydro_last_cuda_error() has the text */
#define HYDRO_ENOMEM (-3)   /* scratch allocation failed */
#define HYDRO_EUNSUP (-4)   /* valid but unsupported configuration */
#define HYDRO_ERANGE (-5)   /* batch larger than hydro_step_static's fixed scratch */

/* ---- device status bits (hydro_status) --------------------------------- */
#define HYDRO_ST_NONPHYS 0x1u  /* rho <= 0, eps <= 0 or NaN seen in a step */
#define HYDRO_ST_TIMEOUT 0x2u  /* a bounded device wait expired; results of that launch are invalid */
#define HYDRO_ST_MESH 0x4u     /* an adaptive mesh violated 2:1 balance where a ghost or flux needed it */

/* ---- precision modes ---------------------------------------------------- */
#define HYDRO_PREC_FP64 0   /* every operation in FP64 (the plain method) */
#define HYDRO_PREC_MIXED 1  /* reconstruction and fluxes in FP32; dual-energy recovery, flux-difference
                               accumulation, sources and update in FP64 */

/* ---- boundary conditions of a uniform mesh ------------------------------ */
#define HYDRO_BC_PERIODIC 0
#define HYDRO_BC_OUTFLOW 1  /* zero-gradient: a ghost copies the nearest interior cell */

typedef struct hydro_ctx hydro_ctx_t;

/* Sub-grid layout.  N is the number of interior cells per edge: 8 (the
 * paper's default sub-grid, Sec. III-B) or 16 (its compile-time alternative,
 * the best-performing configuration of Sec. V); ghost the ghost depth (must
 * be 3: the 5-cell PPM stencil plus the face-adjacent ghost row),
 * n_species >= 1.  With N = 16 the step kernels process each sub-grid as its
 * eight 8^3 octants, each read in place from its 14^3 window of the padded
 * array (no copy), and the fused RK3 step takes each octant as a work
 * unit; the mesh kernels work on the 16^3 layout.  Not available with
 * N = 16: hydro_step_static and hydro_gate_data (EUNSUP). */
typedef struct {
  int N;
  int ghost;
  int n_species;
} hydro_layout_t;

/* Run-time options.  de_eta1: dual-energy selection threshold (eps from
 * E - KE where that exceeds de_eta1*E, else from tau^gamma); de_eta2: tracer
 * resync threshold (tau <- eps^(1/gamma) where eps > de_eta2*E).
 * flux_points: 9 (or 0) for the fluxes at the 9 points of every face summed
 * with Simpson weights (the new hydro module, Sec. III-B), 1 for the flux at
 * the face centre only (the old module the paper compares it with: the
 * same reconstruction, fluxes only at the centres of cell faces).
 * contact: 1 turns on PPM contact-discontinuity detection and steepening of
 * the density and species lines (optional in Sec. III-B; Colella & Woodward
 * 1984: a line whose density jump is a contact, gamma K0 |drho|/min(rho) >=
 * |dp|/min(p) over its two neighbours with K0 = 0.1 (evaluated as gamma K0
 * |drho| min(p) >= |dp| min(rho)), blends both interface
 * values with the neighbours' limited extrapolations by a weight in [0,1]
 * from its second differences, before the monotonicity fix-ups).  With the
 * learned indicator on, cells it marks smooth take the unlimited formula
 * and are not steepened; the others are.
 * spin: 1 feeds each cell's spin angular momentum back into the velocity
 * reconstructed at its quadrature points, read as a rigid rotation of the
 * cell's material: omega = z / I, I = rho h^2 / 6 (a uniform cube about its
 * centre), and v(x_q) += omega x (x_q - x_c), i.e. +-(3 / (rho h)) z x d at
 * the point x_c +- (h/2) d (cell averages rho and z), with omega scaled down
 * where the rotation's corner, at |omega| h sqrt(3)/2, would outrun the
 * cell's sound speed sqrt(gamma (gamma-1) eps / rho), so that it moves at
 * that speed (no feedback for eps <= 0).  The paper defers the spin
 * treatment to the Octo-Tiger method paper, so this is a reading, in the
 * manner of Despres & Labourasse 2015.  Defaults: FP64,
 * cfl 0.4, eta1 1e-3, eta2 0.1, 9 points, contact 0, spin 0. */
typedef struct {
  int precision;   /* HYDRO_PREC_FP64 or HYDRO_PREC_MIXED */
  double cfl;
  double de_eta1;
  double de_eta2;
  int flux_points; /* 9 (0 means 9) or 1 */
  int contact;     /* 0 or 1 */
  int spin;        /* 0 or 1 */
} hydro_mode_t;

/* A batch of leaf sub-grids (device pointers).  g may be NULL. */
typedef struct {
  int n_sub;
  double* U;
  const double* origin;
  const double* h;
  const double* g;
} hydro_batch_t;

/* Create a context for a field layout, ratio of specific heats gamma > 1 and
 * frame angular velocity omega (about +z).  Allocates nothing on the device
 * until the first call that needs scratch.  *out is set on success.
 * Errors: EINVAL (N not in {8, 16}, ghost != 3, n_species < 1, gamma <= 1,
 * non-finite omega, out == NULL), EUNSUP (n_species other than 1). */
int hydro_create(const hydro_layout_t* layout, double gamma, double omega, hydro_ctx_t** out);

/* Replace the run-time options.  Errors: EINVAL (unknown precision, cfl or
 * thresholds outside (0,1], flux_points not in {0, 1, 9}, contact or spin
 * not in {0, 1}). */
int hydro_set_mode(hydro_ctx_t* ctx, const hydro_mode_t* mode);

/* One stage of the semi-discrete operator on every sub-grid of the batch
 * (Sec. III-B; the steps are listed at the top of this file):
 *   dUdt[s] = flux divergence + rotating-frame, gravity and spin sources,
 *   amax[s] = max over all quadrature points of all faces of the sub-grid's
 *             N^3 cells (boundary faces included) of |u_n| + c.
 * B->U must hold filled ghosts.  dt is the stage's time step; the
 * semi-discrete operator does not depend on it (it is accepted for the
 * interface's sake and must be finite and >= 0).  dUdt and amax are written
 * completely.  Alignment: U, dUdt 16-byte aligned.  Precision follows the
 * context's mode: HYDRO_PREC_FP64 matches the FP64 oracle to 1e-12 (error of
 * each field normalised by its largest value in the sub-grid); HYDRO_PREC_MIXED
 * to the FP32 error budget stated in the tests (about 1e-6).
 * face_flux (nullable): the sub-grid boundary faces' sums for coarse-fine
 * flux correction, [n_sub][6][F+3][N][N]: face slot 2a (lower) / 2a+1
 * (upper) of axis a; per face cell [c][b] (b < c the transverse axes) the F
 * face-averaged fluxes and the 3 components of the momentum-flux torque
 * about the adjacent interior cell.
 * Scratch (context-owned, allocated on first need and kept): per persistent
 * CTA 159,744 bytes of flux differences, and in FP64 mode 2,496,000 bytes of
 * line-end buffer (380 MB for one CTA per SM on a 152-SM GPU).
 * Errors: EINVAL (NULL ctx/batch/pointers, n_sub < 0, misaligned U, dt < 0),
 * ENOMEM, ECUDA.
 * n_sub == 0 is a no-op. */
int hydro_step(hydro_ctx_t* ctx, const hydro_batch_t* B, double dt, double* dUdt, double* amax, double* face_flux,
               void* stream);

/* Sub-grid decompositions of the step kernels (launch shape; the results do
 * not depend on it, bit for bit):
 *   HYDRO_DECOMP_ROWS    one thread per row of cells along each axis (192
 *                        threads per sub-grid, two CTAs per SM in mixed
 *                        precision); the edge lines of a cell are
 *                        reconstructed in two axis sweeps and the vertex lines
 *                        in three (27 line evaluations per cell).  The
 *                        learned indicator uses it; the default.  The FP64
 *                        form (ROWS or AUTO; PLANES is mixed only) walks
 *                        each of the 13 lines once per cell along its own
 *                        direction into a per-CTA buffer, then sweeps the
 *                        faces by rows.
 *   HYDRO_DECOMP_PLANES  mixed precision: the sub-grid swept plane by plane
 *                        along z by 768 threads (one CTA per SM), each of the
 *                        13 lines through a cell reconstructed once, the
 *                        primitives in a ring of six planes staged from
 *                        global memory one step ahead, the per-axis flux
 *                        differences kept on chip.
 *   HYDRO_DECOMP_AUTO    the autotuner's choice, else the default. */
#define HYDRO_DECOMP_AUTO 0
#define HYDRO_DECOMP_ROWS 1
#define HYDRO_DECOMP_PLANES 2

/* Autotuner of the step's launch shape for this batch size and the context's
 * precision: times hydro_step (one warm-up, three timed launches each) over
 * the candidate decompositions and persistent grids -- the row sweep with 1,
 * 1.5 and 2 CTAs per SM where they fit and the smallest grid that keeps the
 * number of rounds over the batch; in mixed precision without the indicator
 * also the plane sweep with 1 CTA per SM and its balanced grid -- and keeps
 * the fastest for later steps of this context (*slots_out: its CTAs,
 * nullable; hydro_get_launch gives both).  Overwrites dUdt and amax;
 * synchronises the stream.  Not in the paper. */
int hydro_autotune_step(hydro_ctx_t* ctx, const hydro_batch_t* B, double* dUdt, double* amax, int* slots_out,
                        void* stream);

/* Fix the launch shape of this context's steps in its current precision:
 * the decomposition (HYDRO_DECOMP_*; mixed precision only, the FP64 kernels
 * have rows alone) and the number of persistent CTAs of hydro_step (0: the
 * decomposition's default, one or two per SM).  The fused RK3 step runs the
 * decomposition with as many CTAs as can be resident.  Not in the paper.
 * Errors: EINVAL (unknown decomposition, ctas < 0), EUNSUP (PLANES in FP64). */
int hydro_set_launch(hydro_ctx_t* ctx, int decomposition, int ctas);

/* The launch shape the context's next step will use in its current
 * precision: *decomposition (ROWS or PLANES) and *ctas (either nullable). */
int hydro_get_launch(const hydro_ctx_t* ctx, int* decomposition, int* ctas);

/* SSP-RK3 stage update of the interior cells (ghosts are not touched):
 *   U_new <- alpha_k U0 + beta_k (U + dt dUdt), (alpha, beta) = (0,1), (3/4,1/4),
 *   (1/3,2/3) for stage k = 0, 1, 2; then the tracer resync
 *   tau <- eps_E^(1/gamma) where eps_E = E - |s|^2/(2 rho) exceeds de_eta2 * E.
 * U is B->U.  U_out == NULL: in place on B->U.  Otherwise U_new goes to the
 * interior of U_out (U's padded layout; must not overlap B->U) and B->U is
 * only read, which lets a caller keep the step's initial state without a
 * copy (stage 0 with U0 == B->U writing another buffer).  U0 has U's padded
 * layout (only its interior is read) and may equal B->U.  The time step is
 * *dt_dev (a device scalar, e.g. from hydro_dt) when dt_dev is not NULL,
 * else dt.  FP64 mode: the FP64 oracle's rounding exactly (tau to the
 * library pow's ulps); mixed mode: FMA and an FP32 tracer power.
 * Errors: EINVAL (stage outside 0..2, NULL pointers, overlapping U_out). */
int hydro_update(hydro_ctx_t* ctx, const hydro_batch_t* B, const double* U0, const double* dUdt, double dt,
                 const double* dt_dev, int stage, double* U_out, void* stream);

/* CFL time step on the device: *dt_out = cfl * min_s h[s] / amax[s] (cfl <= 0
 * uses the context's mode).  One launch, no host synchronisation. */
int hydro_dt(hydro_ctx_t* ctx, const double* amax, const double* h, int n_sub, double cfl, double* dt_out,
             void* stream);

/* Interior cells between a compact array and the batch's padded state.  The
 * compact layout holds only the N^3 interior cells of every sub-grid,
 * interior[n_sub][F][N][N][N] FP64 (x fastest; 40,960 bytes per sub-grid
 * instead of the 219,520 of the padded state): the form in which a caller
 * keeps or exchanges the evolved variables of the leaf sub-grids (Sec.
 * III-B), the ghost cells being derived from them by the ghost fill.
 *   hydro_scatter_interior: B->U's interior cells <- interior (ghost cells
 *     untouched);
 *   hydro_gather_interior:  interior <- B->U's interior cells.
 * interior: caller-owned, 16-byte aligned, not overlapping B->U; device
 * memory, or page-locked host memory (cudaHostAlloc / cudaHostRegister),
 * which the kernel then reads or writes directly over the host link (no
 * staging copy; the caller must not touch it until the stream reaches the
 * call).  n_sub == 0 is a no-op; NULL, misaligned or pageable host pointers
 * give HYDRO_EINVAL before any launch.  Pure copies (bitwise), asynchronous
 * on the stream. */
int hydro_scatter_interior(hydro_ctx_t* ctx, const hydro_batch_t* B, const double* interior, void* stream);
int hydro_gather_interior(hydro_ctx_t* ctx, const hydro_batch_t* B, double* interior, void* stream);

/* Ghost fill of a uniform mesh of nbx x nby x nbz sub-grids (sub-grid
 * s = (kz*nby + ky)*nbx + kx, all at one refinement level): every ghost cell
 * copies the cell of the same global position from the neighbouring
 * sub-grid's interior; at the domain boundary the position is wrapped
 * (HYDRO_BC_PERIODIC) or clamped to the nearest interior cell
 * (HYDRO_BC_OUTFLOW).  Ghost exchange between leaf sub-grids, Sec. IV-A.2.
 * Requires B->n_sub == nbx*nby*nbz.  Pure copies (bitwise). */
int hydro_fill_ghosts_uniform(hydro_ctx_t* ctx, const hydro_batch_t* B, int nbx, int nby, int nbz, int bc,
                              void* stream);

/* Global conservation sums over the interior cells of the batch, FP64:
 * sums[k] = sum_s sum_cells U[s][k] h_s^3 for k < F, and
 * sums[F] = sum (x_c s_y - y_c s_x + z_z) h^3 (angular momentum about +z).
 * sums has F+1 device doubles.  Deterministic (fixed reduction order). */
int hydro_conserved_sums(hydro_ctx_t* ctx, const hydro_batch_t* B, double* sums, void* stream);

/* Allocation-free variant of hydro_step.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, such as a host
 * code that gives all device memory to its own pool allocator, or a time
 * loop that cannot afford the device-wide synchronisation an allocation may
 * cause.  It computes exactly what hydro_step computes (FP64 mode only, with
 * the context's flux points, contact steepening and learned indicator), bit
 * for bit, but takes its scratch from a fixed array compiled into
 * the library: HYDRO_STATIC_MAX_SUB slots of 159,744 bytes (30.7 MB), held by
 * every GPU that loads the library until the process exits.
 *   - B->n_sub above HYDRO_STATIC_MAX_SUB returns HYDRO_ERANGE (split the
 *     batch); n_sub == 0 is a no-op; a mixed-precision context returns
 *     HYDRO_EUNSUP.  Other argument errors as hydro_step (EINVAL).
 *   - status: optional device word (caller-owned); it is set to zero, then
 *     receives this call's HYDRO_ST_* bits.  NULL: the bits go to an internal
 *     word nobody reads.
 *   - Calls allocate nothing (no cudaMalloc, no library allocation).  The
 *     first call on a device, with that device current, loads the device
 *     code and looks up the array's address; make that first call before any
 *     stream capture.
 *   - All calls share the array and leave their last contents in it; the
 *     kernel overwrites whatever it later reads.  Calls whose kernels overlap
 *     on the GPU (unordered streams) race on the array: order them. */
#define HYDRO_STATIC_MAX_SUB 192
int hydro_step_static(hydro_ctx_t* ctx, const hydro_batch_t* B, double dt, double* dUdt, double* amax,
                      uint32_t* status, void* stream);

/* ---- adaptive octree meshes -------------------------------------------------
 * Leaves are 8^3 sub-grids of an octree on [-1,1]^3 (Sec. III-B), 2:1 balanced
 * across faces, edges and vertices; leaf s has level leaf_level[s] and integer
 * position leaf_ijk[3s..3s+2] in [0, 2^l)^3 (origin -1 + ijk * 2/2^l, cell
 * width 2/(8 2^l)).  table concatenates, for l = lmin..lmax, the (2^l)^3 entries
 * ((k 2^l) + j) 2^l + i: the leaf index at that position, -1 where it is
 * refined, -2 where it lies inside a coarser leaf.  All device pointers. */
typedef struct {
  int lmin, lmax;
  const int* table;
  const int* leaf_level;
  const int* leaf_ijk;
  int bc;               /* HYDRO_BC_OUTFLOW or HYDRO_BC_PERIODIC */
  /* Optional (NULL: index order): a permutation of 0 .. n_sub-1, the order
   * in which the adaptive-mesh kernels take the leaves.  Results do not
   * depend on it; an order that keeps neighbours close (a space-filling
   * curve) keeps their reads of each other in L2.  An entry outside
   * 0 .. n_sub-1 is skipped and sets HYDRO_ST_MESH. */
  const int* order;
} hydro_amr_t;

/* Ghost fill of the leaves of an adaptive mesh (the ghost exchange of Sec.
 * IV-A.2 across refinement levels), two launches: (1) a ghost cell held by a
 * same-level leaf is copied; one over a refined position is the mean of its 8
 * finer cells (in (dz, dy, dx) order a0..a7, summed ((a0+a1)+(a2+a3)) +
 * ((a4+a5)+(a6+a7)), times 1/8); (2) one inside a
 * coarser leaf is prolonged from the coarse cell: U_C + sum_a s_a o_a with
 * o_a = -1/4 or +1/4 and s_a = minmod(U[C+e_a] - U_C, U_C - U[C-e_a])
 * (conservative).  Outside the domain the position is clamped (outflow) or
 * wrapped (periodic) first.  A 2:1 violation sets HYDRO_ST_MESH. */
int hydro_fill_ghosts_amr(hydro_ctx_t* ctx, const hydro_batch_t* B, const hydro_amr_t* mesh, void* stream);

/* Coarse-fine flux correction of dUdt in place: for a coarse boundary cell
 * whose face borders finer leaves, its face flux is replaced by the mean of
 * the 4 fine sub-face fluxes and its spin torque by the mean of the fine
 * torques moved to the coarse cell centre (T(x_C) = T(x_f) + (x_f - x_C) x
 * F_s).  face_flux: hydro_step's boundary-face output for the same batch.
 * With it the adaptive mesh conserves mass, momentum, energy and angular
 * momentum to round-off. */
int hydro_flux_correct_amr(hydro_ctx_t* ctx, const hydro_batch_t* B, const hydro_amr_t* mesh,
                           const double* face_flux, double* dUdt, void* stream);

/* ---- a whole RK3 time step of a mesh, and its CUDA graphs -----------------
 * One time step (three hydro iterations, Sec. IV-A.2) of a uniform mesh of
 * nbx x nby x nbz sub-grids, state X -> Y:
 *   ghost(X); step(X); dt = cfl min h/amax; Y = X + dt dU      (stage 0)
 *   ghost(Y); step(Y); Y = 3/4 X + 1/4 (Y + dt dU)              (stage 1)
 *   ghost(Y); step(Y); Y = 1/3 X + 2/3 (Y + dt dU)              (stage 2)
 * X and Y are the two state buffers a.U and U_b; the step's initial state is
 * kept in X without a copy and the following step runs Y -> X.
 * dUdt, amax, dt: caller-owned work buffers; *dt holds the step's dt after
 * the step.  All device pointers. */
typedef struct {
  hydro_batch_t a;  /* buffer a: state, origin, h, g (shared by both buffers) */
  double* U_b;      /* buffer b: same layout as a.U, distinct memory */
  int nbx, nby, nbz, bc;
  double* dUdt;     /* [n_sub][F][N][N][N] */
  double* amax;     /* [n_sub] */
  double* dt;       /* one device double */
  double cfl;       /* <= 0: the context's mode */
  /* Adaptive mesh (NULL: the uniform nbx x nby x nbz mesh above).  With a mesh
   * each stage runs hydro_fill_ghosts_amr, hydro_step with face_flux and
   * hydro_flux_correct_amr instead of the uniform ghost fill (nbx, nby, nbz
   * and bc are then ignored).  In HYDRO_PREC_MIXED with 8^3 leaves and the
   * row sweep (no contact steepening or spin feedback) the fill only
   * prolongs the ghost cells inside coarser leaves and the step reads the
   * others where they live: a same-level leaf's interior, or the mean of
   * the eight children in a finer leaf, from a restriction image of every
   * leaf in the context (n_sub x F x 64 doubles).  The new state and *dt
   * equal the full sequence's bit for bit; the ghost cells of the state
   * buffers held by same-level or finer leaves are then not written. */
  const hydro_amr_t* amr;
  double* face_flux;  /* [n_sub][6][F+3][N][N], used with amr */
  /* Nonzero: the whole time step as one persistent launch (uniform mesh and
   * HYDRO_PREC_MIXED only; otherwise the step returns EUNSUP).  Ghost cells
   * are read from the neighbouring sub-grids' interiors instead of being
   * filled (in the context's decomposition, hydro_set_launch), stages 1 and
   * 2 apply their update inside the launch, and a
   * sub-grid's third stage starts as soon as its 27 neighbours have finished
   * their second (bounded waits; HYDRO_ST_TIMEOUT if one expires).  The
   * interiors of the new state and *dt equal the separate launches' bit for
   * bit; the ghost layers of the destination buffer are not written, and
   * dUdt then holds the first stage's rates. */
  int fused;
} hydro_rk3_desc_t;

typedef struct hydro_graph hydro_graph_t;

/* Enqueue one time step on a stream: parity 0 advances a -> b, 1 advances
 * b -> a.  Ten launches on a uniform mesh (two with fused: a clear of the
 * context's sync words and the step); on an adaptive mesh 16 (five per
 * stage and dt), or 15 in the direct-read form (four per stage, two more at
 * the first stage for its restriction images and finer-neighbour tables,
 * and dt).  Errors: EINVAL (inconsistent descriptor, or state
 * buffers a.U and U_b that overlap), EUNSUP (fused with an adaptive mesh or
 * in FP64), ENOMEM. */
int hydro_rk3_step(hydro_ctx_t* ctx, const hydro_rk3_desc_t* d, int parity, void* stream);

/* Capture the two directions of hydro_rk3_step once into CUDA graphs
 * (allocating the context's scratch beforehand, so replays allocate nothing).
 * The state starts in buffer a.  The descriptor's buffers must stay valid
 * and unchanged in address while the graph exists.  A later call on the
 * context that needs larger work buffers (a bigger batch) allocates new
 * ones and keeps the old ones, which the graph uses, until hydro_destroy;
 * the graph and such calls must not run concurrently (one context per
 * stream).  Destroy the graphs before the context. */
int hydro_rk3_graph_create(hydro_ctx_t* ctx, const hydro_rk3_desc_t* d, hydro_graph_t** out);

/* Replay one time step on a stream (alternating a -> b and b -> a). */
int hydro_rk3_graph_launch(hydro_graph_t* g, void* stream);

/* Self-test of the fused step's bounded device wait: one thread waits for
 * `seconds` (0 < seconds <= 1) on a flag that nothing sets, gives up and sets
 * HYDRO_ST_TIMEOUT in the status word, as the fused step does when one of
 * its waits expires.  Asynchronous; read the bit with hydro_status after a
 * synchronise.  Errors: EINVAL, ENOMEM. */
int hydro_selftest_wait(hydro_ctx_t* ctx, double seconds, void* stream);

/* Self-test of the exact FP64 helpers of the FP64 step kernels, which
 * replace FP64 operations by integer operations on the bit patterns (PPM and
 * the MC limiter of Sec. III-B; Colella & Woodward 1984).  For i < n (device
 * arrays x, y of n doubles, out of 2n doubles):
 *   out[2i]     = x_i / 2 as the kernels halve (0.5 x_i rounded to nearest),
 *   out[2i + 1] = the MC-limited slope from the differences (x_i, y_i): 0 if
 *                 x_i y_i <= 0, else sgn(y_i) min(2|x_i|, 2|y_i|, |x_i + y_i|/2).
 * A caller compares them bit for bit with the FP64 operations they stand
 * for.  Asynchronous.  Errors: EINVAL (n < 0, null pointers with n > 0). */
int hydro_selftest_arith(const double* x, const double* y, int n, double* out, void* stream);

/* Which buffer holds the current state: 0 = a, 1 = b. */
int hydro_rk3_graph_state(const hydro_graph_t* g);

/* Release the graphs (after their replays have completed). */
void hydro_rk3_graph_destroy(hydro_graph_t* g);

/* ---- learned smoothness indicator ------------------------------------------
 * A small network (54 -> 32 ReLU -> 32 ReLU -> 1 sigmoid; BF16 parameters,
 * FP32 arithmetic) predicts per cell whether the PPM limiter would change any
 * reconstructed value on the lines through the cell.  In mixed precision with
 * the indicator on, cells predicted smooth use the unlimited interface
 * formula 7/12 (q0 + q1) - 1/12 (q-1 + q2) for every field but the spin
 * (always limited); the rest use the full limited reconstruction (its
 * fallback).  A cell counts as smooth only if every cell of its 3x3x3 block
 * is predicted smooth (the PPM stencils reach two cells out).  Not in the
 * paper: the paper's PPM always
 * limits (Sec. III-B); the indicator is this library's extension.
 * Parameters are packed as W1[32][54], b1[32], W2[32][32], b2[32], w3[32], b3
 * (2849 floats, HYDRO_GATE_NPARAM). */
#define HYDRO_GATE_NPARAM 2849
#define HYDRO_GATE_NIN 54

/* Training data from the method itself, per interior cell of every sub-grid
 * (ghosts filled): X [n_sub*N^3][54] features (density then pressure over the
 * 3x3x3 neighbourhood, (q_k - q_c)/(|q_k| + |q_c|)), y [n_sub*N^3] labels
 * (1 where, on one of the 13 lines and for density, velocity, internal energy,
 * tracer or species, the limited interface pair differs from the unlimited
 * one by more than 1e-4 of the field's scale at the cell -- |q0|, or |v| + c
 * for velocities; FP32 reconstruction).  Either output may be NULL. */
int hydro_gate_data(hydro_ctx_t* ctx, const hydro_batch_t* B, float* X, uint8_t* y, void* stream);

/* Network output (sigmoid) for n samples X [n][54], in the deployed form
 * that hydro_step evaluates: parameters, features and the first hidden
 * layer rounded to BF16, FP32 accumulation. */
int hydro_mlp_forward(const float* params, const float* X, int n, float* out, void* stream);

/* Bytes of work buffer hydro_mlp_loss_grad needs for n samples. */
size_t hydro_mlp_work_bytes(int n);

/* Mean class-weighted binary cross-entropy
 *   L = -mean( w1 y log(out) + w0 (1 - y) log(1 - out) )
 * and its gradient with respect to the FP32 parameters (the forward and
 * backward passes use them rounded to BF16).  grad [HYDRO_GATE_NPARAM],
 * loss (one float, nullable); deterministic (fixed reduction order). */
int hydro_mlp_loss_grad(const float* params, const float* X, const float* y, int n, float w1, float w0, float* grad,
                        float* loss, void* work, size_t work_bytes, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at step count t >= 1. */
int hydro_mlp_adam(float* params, float* m, float* v, const float* grad, int t, float lr, void* stream);

/* Turn the learned smoothness indicator on for this context's steps, in
 * either precision (params: device FP32 parameters, rounded to BF16 into a
 * copy the context owns; cells with output below threshold in (0,1) are
 * predicted smooth), or off (params == NULL).  hydro_step then evaluates
 * the network on the tensor cores (BF16 features and first hidden layer,
 * FP32 accumulation) for the 12^3 block around every sub-grid, and a
 * reconstructed cell whose 3x3x3 block is predicted smooth uses the
 * unlimited interface formula on its lines (spin fields stay limited).
 * Synchronises the stream once (it reads the network's decision for a
 * uniform neighbourhood back to the host).  Changing the parameters while a
 * captured graph of this context may run is the caller's race. */
int hydro_set_indicator(hydro_ctx_t* ctx, const float* params, double threshold, void* stream);

/* Device status bits accumulated since the last call (HYDRO_ST_*), then
 * cleared.  Synchronises nothing: call after the stream has been synchronised. */
int hydro_status(hydro_ctx_t* ctx, uint32_t* flags);

/* Human-readable text of an error code (static storage). */
const char* hydro_strerror(int code);

/* Text of the last CUDA error seen by this thread's calls (static storage per thread). */
const char* hydro_last_cuda_error(void);

/* Release the context and its scratch (after the caller's work on it has completed). */
void hydro_destroy(hydro_ctx_t* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HYDRO_GB300_H */
