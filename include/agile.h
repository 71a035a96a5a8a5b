/*
 * agile.h - C ABI of the GB300 block-AMR finite-volume library (libagile.so).
 *
 * The library advances near-conservation laws dU/dt + div F(U) = S (paper Eq. 1) for
 * Newtonian hydrodynamics (Section 2.3.1, Eqs. 2-6), ideal MHD with GLM divergence
 * cleaning (Section 2.3.3, Eqs. 11-14) and special-relativistic hydrodynamics
 * (Section 2.3.4, Eqs. 15-20) on a block-structured octree of 16^3-cell blocks with two
 * ghost layers (Section 3.1). One call of agile_step is one full SSP Runge-Kutta step of
 * the time loop of Fig. 2: per stage a ghost fill (same-level copy, restriction,
 * prolongation, physical boundaries), the per-block update (primitive recovery, limited
 * linear reconstruction, HLL or TVDLF flux, flux divergence, stage combine; the macro-kernel
 * of Section 2.1.3) and the coarse-fine flux correction; the global CFL time step and the
 * GLM damping (Section 2.3.3) around it. Initialisation follows Fig. 1.
 *
 * Conventions
 *  - Every call returns an agile_status; no call throws, exits or traps. On failure the
 *    message is available from agile_last_error(mesh).
 *  - All host buffers are owned by the caller and only read/written during the call.
 *  - Device memory (state pools, ghost slots, flux registers, descriptors) is owned by
 *    the mesh and comes from the allocator given at creation (cudaMallocAsync on the
 *    mesh's stream when NULL). All kernels run on the mesh's stream.
 *  - Errors found on the device (primitive recovery that does not converge, non-positive
 *    density or pressure) latch into a device status word and are returned by the next
 *    synchronising call (agile_cfl_dt, agile_get_state, agile_conserved_sums,
 *    agile_estimate, agile_regrid, agile_sync).
 *  - Block order: leaves sorted by refinement level, then by Morton (Z-order) index of
 *    their integer block coordinates (x lowest bit). Arrays of per-block data follow it.
 *  - Cell order inside a block: [z][y][x], x fastest, 16 cells per edge, interior only.
 *  - Floating-point data crosses the ABI in FP64, whatever the stencil precision.
 *  - Threads: calls on one mesh or batch must not overlap. Different meshes may be driven
 *    from different host threads once each stage kernel has been launched at least once
 *    (the first launch of a kernel sets its shared-memory attribute in process-wide state);
 *    one process drives one GPU.
 */
#ifndef AGILE_H
#define AGILE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct agile_mesh agile_mesh;

typedef enum {
  AGILE_OK = 0,
  AGILE_EINVAL = 1,     /* invalid argument or configuration */
  AGILE_ENOMEM = 2,     /* the allocator returned NULL */
  AGILE_EBUDGET = 3,    /* a requested size exceeds a documented limit */
  AGILE_ECUDA = 4,      /* a CUDA runtime call failed */
  AGILE_ENOCONV = 5,    /* SRHD primitive recovery did not converge in 50 iterations */
  AGILE_EUNPHYS = 6,    /* non-positive density or pressure, or NaN, met on the device */
  AGILE_ETIMEOUT = 7    /* a bounded device wait gave up */
} agile_status;

enum { AGILE_HD = 0, AGILE_MHD_GLM = 1, AGILE_SRHD = 2, AGILE_FFHD = 3, AGILE_FFHD_HTC = 4 };  /* physics */
enum { AGILE_MINMOD = 0, AGILE_VANLEER = 1 };                  /* limiter */
enum { AGILE_TVDLF = 0, AGILE_HLL = 1, AGILE_HLLC = 2 };        /* Riemann flux */
enum { AGILE_PERIODIC = 0, AGILE_OUTFLOW = 1, AGILE_REFLECT = 2 }; /* boundaries */
enum { AGILE_EOS_IDEAL = 0, AGILE_EOS_SYNGE = 1 };              /* srhd closure */

/* Device allocator: alloc(bytes, stream, ctx) returns device memory or NULL;
 * free(ptr, stream, ctx) releases it in stream order: work already enqueued on `stream` may
 * still read the memory, which the allocator reuses only for work ordered after it (as
 * cudaFreeAsync, or a caching allocator that reuses blocks on the same stream). Both are
 * called only from the calling thread. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* ctx;
} agile_allocator;

/* Problem description.
 *  physics        AGILE_HD | AGILE_MHD_GLM | AGILE_SRHD | AGILE_FFHD (frozen-field
 *                 hydrodynamics, Section 2.3.2: U = (rho, m_par, e, b_x, b_y, b_z) with the
 *                 frozen unit field b set by the initial condition and never updated;
 *                 uniform meshes, TVDLF) | AGILE_FFHD_HTC (the same with hyperbolic
 *                 field-aligned thermal conduction, Eqs. 9-10: U = (rho, m_par, e, q_par,
 *                 b_x, b_y, b_z); q_par relaxes towards htc_kappa0 T^(5/2) b.grad T, T =
 *                 p / rho, over tau = 4 dt and carries energy as -q_par b)
 *  limiter        slope limiter of the piecewise-linear reconstruction on primitives
 *  flux           AGILE_TVDLF (all), AGILE_HLL (hd, mhd), AGILE_HLLC (hd); the
 *                 solvers per module of paper Table 1
 *  rk             2 or 3: SSPRK2 (Heun) or SSPRK3 (Shu-Osher "threestep")
 *  real_bytes     8 (FP64 stencil) or 4 (FP32 stencil; FP64 kept for the SRHD primitive
 *                 recovery, the CFL reduction and the conserved sums)
 *  gamma          ratio of specific heats (ideal gas)
 *  cfl            Courant number: dt = cfl / max_cells sum_d (|v_d| + c_d) / dx_d
 *  glm_alpha      GLM damping parameter alpha (Section 2.3.3; 0.5 in the paper)
 *  base_blocks    level-1 blocks per dimension
 *  xmin, xmax     domain box
 *  bc             boundary kind per face -x, +x, -y, +y, -z, +z; periodic on both faces
 *                 of a dimension or on none
 *  max_level      finest refinement level (1 = uniform grid)
 *  refine_nvars, refine_vars, refine_weights
 *                 conserved variables (indices) and weights of the Loehner estimator
 *  refine_tol     a block refines when its maximum estimate exceeds refine_tol
 *  derefine_ratio a block may coarsen when its maximum estimate is below
 *                 refine_tol * derefine_ratio
 *  lohner_eps     noise filter epsilon of the estimator (0.01)
 *  eos            AGILE_EOS_IDEAL: the ideal gas of every module (Eq. 6, Eq. 21 for srhd);
 *                 AGILE_EOS_SYNGE (srhd only): the Synge gas (Eq. 22) in Mathews'
 *                 approximation h = 5/2 theta + sqrt(9/4 theta^2 + 1), theta = p/rho
 *                 (Section 2.3.4); gamma is then unused by the physics
 *  htc_kappa0     AGILE_FFHD_HTC: conduction coefficient kappa0 >= 0 (ignored otherwise)
 *  eta            AGILE_MHD_GLM: uniform resistivity eta >= 0 (Section 2.3.3: -curl(eta J) in
 *                 the induction equation and div(B x eta J) in the energy equation, J =
 *                 curl B), added in every RK stage as the sources eta lap B and
 *                 eta (J.J + B.lap B) of the stage state, evaluated with the compact
 *                 second-order stencil over the six face neighbours; with eta > 0 the CFL
 *                 step also obeys the diffusive bound: dt = cfl / max(max_cells sum_d
 *                 (|v_d| + c_d) / dx_d, 2 eta sum_d dx_d^-2 at the finest level). Meshes
 *                 only (batches take eta = 0). Must be 0 for the other modules.
 */
typedef struct {
  int physics;
  int limiter;
  int flux;
  int rk;
  int real_bytes;
  double gamma;
  double cfl;
  double glm_alpha;
  int base_blocks[3];
  double xmin[3];
  double xmax[3];
  int bc[6];
  int max_level;
  int refine_nvars;
  int refine_vars[9];
  double refine_weights[9];
  double refine_tol;
  double derefine_ratio;
  double lohner_eps;
  int eos;
  double htc_kappa0;
  double eta;
} agile_config;

/* Create a mesh of level-1 blocks (Fig. 1, "init level one") with uninitialised state.
 * alloc: NULL selects cudaMallocAsync / cudaFreeAsync on the stream. cuda_stream: a
 * cudaStream_t or NULL for the legacy default stream. On success *out owns everything.
 * Errors: AGILE_EINVAL (bad config), AGILE_ENOMEM, AGILE_ECUDA. */
agile_status agile_mesh_create(const agile_config* cfg, const agile_allocator* alloc,
                               void* cuda_stream, agile_mesh** out);

/* Free all device memory of the mesh (through its allocator) and the mesh itself. */
void agile_mesh_destroy(agile_mesh* mesh);

/* Initial condition callback: fill PRIMITIVE variables prim[var * n + i] for the n cell
 * centres (x[i], y[i], z[i]) of one block (the user module's initial condition, Fig. 1).
 * Primitives: hd (rho, vx, vy, vz, p); mhd (rho, v, p, B, psi); srhd (rho, Gamma v, p). */
typedef void (*agile_ic_fn)(const double* x, const double* y, const double* z, int n,
                            double* prim, void* user);

/* Evaluate the initial condition on every leaf and upload it (prim -> cons on the device).
 * The callback is remembered for agile_regrid(init = 1). Errors: AGILE_EINVAL, AGILE_ECUDA,
 * AGILE_EUNPHYS. */
agile_status agile_set_state(agile_mesh* mesh, agile_ic_fn ic, void* user);

/* Set the conserved interiors of all leaves: cons[nblk][nvar][16^3] in block order.
 * nblk must equal the current number of leaves. SRHD auxiliaries are cleared (the next
 * primitive recovery starts from the bracket midpoint). Resuming a run from its
 * agile_get_state output therefore continues it bit for bit for hd, mhd and ffhd, and for
 * srhd within the recovery's tolerance (the converged xi agree to about 1e-14 in FP64).
 * A page-locked cons (cudaHostAlloc, cudaHostRegister) is read in place by the conversion
 * kernel; pageable memory is first copied to a device buffer. Synchronises. */
agile_status agile_set_state_blocks(agile_mesh* mesh, const double* cons, size_t nblk);

/* Initial state from primitive values on the host (Fig. 1, the values an agile_ic_fn
 * returns, evaluated by the caller): prim[nblk][nvar][16][16][16], FP64, the blocks in the
 * mesh's block order (see Conventions; after creation the level-1 blocks in Morton order),
 * nvar primitives per cell: hd 5 (rho, v, p), mhd 9 (rho, v, p, B, psi), srhd 5 (rho,
 * u = Gamma v, p), ffhd 6 (rho, v_par, p, b), ffhd_htc 7 (rho, v_par, p, q_par, b).
 * Converted to conserved variables on the device. nblk must equal the mesh's block count
 * (AGILE_EINVAL otherwise). No callback is kept: agile_regrid(init=1) then has nothing to
 * re-evaluate new blocks with and fills them by prolongation like init=0. A page-locked
 * prim is read in place by the conversion kernel, pageable memory staged in chunks.
 * Synchronises. */
agile_status agile_set_state_prims(agile_mesh* mesh, const double* prim, size_t nblk);

/* Global CFL time step of the current state ("Set dt", Fig. 2):
 * dt = cfl / max over leaf cells of sum_d (|v_d| + c_d) / dx_d, with c_d the sound speed
 * (hd), the fast magnetosonic speed along d (mhd) or the largest |characteristic speed|
 * along d (srhd). Also latches c_max = max_cells,d (|v_d| + c_d), the GLM speed c_h.
 * Synchronises the stream. */
agile_status agile_cfl_dt(agile_mesh* mesh, double* dt_out);

/* The two maxima behind agile_cfl_dt for the current state: sum_over_dx = max over leaf
 * cells of sum_d s_d / dx_d (dt = cfl / sum_over_dx) and cmax = max over cells and d of
 * s_d, the GLM cleaning speed c_h of the next step (Section 2.3.3). Either may be NULL.
 * Synchronises. */
agile_status agile_max_speeds(agile_mesh* mesh, double* sum_over_dx, double* cmax);

/* One full SSPRK step of all leaves with time step dt. dt <= 0 takes the CFL step of the
 * current state from device memory without a host round trip. For MHD the GLM source
 * psi *= exp(-dt/2 c_h alpha / min dx) is applied before and after the step (Strang
 * split, Section 2.3.3) with c_h = c_max of the state at the start of the step.
 * Asynchronous: returns after enqueueing on the mesh's stream. */
agile_status agile_step(agile_mesh* mesh, double dt);

/* Refine and coarsen from the Loehner estimator (Fig. 2, "error estimator",
 * "refine/coarsen", "prolong/restrict"): a leaf below max_level whose maximum estimate
 * exceeds refine_tol refines, and so do its face/edge/corner neighbours at a lower
 * level (2:1 balance); 8 sibling leaves all below refine_tol * derefine_ratio coarsen
 * unless a block adjacent to their parent is refined. New children are prolonged
 * (limited linear, minmod) from the parent; a new parent is the mean of its children.
 * init = 1 evaluates the initial condition on the new blocks instead (Fig. 1).
 * n_refined / n_coarsened (may be NULL) receive the counts of refined leaves and of
 * coarsened parents. Synchronises. */
agile_status agile_regrid(agile_mesh* mesh, int init, int* n_refined, int* n_coarsened);

/* Regrid with caller-chosen flags instead of the estimator: flags[nblk] in block order,
 * +1 refine, -1 coarsen candidate, 0 keep; the same 2:1 rules apply. */
agile_status agile_regrid_flags(agile_mesh* mesh, const int* flags, int init,
                                int* n_refined, int* n_coarsened);

/* Number of leaves and of conserved variables (5 hd/srhd, 9 mhd). */
agile_status agile_get_layout(agile_mesh* mesh, size_t* nblocks, int* nvar);

/* Copy the state to the host: level[nblk] (1-based), ijk[nblk][3] integer block
 * coordinates at that level, cons[nblk][nvar][16^3] (FP64). Any pointer may be NULL. A
 * page-locked cons is written in place by the conversion kernel, pageable memory through a
 * device buffer. Synchronises. */
agile_status agile_get_state(agile_mesh* mesh, int* level, int* ijk, double* cons);

/* SRHD auxiliaries (xi, Gamma) of the interiors: aux[nblk][2][16^3]. AGILE_EINVAL for
 * other physics. Synchronises. */
agile_status agile_get_aux(agile_mesh* mesh, double* aux);

/* Volume integrals of the conserved variables over the leaves (FP64 sums of
 * U * cell volume; the paper's high-cadence mass/energy log, Section 4.1): per block on the
 * device (FP32 pools: each thread's values added in FP32 with the exact error of every
 * addition kept, then FP64), then a deterministic compensated (Neumaier) total over the
 * blocks on the device; only the nvar totals come back. The device scratch (nblk x nvar + 16
 * doubles) is allocated at the first call, kept by the mesh for later calls (a diagnostic
 * read every step allocates nothing after the first), grown when the mesh grows and freed
 * with the mesh. Synchronises. */
agile_status agile_conserved_sums(agile_mesh* mesh, double* sums);

/* Conserved sums like agile_conserved_sums, for callers that cannot allocate device memory
 * at the time of the call: a serving loop that reserved its whole device budget up front
 * and forbids further allocation, or a host whose allocator is not re-entrant from this
 * thread (a callback into a framework allocator that is itself mid-allocation). The paper
 * has no counterpart; this is
 * a property of the library. It allocates nothing: its scratch (per-block partial sums and
 * the totals, about 1.2 MB) is a fixed array in device memory that every GPU that loads the
 * library holds until the process exits. The mesh and sums (host, [nvar]) are the caller's.
 * Limit: meshes of at most 16384 leaves; larger ones return AGILE_EBUDGET with a message.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture. All calls share the one array, so calls
 * whose work overlaps on the GPU (several streams or threads at once) race on it; the
 * array keeps the last call's contents, and every call overwrites what it reads.
 * Synchronises the mesh's stream. Results equal agile_conserved_sums bit for bit. */
agile_status agile_conserved_sums_noalloc(agile_mesh* mesh, double* sums);

/* Optically thin radiative losses (Section 2.3.1, the -n_e n_H Lambda(T) sink of Eq. 4)
 * for the hd and mhd modules, in code units de/dt = -rho^2 Lambda(T) with T = p / rho at
 * fixed rho and momentum, integrated exactly per cell by Townsend's (2009) method for a
 * Lambda that is a power law between the table's nodes (the last segment continues
 * above the table; there are no losses at or below T[0], the temperature floor). The
 * losses are Strang split: half of dt before every agile_step, half after it (the CFL
 * speeds of the next step come from the state after the losses).
 *  T, Lambda  host arrays of n nodes, T strictly increasing, T > 0, Lambda > 0, both
 *             finite, and T_k / Lambda_k and the per-segment integrals of 1/Lambda finite
 *             in the stencil precision (float for real_bytes = 4); copied (the call
 *             synchronises the mesh's stream)
 *  n          2..4096 nodes; n = 0 switches the losses off
 * AGILE_EINVAL for srhd or an invalid table (the previous table stays), AGILE_ENOMEM when
 * the device copy cannot be allocated. Nodes uniform in ln T get an O(1) lookup, others
 * a binary search. */
agile_status agile_set_cooling(agile_mesh* mesh, const double* T, const double* Lambda, int n);

/* Maximum Loehner estimate of every leaf (block order) on the current state after a
 * full ghost fill, computed in FP64 without fused multiply-add so that refinement
 * decisions are reproducible bit for bit. Synchronises. */
agile_status agile_estimate(agile_mesh* mesh, double* emax);

/* Face-ghost view of one leaf after a full ghost fill of the current state:
 * out[nvar + naux][20][20][20] (FP64) with the interior at [2, 18) and the six face-ghost
 * slabs filled; edge and corner cells are NaN (the face-based stencil never reads them).
 * Synchronises. */
agile_status agile_get_halo(agile_mesh* mesh, size_t block, double* out);

/* Wait for all work on the mesh's stream and return any latched device error. */
agile_status agile_sync(agile_mesh* mesh);

/* Kernel timing with CUDA events recorded on the mesh's stream around every launch of the
 * stage (update) kernel (for SRHD together with the primitive-recovery pass before it).
 * enable = 1 resets and starts accumulating; agile_kernel_timing synchronises and returns
 * the summed milliseconds and the launch count of the stage kernel. */
agile_status agile_set_kernel_timing(agile_mesh* mesh, int enable);
agile_status agile_kernel_timing(agile_mesh* mesh, double* stage_ms, long long* stage_launches,
                                 long long* total_launches);

/* Device time per phase of the time loop (Fig. 2), from the same CUDA events (recorded while
 * kernel timing is on, since the last agile_set_kernel_timing(mesh, 1)): ms[0] the stage
 * (update) kernel, ms[1] the coarse-fine ghost fill, ms[2] the coarse-fine flux fix-up,
 * ms[3] the refinement estimator; launches (may be NULL, else 4 values) the timed launches
 * of each. The regrid's own work is partly on the host and is not included. The paper has
 * no counterpart (a profiling aid). Synchronises. */
agile_status agile_phase_timing(agile_mesh* mesh, double* ms, long long* launches);

/* ---------------------------------------------------------------------------------------
 * Batched independent solves. Several problems that share one scheme (physics, limiter,
 * flux, rk, real_bytes, gamma, cfl, glm_alpha, eos) but differ in size, box, boundaries and
 * refinement advance together: one pool holds the blocks of all levels of all solves, every
 * RK stage is one persistent launch of the update kernel over all of them (each block with
 * its solve's CFL dt and GLM speed), the coarse-fine ghost fill and flux fix-up of all
 * solves share one launch each, and from the second step after a (re)layout a whole step is
 * replayed from a captured CUDA graph (dt stays on the device). Each solve's result is the same as when
 * it runs alone as an agile_mesh (same kernels, same per-block arithmetic).
 * The paper runs one problem per job; batching is this library's serving form of the
 * same per-block update (macro-kernel of Section 2.1.3, time loop of Fig. 2 per solve).
 * --------------------------------------------------------------------------------------- */
typedef struct agile_batch agile_batch;

/* Create nsolve solves from cfgs[nsolve], each with its level-1 blocks (refine with
 * agile_batch_regrid). The solves share physics, limiter, flux, rk, real_bytes, gamma, cfl,
 * glm_alpha, eos and htc_kappa0 (AGILE_EINVAL otherwise); grids, boundaries and refinement
 * settings are per solve. alloc as for meshes; it is also called with the batch's own
 * upload stream (a non-blocking stream the batch creates at its first upload), for buffers
 * it frees only after an event behind their last reader on the batch stream has completed.
 * cuda_stream NULL makes the batch create its own non-blocking stream (graphs cannot be
 * captured on the legacy default stream). Errors: AGILE_EINVAL, AGILE_ENOMEM, AGILE_ECUDA. */
agile_status agile_batch_create(const agile_config* cfgs, int nsolve, const agile_allocator* alloc,
                                void* cuda_stream, agile_batch** out);
void agile_batch_destroy(agile_batch* batch);

/* Number of blocks and conserved variables of one solve. */
agile_status agile_batch_layout(agile_batch* batch, int solve, size_t* nblocks, int* nvar);

/* Initial condition of one solve (as agile_set_state). Synchronises. */
agile_status agile_batch_set_state(agile_batch* batch, int solve, agile_ic_fn ic, void* user);

/* agile_set_state_prims for solve `solve` of a batch (its blocks in the solve's order).
 * The host array is copied to a device buffer on the batch's own upload stream before the
 * call returns (it may be released then; the copy does not wait for the steps already
 * enqueued on the batch stream), and its conversion is enqueued on the batch stream behind
 * them. A device error is returned by the next synchronising batch call. */
agile_status agile_batch_set_state_prims(agile_batch* batch, int solve, const double* prim, size_t nblk);

/* One full SSPRK step of every solve with its own on-device CFL dt (as agile_step(dt <= 0)).
 * The first call runs eagerly; later calls launch one captured CUDA graph. Asynchronous. */
agile_status agile_batch_step(agile_batch* batch);

/* CFL time step of every solve: dt[nsolve]. Synchronises. */
agile_status agile_batch_cfl_dt(agile_batch* batch, double* dt);

/* State of one solve, as agile_get_state. Synchronises. */
agile_status agile_batch_get_state(agile_batch* batch, int solve, int* level, int* ijk, double* cons);

/* Refinement of the solves of a batch (Fig. 2 regrid, as agile_regrid / agile_regrid_flags
 * for a mesh): the Loehner estimate after a ghost fill of the batch decides the flags of one
 * solve, or of every solve at once with solve = -1 (agile_batch_regrid; the counts returned
 * are summed over the solves), or the caller gives one flag per block of one solve (-1
 * coarsen, 0 keep, 1 refine; agile_batch_regrid_flags). The batch's pools are laid out once
 * more (the unchanged solves' blocks are copied on the device), its descriptor tables rebuilt
 * and the next step's CUDA graph captured again. init != 0 re-applies the initial condition
 * given to agile_batch_set_state to the blocks a refinement creates. Ghost fill of the
 * coarse-fine faces, the flux fix-up and their launches join every batched step from then
 * on (solves with max_level = 1 never refine). Synchronises. */
agile_status agile_batch_regrid(agile_batch* batch, int solve, int init, int* n_refined, int* n_coarsened);
agile_status agile_batch_regrid_flags(agile_batch* batch, int solve, const int* flags, int init,
                                      int* n_refined, int* n_coarsened);

/* Autotuner of the batched stage launches (no counterpart in the paper): times `trials`
 * launches of the first RK stage (which reads the solution and writes only a stage buffer,
 * so the solution is not modified) for eighteen launch shapes and keeps the fastest for
 * every later step (the CUDA graph of a step is captured again). A shape is a staging layout
 * of the stage kernel's shared memory (1: four raw-plane TMA slots and one face-flux buffer,
 * two CTA barriers per plane; 2: five raw slots and two flux buffers, one barrier per plane,
 * more shared memory per CTA; 3: three raw slots and two flux buffers, one barrier per
 * plane, the update reading its stage input from global memory; FP64 stencils time layout 1
 * only), a persistent grid of 1, 2 or 3 CTAs per SM, and blocks taken from an atomic counter
 * or strided by the grid.
 * Results do not depend on the choice: every block's arithmetic is the same.
 *  trials   1..100 timed launches per shape (after one untimed launch)
 *  grid     out: CTAs of the chosen shape; dynamic: out, 1 for the atomic counter;
 *  layout   out: the chosen staging layout (1, 2 or 3); each may be NULL
 *  ms       out (may be NULL, else 18 floats): mean ms per launch of the shapes in the
 *           order layout 1: (1 CTA/SM, counter), (1, strided), (2, counter), (2, strided),
 *           (3, counter), (3, strided), then the same six for layouts 2 and 3 (-1 where not
 *           timed)
 * Synchronises the batch's stream. */
agile_status agile_batch_autotune(agile_batch* batch, int trials, int* grid, int* dynamic, int* layout,
                                  float* ms);

/* Copy the current state of solve src_solve of batch src into solve dst_solve of batch dst
 * (device to device; no counterpart in the paper: it lets a request loop rebuild its batch
 * when solves join or leave without a host round trip). The two solves must have the same
 * blocks (refinement included), domain, boundaries, physics, EOS and stencil precision. Waits for the
 * source batch's stream and the copy (synchronising both); the next step of dst
 * recomputes its CFL speeds. AGILE_EINVAL when the solves differ. */
agile_status agile_batch_copy_solve(agile_batch* dst, int dst_solve, agile_batch* src, int src_solve);

/* Continuous batching (no counterpart in the paper; the serving loop's admission): attach
 * adds a solve with configuration cfg (the batch's scheme, as for agile_batch_create) to the
 * running batch and returns its index in *solve; detach removes one. Neither moves the other
 * solves' states: a solve occupies a contiguous range of the batch's block pool, a detached
 * solve's range becomes a hole that a later attach may fill (first fit), and the stage
 * launches walk a work list of the attached solves' blocks, so a solve joins or leaves at the
 * next step at the cost of rebuilding the descriptor tables (host, then one upload) and
 * capturing the step's CUDA graph again. Only when no hole fits and the pool is full does
 * attach allocate a new pool (the attached solves, this one and a quarter more) and copy the
 * attached solves into it compactly; a detach that leaves a pool of more than 4096 blocks
 * less than 60% used repacks it the same way to the attached solves and a quarter more, so
 * the pool's capacity follows the attached solves in both directions. A
 * detached solve's index is reused by a later attach; using it otherwise returns
 * AGILE_EINVAL. An attached solve's state is zero until agile_batch_set_state or
 * agile_batch_set_state_prims sets it: set it before the next agile_batch_step (a zero
 * density is reported as AGILE_EUNPHYS). Neither waits for the batch's stream: old tables
 * and buffers are released in stream order (the allocator contract above), a solve's own
 * tables are cached until it is regridded, and where the solve has no coarse-fine faces
 * and fits the pool's free blocks only its own range of the block tables and the work list
 * are written (uploaded on the batch's upload stream, copied into place on the batch
 * stream). Errors: AGILE_EINVAL (a different scheme, a
 * bad index), AGILE_ENOMEM, AGILE_ECUDA; device errors surface at the next synchronising
 * batch call. */
agile_status agile_batch_attach(agile_batch* batch, const agile_config* cfg, int* solve);
agile_status agile_batch_detach(agile_batch* batch, int solve);

/* Wait for the batch stream and return any latched device error. */
agile_status agile_batch_sync(agile_batch* batch);

/* Kernel launches enqueued by agile_batch_step so far (graph nodes counted per step). */
long long agile_batch_launches(const agile_batch* batch);

/* Message of the last failed call on this batch. */
const char* agile_batch_last_error(const agile_batch* batch);

/* Failure-detection check of the bounded device waits: launches one kernel that waits on
 * an mbarrier nothing arrives on, polling it at most `limit` times (1 .. 2^24), then returns
 * AGILE_ETIMEOUT with *timed_out = 1 (AGILE_OK and 0 would mean the barrier completed).
 * The stage kernel bounds its TMA-plane waits the same way (about 2^22 polls) and reports
 * AGILE_ETIMEOUT at the next synchronising call instead of spinning forever; the context
 * stays usable. Synchronises `stream` (a cudaStream_t, NULL for the default stream). */
agile_status agile_selftest_bounded_wait(void* stream, unsigned int limit, int* timed_out);

/* Accuracy check of the FP64 stencil's quotient: every FP64 division of the stencil
 * (limiter, primitive recovery, signal speeds, HLL/HLLC weights, the SRHD Newton iteration)
 * is a * r with r the hardware reciprocal estimate of s refined by one third-order
 * Newton-Raphson step. Evaluates that quotient and the IEEE quotient a / s on the device for
 * the n pairs of the HOST arrays s and a (1 <= n <= 2^26; every |s| normal and below 2^1022,
 * every a finite, else AGILE_EINVAL) and returns the largest distance in units of the last
 * place of the IEEE result (*max_ulps, 0 when all agree) and the largest relative difference
 * (*max_rel). Synchronises `stream` (a cudaStream_t, NULL for the default stream). */
agile_status agile_selftest_rcp64(const double* s, const double* a, size_t n, void* stream, double* max_ulps,
                                  double* max_rel);

/* Message of the last failed call on this mesh (static storage owned by the mesh). */
const char* agile_last_error(const agile_mesh* mesh);

/* Library version string. */
const char* agile_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AGILE_H */
