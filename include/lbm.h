/*
 * lbm.h -- C ABI of the GB300 multilevel octree lattice Boltzmann library.
 *
 * The library runs the data-parallel hot path of the method of Qi, Klimach &
 * Roller, "Implementation of the compact interpolation within the octree based
 * Lattice Boltzmann solver Musubi" (arXiv:1601.06984): per-level pull
 * stream + BGK collide over level-wise, space-filling-curve ordered element
 * arrays (D2Q9 / D3Q19 / D3Q27), ghost filling between levels by compact interpolation
 * (GhostFromCoarser) and by restriction from the children (GhostFromFiner), and
 * the recursive level time stepping with two fine substeps per coarse step.
 *
 * Conventions (all entry points):
 *  - Every function returns an lbm_status; on error lbm_last_error() gives a
 *    one-line message.  No exception crosses the ABI.  After LBM_ERR_ARG,
 *    LBM_ERR_MESH, LBM_ERR_STATE or LBM_ERR_NUMERIC the context stays usable;
 *    after LBM_ERR_CUDA it must be destroyed.
 *  - Host arrays passed in are borrowed for the duration of the call and
 *    copied; host arrays passed out are written before the call returns.
 *  - Element order at the boundary is always the caller's order of the
 *    treeIDs given to lbm_build_mesh.  The internal order (per level,
 *    z-curve sorted, ghosts appended) is hidden.
 *  - Device memory is owned by the caller: lbm_device_bytes() says how much,
 *    the caller allocates it (e.g. with PyTorch) and hands it to lbm_bind()
 *    together with the CUDA stream every kernel is enqueued on.  The library
 *    never allocates or frees device memory itself.
 *  - Calls that produce host results synchronise the bound stream; lbm_step,
 *    lbm_fill_ghosts and lbm_set_force return once their work is enqueued.
 *  - Units: lattice units of each element's own level (dx_L = 1, dt_L = 1);
 *    positions, volumes and forces in reductions as stated per function.
 *  - Direction order of per-direction arrays:
 *      D2Q9 : 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 (+x+y), 6 (-x-y), 7 (+x-y), 8 (-x+y)
 *      D3Q19: 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z, 7 (+x+y), 8 (-x-y),
 *             9 (+x-y), 10 (-x+y), 11 (+x+z), 12 (-x-z), 13 (+x-z), 14 (-x+z),
 *             15 (+y+z), 16 (-y-z), 17 (+y-z), 18 (-y+z)
 *      D3Q27: the D3Q19 directions, then 19 (+x+y+z), 20 (-x-y-z), 21 (+x+y-z),
 *             22 (-x-y+z), 23 (+x-y+z), 24 (-x+y-z), 25 (-x+y+z), 26 (+x-y-z)
 *    Strain-rate components: 2D xx, yy, xy; 3D xx, yy, zz, xy, yz, xz.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque; created by lbm_build_mesh, freed by lbm_destroy */

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,      /* bad argument (null pointer, out-of-range value)        */
  LBM_ERR_MESH = -2,     /* mesh rejected (see lbm_last_error for the rule broken) */
  LBM_ERR_CUDA = -3,     /* a CUDA runtime call failed                             */
  LBM_ERR_OOM = -4,      /* host allocation failed                                 */
  LBM_ERR_STATE = -5,    /* wrong call order (e.g. lbm_step before lbm_bind)       */
  LBM_ERR_NUMERIC = -6,  /* the optional mass check (params.check_every) failed   */
  LBM_ERR_INTERNAL = -7
} lbm_status;

enum { LBM_FP64 = 0, LBM_FP32DEV = 1, LBM_BF16DEV = 2 };
enum { LBM_TIME_LINEAR = 0, LBM_TIME_TWO_LAYER = 1, LBM_TIME_DIFFUSIVE = 2 };
enum { LBM_BC_PERIODIC = 0, LBM_BC_WALL = 1, LBM_BC_VELOCITY_IN = 2, LBM_BC_PRESSURE_OUT = 3 };
enum { LBM_OUTLET_LINEAR = 0, LBM_OUTLET_ZERO_GRADIENT = 1 };
enum { LBM_INLET_UNIFORM = 0, LBM_INLET_PARABOLIC = 1 };

/* Simulation parameters.
 *  stencil       9 (D2Q9), 19 (D3Q19) or 27 (D3Q27, the paper's 3D lattice); Sec. 2.1.
 *                Weights by |c|^2: D2Q9 4/9, 1/9, 1/36; D3Q19 1/3, 1/18, 1/36;
 *                D3Q27 8/27, 2/27, 1/54, 1/216.
 *  precision     LBM_FP64: pdfs stored and computed in double.
 *                LBM_FP32DEV: each pdf stored as float deviation g_i = f_i - w_i rho0,
 *                             arithmetic in float.
 *                LBM_BF16DEV: same deviation stored as bfloat16, arithmetic in float.
 *  time_mode     LBM_TIME_LINEAR: fine ghosts refilled before the second fine substep
 *                from the mean of the coarse source moments at t and t+1.
 *                LBM_TIME_TWO_LAYER: two fine ghost layers filled at the synchronous
 *                step and advanced by the fine kernel (Sec. 2.2, last paragraph).
 *                LBM_TIME_DIFFUSIVE: diffusive scaling, dt proportional to dx^2
 *                (Sec. 2.2 names it as the case for more than two layers): four
 *                fine substeps per coarse step, four fine ghost layers filled at
 *                the synchronous step (the inner three advanced by the fine
 *                kernel), omega the same on every level, and each level in its
 *                own lattice units: for the same flow its velocity is 2^-l,
 *                its density deviation and strain rate 4^-l times the coarsest
 *                level's (l the level index from the coarsest).  The ghost
 *                fills convert between them.
 *  extent        domain box in elements of the coarsest level present (unused axes 1).
 *  bc            per face x-, x+, y-, y+, z-, z+; PERIODIC must be set on both faces of
 *                an axis.  WALL = half-way bounce-back, VELOCITY_IN = velocity
 *                bounce-back with u_in, PRESSURE_OUT = extrapolation outlet with the
 *                normal pdf pressure-corrected to rho0: f_i = f^eq_i(rho0, u) +
 *                f^neq_opp(i), f^neq the pre-collision non-equilibrium part (Sec. 2.3).
 *  omega_coarse  BGK relaxation rate on the coarsest level, in (0,2); finer levels
 *                follow 1/omega_f - 1/2 = 2 (1/omega_c - 1/2) (Sec. 2.2, Eq. fneq_scale),
 *                except in LBM_TIME_DIFFUSIVE, where every level has omega_coarse.
 *  rho0          reference density (outlet density, deviation offset).
 *  u_in          inlet velocity (lattice units of the coarsest level; in
 *                LBM_TIME_DIFFUSIVE a level l inlet applies u_in 2^-l).
 *  use_force     nonzero: a per-element body force (Guo forcing) is applied.
 *  outlet        extrapolation of the outlet's tangential and oblique pdfs:
 *                LBM_OUTLET_LINEAR (0): 2 f(x - n) - f(x - 2n), as in Sec. 2.3;
 *                LBM_OUTLET_ZERO_GRADIENT (1): f(x - n), for relaxation rates
 *                near 2 where the linear rule is unstable.  Other values:
 *                LBM_ERR_ARG from lbm_build_mesh.
 *  inlet_profile LBM_INLET_UNIFORM (0): u_in on every inlet link;
 *                LBM_INLET_PARABOLIC (1): u_in 6 t (1 - t) per axis tangential to
 *                the inlet face, t the position of the link's boundary point
 *                x - c_i / 2 across the domain (mean u_in; Sec. 4.2 inflow).
 *  bouzidi       0: half-way bounce-back on obstacle links; 1: linearly
 *                interpolated bounce-back (Bouzidi, Sec. 2.3) with the wall at
 *                x - q c_i, q per link from lbm_set_link_q (1/2 until set).
 *  n_levels      0: the hierarchy spans the levels of the treeIDs (coarsest to
 *                finest present).  n > 0: exactly n levels from the coarsest
 *                one present; levels beyond the finest present hold no element
 *                (an empty refined region), and the recursive stepping of
 *                Sec. 2.2 still runs through them (each takes its two substeps
 *                per step of the next coarser level, with nothing to update).
 *                n below the span of the treeIDs, or above 16: LBM_ERR_ARG.
 *  check_every   0: no check.  M > 0: lbm_step computes the FP64 mass
 *                (out[0] of lbm_reduce) every M coarse steps, counted across
 *                calls, and returns LBM_ERR_NUMERIC if it is not finite or, with
 *                mass_band > 0, if |mass / mass_ref - 1| > mass_band.  mass_ref
 *                is the mass at the start of the first lbm_step after lbm_bind,
 *                lbm_init or lbm_set_state.  The check synchronises the stream.
 *                Negative: LBM_ERR_ARG.
 *  mass_band     relative band of the mass check (0: finiteness only; negative
 *                or not finite: LBM_ERR_ARG).
 *  adjoint_tape  how lbm_adjoint records the forward steps it reverses (the
 *                gradients are the same either way): 1 records all steps of a
 *                checkpoint segment in one recompute (two forward passes per
 *                step); 2 recomputes the segment, then each step once more
 *                while recording it (three passes, less memory); 0 picks 1
 *                when its workspace holds at most twice the states of 2 or at
 *                most 8 GiB of states, else 2.  Other values: LBM_ERR_ARG. */
typedef struct {
  int32_t stencil;
  int32_t precision;
  int32_t time_mode;
  int32_t extent[3];
  int32_t bc[6];
  double omega_coarse;
  double rho0;
  double u_in[3];
  int32_t use_force;
  int32_t outlet;
  int32_t inlet_profile;
  int32_t bouzidi;
  int32_t n_levels;
  int32_t check_every;
  double mass_band;
  int32_t adjoint_tape;
} lbm_params;

/* Build the multilevel mesh on the host (no device work).
 * Sec. 3.1: every element is a treeID (int64): level L holds ids
 * off(L) .. off(L+1)-1 with off(L) = (2^{dL}-1)/(2^d-1), the remainder being the
 * z-curve (Morton) index at that level, x bit lowest.  levels[k] must equal the
 * level encoded in tree_ids[k].  Boxes not covered by any element inside the
 * domain are solid (half-way bounce-back; their links count toward the
 * obstacle force).  Level interfaces may differ by one level only (Sec. 2.2) and
 * must leave room for the ghost layers; violations return LBM_ERR_MESH.
 * Sec. 3.2: per level the elements are stored as GhostFromCoarser | fluid |
 * GhostFromFiner (inner) | GhostFromFiner (outer), each z-curve sorted.
 * On success *out owns a new context. */
lbm_status lbm_build_mesh(const int64_t* tree_ids, const int8_t* levels, int64_t n,
                          const lbm_params* params, lbm_ctx** out);

/* Per level, 10 int64 each: level, fluid, GFC, GFF inner, GFF outer, padded
 * element count, boundary-value links (outlet links, plus the obstacle links
 * with params.bouzidi), obstacle links, interior bricks, boundary bricks.  An
 * interior brick is an aligned block of 64 fluid elements of the level (4^3
 * in 3D, 8^2 in 2D) whose stencil neighbours are all such blocks; the
 * stream-collide locates their pull sources from a per-brick table instead
 * of the neighbour list; a boundary brick is a block of 64 fluid elements
 * whose links through an incomplete neighbour block use the neighbour list.
 * cap = rows available in info. */
lbm_status lbm_mesh_info(const lbm_ctx* ctx, int64_t* info, int32_t cap, int32_t* nlevels);

/* Obstacle links: fluid elements whose neighbour x - c_i is a solid cell.
 * Per link the caller-order element index and the direction i (lbm.h order),
 * level by level, elements ascending.  Writes min(cap, count) entries (elem and
 * dir may be NULL when cap is 0) and the count to *n. */
lbm_status lbm_obstacle_links(const lbm_ctx* ctx, int64_t* elem, int8_t* dir, int64_t cap, int64_t* n);

/* Wall distance per obstacle link, n = the count of lbm_obstacle_links and q in
 * that order: the wall lies at x - q c_i, q in (0, 1].  Sec. 2.3 interpolated
 * bounce-back; requires params.bouzidi (LBM_ERR_STATE otherwise), q outside
 * (0, 1] or a wrong n give LBM_ERR_ARG.  Host array; may be called before or
 * after lbm_bind. */
lbm_status lbm_set_link_q(lbm_ctx* ctx, const double* q, int64_t n);

/* Bytes of the single device workspace the caller must allocate (256-byte
 * aligned start) before lbm_bind. */
lbm_status lbm_device_bytes(const lbm_ctx* ctx, uint64_t* bytes);

/* Bind the device workspace and CUDA stream (cudaStream_t passed as void*; NULL =
 * legacy default stream) and upload the static mesh tables.  The workspace
 * must stay allocated until lbm_destroy.  All pdfs start at rest equilibrium
 * w_i rho0. */
lbm_status lbm_bind(lbm_ctx* ctx, void* device_workspace, uint64_t bytes, void* stream);

/* Initial state from macroscopic fields (Sec. 4.1):
 *   f*_i = f^eq_i(rho, u) + (1 - omega_L) f^neq_i + df_i,
 *   f^neq_i = -(w_i rho / (c_s^2 omega_L)) (c_i c_i - c_s^2 I) : S,
 * stored as the post-collision state at t = 0.  rho[n], u[n][d], S[n][nS] (level
 * lattice units; may be NULL for S = 0), df[n][Q] (may be NULL).  Host
 * arrays, caller order.  Ghost elements are filled on the next step. */
lbm_status lbm_init(lbm_ctx* ctx, const double* rho, const double* u, const double* S,
                    const double* df);

/* Body force F[n][d] per fluid element (level lattice units), Guo forcing.
 * Requires params.use_force. */
lbm_status lbm_set_force(lbm_ctx* ctx, const double* F);

/* Advance n_coarse coarse time steps (Sec. 2.2 recursive level stepping:
 * GhostFromFiner, then GhostFromCoarser, then stream+collide on the level, then
 * two substeps of the next finer level).  Pairs of coarse steps replay a CUDA
 * graph captured on first use, a remaining single step a one-step graph (one
 * of each per A/B parity state; dropped by lbm_set_params and lbm_bind), on
 * the bound stream; in timing mode 1 every step is launched kernel by kernel
 * (the adjoint's recomputed steps too).  Both paths
 * issue the same kernels; in the graphs the three stream-collide kernels of a
 * level (interior bricks, boundary bricks, neighbour list: disjoint elements,
 * the same source state) run as parallel branches, joined before the next op,
 * which leaves every result bitwise the same.  With params.check_every = M
 * the mass is checked after every M-th coarse step (see lbm_params); a failed
 * check returns LBM_ERR_NUMERIC right after that step, with the state left as
 * it was then (the context stays usable, e.g. for lbm_set_state). */
lbm_status lbm_step(lbm_ctx* ctx, int64_t n_coarse);

/* Fill every ghost element from the current state (the synchronous-time part
 * of a step without stream/collide), coarsest interface first. */
lbm_status lbm_fill_ghosts(lbm_ctx* ctx);

/* Macroscopic fields of every element from the stored post-collision state:
 * rho = sum f*, rho u = sum c f* - F/2, S_ab = -(3 omega / 2 rho) sum c_a c_b f^neq
 * (Sec. 2.1) with f^neq = (f* - f^eq - F_i)/(1 - omega).  rho[n], u[n][d],
 * S[n][nS]; any may be NULL.  Caller order, level lattice units. */
lbm_status lbm_moments(lbm_ctx* ctx, double* rho, double* u, double* S);

/* FP64 reductions over fluid elements, deterministic order:
 * out[0] mass sum rho vol, out[1..3] momentum sum rho u vol, out[4..6] force on
 * solid obstacles by momentum exchange (Sec. 2.3, half-way bounce-back: each
 * link carries 2 c f*), in finest-level lattice units, out[7] kinetic energy
 * sum rho |u|^2 vol / 2; vol = 2^{-d (L - Lmin)}.  In LBM_TIME_DIFFUSIVE the
 * mass, momentum and kinetic energy are in the coarsest level's lattice units
 * (rho0 + 4^l (rho - rho0), 2^l rho u, 4^l rho |u|^2 / 2 per element of level
 * index l) and the force in the finest level's.  Each element's moments are
 * formed in the storage's compute type; with FP32 compute (FP32 and BF16
 * deviation storage) a thread's sum over its elements is kept as a two-float
 * pair (about 48 bits), everything after that in FP64. */
lbm_status lbm_reduce(lbm_ctx* ctx, double out[8]);

/* lbm_reduce_noalloc: the same eight FP64 values as lbm_reduce, computed by the
 * same kernels in the same order (identical results), for callers that cannot
 * allocate device memory when they ask for them -- for instance code running
 * under a host framework that owns every device allocation and forbids raw
 * cudaMalloc, or a monitor that must not grow device memory mid-run.  It
 * allocates nothing and uses no caller scratch: the block partial sums and the
 * result live in a static device array of the library (4096 x 8 + 8 doubles,
 * about 256 KiB), held on every GPU that loads the library until the process
 * exits.  The caller passes the bound context (input) and out[8] (host output).
 *  - Limit: meshes with at most 8 levels (512 partial rows per level); deeper
 *    hierarchies get LBM_ERR_ARG with a message naming lbm_reduce instead.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device made current for the lookup);
 *    make that first call before any CUDA stream capture.
 *  - All calls share the one array and every call overwrites what it reads,
 *    so nothing carries over between calls; calls that overlap on the GPU
 *    (other streams, other threads, other contexts on the same device) race
 *    and must be serialised by the caller.
 * The paper has no counterpart: this is an interface convenience of the
 * library, not a step of the method. */
lbm_status lbm_reduce_noalloc(lbm_ctx* ctx, double out[8]);

/* Post-collision pdfs f*[n][Q] of the fluid elements as FP64 (deviation storage
 * converted back to f), caller order. */
lbm_status lbm_get_state(lbm_ctx* ctx, double* f);

/* Restore a state written by lbm_get_state: f[n][Q] post-collision pdfs of
 * the fluid elements (FP64, caller order), converted to the storage type
 * (deviation storage subtracts w_i rho0).  Ghost elements are refilled on the
 * next step.  With lbm_get_state this is a checkpoint / restart of the
 * simulation state; in FP64 the round trip is exact. */
lbm_status lbm_set_state(lbm_ctx* ctx, const double* f);

/* Ghost elements: count, then info[n][6] (level, kind 1=GFC 2=GFF, layer, x, y, z
 * at the element's level) and f[n][Q] (FP64) of the current state.  In
 * LBM_TIME_LINEAR mode lbm_step does not refill the outer GhostFromCoarser
 * layer (layer 2: no fluid element reads it); lbm_fill_ghosts fills every
 * ghost. */
lbm_status lbm_ghost_count(const lbm_ctx* ctx, int64_t* n);
lbm_status lbm_get_ghosts(lbm_ctx* ctx, int64_t* info, double* f);

/* Host utility, Sec. 3.1 (weight based domain decomposition): z-curve order of
 * the elements, workload weights w = 2^{L - Lmin} (Eq. weight), cumulative
 * weights W, and the part of each sorted element when W is split into nparts
 * equal shares.  order[n] (indices into tree_ids), weights[n], cumulative[n],
 * part[n] in sorted order; any output may be NULL. */
lbm_status lbm_sfc_partition(const int64_t* tree_ids, int64_t n, int32_t d, int32_t nparts,
                             int64_t* order, int64_t* weights, int64_t* cumulative,
                             int32_t* part);

/* Halo plan of a partitioned mesh (Sec. 3.1 weight-based decomposition along
 * the space-filling curve, Sec. 3.2 halo elements); host only, no device work.
 * part[n]: the owning part of every element in caller order, 0 <= part <
 * nparts (for instance the split of lbm_sfc_partition mapped back through its
 * order).  Part `rank` computes its own fluid elements and the ghost elements
 * they depend on; it must receive the other parts' fluid elements that these
 * computations read: pull sources (also the second node of interpolated
 * bounce-back and the outlet's extrapolation sources), GhostFromCoarser
 * sources and GhostFromFiner children of the ghosts it fills, and the pull
 * sources of the ghost layer the time mode advances.  Each such read takes the
 * current state of the read element's level, so exchanging a level's halo
 * after every stream-collide of that level (and after lbm_init) keeps all
 * reads current.
 * Outputs: recv_count[nparts], the number of elements to receive from each
 * part (0 for rank itself); recv, their caller indices grouped by sending part
 * (parts ascending), ascending within a group, up to recv_cap entries (recv
 * may be NULL with recv_cap 0); *n_ghosts, the number of ghosts the part fills
 * itself, and ghosts, their rows in the lbm_get_ghosts order (ascending), up
 * to ghost_cap entries.  The part sending to r sends, in r's order, the list
 * lbm_halo_plan for r gives under the sender.  Errors: LBM_ERR_ARG (null
 * pointers, part values outside [0, nparts), rank outside [0, nparts)). */
lbm_status lbm_halo_plan(const lbm_ctx* ctx, const int32_t* part, int32_t nparts, int32_t rank,
                         int64_t* recv_count, int64_t* recv, int64_t recv_cap, int64_t* n_ghosts,
                         int64_t* ghosts, int64_t ghost_cap);

/* Change the coarsest relaxation rate (finer levels follow Eq. fneq_scale, or
 * keep it in LBM_TIME_DIFFUSIVE) and,
 * if u_in is not NULL, the inlet velocity, without rebuilding the mesh.  The
 * state is kept. */
lbm_status lbm_set_params(lbm_ctx* ctx, double omega_coarse, const double* u_in);

/* Discrete adjoint of n_coarse coarse steps (reverse mode, hand-written
 * kernels for every forward op: pull stream + BGK collide with Guo forcing,
 * outlet values, GhostFromCoarser source moments and compact interpolation,
 * GhostFromFiner restriction; Sec. 2.1-2.3 forward, the paper has no
 * adjoint).  Starting from the current state it runs the n_coarse forward steps
 * (the same arithmetic as lbm_step), evaluates the objective at the end,
 *   objective 0: kinetic energy  sum_fluid vol rho |u|^2 / 2,
 *   objective 1..d: obstacle force component (momentum exchange, as lbm_reduce),
 * and returns J and its gradients with respect to the body-force field
 * dJ_dF[n][d] (caller order, level lattice units), omega_coarse (dJ_domega) and
 * u_in (dJ_duin[3]), all at fixed initial pdfs, and the gradient with respect to
 * those initial post-collision pdfs dJ_df0[n][Q] (caller order; chain it with
 * the derivative of whatever produced the initial state, e.g. the omega
 * dependence of the lbm_init non-equilibrium part); any output may be NULL
 * (with dJ_dF NULL the per-element force adjoint is not accumulated at all).
 * Checkpoints: the state every K
 * coarse steps; each segment is recomputed once, and every step once more while
 * its op inputs are recorded.  adj_ws is a device workspace of
 * lbm_adjoint_bytes(n_coarse, K) bytes owned by the caller.  Afterwards the
 * simulation is at the final state, as after lbm_step(n_coarse).  The
 * gradient with respect to F is that of the forced scheme (also when
 * use_force is 0, where it is taken at F = 0).  LBM_TIME_DIFFUSIVE has no
 * adjoint: both calls return LBM_ERR_STATE there. */
lbm_status lbm_adjoint_bytes(lbm_ctx* ctx, int64_t n_coarse, int32_t K, uint64_t* bytes);
/* The workspace holds, besides the adjoint buffers, ceil(n_coarse / K)
 * checkpoints and the final state, and (params.adjoint_tape) either K step
 * states plus one step's snapshots, or K steps' snapshots plus two states per
 * step but the last (each a full [Q][Ntot] state of the storage type). */
lbm_status lbm_adjoint(lbm_ctx* ctx, int64_t n_coarse, int32_t K, int32_t objective, void* adj_ws,
                       uint64_t bytes, double* J, double* dJ_dF, double* dJ_domega, double* dJ_duin,
                       double* dJ_df0);

/* Launches of library kernels enqueued by this context since it was bound. */
lbm_status lbm_kernel_launches(const lbm_ctx* ctx, int64_t* count);

/* Device timing of the step's kernels with CUDA events on the bound stream.
 *  mode 0: off.
 *  mode 1: every launch of lbm_step is bracketed by events, and the steps are
 *          launched kernel by kernel, not replayed from graphs.
 *  mode 2: lbm_step keeps replaying its captured graphs, which then
 *          also record events around the finest level's stream-collide
 *          launches (kinds 0-2) and around their whole group (kind 7: in the
 *          graphs a level's three stream-collide kernels run as parallel
 *          branches, so their span is the level's stream-collide time);
 *          lbm_timing_read returns those of the most recent replay (its two
 *          coarse steps), if not read before.
 * Changing between mode 2 and the others drops the captured graphs.
 * lbm_timing_read synchronises the stream and returns, in row 8 L + k for level
 * index L (coarsest 0) and kernel kind k, the number of timed launches and
 * their summed device time in milliseconds (rows 0..cap-1), then clears the
 * record.  Enabling clears it too.  Kinds: 0 stream-collide of the interior
 * bricks, 1 stream-collide through the neighbour list, 2 stream-collide of the
 * boundary bricks, 3 GhostFromFiner (L: the coarse level holding the ghosts),
 * 4 source moments (L: the coarse level), 5 GhostFromCoarser (L: the fine
 * level holding the ghosts), 6 outlet values, 7 the span of a level's
 * stream-collide kernels (mode 2 only).  Other modes: LBM_ERR_ARG. */
lbm_status lbm_timing_enable(lbm_ctx* ctx, int32_t mode);
lbm_status lbm_timing_read(lbm_ctx* ctx, int64_t* launches, double* ms, int32_t cap);

/* Measured fused multiply-add rate of the current CUDA device in GFLOP/s
 * (a multiply-add counts as two operations): LBM_FP64 for double,
 * LBM_FP32DEV for float; other precisions LBM_ERR_ARG.  A probe kernel keeps
 * every SM busy with independent register-only multiply-add chains, timed with
 * CUDA events on a private stream (one warm-up launch, then five timed).
 * device_scratch: caller-owned device memory of at least
 * 16 x SMs x 256 x 8 bytes (the probe stores one value per thread there);
 * smaller: LBM_ERR_ARG.  Synchronous.  It is the denominator of the FP64
 * stream-collide's ALU roofline; the paper has no counterpart. */
lbm_status lbm_alu_peak(int32_t precision, void* device_scratch, uint64_t bytes, double* gflops);

const char* lbm_last_error(const lbm_ctx* ctx);
void lbm_destroy(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
